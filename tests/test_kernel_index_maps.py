"""Index arithmetic of the CUDA kernels, checked on the CPU against the kernels' own tables (parsed from the
sources, so that a change there is checked too): every output position is written exactly once and every
read stays inside its buffer.  These are the checks that precede a new kernel's first GPU run, kept as
regression tests."""

import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1703_01216_gb300", "csrc")


def _read(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def plans():
    """FR3D_PLAN(L, NP, R0, R1, R2) entries of fft_engine.cuh -> {L: [radices]}."""
    out = {}
    for m in re.finditer(r"FR3D_PLAN\((\d+), (\d+), (\d+), (\d+), (\d+)\)", _read("fft_engine.cuh")):
        L, npass, *r = map(int, m.groups())
        out[L] = r[:npass]
    return out


def fused_cfgs():
    """FusedCfg<N> entries of fused.cuh -> {N: (CL, NT, RB, MINB)}."""
    pat = (r"template <> struct FusedCfg<(\d+)> : FusedCfgBase \{ static constexpr int CL = (\d+), NT = (\d+), "
           r"RB = (\d+), MINB = (\d+); \};")
    return {int(m.group(1)): tuple(map(int, m.groups()[1:])) for m in re.finditer(pat, _read("fused.cuh"))}


def passtw_offset(radices, p):
    off, ns = 0, 1
    for i in range(p):
        if ns > 1:
            off += (radices[i] - 1) * ns
        ns *= radices[i]
    return off


def test_tables_parse_and_every_plan_multiplies_out():
    P, C = plans(), fused_cfgs()
    assert len(P) >= 12 and len(C) >= 10
    for L, rad in P.items():
        assert int(np.prod(rad)) == L, (L, rad)
    for N in C:
        assert N in P and N // 2 in P, N            # column length N and row length N/2 both planned


@pytest.mark.parametrize("L", sorted(plans()))
def test_last_pass_outputs_are_a_bijection_and_twiddles_stay_in_their_table(L):
    """last_pass_to: butterfly b of NSEQ sequences owns outputs t = j + r NS (j = b mod BPS) of sequence
    s = b / BPS; reads j + r BPS; twiddle (r - 1) NS + j of the last pass's block."""
    rad = plans()[L]
    R = rad[-1]
    BPS = NS = L // R
    for nseq in (1, 3, 16):
        hits = np.zeros(nseq * L, int)
        for b in range(nseq * BPS):
            s, j = divmod(b, BPS)
            for r in range(R):
                assert 0 <= j + r * BPS < L                       # the read
                hits[s * L + j + r * NS] += 1                       # the emitted output
        assert np.all(hits == 1)
    # the last pass's twiddle block is the end of the table, and every index falls inside it
    off = passtw_offset(rad, len(rad) - 1)
    size = passtw_offset(rad, len(rad))
    if NS > 1:
        idx = [(r - 1) * NS + j for r in range(1, R) for j in range(BPS)]
        assert off + max(idx) < size and off + (R - 1) * NS == size


@pytest.mark.parametrize("N", sorted(fused_cfgs()))
def test_register_accumulator_covers_the_ctas_rows_once(N):
    """Variant 3 of the fused inverse: one row batch of all N / CL rows; butterfly bb = tid + k NT of the
    last row pass keeps its R outputs in registers for every q and writes them at the end to
    ov[sr L + jq + rr NS] (float2 units; a row is L float2).  Every position of the CTA's rows must be
    written exactly once, and the accumulator array [KRA][R] must hold every butterfly."""
    CL, NT, RB0, MINB = fused_cfgs()[N]
    L = N // 2
    RB = N // CL                                                   # variant 3
    R = plans()[L][-1]
    BPS = NS = L // R
    KRA = (RB * BPS + NT - 1) // NT
    assert (RB * L) % NT == 0 and L % CL == 0
    hits = np.zeros(RB * L, int)
    for tid in range(NT):
        for k in range(KRA):
            bb = tid + k * NT
            if bb < RB * BPS:
                sr, jq = divmod(bb, BPS)
                for rr in range(R):
                    hits[sr * L + jq + rr * NS] += 1
    assert np.all(hits == 1)


@pytest.mark.parametrize("N", sorted(fused_cfgs()))
def test_column_owner_of_every_spectrum_column_is_in_the_cluster(N):
    """The row phase gathers column c (kx = n/2 folded onto packed column 0) from CTA c / CPC of the
    cluster through distributed shared memory: the owner rank must be < CL and the offset inside the
    owner's CPC columns."""
    CL = fused_cfgs()[N][0]
    L = N // 2
    CPC = L // CL
    for kx in range(L + 1):
        c = 0 if kx == L else kx
        o = c // CPC
        assert 0 <= o < CL and 0 <= c - o * CPC < CPC


@pytest.mark.parametrize("n,planes", [(16, 1), (24, 3), (48, 2)])
def test_padded_box_embed_and_crop_stay_in_bounds(n, planes):
    """pad.cu: k_embed writes every element of planes x 2n x 2n once and reads the n x n source only in
    the low corner; k_crop reads the box's low corner and writes every element of planes x n x n once."""
    N2 = 2 * n
    dst_hits = np.zeros(planes * N2 * N2, int)
    src_hits = np.zeros(planes * n * n, int)
    for e in range(planes * N2 * N2):
        p, r = divmod(e, N2 * N2)
        y, x = divmod(r, N2)
        dst_hits[e] += 1
        if y < n and x < n:
            src_hits[(p * n + y) * n + x] += 1
    assert np.all(dst_hits == 1) and np.all(src_hits == 1)
    out_hits = np.zeros(planes * n * n, int)
    box_reads = np.zeros(planes * N2 * N2, int)
    for e in range(planes * n * n):
        p, r = divmod(e, n * n)
        y, x = divmod(r, n)
        out_hits[e] += 1
        box_reads[(p * N2 + y) * N2 + x] += 1
    assert np.all(out_hits == 1)
    corner = np.zeros((planes, N2, N2), int)
    corner[:, :n, :n] = 1
    assert np.array_equal(box_reads, corner.ravel())
