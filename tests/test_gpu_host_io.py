"""The host-buffer entry point (fr3d_invert_host) at one observation depth: page-locked buffers are
read and written in place by the kernels, pageable or unaligned buffers go through staging copies,
and every form gives the bits of the device entry point (and the oracle's result).  With the output
in page-locked memory the autotuner keeps to the fused variants that write every output once."""

import numpy as np
import pytest

import oracle as O
from paper_1703_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    from paper_1703_01216_gb300 import build, fr3d
    assert torch.cuda.is_available()
    build.build()
    fr3d.load()
    prev = fr3d.autotune_mode()
    yield fr3d
    fr3d.autotune_mode(prev)


def _problem(F, n, mp, q, seed):
    w = I.make_workload(n, mp, q=q, n_incl=3, noise_level=0.02, n_alpha=16, seed=seed)
    zeta = O.zeta_from_xi(w.xi_true, w.sources, n, w.x0, w.h, w.zr)
    U = O.forward_dft(zeta, n, w.h, w.zy, w.zr, w.nu)
    nz = w.noise * (w.noise_level * np.linalg.norm(U) / np.linalg.norm(w.noise))
    U = U + nz
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu)
    return w, H, U, float(np.linalg.norm(nz))


def _host_buffers(shape, pinned, misalign):
    """A float32 host tensor of `shape` (pinned or pageable); misalign shifts it by one element
    inside a larger buffer (4-byte aligned only)."""
    size = int(np.prod(shape))
    base = torch.empty(size + 1, dtype=torch.float32)
    if pinned:
        base = base.pin_memory()
    return base[1:].view(shape) if misalign else base[:size].view(shape)


# (128, 150, 2) and (256, 70, 2) run the fused inverse in several waves of resident clusters
@pytest.mark.parametrize("n,mp,q", [(64, 5, 3), (256, 3, 2), (512, 2, 1), (128, 150, 2), (256, 70, 2)])
@pytest.mark.parametrize("output", ["xi", "zeta"])
def test_host_forms_match_device_bits(F, n, mp, q, output):
    F.autotune_mode(1)
    w, H, U, delta = _problem(F, n, mp, q, seed=700 + n + mp)
    kind = F.OUT_XI if output == "xi" else F.OUT_ZETA
    shape = (mp, n, n) if output == "xi" else (q, mp, n, n)
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    opts = F.Opts(alphas=w.alphas, delta=delta, tau=1.1, output=kind, points=w.sources, alpha_idx=idx)
    Ud = torch.as_tensor(U, dtype=torch.float32, device="cuda")
    od = torch.full(shape, float("nan"), device="cuda")
    F.invert(H, Ud, q, od, opts)
    torch.cuda.synchronize()
    ref = od.cpu()
    for pinned, misalign in [(True, False), (False, False), (True, True)]:
        uh = _host_buffers(U.shape, pinned, misalign)
        uh.copy_(torch.as_tensor(U, dtype=torch.float32))
        oh = _host_buffers(shape, pinned, misalign)
        oh.fill_(float("nan"))
        F.invert_host(H, uh, q, oh, opts)
        assert torch.equal(oh, ref), (pinned, misalign)
    # and the device result is the oracle's at the chosen alpha
    k = int(idx.item())
    want = O.invert(U, n, w.x0, w.h, w.zy, w.zr, w.nu, alpha=float(w.alphas[k]), sources=w.sources,
                    output=output)[output]
    got = ref.double().numpy()
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)


def test_host_result_in_fp64(F):
    """FP64 (whole copies through the workspace): the device entry point's bits."""
    w, H, U, delta = _problem(F, 64, 9, 2, seed=91)
    opts = F.Opts(alpha=1e-3, points=w.sources, precision=F.PREC_FP64)
    od = torch.empty((9, 64, 64), dtype=torch.float64, device="cuda")
    F.invert(H, torch.as_tensor(U, dtype=torch.float64, device="cuda"), 2, od, opts)
    torch.cuda.synchronize()
    uh = torch.as_tensor(U, dtype=torch.float64).pin_memory()
    oh = torch.full((9, 64, 64), float("nan"), dtype=torch.float64).pin_memory()
    F.invert_host(H, uh, 2, oh, opts)
    assert torch.equal(oh, od.cpu())


def test_tuner_keeps_write_once_variants_for_mapped_output(F):
    F.autotune_mode(1)
    # a shape no other test tunes: n = 96, M' = 7, Q = 3
    w, H, U, delta = _problem(F, 96, 7, 3, seed=77)
    opts = F.Opts(alpha=1e-3, points=w.sources)
    uh = torch.as_tensor(U, dtype=torch.float32).pin_memory()
    oh = torch.empty((7, 96, 96), dtype=torch.float32).pin_memory()
    F.invert_host(H, uh, 3, oh, opts)
    v, ms = F.autotune_query(H)
    assert v in (0, 3, 4, 5)                 # the variants that write every output once
    assert ms[1] == 0 and ms[2] == 0 and ms[0] > 0 and ms[3] > 0 and ms[4] > 0
    od = torch.empty((7, 96, 96), device="cuda")
    F.invert(H, torch.as_tensor(U, dtype=torch.float32, device="cuda"), 3, od, opts)
    torch.cuda.synchronize()
    assert torch.equal(od.cpu(), oh)
