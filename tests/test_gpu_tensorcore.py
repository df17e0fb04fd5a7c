"""The per-class dense products of Eq. (6) on the tensor cores (FR3D_PREC_BF16TC and FR3D_PREC_BF16X3, M > 1)
against the FP64 oracle: the forward operator, fixed-alpha inversions (Tikhonov and TSVD) and the
discrepancy rule, at the paper's depth counts (M = M' = 51) and at smaller ones.

Error model (relative, per product of a table entry and a right-hand-side value): BF16 rounding of both
operands, 2^-8 (BF16TC); the hi + lo split keeps about 16 bits of each, and the dropped lo * lo term and
the remainders leave about 3 * 2^-18 (BF16X3).  Accumulation is FP32.  Bounds: BF16X3 is held to the FP32
path's own bounds (forward 1e-5, reconstruction 1e-4; measured on GB300: forward <= 1.7e-6, reconstruction
<= 1.7e-5 at alpha = 1e-4 and 1e-2); BF16TC to its per-product error, forward 2^-8 and reconstruction
5 * 2^-8 (measured: forward <= 8.7e-4, reconstruction <= 6.5e-3).  Each test prints its measured errors.
"""

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
    return fr3d


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _problem(case, noise=0.05, n_alpha=16):
    if case == "paper51":
        n, q = 16, 1
        w = I.paper_workload(n, 51, 51, noise_level=noise, n_alpha=n_alpha)
    elif case == "m40x64":
        n, q = 32, 2
        w = I.make_workload(n, 64, q=q, m_obs=40, n_incl=3, noise_level=noise, n_alpha=n_alpha, seed=4242)
    else:
        n, q = 48, 3
        w = I.make_workload(n, 6, q=q, m_obs=4, n_incl=3, noise_level=noise, n_alpha=n_alpha, seed=4343)
    A = O.A_matrices(n, w.h, w.zy, w.zr, w.nu)
    zeta = O.zeta_from_xi(w.xi_true, w.sources, n, w.x0, w.h, w.zr)
    U = O.forward_dft(zeta, n, w.h, w.zy, w.zr, w.nu, A=A)
    nz = w.noise * (noise * np.linalg.norm(U) / np.linalg.norm(w.noise))
    return n, q, w, A, zeta, U + nz, float(np.linalg.norm(nz))


def _levels_away_from_spectrum(A, s2, alphas, gap=1e-3):
    """TSVD levels with no squared singular value within `gap` (relative) of a level: the keep decision
    is then the same for the oracle's SVD and the GPU's Gram eigenvalues."""
    L = A.shape[0]
    sig2 = np.linalg.svd(A.reshape(L * L, A.shape[2], A.shape[3]), compute_uv=False).ravel() ** 2
    out = []
    for a in alphas:
        while np.min(np.abs(sig2 - a * s2)) <= gap * a * s2:
            a *= 1.0 + 3 * gap
        out.append(a)
    return np.array(out)


CASES = ["paper51", "m40x64", "m4x6"]
FWD_TOL = {"BF16X3": 1e-5, "BF16TC": 2.0 ** -8}


@pytest.mark.parametrize("case", CASES)
def test_forward_operator_on_tensor_cores(F, case):
    n, q, w, A, zeta, U, delta = _problem(case)
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu)
    ref = O.forward_dft(zeta, n, w.h, w.zy, w.zr, w.nu, A=A)
    errs = {}
    for name, prec in (("BF16X3", F.PREC_BF16X3), ("BF16TC", F.PREC_BF16TC)):
        u = torch.full((q, H.M, n, n), float("nan"), device="cuda")
        F.fwd_apply(H, dev(zeta), q, u, prec)
        errs[name] = rel(host(u), ref)
    print(f"forward {case}: {errs}")
    for name, e in errs.items():
        assert e <= FWD_TOL[name], errs


# fixed alpha: BF16X3 meets the FP32 path's 1e-4 at both alphas; BF16TC 5 * 2^-8
INV_TOL = {("BF16X3", 1e-2): 1e-4, ("BF16X3", 1e-4): 1e-4, ("BF16TC", 1e-2): 5 * 2.0 ** -8,
           ("BF16TC", 1e-4): 5 * 2.0 ** -8}


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("ra", ["tikhonov", "tsvd"])
def test_fixed_alpha_inversion_on_tensor_cores(F, case, ra):
    n, q, w, A, zeta, U, delta = _problem(case)
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu)
    s2 = O.alpha_scale(A)
    levels = [1e-4, 1e-2] if ra == "tikhonov" else list(_levels_away_from_spectrum(A, s2, [1e-4, 1e-2]))
    errs = {}
    for alpha, nominal in zip(levels, (1e-4, 1e-2)):
        ref = O.invert(U, n, w.x0, w.h, w.zy, w.zr, w.nu, alpha=alpha, sources=w.sources, A=A, ra=ra)
        for name, prec in (("BF16X3", F.PREC_BF16X3), ("BF16TC", F.PREC_BF16TC)):
            info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            for output in ("xi", "zeta"):
                shape = (w.zr.size, n, n) if output == "xi" else (q, w.zr.size, n, n)
                o = torch.full(shape, float("nan"), device="cuda")
                F.invert(H, dev(U), q, o, F.Opts(alpha=alpha, output=F.OUT_XI if output == "xi" else F.OUT_ZETA,
                                                 points=w.sources, precision=prec, info=info,
                                                 ra=F.RA_TSVD if ra == "tsvd" else F.RA_TIKHONOV))
                errs[(name, nominal, output)] = rel(host(o), ref[output])
                assert int(info.item()) == 0                 # no bounded wait gave up
    print(f"fixed alpha {case} {ra}: {errs}")
    for (name, nominal, output), e in errs.items():
        assert e <= INV_TOL[(name, nominal)], errs


@pytest.mark.parametrize("case", ["paper51", "m40x64"])
def test_discrepancy_rule_on_tensor_cores(F, case):
    """BF16X3: residual curves within 1e-4 of the oracle's, the oracle's choice (or a near-tie), and xi at
    that choice within the fixed-alpha bound of its alpha."""
    n, q, w, A, zeta, U, delta = _problem(case)
    ref = O.invert(U, n, w.x0, w.h, w.zy, w.zr, w.nu, alphas=w.alphas, delta=delta, tau=1.1, sources=w.sources, A=A)
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu)
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    res = torch.zeros(w.alphas.size, dtype=torch.float64, device="cuda")
    info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    xi = torch.full((w.zr.size, n, n), float("nan"), device="cuda")
    F.invert(H, dev(U), q, xi, F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources, alpha_idx=idx,
                                      residuals=res, info=info, precision=F.PREC_BF16X3))
    r = host(res)
    err_curve = float(np.max(np.abs(r - ref["res2"]) / ref["res2"]))
    print(f"discrepancy {case}: curve {err_curve:.2e}, index {int(idx.item())} vs {ref['alpha_index']}")
    assert err_curve <= 1e-4, err_curve
    k = int(idx.item())
    thr2 = (1.1 * delta) ** 2
    if k != ref["alpha_index"]:
        lo, hi = sorted((k, ref["alpha_index"]))
        assert np.any(np.abs(ref["res2"][lo:hi + 1] - thr2) <= 1e-3 * thr2), (k, ref["alpha_index"])
        ref = O.invert(U, n, w.x0, w.h, w.zy, w.zr, w.nu, alpha=w.alphas[k], sources=w.sources, A=A)
    assert int(info.item()) == 0
    assert w.alphas[k] >= 1e-4
    assert rel(host(xi), ref["xi"]) <= 1e-4, rel(host(xi), ref["xi"])
    # the standalone rule runs the same projection and sums
    idx2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    res2 = torch.zeros(w.alphas.size, dtype=torch.float64, device="cuda")
    F.choose_alpha(H, dev(U), q, w.alphas, delta, 1.1, idx2, res2, precision=F.PREC_BF16X3)
    assert int(idx2.item()) == k and np.array_equal(host(res2), r)


def test_tensor_core_inversion_replays_in_a_cuda_graph(F):
    n, q, w, A, zeta, U, delta = _problem("m4x6")
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu)
    Ud = dev(U)
    out = torch.empty((w.zr.size, n, n), device="cuda")
    opts = F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources, precision=F.PREC_BF16X3)
    F.invert(H, Ud, q, out, opts)              # tables and workspace are built outside the capture
    torch.cuda.synchronize()
    ref = out.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            F.invert(H, Ud, q, out, opts)
    torch.cuda.current_stream().wait_stream(s)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_tensor_core_precisions_are_rejected_where_they_do_not_apply(F):
    w = I.make_workload(32, 4, q=1, seed=5)          # one observation depth: no per-class contraction
    H = F.kernel_transform(32, w.x0, w.h, w.zr, w.zy, w.nu)
    z = torch.zeros((1, 4, 32, 32), device="cuda")
    u = torch.zeros((1, 1, 32, 32), device="cuda")
    for prec in (F.PREC_BF16TC, F.PREC_BF16X3):
        with pytest.raises(F.Fr3dError):
            F.fwd_apply(H, z, 1, u, prec)
        with pytest.raises(F.Fr3dError):
            F.invert(H, u, 1, torch.empty((4, 32, 32), device="cuda"),
                     F.Opts(alpha=1e-2, points=w.sources, precision=prec))
    w2 = I.make_workload(16, 4, q=17, m_obs=2, seed=6)  # 17 source parameters: above the 16 of one MMA tile
    H2 = F.kernel_transform(16, w2.x0, w2.h, w2.zr, w2.zy, w2.nu)
    with pytest.raises(F.Fr3dError):
        F.invert(H2, torch.zeros((17, 2, 16, 16), device="cuda"), 17, torch.empty((4, 16, 16), device="cuda"),
                 F.Opts(alpha=1e-2, points=w2.sources, precision=F.PREC_BF16X3))
