"""The zero-padded box (pad = 2): the GPU path against the FP64 oracle's pad = 2 (data and unknowns in
the low corner of the 2n x 2n box, whose circular sums are the aperiodic ones over R; the inversion on
the box, cropped to R).  Tolerances as in test_gpu_parity.py: forward 1e-5 (FP32) and 1e-12 (FP64),
reconstruction 1e-4 at the chosen alpha (FP32), residual curves 1e-5 per candidate."""

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


def _problem(n, mp, q, m, seed, n_alpha=16, noise=0.02):
    w = I.make_workload(n, mp, q=q, m_obs=m, n_incl=3, noise_level=noise, n_alpha=n_alpha, seed=seed)
    A = O.A_matrices(n, w.h, w.zy, w.zr, w.nu, pad=2)
    zeta = O.zeta_from_xi(w.xi_true, w.sources, n, w.x0, w.h, w.zr)
    U = O.forward_dft(zeta, n, w.h, w.zy, w.zr, w.nu, pad=2, A=A)
    nz = w.noise * (noise * np.linalg.norm(U) / np.linalg.norm(w.noise))
    return w, A, U + nz, float(np.linalg.norm(nz))


@pytest.mark.parametrize("n,mp,q,m", [(32, 4, 2, 1), (48, 3, 1, 2)])
def test_forward_and_zeta_match_oracle(F, n, mp, q, m):
    w, A, U, delta = _problem(n, mp, q, m, seed=1100 + n)
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu, pad=2)
    assert H.n == n and abs(H.s2 - O.alpha_scale(A)) <= 1e-12 * O.alpha_scale(A)
    rng = np.random.default_rng(n)
    zeta = rng.standard_normal((q, mp, n, n))
    ref = O.forward_dft(zeta, n, w.h, w.zy, w.zr, w.nu, pad=2, A=A)
    for prec, dt, tol in [(F.PREC_FP32, torch.float32, 1e-5), (F.PREC_FP64, torch.float64, 1e-12)]:
        out = torch.empty((q, m, n, n), dtype=dt, device="cuda")
        F.fwd_apply(H, dev(zeta, dt), q, out, prec)
        assert rel(host(out), ref) <= tol, (prec, rel(host(out), ref))
    zref = O.zeta_from_xi(w.xi_true, w.sources, n, w.x0, w.h, w.zr)
    z = torch.empty((q, mp, n, n), device="cuda")
    F.zeta_from_xi(H, dev(w.xi_true), w.sources, z)
    assert rel(host(z), zref) <= 1e-6


@pytest.mark.parametrize("n,mp,q,m", [(32, 6, 2, 1), (32, 4, 1, 3)])
@pytest.mark.parametrize("output", ["xi", "zeta"])
def test_fixed_alpha_inversion_matches_oracle(F, n, mp, q, m, output):
    w, A, U, delta = _problem(n, mp, q, m, seed=1200 + n + m)
    H = F.kernel_transform(n, w.x0, w.h, w.zr, w.zy, w.nu, pad=2)
    kind = F.OUT_XI if output == "xi" else F.OUT_ZETA
    shape = (mp, n, n) if output == "xi" else (q, mp, n, n)
    for alpha in (1e-4, 1e-2):
        ref = O.invert(U, n, w.x0, w.h, w.zy, w.zr, w.nu, pad=2, alpha=alpha, sources=w.sources, A=A,
                       output=output)
        o = torch.full(shape, float("nan"), device="cuda")
        F.invert(H, dev(U), q, o, F.Opts(alpha=alpha, output=kind, points=w.sources))
        assert rel(host(o), ref[output]) <= 1e-4, (alpha, rel(host(o), ref[output]))


@pytest.mark.parametrize("m", [1, 2])
def test_discrepancy_and_host_buffers_match_oracle(F, m):
    w, A, U, delta = _problem(32, 5, 2, m, seed=1300 + m, n_alpha=16)
    H = F.kernel_transform(32, w.x0, w.h, w.zr, w.zy, w.nu, pad=2)
    ref = O.invert(U, 32, w.x0, w.h, w.zy, w.zr, w.nu, pad=2, alphas=w.alphas, delta=delta, tau=1.1,
                   sources=w.sources, A=A)
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    res = torch.zeros(w.alphas.size, dtype=torch.float64, device="cuda")
    xi = torch.empty((5, 32, 32), device="cuda")
    opts = F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources, alpha_idx=idx, residuals=res)
    F.invert(H, dev(U), 2, xi, opts)
    r = host(res)
    assert np.max(np.abs(r - ref["res2"]) / ref["res2"]) <= 1e-5
    k = int(idx.item())
    thr2 = (1.1 * delta) ** 2
    if k != ref["alpha_index"]:
        lo, hi = min(k, ref["alpha_index"]), max(k, ref["alpha_index"])
        assert np.all(np.abs(ref["res2"][lo:hi + 1] - thr2) <= 1e-4 * thr2)
    else:
        assert rel(host(xi), ref["xi"]) <= 1e-4
    # the standalone choice and the host-buffer entry point agree with the device call
    idx2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    res2 = torch.zeros(w.alphas.size, dtype=torch.float64, device="cuda")
    F.choose_alpha(H, dev(U), 2, w.alphas, delta, 1.1, idx2, res2)
    assert int(idx2.item()) == k and np.allclose(host(res2), r, rtol=1e-9, atol=0)
    xh = torch.empty((5, 32, 32), dtype=torch.float32).pin_memory()
    F.invert_host(H, torch.as_tensor(U, dtype=torch.float32).pin_memory(), 2, xh,
                  F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources))
    assert torch.equal(xh, xi.cpu())


def test_padded_box_differs_from_the_periodic_one_and_unsupported_calls_are_rejected(F):
    w, A, U, delta = _problem(32, 4, 1, 1, seed=1400)
    Hp = F.kernel_transform(32, w.x0, w.h, w.zr, w.zy, w.nu, pad=2)
    H1 = F.kernel_transform(32, w.x0, w.h, w.zr, w.zy, w.nu, pad=1)
    zeta = dev(np.random.default_rng(3).standard_normal((1, 4, 32, 32)))
    u2 = torch.empty((1, 1, 32, 32), device="cuda")
    u1 = torch.empty((1, 1, 32, 32), device="cuda")
    F.fwd_apply(Hp, zeta, 1, u2)
    F.fwd_apply(H1, zeta, 1, u1)
    assert rel(host(u2), host(u1)) > 1e-3          # the wrap-around terms are gone
    with pytest.raises(F.Fr3dError):
        F.fwd_apply_noalloc(Hp, zeta, 1, u2)
    with pytest.raises(F.Fr3dError):
        F.band_features(Hp, dev(U), 1, 4, delta, torch.empty(4, device="cuda"))


def test_per_band_discrepancy_uses_the_box_bands(F):
    nb = 4
    w, A, U, delta = _problem(32, 6, 1, 1, seed=1500)
    H = F.kernel_transform(32, w.x0, w.h, w.zr, w.zy, w.nu, pad=2)
    ref = O.invert(U, 32, w.x0, w.h, w.zy, w.zr, w.nu, pad=2, alphas=w.alphas, delta=delta, tau=1.1,
                   sources=w.sources, A=A, n_bands=nb)
    idx = torch.zeros(nb, dtype=torch.int32, device="cuda")
    res = torch.zeros((nb, w.alphas.size), dtype=torch.float64, device="cuda")
    xi = torch.empty((6, 32, 32), device="cuda")
    F.invert(H, dev(U), 1, xi, F.Opts(alphas=w.alphas, delta=delta, tau=1.1, points=w.sources, alpha_idx=idx,
                                      residuals=res, n_bands=nb))
    assert np.max(np.abs(host(res) - ref["res2"]) / np.maximum(ref["res2"], 1e-300)) <= 1e-5
    got = [int(v) for v in idx.cpu().numpy()]
    count = np.bincount(O.radial_bands(64, nb), minlength=nb)          # the bands of the 64 x 64 box
    for b in range(nb):
        if got[b] != ref["alpha_index"][b]:
            thr2 = (1.1 * delta) ** 2 * count[b] / 64 ** 2
            lo, hi = sorted((got[b], ref["alpha_index"][b]))
            assert np.all(np.abs(ref["res2"][b][lo:hi + 1] - thr2) <= 1e-4 * thr2)
    if got != ref["alpha_index"]:   # a proven near-tie: the oracle at the GPU's per-band choice
        ref = O.invert(U, 32, w.x0, w.h, w.zy, w.zr, w.nu, pad=2, alphas=w.alphas, sources=w.sources, A=A,
                       n_bands=nb, band_alpha_index=got)
    assert rel(host(xi), ref["xi"]) <= 1e-4
    # the learned rule has no padded-box features: rejected before any launch
    net = F.Mlp(nb, 16, nb, seed=1)
    with pytest.raises(F.Fr3dError):
        F.invert(H, dev(U), 1, xi, F.Opts(alphas=w.alphas, delta=delta, points=w.sources, n_bands=nb, net=net))
