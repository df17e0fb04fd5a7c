"""The discrepancy rule reduces its block sums with two levels of atomic tickets (per group of eight
blocks, then over the groups) kept in the handle's partial-sum buffer.  Every ticket must be zero
again when a launch ends, whatever the candidate and band counts.  On one handle, calls that change
both counts from call to call return the same choices, residual curves and xi as the same calls on a
fresh handle; the largest output count (128 candidates in 16 bands) is among them."""

import numpy as np
import pytest

from paper_1703_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# (candidates, bands); at n = 128 the rule runs 34 blocks of 64 classes (2145 classes) in 5 groups
SEQUENCE = [(40, 1), (17, 4), (128, 16), (40, 1), (5, 2), (64, 8), (40, 1)]


@pytest.fixture(scope="module")
def F():
    from paper_1703_01216_gb300 import build, fr3d
    assert torch.cuda.is_available()
    build.build()
    fr3d.load()
    return fr3d


def _call(F, H, U, w, delta, na, nb):
    alphas = np.geomspace(1e-7, 1e-1, na)
    idx = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
    res = torch.full((nb * na,), float("nan"), dtype=torch.float64, device="cuda")
    out = torch.full((w.Mp, w.n, w.n), float("nan"), device="cuda")
    F.invert(H, U, w.Q, out, F.Opts(alphas=alphas, delta=delta, tau=1.1, points=w.sources, alpha_idx=idx,
                                    residuals=res, n_bands=nb))
    torch.cuda.synchronize()
    return idx, res, out


def test_changing_counts_on_one_handle_match_fresh_handles(F):
    w = I.make_workload(128, 6, q=2, n_incl=3, noise_level=0.02, n_alpha=8, seed=1310)
    H = F.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
    zeta = torch.empty((w.Q, w.Mp, w.n, w.n), device="cuda")
    F.zeta_from_xi(H, torch.as_tensor(w.xi_true, dtype=torch.float32, device="cuda"), w.sources, zeta)
    U = torch.empty((w.Q, 1, w.n, w.n), device="cuda")
    F.fwd_apply(H, zeta, w.Q, U)
    nz = torch.as_tensor(w.noise, dtype=torch.float32, device="cuda")
    nz *= w.noise_level * U.norm() / nz.norm()
    U = U + nz
    delta = float(nz.norm())
    for na, nb in SEQUENCE:
        got = _call(F, H, U, w, delta, na, nb)
        H2 = F.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
        ref = _call(F, H2, U, w, delta, na, nb)
        H2.close()
        assert int(got[0].min()) >= 0, (na, nb)
        assert torch.equal(got[0], ref[0]), (na, nb)
        assert torch.equal(got[1], ref[1]), (na, nb)
        assert torch.equal(got[2], ref[2]), (na, nb)
