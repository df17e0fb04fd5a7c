"""Pins of the FP64 oracle to what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form,
a brute-force sum, a library routine used as an independent check, an
invariant, or a special case with a known answer.
"""

import json
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
rng0 = np.random.default_rng(12345)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ------------------------------------------------------------------ kernel (Sec. 3)
def test_kernel_is_z_derivative_of_inverse_distance():
    """K = d/dz (1/r): compare with a central difference of 1/r (fixes sign and the 3/2 power)."""
    pts = rng0.uniform(-2, 2, size=(50, 3))
    pts[:, 2] = np.where(np.abs(pts[:, 2]) < 0.2, 0.5, pts[:, 2])
    e = 1e-5
    inv_r = lambda x, y, z: 1.0 / np.sqrt(x * x + y * y + z * z)
    fd = (inv_r(pts[:, 0], pts[:, 1], pts[:, 2] + e) - inv_r(pts[:, 0], pts[:, 1], pts[:, 2] - e)) / (2 * e)
    assert rel(O.kernel_K(pts[:, 0], pts[:, 1], pts[:, 2]), fd) < 1e-8


def _rect_solid_angle(x1, x2, y1, y2, z):
    """integral over [x1,x2]x[y1,y2] of |z| / (x^2+y^2+z^2)^(3/2) (closed form of the rectangle's solid angle)."""
    z = abs(z)
    F = lambda x, y: np.arctan(x * y / (z * np.sqrt(x * x + y * y + z * z)))
    return F(x2, y2) - F(x1, y2) - F(x2, y1) + F(x1, y1)


@pytest.mark.parametrize("dz", [-0.5, -0.3, 0.4])
def test_kernel_hat_dc_bin_equals_rectangle_closed_form(dz):
    """h^2 * DFT at k = 0 is the midpoint rule for the kernel's integral over the periodic box;
    the integral has the closed form -sgn(z) * solid angle of the box's square."""
    n, h = 256, 0.01
    Kh = O.kernel_hat(n, h, [0.0], [-dz])[0, 0]           # z_i - z'_j = dz
    # wrapped lags run from -n/2 to n/2 - 1: cells cover [-(n/2 + 1/2) h, (n/2 - 1/2) h]
    lo, hi = -(n / 2 + 0.5) * h, (n / 2 - 0.5) * h
    exact = -np.sign(dz) * _rect_solid_angle(lo, hi, lo, hi, dz)
    assert abs(Kh[0, 0] - exact) <= 1e-4 * abs(exact)
    # and the whole-plane value -2 pi sgn(z) is approached as the box grows
    assert abs(Kh[0, 0] + 2 * np.pi * np.sign(dz)) < 2 * np.pi * abs(dz) / (n / 2 * h) * 1.5


def test_kernel_hat_matches_continuum_transform():
    """K~(w, z) = -2 pi sgn(z) exp(-|w||z|) (Fourier transform of d/dz 1/r with the e^{-i w x}
    convention of Lemma 1's 1/(4 pi^2) Plancherel identity).  On a large box the discrete
    transform h^2 DFT must agree to within the box-truncation error, which is bounded by the
    kernel's L1 mass outside the inscribed disk, 2 pi |z| / half-width."""
    n, h, dz = 512, 0.05, -0.5
    Kh = O.kernel_hat(n, h, [0.0], [-dz])[0, 0]
    k = np.fft.fftfreq(n, d=h) * 2 * np.pi
    W = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    exact = -2 * np.pi * np.sign(dz) * np.exp(-W * abs(dz))
    bound = 2 * np.pi * abs(dz) / (n / 2 * h)
    sel = W < 12.0
    assert np.max(np.abs(Kh[sel] - exact[sel])) < bound
    # away from k = 0 the truncation error oscillates away; the agreement is much tighter
    mid = (W > 2.0) & (W < 12.0)
    assert np.max(np.abs(Kh[mid] - exact[mid])) < 0.1 * bound
    # a wrong decay law (e.g. exp(-|w||z|/2)) or a dropped 2 pi would fail these bounds
    wrong = -2 * np.pi * np.sign(dz) * np.exp(-W * abs(dz) / 2)
    assert np.max(np.abs(Kh[mid] - wrong[mid])) > 10 * (0.1 * bound)


@pytest.mark.parametrize("n,pad", [(8, 1), (6, 1), (6, 2)])
def test_kernel_hat_is_real_and_has_eightfold_symmetry(n, pad):
    Kh = O.kernel_hat(n, 0.3, [0.0, 0.1], [0.5, 0.7], pad)
    L = n * pad
    for i in range(2):
        for j in range(2):
            K = Kh[i, j]
            assert np.allclose(K, K.T, rtol=0, atol=1e-13 * np.abs(K).max())                 # kx <-> ky
            idx = (-np.arange(L)) % L
            assert np.allclose(K, K[idx][:, idx], rtol=0, atol=1e-13 * np.abs(K).max())      # k -> -k
            assert np.allclose(K, K[:, idx], rtol=0, atol=1e-13 * np.abs(K).max())           # kx -> -kx


# ------------------------------------------------------------------ DFT
@pytest.mark.parametrize("shape", [(4, 4), (6, 6), (3, 5)])
def test_dft2_equals_definition_double_sum(shape):
    f = rng0.standard_normal(shape) + 1j * rng0.standard_normal(shape)
    Ly, Lx = shape
    F = np.zeros(shape, complex)
    for ky in range(Ly):
        for kx in range(Lx):
            for y in range(Ly):
                for x in range(Lx):
                    F[ky, kx] += f[y, x] * np.exp(-2j * np.pi * (ky * y / Ly + kx * x / Lx))
    assert rel(O.dft2(f), F) < 1e-13
    assert rel(O.idft2(F), f) < 1e-13


def test_dft2_agrees_with_library_fft_and_parseval():
    f = rng0.standard_normal((3, 24, 24))
    F = O.dft2(f)
    assert rel(F, np.fft.fft2(f)) < 1e-13
    # Parseval: sum |f|^2 = L^-2 sum |F|^2 (the discrete form of Lemma 1's Plancherel identity)
    assert abs(np.sum(f ** 2) - np.sum(np.abs(F) ** 2) / 24 ** 2) < 1e-10 * np.sum(f ** 2)


# ------------------------------------------------------------------ convolution theorem (Eq. (5))
@pytest.mark.parametrize("n", [6, 8])
@pytest.mark.parametrize("kind", ["dz_inv_r", "inv_r"])
def test_forward_dft_equals_direct_quadrature_periodic(n, kind):
    h, zy, zr, nu = 0.25, [0.0, 0.1], [0.5, 0.6, 0.8], [0.1, 0.1, 0.2]
    zeta = rng0.standard_normal((2, 3, n, n))
    Ud = O.forward_direct(zeta, n, h, zy, zr, nu, kind=kind)
    Uf = O.forward_dft(zeta, n, h, zy, zr, nu, kind=kind)
    assert rel(Uf, Ud) < 1e-12


def test_pad2_gives_the_aperiodic_sum_over_R():
    n, h, zy, zr, nu = 5, 0.3, [0.0], [0.5, 0.9], [0.2, 0.2]
    zeta = rng0.standard_normal((2, n, n))
    # brute force aperiodic sum, no wrapping at all
    U = np.zeros((1, n, n))
    for b in range(n):
        for a in range(n):
            for j in range(2):
                for bb in range(n):
                    for aa in range(n):
                        U[0, b, a] += h * h * nu[j] * O.kernel_K((a - aa) * h, (b - bb) * h, zy[0] - zr[j]) * zeta[j, bb, aa]
    assert rel(O.forward_direct(zeta, n, h, zy, zr, nu, pad=2), U) < 1e-13
    assert rel(O.forward_dft(zeta, n, h, zy, zr, nu, pad=2), U) < 1e-12


def _operator_matrix(n, h, zy, zr, nu, pad=1):
    """The full discrete operator of Eq. (4) as a dense matrix, column by column from unit inputs."""
    Mp = len(zr)
    cols = []
    for j in range(Mp):
        for b in range(n):
            for a in range(n):
                e = np.zeros((Mp, n, n))
                e[j, b, a] = 1.0
                cols.append(O.forward_direct(e, n, h, zy, zr, nu, pad).ravel())
    return np.array(cols).T


# ------------------------------------------------------------------ Tikhonov (Sec. 5)
def test_tikhonov_optimality_pinv_limit_and_dual_identity():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((20, 3, 5))
    u = rng.standard_normal((20, 3, 2)) + 1j * rng.standard_normal((20, 3, 2))
    for a in [1e-3, 0.1, 3.0]:
        x = O.tikhonov_qr(A, u, a)
        g = np.swapaxes(A, 1, 2) @ (A @ x - u) + a * x              # gradient of the Tikhonov functional
        assert np.max(np.abs(g)) < 1e-12 * max(1, np.max(np.abs(u)))
        # dual form A^T (A A^T + a I)^{-1} u (a different formula for the same minimiser)
        xd = np.swapaxes(A, 1, 2) @ np.linalg.solve(A @ np.swapaxes(A, 1, 2) + a * np.eye(3), u)
        assert rel(x, xd) < 1e-11
    x0 = O.tikhonov_qr(A, u, 1e-13)
    assert rel(x0, np.linalg.pinv(A) @ u) < 1e-8                   # normal (minimum-norm) solution
    # the residual grows and the norm shrinks with alpha
    res = [np.linalg.norm(A @ O.tikhonov_qr(A, u, a) - u) for a in np.logspace(-6, 2, 12)]
    nrm = [np.linalg.norm(O.tikhonov_qr(A, u, a)) for a in np.logspace(-6, 2, 12)]
    assert np.all(np.diff(res) >= -1e-12) and np.all(np.diff(nrm) <= 1e-12)


@pytest.mark.parametrize("zy", [[0.0], [0.0, -0.15]])
def test_algorithm1_equals_dense_tikhonov_of_full_operator(zy):
    """Per-frequency Tikhonov + inverse DFT (Algorithm 1, Lemma 1) equals Tikhonov on the whole
    discretised operator of Eq. (4), assembled by brute force from the direct quadrature (one and two
    observation planes)."""
    n, h, zr, nu = 4, 0.3, [0.5, 0.7, 0.9], [0.2, 0.2, 0.2]
    Aop = _operator_matrix(n, h, zy, zr, nu)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((1, len(zy), n, n))
    A = O.A_matrices(n, h, zy, zr, nu)
    s2 = O.alpha_scale(A)
    for alpha in [1e-12, 1e-3, 0.5]:
        out = O.invert(U, n, -0.6, h, zy, zr, nu, alpha=alpha, output="zeta")
        stacked = np.vstack([Aop, np.sqrt(alpha * s2) * np.eye(Aop.shape[1])])
        rhs = np.concatenate([U.ravel(), np.zeros(Aop.shape[1])])
        z = np.linalg.lstsq(stacked, rhs, rcond=None)[0]
        assert rel(out["zeta"].ravel(), z) < 1e-9
    # the alpha -> 0 limit is the normal solution (Assumption U): the pseudo-inverse of the operator
    out = O.invert(U, n, -0.6, h, zy, zr, nu, alpha=1e-14, output="zeta")
    assert rel(out["zeta"].ravel(), np.linalg.pinv(Aop) @ U.ravel()) < 1e-6


def test_pad2_inversion_is_dense_tikhonov_on_the_box_with_zero_data_outside_R():
    """pad = 2: Algorithm 1 on the 2n x 2n box equals Tikhonov of the box's whole discrete operator
    (brute force from the direct quadrature on the box) with the data zero-padded and the unknown free
    over the box, cropped to R; the discrepancy residual is the spatial one over the whole box, the
    padded zeros included."""
    n, h, zy, zr, nu = 4, 0.3, [0.0, -0.15], [0.5, 0.8], [0.25, 0.25]
    L = 2 * n
    Abox = _operator_matrix(L, h, zy, zr, nu)
    rng = np.random.default_rng(11)
    U = rng.standard_normal((1, len(zy), n, n))
    Ubox = np.zeros((len(zy), L, L))
    Ubox[:, :n, :n] = U[0]
    s2 = O.alpha_scale(O.A_matrices(n, h, zy, zr, nu, pad=2))
    assert abs(s2 - O.alpha_scale(O.A_matrices(L, h, zy, zr, nu))) < 1e-14 * s2
    for alpha in [1e-6, 1e-2]:
        out = O.invert(U, n, -0.6, h, zy, zr, nu, pad=2, alpha=alpha, output="zeta")
        stacked = np.vstack([Abox, np.sqrt(alpha * s2) * np.eye(Abox.shape[1])])
        z = np.linalg.lstsq(stacked, np.concatenate([Ubox.ravel(), np.zeros(Abox.shape[1])]), rcond=None)[0]
        z = z.reshape(len(zr), L, L)
        assert rel(out["zeta"][0], z[:, :n, :n]) < 1e-9
    out = O.invert(U, n, -0.6, h, zy, zr, nu, pad=2, alphas=[1e-6, 1e-2], delta=1.0, tau=1.1, output="zeta")
    zfull = np.linalg.lstsq(np.vstack([Abox, np.sqrt(1e-2 * s2) * np.eye(Abox.shape[1])]),
                            np.concatenate([Ubox.ravel(), np.zeros(Abox.shape[1])]), rcond=None)[0]
    assert abs(out["res2"][1] - np.sum((Abox @ zfull - Ubox.ravel()) ** 2)) < 1e-10 * np.sum(U ** 2)


def test_restricting_the_solve_to_the_occupied_bins_is_exact():
    """A zero right-hand side has the zero Tikhonov solution, so on data whose spectrum occupies a few
    bins, solving those bins only (``bins``, used by the full-size parity test and the CPU baseline's
    sample) gives the full inversion's zeta, residuals and choice; on data with a full spectrum it does
    not."""
    n, h, zy, zr, nu = 12, 0.2, [0.0], [0.5, 0.7, 0.9], [0.2] * 3
    a = np.arange(n)
    U = np.zeros((2, 1, n, n))
    for q, (kx, ky, ph) in enumerate([(1, 2, 0.3), (3, 0, 1.1)]):
        U[q, 0] = np.cos(2 * np.pi * (kx * a[None, :] + ky * a[:, None]) / n + ph)
    sel = np.nonzero(np.abs(O.dft2(U)[:, 0]).max(axis=0).ravel() > 1e-9)[0]
    assert sel.size == 4
    al = np.logspace(-6, 0, 7)
    full = O.invert(U, n, -1.2, h, zy, zr, nu, alphas=al, delta=0.3, tau=1.1, output="zeta")
    part = O.invert(U, n, -1.2, h, zy, zr, nu, alphas=al, delta=0.3, tau=1.1, output="zeta", bins=sel)
    assert np.allclose(part["res2"], full["res2"], rtol=1e-12, atol=1e-14)
    assert part["alpha_index"] == full["alpha_index"]
    assert rel(part["zeta"], full["zeta"]) < 1e-12
    Un = U + 0.1 * np.random.default_rng(5).standard_normal(U.shape)
    f2 = O.invert(Un, n, -1.2, h, zy, zr, nu, alpha=1e-3, output="zeta")
    p2 = O.invert(Un, n, -1.2, h, zy, zr, nu, alpha=1e-3, output="zeta", bins=sel)
    assert rel(p2["zeta"], f2["zeta"]) > 1e-3


def test_frequency_residual_equals_spatial_residual():
    """Parseval: the residual summed over frequencies / L^2 is the spatial residual ||A zeta - U||^2."""
    n, h, zy, zr, nu = 6, 0.3, [0.0], [0.5, 0.8], [0.25, 0.25]
    rng = np.random.default_rng(4)
    U = rng.standard_normal((1, 1, n, n))
    out = O.invert(U, n, -0.9, h, zy, zr, nu, alphas=[1e-4, 1e-2], delta=1.0, tau=1.1, output="zeta")
    k = out["alpha_index"]
    Ufit = O.forward_direct(out["zeta"], n, h, zy, zr, nu)
    assert abs(out["res2"][k] - np.sum((Ufit - U) ** 2)) < 1e-10 * np.sum(U ** 2)


def test_exact_recovery_tiny_well_conditioned():
    """M = M' = 1, coarse grid, small |dz|: noise-free data are inverted essentially exactly."""
    n, h, zy, zr, nu = 8, 0.25, [0.0], [0.1], [1.0]
    A = O.A_matrices(n, h, zy, zr, nu)
    cond = np.abs(A).max() / np.abs(A).min()
    assert cond < 50
    zt = np.random.default_rng(5).standard_normal((1, 1, n, n))
    U = O.forward_direct(zt, n, h, zy, zr, nu)
    out = O.invert(U, n, -1.0, h, zy, zr, nu, alpha=1e-14, output="zeta")
    assert rel(out["zeta"], zt) < 1e-9


def test_discrepancy_rule():
    r2 = np.array([0.5, 1.0, 1.2, 4.0, 9.0])
    assert O.choose_alpha_index(r2, 1.0, 1.1) == (2, 0)        # 1.2 <= 1.21 < 4
    assert O.choose_alpha_index(r2, 0.1, 1.1) == (0, 1)        # nothing admissible: smallest, flagged
    assert O.choose_alpha_index(r2, 10.0, 1.1) == (4, 2)       # everything admissible: largest, flagged


def test_convergence_as_noise_vanishes():
    """Theorem 1: with the discrepancy principle the error to the normal solution decreases as
    delta -> 0.  The truth is built in range(A^T) per frequency, so it is its own normal solution."""
    n, h, zy, zr, nu = 16, 0.125, [0.0], list(0.5 + 0.05 * np.arange(6)), [0.05] * 6
    A = O.A_matrices(n, h, zy, zr, nu)
    rng = np.random.default_rng(11)
    w = O.dft2(rng.standard_normal((1, n, n)))                       # Hermitian weights
    Zh = np.einsum("yxij,iyx->jyx", A, w)
    zt = O.idft2(Zh).real[None]
    U = O.forward_dft(zt, n, h, zy, zr, nu, A=A)
    noise = rng.standard_normal(U.shape)
    errs = []
    for lev in [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]:
        d = lev * np.linalg.norm(U)
        Un = U + d * noise / np.linalg.norm(noise)
        out = O.invert(Un, n, -1.0, h, zy, zr, nu, alphas=np.logspace(-12, 0, 25), delta=d, tau=1.1,
                       output="zeta", A=A)
        errs.append(rel(out["zeta"], zt))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] < 0.05


# ------------------------------------------------------------------ sources and V0 (Sec. 2, Sec. 6)
def test_A0_A2_for_exponential_source_pulse():
    g = json.load(open(os.path.join(GOLD, "paper_model_example.json")))
    assert abs(O.A0_of(lambda t: np.exp(-t)) - g["A0_for_g"]) < 1e-10
    assert abs(O.A2_of(lambda t: np.exp(-t)) - g["A2_for_g"]) < 1e-10


def test_V0_solves_poisson_equation_for_point_sources():
    """Delta V0 = A0 phi: V0 is harmonic away from the sources and the flux of grad V0 through a
    sphere around one source is A0 (fixes the sign and the 1/(4 pi))."""
    pts = np.array([[0.1, -0.2, -0.3], [0.5, 0.5, -0.4]])
    A0 = 1.7
    e = 1e-3
    X, Y, Z = 0.3, 0.2, 0.6
    lap = (O.V0(pts, X + e, Y, Z, A0) + O.V0(pts, X - e, Y, Z, A0) + O.V0(pts, X, Y + e, Z, A0)
           + O.V0(pts, X, Y - e, Z, A0) + O.V0(pts, X, Y, Z + e, A0) + O.V0(pts, X, Y, Z - e, A0)
           - 6 * O.V0(pts, X, Y, Z, A0)) / e ** 2
    assert abs(lap) < 1e-4
    # flux through a sphere of radius 0.05 around the first source (midpoint rule in angles)
    r, c = 0.05, pts[0]
    th = (np.arange(200) + 0.5) * np.pi / 200
    ph = (np.arange(400) + 0.5) * 2 * np.pi / 400
    T, P = np.meshgrid(th, ph, indexing="ij")
    nrm = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)])
    x = c[:, None, None] + r * nrm
    grad = np.stack([(O.V0(pts, x[0] + s[0] * e, x[1] + s[1] * e, x[2] + s[2] * e, A0)
                      - O.V0(pts, x[0] - s[0] * e, x[1] - s[1] * e, x[2] - s[2] * e, A0)) / (2 * e)
                     for s in np.eye(3)])
    flux = np.sum(np.sum(grad * nrm, axis=0) * r * r * np.sin(T)) * (np.pi / 200) * (2 * np.pi / 400)
    assert abs(flux - A0) < 1e-3 * A0


def test_combination_recovers_shared_xi_exactly():
    from paper_1703_01216_gb300.inputs import cross_sources
    n, x0, h = 8, -1.0, 0.25
    zr = [0.6, 0.8]
    xi = np.random.default_rng(2).standard_normal((2, n, n))
    S = cross_sources(3)
    zeta = O.zeta_from_xi(xi, S, n, x0, h, zr)
    assert rel(O.combine_sources(zeta, S, n, x0, h, zr), xi) < 1e-14
    # single source: xi = zeta / V0 (Algorithm 1 step 4)
    c = x0 + (np.arange(n) + 0.5) * h
    v = O.V0(S[0], c[None, None, :], c[None, :, None], np.array(zr)[:, None, None])
    assert rel(O.combine_sources(zeta[:1], S[:1], n, x0, h, zr), zeta[0] / v) < 1e-14


def test_band_residuals_partition_the_global_residual():
    """Per-band residuals add up to the global one; the bands partition the grid; one band is the
    global rule."""
    n, h, zy, zr, nu = 12, 0.2, [0.0], [0.5, 0.7, 0.9], [0.2] * 3
    rng = np.random.default_rng(21)
    U = rng.standard_normal((2, 1, n, n))
    al = np.logspace(-6, 0, 7)
    g = O.invert(U, n, -1.2, h, zy, zr, nu, alphas=al, delta=0.5, tau=1.1, output="none")
    b = O.invert(U, n, -1.2, h, zy, zr, nu, alphas=al, delta=0.5, tau=1.1, output="none", n_bands=4)
    assert np.allclose(b["res2"].sum(axis=0), g["res2"], rtol=1e-12)
    assert np.bincount(O.radial_bands(n, 4), minlength=4).sum() == n * n
    assert np.all(np.bincount(O.radial_bands(n, 4), minlength=4) > 0)
    one = O.invert(U, n, -1.2, h, zy, zr, nu, alphas=al, delta=0.5, tau=1.1, output="zeta", band_alpha_index=[3])
    fix = O.invert(U, n, -1.2, h, zy, zr, nu, alpha=al[3], output="zeta")
    assert np.allclose(one["zeta"], fix["zeta"], rtol=0, atol=1e-13 * np.abs(fix["zeta"]).max())


def test_radial_bands_are_symmetric_monotone_and_hand_evaluated():
    """The bands depend only on the folded |k| (so every 8-fold symmetry class lies in one band), grow
    with it, start at DC and end at the corner; two values by hand: L = 16, 4 bands, band width
    sqrt(2) * 8 / 4 = 2.83 in |k'|."""
    L, nb = 16, 4
    B = O.radial_bands(L, nb).reshape(L, L)
    neg = (-np.arange(L)) % L
    assert np.array_equal(B, B.T) and np.array_equal(B, B[neg]) and np.array_equal(B, B[:, neg])
    kf = np.minimum(np.arange(L), L - np.arange(L))
    rho = np.sqrt(kf[None, :] ** 2 + kf[:, None] ** 2).ravel()
    order = np.argsort(rho, kind="stable")
    assert np.all(np.diff(B.ravel()[order]) >= 0)
    assert B[0, 0] == 0 and B[L // 2, L // 2] == nb - 1
    assert B[0, 3] == 1                      # |k'| = 3: 3 / 2.83 = 1.06
    assert B[5, 5] == 2                      # |k'| = 7.07: 2.5


def test_alpha_scale_is_the_dc_norm_in_closed_form():
    """At M = 1 the kernel samples of one depth difference share one sign, so the DC bin has the largest
    modulus of its transform (triangle inequality) and s^2 = sum_j (nu_j K~(0, dz_j))^2, with K~(0, dz)
    the box integral of the kernel: minus the sign of dz times the solid angle of the box's square."""
    n, h = 256, 0.01
    zr, nu = [0.3, 0.5], [0.2, 0.1]
    A = O.A_matrices(n, h, [0.0], zr, nu)
    lo, hi = -(n / 2 + 0.5) * h, (n / 2 - 0.5) * h
    exact = sum((v * _rect_solid_angle(lo, hi, lo, hi, -z)) ** 2 for z, v in zip(zr, nu))
    assert abs(O.alpha_scale(A) - exact) <= 1e-3 * exact
    assert np.argmax(np.sum(A * A, axis=(-2, -1))) == 0


# ------------------------------------------------------------------ truncated SVD (Sec. 5, the paper's best RA)
def test_tsvd_matches_library_pseudo_inverse_and_limits():
    """tsvd_solve against numpy.linalg.pinv with the matching cut-off, and its two limits."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((5, 3, 6)) * np.array([1.0, 0.1, 1e-3])[None, :, None]
    Uh = rng.standard_normal((5, 3, 2)) + 1j * rng.standard_normal((5, 3, 2))
    sig = np.linalg.svd(A, compute_uv=False)
    for b in range(5):
        for keep in (1, 2, 3):
            # a level strictly between the kept and the dropped squared singular values
            t = sig[b, keep - 1] ** 2 * 0.5 if keep == 3 else np.sqrt(sig[b, keep - 1] ** 2 * sig[b, keep] ** 2)
            x = O.tsvd_solve(A[b:b + 1], Uh[b:b + 1], t)[0]
            P = np.linalg.pinv(A[b], rcond=np.sqrt(t) / sig[b, 0])
            assert rel(x, P @ Uh[b]) < 1e-10
    assert np.allclose(O.tsvd_solve(A, Uh, 1e-30), np.linalg.pinv(A) @ Uh, rtol=0, atol=1e-9 * np.abs(np.linalg.pinv(A) @ Uh).max())
    assert np.all(O.tsvd_solve(A, Uh, 10 * sig.max() ** 2) == 0)


def test_single_observation_depth_has_closed_form_solutions():
    """M = 1: A^(m) is one row a, so the Tikhonov minimiser is a (a . u) / (|a|^2 + alpha s^2) (the
    Sherman-Morrison form of (a^T a + c I)^-1 a^T) and the truncated SVD keeps a u / |a|^2 when
    |a|^2 >= t, else 0; the squared residual of the Tikhonov solution is (c / (|a|^2 + c))^2 |u|^2."""
    rng = np.random.default_rng(9)
    A = rng.standard_normal((30, 1, 7)) * np.exp(-rng.uniform(0, 4, (30, 1, 1)))
    u = rng.standard_normal((30, 1, 3)) + 1j * rng.standard_normal((30, 1, 3))
    a2 = np.sum(A[:, 0, :] ** 2, axis=1)
    for c in (1e-3, 0.2):
        x = O.tikhonov_qr(A, u, c)
        closed = A[:, 0, :, None] * u[:, :, :] / (a2 + c)[:, None, None]
        assert rel(x, closed) < 1e-12
        r2 = np.sum(np.abs(A @ x - u) ** 2, axis=(1, 2))
        assert np.allclose(r2, (c / (a2 + c)) ** 2 * np.sum(np.abs(u) ** 2, axis=(1, 2)), rtol=1e-10)
    t = float(np.median(a2))
    x = O.tsvd_solve(A, u, t)
    keep = a2 >= t
    closed = np.where(keep[:, None, None], A[:, 0, :, None] * u / a2[:, None, None], 0.0)
    assert rel(x, closed) < 1e-12


def test_tsvd_inversion_residual_is_monotone_and_reaches_the_data_norm():
    """The squared residual grows with the truncation level; with every singular value truncated it is
    ||U||^2 (the zero solution), and at M = 1 with none truncated it is 0 (an exact fit)."""
    n, h, zy, zr, nu = 8, 0.25, [0.0], [0.3, 0.45, 0.6], [0.15] * 3
    rng = np.random.default_rng(12)
    U = rng.standard_normal((2, 1, n, n))
    al = np.logspace(-9, 1, 11)
    out = O.invert(U, n, -1.0, h, zy, zr, nu, alphas=al, delta=1.0, tau=1.1, output="none", ra="tsvd")
    r = out["res2"]
    assert np.all(np.diff(r) >= -1e-12 * r.max())
    assert abs(r[-1] - np.sum(U ** 2)) < 1e-10 * np.sum(U ** 2)
    assert r[0] < 1e-20 * np.sum(U ** 2)


# ------------------------------------------------------------------ the 1/r kernel of the first equation (Sec. 3)
def test_inv_r_kernel_z_derivative_is_the_solved_kernel():
    """d/dz of the 1/r kernel's discrete transform is the transform of d/dz (1/r), at every frequency
    (central difference in the depth difference; the two kinds share grid, box and DFT)."""
    n, h, e = 16, 0.125, 1e-4
    for dz in (-0.6, -0.25, 0.4):
        up = O.kernel_hat(n, h, [0.0], [-(dz + e)], kind="inv_r")[0, 0]
        dn = O.kernel_hat(n, h, [0.0], [-(dz - e)], kind="inv_r")[0, 0]
        want = O.kernel_hat(n, h, [0.0], [-dz])[0, 0]
        assert rel((up - dn) / (2 * e), want) < 1e-6


def test_inv_r_dc_bin_is_the_integral_over_the_box():
    """h^2 * DFT at k = 0 of the sampled 1/r is the midpoint rule for its integral over the periodic
    box's square; compare with scipy's adaptive quadrature of the same integral."""
    from scipy.integrate import dblquad
    n, h, dz = 64, 0.05, 0.3
    Kh = O.kernel_hat(n, h, [0.0], [-dz], kind="inv_r")[0, 0]
    lo, hi = -(n / 2 + 0.5) * h, (n / 2 - 0.5) * h
    val = dblquad(lambda y, x: 1.0 / np.sqrt(x * x + y * y + dz * dz), lo, hi, lo, hi, epsabs=1e-11, epsrel=1e-11)[0]
    assert abs(Kh[0, 0] - val) <= 2e-4 * val


# ------------------------------------------------------------------ right-hand side of Eq. (7)
def test_rhs_source_term_is_the_z_derivative_of_the_inverse_distances():
    """S = sum_l d/dx3 (1/|x - x_l|): central difference in the observation depth of the 1/r field."""
    n, x0, h, zy = 8, -1.0, 0.25, [0.1, 0.3]
    src = np.array([[[0.05, -0.2, -0.4], [0.6, 0.3, -0.7]]])
    S, _ = O.rhs_terms(n, x0, h, zy, src, 4, 1.0)
    c = x0 + (np.arange(n) + 0.5) * h
    e = 1e-5
    field = lambda z: sum(1.0 / np.sqrt((c[None, :] - p[0]) ** 2 + (c[:, None] - p[1]) ** 2 + (z - p[2]) ** 2)
                          for p in src[0])
    for i, z in enumerate(zy):
        assert rel(S[0, i], (field(z + e) - field(z - e)) / (2 * e)) < 1e-8


def test_pi_depth_grid_is_the_midpoint_rule_of_the_box_height():
    """Pi's vertical grid: n_pi cells of equal height covering [-half, half] once, one node at each cell's
    centre, so it integrates polynomials of degree 1 exactly and z^2 with the midpoint rule's known
    defect, (2 half) dz^2 / 12 too little."""
    for n_pi, half in [(4, 0.75), (16, 1.28), (2, 3.0)]:
        zp, nup = O.pi_depths(n_pi, half)
        dz = 2 * half / n_pi
        assert zp.size == nup.size == n_pi and np.allclose(nup, dz)
        assert np.allclose(np.sort(zp), zp) and np.allclose(zp + zp[::-1], 0.0)
        assert abs(zp[0] - (-half + dz / 2)) < 1e-15 and abs(np.sum(nup) - 2 * half) < 1e-14
        assert abs(np.sum(nup * zp)) < 1e-14                                   # odd moment
        exact2 = 2 * half ** 3 / 3
        assert abs(np.sum(nup * zp ** 2) - (exact2 - 2 * half * dz ** 2 / 12)) < 1e-12


def test_pi_integral_of_a_constant_density_is_a_sum_of_solid_angles():
    """The discrete operator on Pi's depth grid applied to a constant density: each layer contributes
    -sgn(z - z') times the solid angle of the periodic square seen from distance |z - z'| (midpoint rule,
    the closed form of the kernel's plane integral), times the layer thickness."""
    n, h, half, n_pi = 128, 0.02, 1.28, 16
    zp, nup = O.pi_depths(n_pi, half)
    zy = [0.37]
    U = O.forward_dft(np.ones((n_pi, n, n)), n, h, zy, zp, nup)
    lo, hi = -(n / 2 + 0.5) * h, (n / 2 - 0.5) * h
    want = sum(-np.sign(zy[0] - z) * _rect_solid_angle(lo, hi, lo, hi, zy[0] - z) * dz for z, dz in zip(zp, nup))
    # the operator's horizontal sum is the midpoint rule of the plane integral: agreement to its error
    assert np.max(np.abs(U - want)) <= 1e-3 * np.abs(want)


def test_rhs_integral_term_equals_brute_force_quadrature_and_round_trip():
    """I is the direct quadrature over Pi of K times sum_l 1/|x' - x_l| (built here from the definition),
    and assembling the simulated measurement returns the left-hand side it was made from."""
    n, x0, h, zy, half, n_pi = 6, -0.75, 0.25, [0.2], 0.75, 4
    src = np.array([[[0.03, 0.01, -0.33]], [[-0.4, 0.2, -0.5]]])
    S, I = O.rhs_terms(n, x0, h, zy, src, n_pi, half)
    zp, nup = O.pi_depths(n_pi, half)
    c = x0 + (np.arange(n) + 0.5) * h
    for q in range(2):
        p = src[q, 0]
        f = 1.0 / np.sqrt((c[None, None, :] - p[0]) ** 2 + (c[None, :, None] - p[1]) ** 2 + (zp[:, None, None] - p[2]) ** 2)
        assert rel(I[q], O.forward_direct(f, n, h, zy, zp, nup)) < 1e-12
    U = np.random.default_rng(3).standard_normal((2, 1, n, n))
    d = O.simulate_dV2dz(U, n, x0, h, zy, src, 1.0, 2.0, 0.5, n_pi, half)
    assert rel(O.assemble_rhs(d, n, x0, h, zy, src, 1.0, 2.0, 0.5, n_pi, half), U) < 1e-12


def test_rhs_coefficients_follow_from_the_wave_equation_moments():
    """The coefficients of Eq. (7) (2 pi, A2 / 2 and -A0 / (4 pi c0^2)) pinned without their printed form.
    The time moments of the wave equation (Sec. 2) give Delta V0 = A0 phi (the zeroth moment, whatever c is)
    and Delta V2 = 2 V0 / c^2 + A2 phi (the second, with int t^2 u_tt dt = 2 V0 and int t^2 g dt = A2).
    Inverting the Laplacian with its Green function -1/(4 pi |x|), with 1/c^2 = 1/c0^2 - xi and zeta = xi V0:
        V2 = -(1/(4 pi)) [ (2 / c0^2) int V0 / |x - x'| - 2 int zeta / |x - x'| + A2 sum_l 1/|x - x_l| ],
    so d/dx3 V2 is built here from three independent pieces: the forward operator of zeta over R, the same
    operator over the box Pi (R^3 replaced by Pi, Sec. 5) applied to the Poisson-pinned V0, and a central
    difference of the sources' 1/r field.  Assembling Eq. (7) from that measurement must return the
    left-hand side, the forward operator of zeta."""
    n, x0, h, half, n_pi = 6, -0.75, 0.25, 0.75, 4
    zy = [0.2, 0.35]
    zr, nu = np.array([-0.6, -0.45]), np.array([0.15, 0.15])
    A0, A2, c0 = 1.3, 2.0, 0.7
    src = np.array([[[0.03, 0.01, -0.33], [-0.2, 0.3, -0.52]]])
    rng = np.random.default_rng(11)
    zeta = rng.standard_normal((1, zr.size, n, n))
    c = x0 + (np.arange(n) + 0.5) * h
    Xc, Yc = c[None, None, :], c[None, :, None]
    lhs = O.forward_direct(zeta, n, h, zy, zr, nu)                          # int_R d/dx3(1/|x - x'|) zeta
    zp, nup = O.pi_depths(n_pi, half)
    v0 = O.V0(src[0], Xc, Yc, np.asarray(zp)[:, None, None], A0)            # V0 on Pi's grid
    j_v0 = O.forward_direct(v0[None], n, h, zy, zp, nup)                    # int_Pi d/dx3(1/|x - x'|) V0
    e = 1e-5
    inv_r = lambda z: sum(1.0 / np.sqrt((Xc - p[0]) ** 2 + (Yc - p[1]) ** 2 + (z - p[2]) ** 2) for p in src[0])
    zyc = np.asarray(zy)[:, None, None]
    dsrc = ((inv_r(zyc + e) - inv_r(zyc - e)) / (2 * e))[None]              # sum_l d/dx3 (1/|x - x_l|)
    dV2dz = -(1.0 / (4.0 * np.pi)) * ((2.0 / c0 ** 2) * j_v0 - 2.0 * lhs + A2 * dsrc)
    U = O.assemble_rhs(dV2dz, n, x0, h, zy, src, A0, A2, c0, n_pi, half)
    assert rel(U, lhs) < 1e-6                    # the central difference's error; a wrong coefficient is O(1)
