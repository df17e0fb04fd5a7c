"""Plain FP64 CPU oracle for the FFT-Tikhonov method of Leonov & Bakushinsky,
"Economic numerical method of solving coefficient inverse problem for 3D wave
equation" (arXiv 1703.01216).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm), and by nothing else.  The product path
(``paper_1703_01216_gb300``) never imports, links or calls it, and this module
shares no code with the CUDA path: it only consumes plain numpy arrays.

Everything here is written to be checked by eye against the paper:

* the kernel K = d/dz (1/r) of Eq. (4), sampled on the discrete grid of Sec. 5;
* a naive separable DFT (twiddle matrices, one matrix product per axis) for the
  2D Fourier transforms of Algorithm 1 steps 1 and 3;
* the direct quadrature sum of the discretised operator of Eq. (4), the
  definition the DFT route must reproduce (convolution theorem, Eq. (5));
* the N^2 small systems A^(m) zeta^(m) = U^(m) of Eq. (6), solved by Tikhonov
  regularisation (Sec. 5) as a damped least-squares problem through a
  Householder QR of the stacked matrix [A; sqrt(alpha s^2) I] (no normal
  equations, no symmetry folding: every frequency is solved separately);
* the discrepancy principle for alpha (Sec. 4, remark after Algorithm 1);
* the inverse DFT, V0 of the point-source model (Sec. 6) and
  xi = zeta / V0 (Algorithm 1 step 4).

Array conventions (shared with the CUDA path only through the test harness):
planes are ``[..., y, x]`` with x fastest; spectra are ``[..., ky, kx]`` on the
full PN x PN grid; the forward DFT is unnormalised and the inverse carries
1/(PN)^2.

Readings of the paper that this oracle fixes (the paper is silent there):
voxel-centred grids, periodic box (pad P = 1) or zero padded box (P = 2),
midpoint quadrature weights nu_j, the alpha scale s^2 = max_m ||A^(m)||_F^2,
the discrepancy threshold tau * delta with the largest admissible alpha, and the
pointwise least-squares combination of several source parameters q.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "KINDS", "kernel_K", "wrapped_lags", "kernel_samples", "dft_matrix", "dft2", "idft2",
    "kernel_hat", "A_matrices", "alpha_scale", "forward_direct", "forward_dft",
    "tikhonov_qr", "tsvd_solve", "residual_sq", "radial_bands", "choose_alpha_index", "V0", "zeta_from_xi",
    "combine_sources", "invert", "A0_of", "A2_of", "pi_depths", "rhs_terms", "assemble_rhs", "simulate_dV2dz",
]


# --------------------------------------------------------------------------- kernel
KINDS = ("dz_inv_r", "inv_r")


def kernel_K(x, y, z, kind: str = "dz_inv_r"):
    """K(x, y, z) = d/dz (1/r) = -z / (x^2 + y^2 + z^2)^(3/2)  (Sec. 3, the kernel of Eq. (4) and of the
    equation the paper solves), or with kind="inv_r" K = 1/r, the kernel of the first equation the paper
    derives (for data V2 instead of its z-derivative, Sec. 3)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    r2 = x * x + y * y + z * z
    if kind == "inv_r":
        return 1.0 / np.sqrt(r2)
    if kind != "dz_inv_r":
        raise ValueError(kind)
    return -z / (r2 * np.sqrt(r2))


def wrapped_lags(n: int, pad: int = 1) -> np.ndarray:
    """Integer lags d of the L = pad*n periodic grid, stored in DFT order.

    Position t of an L-point DFT stands for the lag t when t < L/2 and t - L
    otherwise, so the lags cover [-L/2, L/2).  This is the periodisation of
    Sec. 5 (the space R^2 replaced by the square Pi_xy); with pad = 2 and data
    zero-padded to 2n, the circular sum equals the aperiodic one over R.
    """
    L = pad * n
    t = np.arange(L)
    return np.where(t < L // 2, t, t - L)


def kernel_samples(n: int, h: float, dz: float, pad: int = 1, kind: str = "dz_inv_r") -> np.ndarray:
    """K at the wrapped lags (dy, dx) * h for one depth difference dz, shape [L, L] ([y, x])."""
    lag = wrapped_lags(n, pad) * h
    return kernel_K(lag[None, :], lag[:, None], dz, kind)


# --------------------------------------------------------------------------- DFT
def dft_matrix(L: int) -> np.ndarray:
    """W[k, t] = exp(-2 pi i ((k t) mod L) / L): the DFT as a plain matrix (index reduced first)."""
    k = np.arange(L)
    kt = np.outer(k, k) % L
    return np.exp(-2j * np.pi * kt / L)


def dft2(f: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT over the last two axes, one matrix product per axis (naive, O(L^3))."""
    Ly, Lx = f.shape[-2:]
    Wy, Wx = dft_matrix(Ly), dft_matrix(Lx)
    return Wy @ f.astype(np.complex128) @ Wx.T


def idft2(F: np.ndarray) -> np.ndarray:
    """Inverse of dft2: conjugate twiddles and the factor 1/(Ly Lx)."""
    Ly, Lx = F.shape[-2:]
    Wy, Wx = dft_matrix(Ly).conj(), dft_matrix(Lx).conj()
    return (Wy @ F.astype(np.complex128) @ Wx.T) / (Ly * Lx)


# --------------------------------------------------------------------------- Eq. (6)
def kernel_hat(n: int, h: float, zy, zr, pad: int = 1, kind: str = "dz_inv_r") -> np.ndarray:
    """Discrete analogue of K~(w1, w2, z_i - z'_j) (Algorithm 1 step 1, Sec. 5).

    Returns h^2 * DFT of the sampled kernel, shape [M, M', L, L] ([i, j, ky, kx]).
    The sampled kernel is even in x and y, so the DFT is real; the imaginary
    part (rounding only) is checked and dropped.
    """
    zy = np.atleast_1d(np.asarray(zy, np.float64))
    zr = np.atleast_1d(np.asarray(zr, np.float64))
    L = pad * n
    out = np.empty((zy.size, zr.size, L, L))
    for i, zi in enumerate(zy):
        for j, zj in enumerate(zr):
            Kh = h * h * dft2(kernel_samples(n, h, zi - zj, pad, kind))
            assert np.max(np.abs(Kh.imag)) <= 1e-9 * max(1.0, np.max(np.abs(Kh.real)))
            out[i, j] = Kh.real
    return out


def A_matrices(n: int, h: float, zy, zr, nu, pad: int = 1, kind: str = "dz_inv_r") -> np.ndarray:
    """A^(m) = [nu_j K~(w^(m), z_i - z'_j)] of Eq. (6) for every frequency m.

    Shape [L, L, M, M'] ([ky, kx, i, j]): one M x M' matrix per grid frequency.
    """
    nu = np.asarray(nu, np.float64)
    Kh = kernel_hat(n, h, zy, zr, pad, kind)                # [i, j, ky, kx]
    A = Kh * nu[None, :, None, None]
    return np.ascontiguousarray(np.transpose(A, (2, 3, 0, 1)))


def alpha_scale(A: np.ndarray) -> float:
    """s^2 = max over frequencies of ||A^(m)||_F^2, which makes alpha dimensionless (a reading)."""
    return float(np.max(np.sum(A * A, axis=(-2, -1))))


# --------------------------------------------------------------------------- forward operator
def forward_direct(zeta: np.ndarray, n: int, h: float, zy, zr, nu, pad: int = 1, kind: str = "dz_inv_r") -> np.ndarray:
    """Direct quadrature of the discretised Eq. (4) (the definition; O(n^4 M M')).

    U(b, a, i) = sum_{b', a', j} h^2 nu_j K(lag(a - a') h, lag(b - b') h, z_i - z'_j) zeta(b', a', j)

    with lag() the wrapped lag of the pad*n periodic box.  ``zeta`` is
    [..., M', n, n]; the result is [..., M, n, n].  Small n only.
    """
    zy = np.atleast_1d(np.asarray(zy, np.float64))
    zr = np.atleast_1d(np.asarray(zr, np.float64))
    nu = np.asarray(nu, np.float64)
    L = pad * n
    idx = np.arange(n)
    diff = idx[:, None] - idx[None, :]                       # a - a'
    lag = (((diff + L // 2) % L) - L // 2) * h               # wrapped into [-L/2, L/2)
    lead = zeta.shape[:-3]
    out = np.zeros(lead + (zy.size, n, n))
    for i, zi in enumerate(zy):
        for j, zj in enumerate(zr):
            # Kmat[b, a, b', a'] = K(lag[a, a'], lag[b, b'], dz)
            Kmat = kernel_K(lag[None, :, None, :], lag[:, None, :, None], zi - zj, kind)
            out[..., i, :, :] += h * h * nu[j] * np.einsum("bacd,...cd->...ba", Kmat, zeta[..., j, :, :])
    return out


def _embed(f: np.ndarray, n: int, pad: int) -> np.ndarray:
    """Zero-pad [..., n, n] into the [..., pad*n, pad*n] box (data in the low corner)."""
    if pad == 1:
        return np.asarray(f, np.float64)
    L = pad * n
    g = np.zeros(f.shape[:-2] + (L, L))
    g[..., :n, :n] = f
    return g


def forward_dft(zeta: np.ndarray, n: int, h: float, zy, zr, nu, pad: int = 1, A=None,
                kind: str = "dz_inv_r") -> np.ndarray:
    """The same operator through the DFT (Eq. (5) discretised, Eq. (6)):

    U~_i(m) = sum_j A^(m)_ij zeta~_j(m),   U = IDFT2(U~) cropped to the n x n grid.
    ``zeta`` is [..., M', n, n]; the result is [..., M, n, n].
    """
    if A is None:
        A = A_matrices(n, h, zy, zr, nu, pad, kind)          # [ky, kx, i, j]
    Zh = dft2(_embed(zeta, n, pad))                          # [..., j, ky, kx]
    Uh = np.einsum("yxij,...jyx->...iyx", A, Zh)
    U = idft2(Uh)
    return U.real[..., :n, :n]


# --------------------------------------------------------------------------- Tikhonov (Sec. 5)
def tikhonov_qr(A: np.ndarray, Uh: np.ndarray, alpha_s2: float) -> np.ndarray:
    """Tikhonov-regularised normal solution of A x = u for a batch of small systems.

    x_alpha = argmin ||A x - u||^2 + alpha s^2 ||x||^2, computed as the least-squares
    solution of the stacked system [A; sqrt(alpha s^2) I] x = [u; 0] through a
    Householder QR (LAPACK geqrf via numpy.linalg.qr).  A is real, so the real
    and imaginary parts of a complex right-hand side are two real columns.

    A: [B, M, M'] real.  Uh: [B, M, K] complex (K right-hand sides).  Returns [B, M', K].
    """
    A = np.asarray(A, np.float64)
    B, M, Mp = A.shape
    K = Uh.shape[-1]
    S = np.concatenate([A, np.broadcast_to(np.sqrt(alpha_s2) * np.eye(Mp), (B, Mp, Mp))], axis=1)
    rhs = np.concatenate([Uh.real, Uh.imag], axis=-1)                  # [B, M, 2K]
    rhs = np.concatenate([rhs, np.zeros((B, Mp, 2 * K))], axis=1)     # [B, M+M', 2K]
    Qm, R = np.linalg.qr(S)                                           # reduced QR
    x = np.linalg.solve(R, np.swapaxes(Qm, -1, -2) @ rhs)
    return x[..., :K] + 1j * x[..., K:]


def tsvd_solve(A: np.ndarray, Uh: np.ndarray, t: float) -> np.ndarray:
    """Truncated-SVD solution of A x = u for a batch of small systems (the regularising algorithm the
    paper reports as its best, Sec. 5): with A = W diag(sigma) V^T (numpy.linalg.svd, LAPACK gesdd),
    x_t = sum over the singular values with sigma^2 >= t of v_i (w_i^T u) / sigma_i, so that t plays the
    role of alpha s^2 (a reading: the paper does not say how the truncation level is chosen; here the
    discrepancy principle picks it from the same candidate list).

    A: [B, M, M'] real.  Uh: [B, M, K] complex.  Returns [B, M', K]."""
    A = np.asarray(A, np.float64)
    W, sig, Vt = np.linalg.svd(A, full_matrices=False)              # [B,M,r], [B,r], [B,r,M']
    keep = sig * sig >= t
    inv = np.where(keep, 1.0 / np.where(sig > 0, sig, 1.0), 0.0)
    proj = np.swapaxes(W, -1, -2) @ Uh                                # [B, r, K]
    return np.swapaxes(Vt, -1, -2) @ (inv[..., None] * proj)


def residual_sq(A: np.ndarray, Zh: np.ndarray, Uh: np.ndarray, n_freq: int | None = None) -> float:
    """sum over frequencies and right-hand sides of |A^(m) zeta~ - U~|^2, divided by L^2.

    By Parseval this is the squared residual ||A zeta - U||^2 on the spatial grid
    (the data norm of the discrepancy principle).  A: [B, M, M'], Zh: [B, M', K],
    Uh: [B, M, K]; ``n_freq`` = L^2, the number of grid frequencies (default B).
    """
    r = A @ Zh - Uh
    return float(np.sum(np.abs(r) ** 2) / (A.shape[0] if n_freq is None else n_freq))


def radial_bands(L: int, n_bands: int) -> np.ndarray:
    """Band of every frequency of the L x L DFT grid, flattened [ky, kx]: with the folded indices
    k' = min(k, L - k) per axis, band = floor(n_bands |k'| / (sqrt(2) L/2)), clamped to n_bands - 1
    (a reading: the paper only says step 2 is done per frequency; bands group frequencies by |w|)."""
    k = np.arange(L)
    kf = np.minimum(k, L - k)
    rho = np.sqrt(kf[None, :] ** 2 + kf[:, None] ** 2)
    b = np.floor(n_bands * rho / (np.sqrt(2.0) * (L // 2))).astype(int)
    return np.minimum(b, n_bands - 1).ravel()


def choose_alpha_index(res2, delta: float, tau: float):
    """Discrepancy principle (Sec. 4): the largest alpha_k whose residual is <= tau * delta.

    ``res2`` holds squared residuals for increasing alphas.  Returns (index, flag) where
    flag = 0 normally, 1 when no alpha satisfies the bound (the smallest is used) and
    2 when every alpha does (the largest is used).
    """
    res2 = np.asarray(res2, np.float64)
    ok = res2 <= (tau * delta) ** 2
    if not ok.any():
        return 0, 1
    k = int(np.max(np.nonzero(ok)[0]))
    return k, (2 if ok.all() else 0)


# --------------------------------------------------------------------------- sources (Sec. 2, Sec. 6)
def A0_of(g, t_max: float = 60.0) -> float:
    """A0 = integral_0^inf g(t) dt (Sec. 2, Assumption 5)."""
    from scipy.integrate import quad
    return quad(g, 0.0, t_max, limit=200)[0]


def A2_of(g, t_max: float = 60.0) -> float:
    """A2 = integral_0^inf t^2 g(t) dt (Sec. 2, Assumption 5)."""
    from scipy.integrate import quad
    return quad(lambda t: t * t * g(t), 0.0, t_max, limit=200)[0]


def V0(points: np.ndarray, X, Y, Z, A0: float = 1.0) -> np.ndarray:
    """V0(x) = -A0/(4 pi) sum_l 1/|x - x_l| for delta-shaped sources at ``points`` [L, 3] (Sec. 6)."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    Z = np.asarray(Z, np.float64)
    acc = np.zeros(np.broadcast(X, Y, Z).shape)
    for (px, py, pz) in np.asarray(points, np.float64).reshape(-1, 3):
        acc += 1.0 / np.sqrt((X - px) ** 2 + (Y - py) ** 2 + (Z - pz) ** 2)
    return -A0 / (4.0 * np.pi) * acc


def _grid_xyz(n: int, x0: float, h: float, zr):
    c = x0 + (np.arange(n) + 0.5) * h
    Z = np.asarray(zr, np.float64)[:, None, None]
    return c[None, None, :], c[None, :, None], Z             # X [1,1,n], Y [1,n,1], Z [M',1,1]


def zeta_from_xi(xi: np.ndarray, sources: np.ndarray, n: int, x0: float, h: float, zr, A0: float = 1.0):
    """zeta_q = xi * V0_q on the R grid (Sec. 2: zeta = xi V0), one plane set per source parameter q.

    xi: [M', n, n]; sources: [Q, L, 3].  Returns [Q, M', n, n].
    """
    X, Y, Z = _grid_xyz(n, x0, h, zr)
    return np.stack([xi * V0(s, X, Y, Z, A0) for s in np.asarray(sources, np.float64)])


def combine_sources(zeta: np.ndarray, sources: np.ndarray, n: int, x0: float, h: float, zr, A0: float = 1.0):
    """Algorithm 1 step 4 for several source parameters q sharing one xi.

    Each q gives zeta_q = xi V0_q; the pointwise least-squares xi is
    sum_q V0_q zeta_q / sum_q V0_q^2, which is zeta / V0 when Q = 1.
    zeta: [Q, M', n, n].  Returns [M', n, n].
    """
    X, Y, Z = _grid_xyz(n, x0, h, zr)
    num = np.zeros(zeta.shape[1:])
    den = np.zeros(zeta.shape[1:])
    for q, s in enumerate(np.asarray(sources, np.float64)):
        v = V0(s, X, Y, Z, A0)
        num += v * zeta[q]
        den += v * v
    return num / den


# --------------------------------------------------------------------------- right-hand side of Eq. (7)
def pi_depths(n_pi: int, half: float):
    """Midpoint grid of the vertical extent [-half, half] of the box Pi (Sec. 5: R^3 replaced by the
    cube Pi = [-r, r]^3; horizontally the periodic box of the R grid) and its quadrature weights."""
    dz = 2.0 * half / n_pi
    return -half + (np.arange(n_pi) + 0.5) * dz, np.full(n_pi, dz)


def rhs_terms(n: int, x0: float, h: float, zy, sources: np.ndarray, n_pi: int, half: float):
    """The a-priori terms of Eq. (7) for point sources x_{q,l} (Sec. 6), on the observation grid:
        S_q(x) = sum_l d/dx3 (1/|x - x_l|) = sum_l K(x - x_l),
        I_q(x) = sum_l integral over Pi of d/dx3 (1/|x - x'|) / |x' - x_l| dx'
    (R^3 replaced by Pi as the paper does when it simulates its data, Sec. 6); I_q is the discrete
    operator of Eq. (4) with Pi's depth grid in place of R's, applied to f_q(x') = sum_l 1/|x' - x_l|.
    Returns S, I of shape [Q, M, n, n]."""
    zy = np.atleast_1d(np.asarray(zy, np.float64))
    src = np.asarray(sources, np.float64)
    X, Y, Zy = _grid_xyz(n, x0, h, zy)
    zp, nup = pi_depths(n_pi, half)
    Xp, Yp, Zp = _grid_xyz(n, x0, h, zp)
    S = np.zeros((src.shape[0], zy.size, n, n))
    f = np.zeros((src.shape[0], zp.size, n, n))
    for q, pts in enumerate(src):
        for (px, py, pz) in pts:
            S[q] += kernel_K(X - px, Y - py, Zy - pz)
            f[q] += 1.0 / np.sqrt((Xp - px) ** 2 + (Yp - py) ** 2 + (Zp - pz) ** 2)
    I = forward_dft(f, n, h, zy, zp, nup)
    return S, I


def assemble_rhs(dV2dz: np.ndarray, n: int, x0: float, h: float, zy, sources, A0: float, A2: float, c0: float,
                 n_pi: int, half: float) -> np.ndarray:
    """Right-hand side of Eq. (7) from the measured dV2/dx3 on Y:
        U = 2 pi dV2/dx3 + (A2 / 2) S - A0 / (4 pi c0^2) I."""
    S, I = rhs_terms(n, x0, h, zy, sources, n_pi, half)
    return 2.0 * np.pi * np.asarray(dV2dz, np.float64) + 0.5 * A2 * S - A0 / (4.0 * np.pi * c0 * c0) * I


def simulate_dV2dz(U: np.ndarray, n: int, x0: float, h: float, zy, sources, A0: float, A2: float, c0: float,
                   n_pi: int, half: float) -> np.ndarray:
    """The paper's simulated measurement (Sec. 6) for a given left-hand side U = integral over R of
    K zeta: dV2/dx3 = (U - (A2 / 2) S + A0 / (4 pi c0^2) I) / (2 pi)."""
    S, I = rhs_terms(n, x0, h, zy, sources, n_pi, half)
    return (np.asarray(U, np.float64) - 0.5 * A2 * S + A0 / (4.0 * np.pi * c0 * c0) * I) / (2.0 * np.pi)


# --------------------------------------------------------------------------- Algorithm 1
def invert(U: np.ndarray, n: int, x0: float, h: float, zy, zr, nu, *, pad: int = 1,
           alpha=None, alphas=None, delta=None, tau: float = 1.1, sources=None, A0: float = 1.0,
           output: str = "xi", chunk: int = 4096, bins=None, A=None, n_bands: int = 1, band_alpha_index=None,
           ra: str = "tikhonov", kind: str = "dz_inv_r"):
    """Algorithm 1 (Sec. 4) in its finite-dimensional form (Sec. 5).

    U: [Q, M, n, n] data for Q source parameters.
    Step 1: 2D DFT of the data; the DFT of the kernel gives A^(m) (Eq. (6)).
    Step 2: per frequency, a Tikhonov solution of Eq. (6), alpha either fixed
            (``alpha``) or chosen from ``alphas`` by the discrepancy principle
            with ``delta`` and ``tau``; the residual is summed over all frequencies
            and all q (one global alpha).
    Step 3: inverse 2D DFT per depth z'_j (cropped to n x n when pad = 2).
    Step 4: xi = zeta / V0 (several q: pointwise least squares).

    Returns a dict with ``zeta`` [Q, M', n, n], ``xi`` [M', n, n] (if sources are given and
    output == "xi"), ``alpha_index``, ``flag`` and ``res2`` (squared residual per candidate).
    ``output="none"`` stops after step 2.  ``bins`` (optional) restricts step 2 to a subset of
    the flattened frequencies; every other frequency gets the zero solution, which is exact when
    the data spectrum vanishes there (a zero right-hand side has the zero Tikhonov solution).
    ``ra="tsvd"`` replaces the Tikhonov solution by the truncated SVD with truncation level alpha s^2
    (tsvd_solve); everything else is unchanged.
    ``n_bands`` > 1 applies the discrepancy principle per radial band of frequencies (see
    radial_bands): band b gets its own alpha, the largest with residual_b <= tau delta_b, where
    delta_b^2 = delta^2 (frequencies in b) / L^2 (the share of white noise in the band); ``res2``
    is then [n_bands, n_alpha] and ``alpha_index`` a list.  ``band_alpha_index`` (with
    ``alphas``) imposes the per-band indices instead of choosing them.
    """
    zy = np.atleast_1d(np.asarray(zy, np.float64))
    zr = np.atleast_1d(np.asarray(zr, np.float64))
    Q, M = U.shape[0], U.shape[1]
    Mp = zr.size
    L = pad * n
    if A is None:
        A = A_matrices(n, h, zy, zr, nu, pad, kind)
    s2 = alpha_scale(A)
    Af = A.reshape(L * L, M, Mp)
    Uh = dft2(_embed(U, n, pad))                                     # [Q, M, L, L]
    Uf = np.transpose(Uh.reshape(Q, M, L * L), (2, 1, 0))             # [B, M, Q]
    sel = np.arange(L * L) if bins is None else np.asarray(bins)

    def solve(a):
        """Tikhonov solutions on the selected frequencies, [len(sel), M', Q]."""
        Z = np.empty((sel.size, Mp, Q), np.complex128)
        for s in range(0, sel.size, chunk):
            b = sel[s:s + chunk]
            Z[s:s + b.size] = (tsvd_solve if ra == "tsvd" else tikhonov_qr)(Af[b], Uf[b], a * s2)
        return Z

    res2 = None
    flag = 0
    if alpha is not None:
        k = -1
        Zs = solve(float(alpha))
    elif n_bands <= 1 and band_alpha_index is None:
        alphas = np.asarray(alphas, np.float64)
        res2 = np.array([residual_sq(Af[sel], solve(float(a)), Uf[sel], L * L) for a in alphas])
        k, flag = choose_alpha_index(res2, float(delta), tau)
        Zs = solve(float(alphas[k]))
    else:
        alphas = np.asarray(alphas, np.float64)
        nb = max(int(n_bands), 1)
        band = radial_bands(L, nb)[sel]
        if band_alpha_index is None:
            res2 = np.zeros((nb, alphas.size))
            for t, a in enumerate(alphas):
                r = np.sum(np.abs(Af[sel] @ solve(float(a)) - Uf[sel]) ** 2, axis=(1, 2)) / (L * L)
                res2[:, t] = np.bincount(band, weights=r, minlength=nb)
            count = np.bincount(radial_bands(L, nb), minlength=nb)
            k, flag = [], 0
            for b in range(nb):
                kb, fb = choose_alpha_index(res2[b], float(delta) * np.sqrt(count[b] / (L * L)), tau)
                k.append(kb)
                flag |= fb
        else:
            k = [int(v) for v in band_alpha_index]
        Zs = np.empty((sel.size, Mp, Q), np.complex128)
        for kb in sorted(set(k)):
            use = np.isin(band, [b for b in range(nb) if k[b] == kb])
            full = solve(float(alphas[kb]))
            Zs[use] = full[use]
    out = {"alpha_index": k, "flag": flag, "res2": res2, "s2": s2}
    if output == "none":
        return out
    Zh = np.zeros((L * L, Mp, Q), np.complex128)
    Zh[sel] = Zs
    Zq = np.transpose(Zh, (2, 1, 0)).reshape(Q, Mp, L, L)
    zeta = idft2(Zq).real[..., :n, :n]
    out["zeta"] = zeta
    if sources is not None and output == "xi":
        out["xi"] = combine_sources(zeta, sources, n, x0, h, zr, A0)
    return out
