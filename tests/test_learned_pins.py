"""Pins of the learned-alpha oracle (CPU only): closed forms, finite differences, Parseval and
invariants that a dropped term, a transposed operand or a wrong sign in it would break."""

import numpy as np
import pytest

import oracle as O


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ------------------------------------------------------------------ features
def test_features_single_cosine_closed_form():
    """U = A cos(2 pi k x / n): its spectrum is A n^2 / 2 at +-k (two frequencies), so the band
    holding |k| has power A^2 n^4 / 2 and f_b = log10(A^2 n^4 / (2 count_b delta^2))."""
    n, k, amp, delta, nb = 16, 3, 0.7, 0.05, 4
    x = np.arange(n)
    U = np.broadcast_to(amp * np.cos(2 * np.pi * k * x / n)[None, :], (n, n))[None, None]
    f = O.band_features(U, nb, delta)
    band = O.radial_bands(n, nb)
    b = band[k]                                   # frequency (ky = 0, kx = k), flattened [ky, kx]
    count = np.bincount(band, minlength=nb)[b]
    assert abs(f[b] - np.log10(amp ** 2 * n ** 4 / (2 * count * delta ** 2))) < 1e-12
    assert all(f[c] < f[b] - 20 for c in range(nb) if c != b)


def test_features_parseval_and_white_noise_level():
    """sum_b count_b delta^2 10^f_b = sum |U~|^2 = n^2 ||U||^2; white noise of norm delta gives f ~ 0."""
    rng = np.random.default_rng(7)
    n, nb = 64, 6
    U = rng.standard_normal((4, 1, n, n))
    delta = float(np.linalg.norm(U))
    f = O.band_features(U, nb, delta)
    count = np.bincount(O.radial_bands(n, nb), minlength=nb)
    assert abs(np.sum(count * delta ** 2 * 10.0 ** f) - n * n * np.sum(U ** 2)) < 1e-9 * n * n * np.sum(U ** 2)
    assert np.all(np.abs(f) < 0.1)


# ------------------------------------------------------------------ targets
def _tiny_problem(seed=3):
    n, h, zy, zr, nu = 8, 0.25, [0.0], [0.3, 0.45, 0.6], [0.15] * 3
    rng = np.random.default_rng(seed)
    zt = rng.standard_normal((2, 3, n, n))
    U = O.forward_direct(zt, n, h, zy, zr, nu) + 0.05 * rng.standard_normal((2, 1, n, n))
    return n, h, zy, zr, nu, zt, U


def test_band_errors_equal_spatial_errors_of_the_full_inversion():
    """One band: E(alpha) is L^2 times the spatial ||zeta_alpha - zeta_true||^2 of Algorithm 1
    run at that alpha (Parseval for the unnormalised DFT); bands partition the total."""
    n, h, zy, zr, nu, zt, U = _tiny_problem()
    A = O.A_matrices(n, h, zy, zr, nu)
    al = np.logspace(-5, 0, 6)
    E1 = O.band_error_curves(A, U, zt, al, 1)
    for k, a in enumerate(al):
        z = O.invert(U, n, -1.0, h, zy, zr, nu, alpha=a, output="zeta")["zeta"]
        assert abs(E1[0, k] - n * n * np.sum((z - zt) ** 2)) < 1e-9 * E1[0, k]
    E4 = O.band_error_curves(A, U, zt, al, 4)
    assert np.allclose(E4.sum(axis=0), E1[0], rtol=1e-12)
    idx = O.band_optimal_alpha(E4)
    assert all(E4[b, idx[b]] == E4[b].min() for b in range(4))


def test_band_optimal_alphas_beat_every_global_alpha():
    """Per-band minimisers give a total error no larger than the best single alpha (the global
    choice is one of the per-band choices)."""
    n, h, zy, zr, nu, zt, U = _tiny_problem(5)
    A = O.A_matrices(n, h, zy, zr, nu)
    al = np.logspace(-6, 0, 13)
    E = O.band_error_curves(A, U, zt, al, 3)
    idx = O.band_optimal_alpha(E)
    assert E[np.arange(3), idx].sum() <= E.sum(axis=0).min() * (1 + 1e-12)
    y = O.log_alpha_target(al, idx)
    assert np.allclose(y * O.LOG_SCALE - O.LOG_SHIFT, np.log10(al[idx]))


# ------------------------------------------------------------------ network
def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(11)
    nin, nh, nout, B = 3, 5, 2, 4
    npar = O.mlp_offsets(nin, nh, nout)["np"]
    assert npar == nh * nin + nh + nh * nh + nh + nout * nh + nout
    p = rng.standard_normal(npar) * 0.7
    X = rng.standard_normal((B, nin))
    T = rng.standard_normal((B, nout))
    loss, g = O.mlp_loss_grad(p, X, T, nin, nh, nout)
    fd = np.empty(npar)
    e = 1e-6
    for i in range(npar):
        d = np.zeros(npar)
        d[i] = e
        fd[i] = (O.mlp_loss_grad(p + d, X, T, nin, nh, nout)[0] - O.mlp_loss_grad(p - d, X, T, nin, nh, nout)[0]) / (2 * e)
    assert rel(g, fd) < 1e-7
    Y, _ = O.mlp_forward(p, X, nin, nh, nout)
    assert abs(loss - np.mean((Y - T) ** 2)) < 1e-14


def test_mlp_forward_by_hand_and_zero_output_layer():
    """A hand-evaluated 1-1-1 network, and W3 = 0: y = b3, gradient only in b3 (closed form)."""
    p = np.array([0.5, 0.1, -2.0, 0.3, 1.5, -0.2])        # W1 b1 W2 b2 W3 b3 (nin = nh = nout = 1)
    x = 0.8
    h1 = np.tanh(0.5 * x + 0.1)
    h2 = np.tanh(-2.0 * h1 + 0.3)
    y, _ = O.mlp_forward(p, np.array([[x]]), 1, 1, 1)
    assert abs(y[0, 0] - (1.5 * h2 - 0.2)) < 1e-15
    rng = np.random.default_rng(2)
    nin, nh, nout, B = 4, 6, 3, 5
    o = O.mlp_offsets(nin, nh, nout)
    p = rng.standard_normal(o["np"])
    p[o["W3"]:o["b3"]] = 0.0
    X, T = rng.standard_normal((B, nin)), rng.standard_normal((B, nout))
    Y, _ = O.mlp_forward(p, X, nin, nh, nout)
    assert np.allclose(Y, p[o["b3"]:][None, :], rtol=0, atol=0)
    _, g = O.mlp_loss_grad(p, X, T, nin, nh, nout)
    assert np.all(g[:o["W3"]] == 0.0)
    assert np.allclose(g[o["b3"]:], 2.0 * (p[o["b3"]:][None, :] - T).sum(axis=0) / (B * nout), rtol=1e-14)


def test_adam_first_step_is_signed_learning_rate():
    """With zero moments, the bias-corrected first step is -lr g / (|g| + eps) ~ -lr sign(g)."""
    g = np.array([0.3, -2.0, 1e-3, -5e-2])
    p, m, v = O.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_ties_to_even():
    vals = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -3.0, 1 + 2.0 ** -8 + 2.0 ** -20])
    want = np.array([1.0, 1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -3.0, 1 + 2.0 ** -7])
    assert np.array_equal(O.bf16_round(vals), want)


def test_nearest_candidate_rule():
    """Zero hidden layers' effect (W3 = 0): y = b3, so log10 alpha = 3.5 b3 - 4.5 picks the nearest
    candidate on the log grid."""
    nb, nh = 3, 4
    o = O.mlp_offsets(nb, nh, nb)
    p = np.zeros(o["np"])
    al = np.logspace(-8, -1, 8)
    want_log = np.array([-7.9, -4.4, -0.2])
    p[o["b3"]:] = (want_log + O.LOG_SHIFT) / O.LOG_SCALE
    y, la, idx = O.learned_alpha_index(p, np.ones(nb), al, nh)
    assert np.allclose(la, want_log)
    assert list(idx) == [0, 4, 7]
