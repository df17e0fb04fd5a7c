"""The oracle's pins have teeth (CPU only): each test plants one plausible mistake in the oracle -- a flipped
sign, a dropped factor or term, a wrong index range, a wrong normalisation, the wrong end of a rule -- and
checks that at least one pin of tests/test_oracle_pins.py or tests/test_learned_pins.py then fails.  The
mistakes are planted by monkeypatching the oracle's functions for the duration of one test; the oracle's
files are not touched."""

import importlib.util
import os

import numpy as np
import pytest

import oracle
from oracle import fr3d_oracle as FO
from oracle import learned_oracle as LO
from oracle import unet_oracle as UO

HERE = os.path.dirname(os.path.abspath(__file__))


def _load(name):
    spec = importlib.util.spec_from_file_location(f"_pins_{name}", os.path.join(HERE, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


P = _load("test_oracle_pins")
LP = _load("test_learned_pins")
UP = _load("test_unet_pins")


def _plant(monkeypatch, module, name, fn):
    """Replace oracle function ``name`` in its defining module (for the oracle's internal calls) and in
    the package namespace (for the pins' calls)."""
    monkeypatch.setattr(module, name, fn)
    if hasattr(oracle, name):
        monkeypatch.setattr(oracle, name, fn)


def _some_pin_fails(pins):
    failed = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed.append(pin)
    return failed


# ------------------------------------------------------------------ the planted mistakes
def _kernel_sign(mp):
    orig = FO.kernel_K
    _plant(mp, FO, "kernel_K", lambda x, y, z, kind="dz_inv_r": -orig(x, y, z, kind) if kind == "dz_inv_r"
           else orig(x, y, z, kind))


def _kernel_power(mp):
    orig = FO.kernel_K

    def bad(x, y, z, kind="dz_inv_r"):
        if kind != "dz_inv_r":
            return orig(x, y, z, kind)
        z = np.asarray(z, np.float64)
        return -z / (np.asarray(x) ** 2 + np.asarray(y) ** 2 + z * z)          # r^2 instead of r^3
    _plant(mp, FO, "kernel_K", bad)


def _dft_exponent_sign(mp):
    def bad(L):
        k = np.arange(L)
        return np.exp(2j * np.pi * (np.outer(k, k) % L) / L)
    _plant(mp, FO, "dft_matrix", bad)


def _idft_unnormalised(mp):
    def bad(F):
        Ly, Lx = F.shape[-2:]
        return FO.dft_matrix(Ly).conj() @ F.astype(np.complex128) @ FO.dft_matrix(Lx).conj().T
    _plant(mp, FO, "idft2", bad)


def _quadrature_weights_dropped(mp):
    orig = FO.A_matrices
    _plant(mp, FO, "A_matrices", lambda n, h, zy, zr, nu, pad=1, kind="dz_inv_r":
           orig(n, h, zy, zr, np.ones(np.atleast_1d(zr).size), pad, kind))


def _cell_area_dropped(mp):
    orig = FO.kernel_hat
    _plant(mp, FO, "kernel_hat", lambda n, h, zy, zr, pad=1, kind="dz_inv_r": orig(n, h, zy, zr, pad, kind) / (h * h))


def _alpha_scale_not_squared(mp):
    _plant(mp, FO, "alpha_scale", lambda A: float(np.max(np.sqrt(np.sum(A * A, axis=(-2, -1))))))


def _alpha_scale_summed(mp):
    _plant(mp, FO, "alpha_scale", lambda A: float(np.sum(A * A)))


def _tikhonov_unrooted(mp):
    orig = FO.tikhonov_qr
    _plant(mp, FO, "tikhonov_qr", lambda A, Uh, a: orig(A, Uh, a * a))        # [A; a I] instead of [A; sqrt(a) I]


def _tikhonov_drops_imaginary_part(mp):
    orig = FO.tikhonov_qr
    _plant(mp, FO, "tikhonov_qr", lambda A, Uh, a: orig(A, Uh.real + 0j, a))


def _residual_unnormalised(mp):
    orig = FO.residual_sq
    _plant(mp, FO, "residual_sq", lambda A, Zh, Uh, n_freq=None: orig(A, Zh, Uh, 1))


def _discrepancy_smallest_admissible(mp):
    def bad(res2, delta, tau):
        ok = np.asarray(res2) <= (tau * delta) ** 2
        if not ok.any():
            return 0, 1
        return int(np.min(np.nonzero(ok)[0])), (2 if ok.all() else 0)
    _plant(mp, FO, "choose_alpha_index", bad)


def _discrepancy_bound_not_squared(mp):
    def bad(res2, delta, tau):
        ok = np.asarray(res2) <= tau * delta
        if not ok.any():
            return 0, 1
        return int(np.max(np.nonzero(ok)[0])), (2 if ok.all() else 0)
    _plant(mp, FO, "choose_alpha_index", bad)


def _v0_sign(mp):
    orig = FO.V0
    _plant(mp, FO, "V0", lambda points, X, Y, Z, A0=1.0: -orig(points, X, Y, Z, A0))


def _v0_without_four_pi(mp):
    orig = FO.V0
    _plant(mp, FO, "V0", lambda points, X, Y, Z, A0=1.0: 4.0 * np.pi * orig(points, X, Y, Z, A0))


def _combination_without_squares(mp):
    def bad(zeta, sources, n, x0, h, zr, A0=1.0):
        X, Y, Z = FO._grid_xyz(n, x0, h, zr)
        num = np.zeros(zeta.shape[1:])
        den = np.zeros(zeta.shape[1:])
        for q, s in enumerate(np.asarray(sources, np.float64)):
            v = FO.V0(s, X, Y, Z, A0)
            num += v * zeta[q]
            den += np.abs(v)
        return num / den
    _plant(mp, FO, "combine_sources", bad)


def _zeta_divides_by_v0(mp):
    def bad(xi, sources, n, x0, h, zr, A0=1.0):
        X, Y, Z = FO._grid_xyz(n, x0, h, zr)
        return np.stack([xi / FO.V0(s, X, Y, Z, A0) for s in np.asarray(sources, np.float64)])
    _plant(mp, FO, "zeta_from_xi", bad)


def _padding_centred(mp):
    def bad(f, n, pad):
        if pad == 1:
            return np.asarray(f, np.float64)
        L, o = pad * n, n // 2
        g = np.zeros(f.shape[:-2] + (L, L))
        g[..., o:o + n, o:o + n] = f
        return g
    _plant(mp, FO, "_embed", bad)


def _padded_lags_wrapped_at_half_the_grid(mp):
    def bad(n, pad=1):
        L = pad * n
        t = np.arange(L)
        return np.where(t < n // 2, t, t - L)
    _plant(mp, FO, "wrapped_lags", bad)


def _tsvd_cut_on_sigma(mp):
    orig = FO.tsvd_solve
    _plant(mp, FO, "tsvd_solve", lambda A, Uh, t: orig(A, Uh, t * t))          # sigma >= t instead of sigma^2 >= t


def _bands_unfolded(mp):
    def bad(L, n_bands):
        k = np.arange(L)
        rho = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
        b = np.floor(n_bands * rho / (np.sqrt(2.0) * (L // 2))).astype(int)
        return np.minimum(b, n_bands - 1).ravel()
    _plant(mp, FO, "radial_bands", bad)


def _rhs_integral_sign(mp):
    def bad(dV2dz, n, x0, h, zy, sources, A0, A2, c0, n_pi, half):
        S, I = FO.rhs_terms(n, x0, h, zy, sources, n_pi, half)
        return 2.0 * np.pi * np.asarray(dV2dz, np.float64) + 0.5 * A2 * S + A0 / (4.0 * np.pi * c0 * c0) * I
    _plant(mp, FO, "assemble_rhs", bad)


def _rhs_source_coefficient_in_both(mp):
    """A2 instead of A2 / 2 in both the assembly and the simulated measurement: the round trip still closes."""
    def bad_assemble(dV2dz, n, x0, h, zy, sources, A0, A2, c0, n_pi, half):
        S, I = FO.rhs_terms(n, x0, h, zy, sources, n_pi, half)
        return 2.0 * np.pi * np.asarray(dV2dz, np.float64) + A2 * S - A0 / (4.0 * np.pi * c0 * c0) * I

    def bad_simulate(U, n, x0, h, zy, sources, A0, A2, c0, n_pi, half):
        S, I = FO.rhs_terms(n, x0, h, zy, sources, n_pi, half)
        return (np.asarray(U, np.float64) - A2 * S + A0 / (4.0 * np.pi * c0 * c0) * I) / (2.0 * np.pi)
    _plant(mp, FO, "assemble_rhs", bad_assemble)
    _plant(mp, FO, "simulate_dV2dz", bad_simulate)


def _rhs_integral_coefficient_in_both(mp):
    """1/(4 pi c0^2) without its 4 pi in both functions: the round trip still closes."""
    def bad_assemble(dV2dz, n, x0, h, zy, sources, A0, A2, c0, n_pi, half):
        S, I = FO.rhs_terms(n, x0, h, zy, sources, n_pi, half)
        return 2.0 * np.pi * np.asarray(dV2dz, np.float64) + 0.5 * A2 * S - A0 / (c0 * c0) * I

    def bad_simulate(U, n, x0, h, zy, sources, A0, A2, c0, n_pi, half):
        S, I = FO.rhs_terms(n, x0, h, zy, sources, n_pi, half)
        return (np.asarray(U, np.float64) - 0.5 * A2 * S + A0 / (c0 * c0) * I) / (2.0 * np.pi)
    _plant(mp, FO, "assemble_rhs", bad_assemble)
    _plant(mp, FO, "simulate_dV2dz", bad_simulate)


def _gradient_sign(mp):
    orig = LO.mlp_loss_grad

    def bad(*a, **k):
        loss, g = orig(*a, **k)
        return loss, -g
    _plant(mp, LO, "mlp_loss_grad", bad)


def _adam_without_bias_correction(mp):
    def bad(p, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        return p - lr * m / (np.sqrt(v) + eps), m, v
    _plant(mp, LO, "adam_step", bad)


def _bf16_truncates(mp):
    def bad(x):
        f = np.ascontiguousarray(np.asarray(x, np.float32))
        u = f.view(np.uint32)
        return ((u >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)
    _plant(mp, LO, "bf16_round", bad)


def _features_natural_log(mp):
    orig = LO.band_features
    _plant(mp, LO, "band_features", lambda U, n_bands, delta: orig(U, n_bands, delta) * np.log(10.0))


def _band_errors_normalised(mp):
    orig = LO.band_error_curves
    _plant(mp, LO, "band_error_curves",
           lambda A, U, zeta_true, alphas, n_bands: orig(A, U, zeta_true, alphas, n_bands) / U.shape[-1] ** 2)


def _second_layer_linear(mp):
    def bad(p, X, nin, nh, nout):
        W1, b1, W2, b2, W3, b3 = LO.mlp_unpack(p, nin, nh, nout)
        h1 = np.tanh(np.asarray(X, np.float64) @ W1.T + b1)
        h2 = h1 @ W2.T + b2                                   # tanh dropped
        return h2 @ W3.T + b3, (h1, h2)
    _plant(mp, LO, "mlp_forward", bad)


def _candidate_below_instead_of_nearest(mp):
    def bad(p, feat, alphas, nh):
        feat = np.asarray(feat, np.float64)
        nb = feat.size
        y, _ = LO.mlp_forward(p, (feat * LO.FEAT_SCALE)[None, :], nb, nh, nb)
        la = y[0] * LO.LOG_SCALE - LO.LOG_SHIFT
        lg = np.log10(np.asarray(alphas, np.float64))
        idx = np.clip(np.searchsorted(lg, la) - 1, 0, lg.size - 1)   # the candidate below, not the nearest
        return y[0], la, idx
    _plant(mp, LO, "learned_alpha_index", bad)


def _unet_skip_gradient_dropped(mp):
    """the encoder output's gradient takes the pooled path only: the decoder convolution's input gradient
    loses its skip-connection half (the input has more channels than the output only there)"""
    orig = UO.conv3_backward

    def bad(x, w, dy):
        dx, dw, db = orig(x, w, dy)
        if x.shape[1] > w.shape[0]:
            dx = dx.copy()
            dx[:, x.shape[1] - w.shape[0]:] = 0.0
        return dx, dw, db
    mp.setattr(UO, "conv3_backward", bad)


def _unet_pool_backward_unscaled(mp):
    mp.setattr(UO, "pool2_backward", lambda dy: UO.up2(dy))


def _unet_leaky_backward_identity(mp):
    mp.setattr(UO, "leaky_backward", lambda y, dy: np.asarray(dy, np.float64))


def _unet_conv_dx_unflipped(mp):
    """the input gradient taken as the forward correlation of dy with the weights (not their adjoint)"""
    orig = UO.conv3_backward

    def bad(x, w, dy):
        _, dw, db = orig(x, w, dy)
        wt = np.transpose(w, (1, 0, 2, 3, 4))
        return UO.conv3(dy, wt, np.zeros(wt.shape[0])), dw, db
    mp.setattr(UO, "conv3_backward", bad)


def _unet_loss_gradient_halved(mp):
    orig = UO.loss_and_grad
    mp.setattr(UO, "loss_and_grad", lambda y, t: (orig(y, t)[0], 0.5 * orig(y, t)[1]))


MUTATIONS = {
    "kernel sign": (_kernel_sign, [P.test_kernel_is_z_derivative_of_inverse_distance]),
    "kernel power": (_kernel_power, [P.test_kernel_is_z_derivative_of_inverse_distance]),
    "DFT exponent sign": (_dft_exponent_sign, [lambda: P.test_dft2_equals_definition_double_sum((4, 4))]),
    "inverse DFT without 1/L^2": (_idft_unnormalised,
                                  [lambda: P.test_forward_dft_equals_direct_quadrature_periodic(6, "dz_inv_r")]),
    "quadrature weights dropped": (_quadrature_weights_dropped,
                                   [lambda: P.test_forward_dft_equals_direct_quadrature_periodic(6, "dz_inv_r")]),
    "cell area h^2 dropped": (_cell_area_dropped, [lambda: P.test_kernel_hat_dc_bin_equals_rectangle_closed_form(-0.5)]),
    "alpha scale not squared": (_alpha_scale_not_squared, [P.test_alpha_scale_is_the_dc_norm_in_closed_form]),
    "alpha scale summed": (_alpha_scale_summed, [P.test_alpha_scale_is_the_dc_norm_in_closed_form]),
    "Tikhonov weight not rooted": (_tikhonov_unrooted, [P.test_tikhonov_optimality_pinv_limit_and_dual_identity]),
    "Tikhonov drops Im": (_tikhonov_drops_imaginary_part, [P.test_tikhonov_optimality_pinv_limit_and_dual_identity]),
    "residual without 1/L^2": (_residual_unnormalised, [P.test_frequency_residual_equals_spatial_residual]),
    "smallest admissible alpha": (_discrepancy_smallest_admissible, [P.test_discrepancy_rule]),
    "bound not squared": (_discrepancy_bound_not_squared, [P.test_discrepancy_rule]),
    "V0 sign": (_v0_sign, [P.test_V0_solves_poisson_equation_for_point_sources]),
    "V0 without 4 pi": (_v0_without_four_pi, [P.test_V0_solves_poisson_equation_for_point_sources]),
    "combination without squares": (_combination_without_squares, [P.test_combination_recovers_shared_xi_exactly]),
    "zeta = xi / V0": (_zeta_divides_by_v0, [P.test_combination_recovers_shared_xi_exactly]),
    "padding centred": (_padding_centred, [P.test_pad2_gives_the_aperiodic_sum_over_R]),
    "padded lags wrapped at n/2": (_padded_lags_wrapped_at_half_the_grid, [P.test_pad2_gives_the_aperiodic_sum_over_R]),
    "TSVD cut on sigma": (_tsvd_cut_on_sigma, [P.test_tsvd_matches_library_pseudo_inverse_and_limits]),
    "bands of unfolded k": (_bands_unfolded, [P.test_radial_bands_are_symmetric_monotone_and_hand_evaluated]),
    "RHS integral sign": (_rhs_integral_sign, [P.test_rhs_integral_term_equals_brute_force_quadrature_and_round_trip]),
    "RHS A2 coefficient in both": (_rhs_source_coefficient_in_both,
                                   [P.test_rhs_integral_term_equals_brute_force_quadrature_and_round_trip,
                                    P.test_rhs_coefficients_follow_from_the_wave_equation_moments]),
    "RHS Pi coefficient in both": (_rhs_integral_coefficient_in_both,
                                   [P.test_rhs_integral_term_equals_brute_force_quadrature_and_round_trip,
                                    P.test_rhs_coefficients_follow_from_the_wave_equation_moments]),
    "MLP gradient sign": (_gradient_sign, [LP.test_mlp_gradient_matches_central_differences]),
    "Adam without bias correction": (_adam_without_bias_correction, [LP.test_adam_first_step_is_signed_learning_rate]),
    "BF16 truncation": (_bf16_truncates, [LP.test_bf16_rounding_ties_to_even]),
    "features in natural log": (_features_natural_log, [LP.test_features_single_cosine_closed_form]),
    "band errors divided by L^2": (_band_errors_normalised, [LP.test_band_errors_equal_spatial_errors_of_the_full_inversion]),
    "second layer without tanh": (_second_layer_linear, [LP.test_mlp_forward_by_hand_and_zero_output_layer]),
    "candidate below, not nearest": (_candidate_below_instead_of_nearest, [LP.test_nearest_candidate_rule]),
    "U-Net skip gradient dropped": (_unet_skip_gradient_dropped, [UP.test_network_gradient_matches_central_differences]),
    "U-Net pool backward without 1/8": (_unet_pool_backward_unscaled,
                                        [UP.test_pool_and_upsample_adjoints_and_round_trip]),
    "U-Net leaky backward identity": (_unet_leaky_backward_identity, [UP.test_leaky_and_its_derivative]),
    "U-Net conv input gradient unflipped": (_unet_conv_dx_unflipped,
                                            [UP.test_conv3_backward_is_the_adjoint_and_the_weight_derivative]),
    "U-Net loss gradient halved": (_unet_loss_gradient_halved, [UP.test_network_gradient_matches_central_differences]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    plant, pins = MUTATIONS[name]
    assert not _some_pin_fails(pins), "the pins must pass on the unmodified oracle"
    plant(monkeypatch)
    assert _some_pin_fails(pins), f"no pin caught the planted mistake: {name}"
