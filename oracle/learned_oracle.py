"""Plain FP64 CPU oracle of the learned per-band choice of alpha.

TEST INFRASTRUCTURE ONLY, like fr3d_oracle: imported by ``tests/`` (and through
the package ``oracle``) and by nothing on the product path; it shares no code
with the CUDA path and only consumes plain numpy arrays.

The paper chooses one alpha for the whole spectrum by the discrepancy principle
(Sec. 4).  The learned rule replaces that choice by a small network that maps
per-band statistics of the data to one alpha per radial band of frequencies
(the bands of ``fr3d_oracle.radial_bands``); step 2 then solves every frequency
of band b with alpha_b, exactly as ``fr3d_oracle.invert(band_alpha_index=...)``.
What is defined here, each written out from its definition:

* band features  f_b = log10( sum_{k in b} sum_planes |U~_k|^2 / (count_b delta^2) ):
  the data power per frequency of band b over the power per frequency of white
  noise of total norm delta (Parseval: the unnormalised spectrum of noise with
  ||noise|| = delta has expected power delta^2 per frequency, summed over planes);
* training targets: for data made by the discrete operator from a known zeta,
  the candidate alpha that minimises, per band, the squared error of the
  Tikhonov solution's spectrum E_b(alpha) = sum_{k in b} ||zeta~_alpha,k - zeta~_true,k||^2
  (explicit solves, nothing folded);
* the network: y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with x = f / 4 and
  y_b = (log10 alpha_b + 4.5) / 3.5 (so that alpha in [1e-8, 1e-1] maps to [-1, 1]);
  parameters in one flat vector [W1 (nh x nin, row-major), b1, W2 (nh x nh), b2,
  W3 (nout x nh), b3]; the mean squared error loss, its gradient by the chain
  rule, and one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected);
* the inference rule: the candidate alpha nearest to the network's log10 alpha.

The kernels store the weights in bfloat16, so the parity tests round the
oracle's weights with ``bf16_round`` (round to nearest, ties to even) and
compute everything else in FP64.
"""

from __future__ import annotations

import numpy as np

from .fr3d_oracle import dft2, radial_bands, tikhonov_qr, alpha_scale

FEAT_SCALE = 0.25
LOG_SHIFT = 4.5
LOG_SCALE = 3.5


# --------------------------------------------------------------------------- features and targets
def band_features(U: np.ndarray, n_bands: int, delta: float) -> np.ndarray:
    """f_b for data U [Q, M, n, n] (periodic box, L = n)."""
    U = np.asarray(U, np.float64)
    L = U.shape[-1]
    P = np.sum(np.abs(dft2(U)) ** 2, axis=tuple(range(U.ndim - 2))).ravel()   # [L*L], [ky, kx]
    band = radial_bands(L, n_bands)
    S = np.bincount(band, weights=P, minlength=n_bands)
    count = np.bincount(band, minlength=n_bands).astype(np.float64)
    return np.log10(np.maximum(S, 1e-300) / (count * delta * delta))


def band_error_curves(A: np.ndarray, U: np.ndarray, zeta_true: np.ndarray, alphas, n_bands: int) -> np.ndarray:
    """E[b, k] = sum over the frequencies of band b, the depths and the source parameters of
    |zeta~_alpha_k - zeta~_true|^2 (unnormalised spectra), with zeta~_alpha_k the Tikhonov solution
    of each frequency's system (alpha_k s^2, s^2 = max ||A^(m)||_F^2).  A: [L, L, M, M'];
    U: [Q, M, L, L]; zeta_true: [Q, M', L, L]."""
    L = U.shape[-1]
    Q, M = U.shape[0], U.shape[1]
    Mp = zeta_true.shape[1]
    s2 = alpha_scale(A)
    Af = A.reshape(L * L, M, Mp)
    Uf = np.transpose(dft2(np.asarray(U, np.float64)).reshape(Q, M, L * L), (2, 1, 0))       # [B, M, Q]
    Zt = np.transpose(dft2(np.asarray(zeta_true, np.float64)).reshape(Q, Mp, L * L), (2, 1, 0))
    band = radial_bands(L, n_bands)
    E = np.zeros((n_bands, len(alphas)))
    for k, a in enumerate(alphas):
        Z = tikhonov_qr(Af, Uf, float(a) * s2)
        e = np.sum(np.abs(Z - Zt) ** 2, axis=(1, 2))
        E[:, k] = np.bincount(band, weights=e, minlength=n_bands)
    return E


def band_optimal_alpha(E: np.ndarray) -> np.ndarray:
    """Per band, the index of the candidate with the smallest error (first one on ties)."""
    return np.argmin(E, axis=1)


def log_alpha_target(alphas, idx) -> np.ndarray:
    """Network target y_b for candidate index idx_b."""
    return (np.log10(np.asarray(alphas, np.float64)[np.asarray(idx)]) + LOG_SHIFT) / LOG_SCALE


# --------------------------------------------------------------------------- the network
def mlp_offsets(nin: int, nh: int, nout: int):
    """Start of each parameter block in the flat vector, and its length."""
    o = {}
    off = 0
    for name, size in (("W1", nh * nin), ("b1", nh), ("W2", nh * nh), ("b2", nh), ("W3", nout * nh), ("b3", nout)):
        o[name] = off
        off += size
    o["np"] = off
    return o


def mlp_unpack(p: np.ndarray, nin: int, nh: int, nout: int):
    o = mlp_offsets(nin, nh, nout)
    p = np.asarray(p, np.float64)
    return (p[o["W1"]:o["b1"]].reshape(nh, nin), p[o["b1"]:o["W2"]],
            p[o["W2"]:o["b2"]].reshape(nh, nh), p[o["b2"]:o["W3"]],
            p[o["W3"]:o["b3"]].reshape(nout, nh), p[o["b3"]:o["np"]])


def mlp_forward(p: np.ndarray, X: np.ndarray, nin: int, nh: int, nout: int):
    """Y [B, nout] for inputs X [B, nin]; also returns the hidden activations (h1, h2)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(p, nin, nh, nout)
    X = np.asarray(X, np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (h1, h2)


def mlp_loss_grad(p: np.ndarray, X: np.ndarray, T: np.ndarray, nin: int, nh: int, nout: int):
    """Mean squared error over all B * nout outputs and its gradient (chain rule, layer by layer)."""
    W1, b1, W2, b2, W3, b3 = mlp_unpack(p, nin, nh, nout)
    X = np.asarray(X, np.float64)
    Y, (h1, h2) = mlp_forward(p, X, nin, nh, nout)
    B = X.shape[0]
    R = Y - np.asarray(T, np.float64)
    loss = float(np.sum(R * R) / (B * nout))
    dY = 2.0 * R / (B * nout)                       # dL/dY
    gW3 = dY.T @ h2
    gb3 = dY.sum(axis=0)
    dz2 = (dY @ W3) * (1.0 - h2 * h2)               # through tanh
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(p, m, v, g, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; ``step`` counts from 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (8 exponent bits, 7 stored mantissa bits), ties to even,
    by integer arithmetic on the FP32 bit pattern; returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def learned_alpha_index(p: np.ndarray, feat: np.ndarray, alphas, nh: int):
    """Network output y [nb], its log10 alpha and the nearest candidate index per band."""
    feat = np.asarray(feat, np.float64)
    nb = feat.size
    y, _ = mlp_forward(p, (feat * FEAT_SCALE)[None, :], nb, nh, nb)
    la = y[0] * LOG_SCALE - LOG_SHIFT
    lg = np.log10(np.asarray(alphas, np.float64))
    idx = np.argmin(np.abs(lg[None, :] - la[:, None]), axis=1)
    return y[0], la, idx
