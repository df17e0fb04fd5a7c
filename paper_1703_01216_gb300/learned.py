"""Training and use of the learned per-band alpha rule (FR3D_ALPHA_LEARNED).

Every step that computes runs in libfr3d's kernels: the forward operator that makes the training
data (fr3d_zeta_from_xi, fr3d_fwd_apply), the band features and the per-band error-optimal targets
(fr3d_band_features, fr3d_band_alpha_targets), the network's forward and backward passes and its
Adam update (fr3d_mlp_*), and the inversion that uses it (fr3d_invert).  Torch supplies device
buffers, the seeded noise draws of the synthetic data and the minibatch gathers.

Training pairs follow the paper's model experiment (Sec. 6): a contrast of localised inclusions in
the slab R, data on the observation plane from the point sources, relative Gaussian noise; the
network learns, per radial band, the candidate alpha that minimises the error of that band's
Tikhonov solution, from the band's data-to-noise power.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fr3d
from .synth import PhantomSampler


@dataclass
class PairSet:
    x: object          # [count, nb] float32 (device): network inputs f_b / 4
    y: object          # [count, nb] float32 (device): targets (log10 alpha_b + 4.5) / 3.5
    idx: object        # [count, nb] int32 (device): error-optimal candidate per band


def make_pairs(H: fr3d.Handle, n: int, x0: float, h: float, zr, points, alphas, n_bands: int, count: int,
               seed: int, device, n_incl=(1, 12), noise=(0.005, 0.05), kinds=("gauss", "ellipsoid")) -> PairSet:
    """``count`` seeded (data, coefficient) pairs made by the forward operator, reduced to features and
    per-band targets.  Sample i uses NumPy seed ``seed + i`` for the phantom and the noise level and a
    torch generator seeded the same way for the noise."""
    import torch
    pts = np.asarray(points, np.float64)
    Q = pts.shape[0]
    Mp = len(zr)
    samp = PhantomSampler(n, x0, h, zr, device, kinds=kinds)
    zeta = torch.empty((Q, Mp, n, n), device=device)
    Uc = torch.empty((Q, 1, n, n), device=device)
    X = torch.empty((count, n_bands), device=device)
    Y = torch.empty((count, n_bands), device=device)
    I = torch.empty((count, n_bands), dtype=torch.int32, device=device)
    gen = torch.Generator(device=device)
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        xi = samp.draw(rng, int(rng.integers(n_incl[0], n_incl[1] + 1)))
        level = float(rng.uniform(*noise))
        fr3d.zeta_from_xi(H, xi, pts, zeta)
        fr3d.fwd_apply(H, zeta, Q, Uc)
        gen.manual_seed(seed + i)
        nz = torch.randn(Uc.shape, generator=gen, device=device)
        nz *= level * Uc.norm() / nz.norm()
        delta = float(nz.norm())
        U = Uc + nz
        fr3d.band_features(H, U, Q, n_bands, delta, X[i])
        fr3d.band_alpha_targets(H, U, zeta, Q, alphas, n_bands, I[i], Y[i])
    return PairSet(X, Y, I)


def train(net: fr3d.Mlp, pairs: PairSet, steps: int, batch: int = 256, lr: float = 3e-3, seed: int = 0,
          lr_final: float | None = None):
    """Minibatch Adam on the mean squared error of y; returns the loss of every 100th step (host)."""
    import torch
    N = pairs.x.shape[0]
    gen = torch.Generator(device=pairs.x.device)
    gen.manual_seed(seed)
    loss = torch.zeros(1, device=pairs.x.device)
    hist = []
    for s in range(steps):
        sel = torch.randint(N, (min(batch, N),), generator=gen, device=pairs.x.device)
        xb = pairs.x.index_select(0, sel).contiguous()
        yb = pairs.y.index_select(0, sel).contiguous()
        a = lr if lr_final is None else lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        net.train_step(xb, yb, a, loss)
        if s % 100 == 0 or s == steps - 1:
            hist.append(float(loss))
    return hist


def loss_on(net: fr3d.Mlp, pairs: PairSet) -> float:
    """Mean squared error of the network on a pair set."""
    import torch
    l = torch.zeros(1, device=pairs.x.device)
    net.gradient(pairs.x, pairs.y, None, l)
    return float(l)
