"""Seeded synthetic contrasts evaluated on the GPU, for generating training pairs of the learned
alpha rule at a rate the host cannot reach at 256^2 x 64.

This module holds none of the method's arithmetic (no kernel, transform, solve or V0).  It draws
the same family of phantoms as ``inputs.inclusion_phantom`` -- localised Gaussian and ellipsoidal
inclusions, centres uniform in R, contrast amplitudes uniform in [-0.5, 0.5], Gaussian widths in
[0.1, 0.2], ellipsoid semi-axes in [0.1, 0.3] with a random rotation about z and profile
(1 - q^2)_+^2, all modulated in depth by (1 - 4 (z~ - 1/2)^2)^2 -- with the shape parameters drawn
on the host by a seeded NumPy generator and the volume evaluated by torch on the device.
"""

from __future__ import annotations

import numpy as np


class PhantomSampler:
    """xi = 1/c0^2 - 1/c^2 volumes [M', n, n] (float32, on ``device``) for one grid."""

    def __init__(self, n: int, x0: float, h: float, zr, device, kinds=("gauss", "ellipsoid"),
                 amp=(-0.5, 0.5), width=(0.1, 0.2), semi=(0.1, 0.3)):
        import torch
        self.torch = torch
        zr = np.asarray(zr, np.float64)
        self.n, self.x0, self.h, self.zr = n, x0, h, zr
        self.kinds, self.amp, self.width, self.semi = kinds, amp, width, semi
        self.dev = device
        c = torch.tensor(x0 + (np.arange(n) + 0.5) * h, dtype=torch.float32, device=device)
        self.X = c[None, None, :]
        self.Y = c[None, :, None]
        self.Z = torch.tensor(zr, dtype=torch.float32, device=device)[:, None, None]
        dz = float(zr[1] - zr[0]) if zr.size > 1 else 0.5
        ztop, zbot = zr[0] - 0.5 * dz, zr[-1] + 0.5 * dz
        zt = (zr - ztop) / max(zbot - ztop, 1e-12)
        bump = (1 - 4 * (zt - 0.5) ** 2) ** 2 if zr.size > 1 else np.ones_like(zr)
        self.bump = torch.tensor(bump, dtype=torch.float32, device=device)[:, None, None]

    def draw(self, rng: np.random.Generator, n_incl: int):
        torch = self.torch
        lo, hi = self.x0, self.x0 + self.n * self.h
        con = torch.zeros((self.zr.size, self.n, self.n), dtype=torch.float32, device=self.dev)
        for _ in range(n_incl):
            kind = self.kinds[rng.integers(len(self.kinds))]
            cx, cy = rng.uniform(lo, hi, size=2)
            cz = rng.uniform(self.zr[0], self.zr[-1])
            a = rng.uniform(*self.amp)
            if kind == "gauss":
                s = rng.uniform(*self.width)
                gx = torch.exp(-(self.X - cx) ** 2 / (2 * s * s))
                gy = torch.exp(-(self.Y - cy) ** 2 / (2 * s * s))
                gz = torch.exp(-(self.Z - cz) ** 2 / (2 * s * s))
                con += (a * gz) * gy * gx
            else:
                ax, ay, az = rng.uniform(*self.semi, size=3)
                th = rng.uniform(0, np.pi)
                u = (self.X - cx) * np.cos(th) + (self.Y - cy) * np.sin(th)
                v = -(self.X - cx) * np.sin(th) + (self.Y - cy) * np.cos(th)
                qq = (u / ax) ** 2 + (v / ay) ** 2 + ((self.Z - cz) / az) ** 2
                con += a * torch.clamp(1 - qq, min=0) ** 2
        return -(con * self.bump)
