"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds NONE of the method's arithmetic (no kernel, no transform, no
solve, no V0): only the description of a workload (grid coordinates, depths,
quadrature weights, source positions) and random draws (inclusion phantoms,
standard-normal noise).  Both the CUDA path and the oracle consume what it
returns, so the two sides see identical inputs.

Workload shapes follow the paper's experiment (Sec. 6): a horizontal slab R of
scatterers, a disjoint observation plane, delta-shaped point sources outside
both, and a smooth contrast made of a few localised inclusions whose amplitude
is modulated in depth by the bump (1 - 4 (z~ - 1/2)^2)^2 of the model solution.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    """One inversion instance: grid, depths, sources and ground truth."""

    n: int                       # horizontal grid n x n
    x0: float                    # x_a = x0 + (a + 1/2) h (same in y)
    h: float
    zr: np.ndarray               # M' depths of R (voxel centres)
    nu: np.ndarray               # M' quadrature weights (midpoint: dz')
    zy: np.ndarray               # M observation depths
    sources: np.ndarray          # [Q, L, 3] point-source positions per source parameter q
    xi_true: np.ndarray          # [M', n, n] xi = 1/c0^2 - 1/c^2 (float64)
    noise: np.ndarray            # [Q, M, n, n] standard-normal draws
    noise_level: float           # relative noise (e.g. 0.01 for 1 %)
    alphas: np.ndarray           # candidate alphas, increasing
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def Q(self):
        return int(self.sources.shape[0])

    @property
    def M(self):
        return int(self.zy.size)

    @property
    def Mp(self):
        return int(self.zr.size)


def slab_depths(mp: int, top: float = 0.5, bottom: float = 1.0):
    """Voxel-centred depths of R = [top, bottom] and midpoint weights."""
    dz = (bottom - top) / mp
    zr = top + (np.arange(mp) + 0.5) * dz
    return zr, np.full(mp, dz)


def cross_sources(q: int, offset: float = 0.8, z_step: float = 0.1, L: int = 5):
    """Source parameter q = 0..Q-1: the paper's 5-point cross (0,0), (+-r,0), (0,+-r)
    (Sec. 6, r = 8 on half-width 10, here scaled to half-width 1) on the plane
    z = -z_step (q + 1), above the observation plane z = 0."""
    base = np.array([(0.0, 0.0), (-offset, 0.0), (offset, 0.0), (0.0, -offset), (0.0, offset)])[:L]
    out = np.zeros((q, base.shape[0], 3))
    for k in range(q):
        out[k, :, :2] = base
        out[k, :, 2] = -z_step * (k + 1)
    return out


def inclusion_phantom(rng, n, x0, h, zr, n_incl, *, kinds=("gauss",), amp=(-0.5, 0.5),
                      width=(0.1, 0.2), semi=(0.1, 0.3), depth_bump=True):
    """Sum of localised inclusions in R; returns xi = 1/c0^2 - 1/c^2 = -(contrast), [M', n, n].

    Each inclusion draws a centre uniform in R, an amplitude (of the contrast
    1/c^2 - 1/c0^2) uniform in ``amp`` and, by kind, a Gaussian width in
    ``width`` or ellipsoid semi-axes in ``semi`` with a random rotation about z;
    an ellipsoid's profile is (1 - q^2)_+^2.
    """
    c = x0 + (np.arange(n) + 0.5) * h
    X = c[None, None, :]
    Y = c[None, :, None]
    Z = np.asarray(zr)[:, None, None]
    lo, hi = x0, x0 + n * h
    dz = float(zr[1] - zr[0]) if zr.size > 1 else 0.5
    ztop, zbot = zr[0] - 0.5 * dz, zr[-1] + 0.5 * dz
    contrast = np.zeros((zr.size, n, n))
    for _ in range(n_incl):
        kind = kinds[rng.integers(len(kinds))]
        cx, cy = rng.uniform(lo, hi, size=2)
        cz = rng.uniform(zr[0], zr[-1])
        a = rng.uniform(*amp)
        if kind == "gauss":
            s = rng.uniform(*width)
            contrast += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2 * s * s))
        else:
            ax, ay, az = rng.uniform(*semi, size=3)
            th = rng.uniform(0, np.pi)
            u = (X - cx) * np.cos(th) + (Y - cy) * np.sin(th)
            v = -(X - cx) * np.sin(th) + (Y - cy) * np.cos(th)
            qq = (u / ax) ** 2 + (v / ay) ** 2 + ((Z - cz) / az) ** 2
            contrast += a * np.clip(1 - qq, 0, None) ** 2
    if depth_bump and zr.size > 1:
        zt = (Z - ztop) / max(zbot - ztop, 1e-12)
        contrast *= (1 - 4 * (zt - 0.5) ** 2) ** 2
    return -contrast


def make_workload(n: int, mp: int, *, q: int = 1, m_obs: int = 1, n_incl: int = 2, kinds=("gauss",),
                  noise_level: float = 0.01, n_alpha: int = 16, seed: int = 0,
                  half_width: float = 1.0, depth=(0.5, 1.0), z_obs=0.0, alpha_range=(1e-8, 1e-1)):
    """A seeded instance shaped like the paper's flat-layer scheme (Sec. 3, Sec. 6)."""
    rng = np.random.default_rng(seed)
    h = 2.0 * half_width / n
    x0 = -half_width
    zr, nu = slab_depths(mp, *depth)
    zy = (np.asarray([z_obs], np.float64) if m_obs == 1
          else np.linspace(z_obs - 0.2, z_obs, m_obs))
    sources = cross_sources(q)
    xi = inclusion_phantom(rng, n, x0, h, zr, n_incl, kinds=kinds)
    noise = rng.standard_normal((q, zy.size, n, n))
    alphas = np.logspace(np.log10(alpha_range[0]), np.log10(alpha_range[1]), n_alpha)
    return Workload(n=n, x0=x0, h=h, zr=zr, nu=nu, zy=zy, sources=sources, xi_true=xi,
                    noise=noise, noise_level=noise_level, alphas=alphas, seed=seed)


def paper_model_xi(n: int, x0: float, h: float, zr) -> np.ndarray:
    """The model solution of Sec. 6 on the voxel-centred grid, [M', n, n], with the readings of its
    garbled terms: a2 and a3 take the depth z (printed with the source height z0, which would make a2
    vanish), a3's exponent takes +(y + 4)^2 (printed with a minus, indefinite and growing in y), and
    a3's envelope is max{1 - (z - 1.7)^2, 0}^2."""
    c = x0 + (np.arange(n) + 0.5) * h
    X = c[None, None, :]
    Y = c[None, :, None]
    Z = np.asarray(zr, np.float64)[:, None, None]
    a1 = (1.0 - 4.0 * (Z - 1.5) ** 2) ** 2
    a2 = 0.4 * np.maximum(1.0 - (Z - 1.3) ** 2, 0.0)
    a3 = 0.2 * np.maximum(1.0 - (Z - 1.7) ** 2, 0.0) ** 2
    return (a1 * np.exp(-X ** 2 - 2.0 * Y ** 2)
            + a2 * np.exp(-3.0 * (X + 4.0) ** 2 - (Y - 5.0) ** 2 + (X + 4.0) * (Y - 5.0))
            + a3 * np.exp(-0.9 * ((X - 4.0) ** 2 + (Y + 4.0) ** 2 + (X - 4.0) * (Y + 4.0))))


def paper_workload(n: int = 512, m: int = 51, mp: int = 51, *, noise_level: float = 1e-4, n_alpha: int = 32,
                   seed: int = 7000):
    """The experiment of Sec. 6 in the paper's own coordinates: R = [-10, 10]^2 x [1, 2] with mp depths,
    Y = [-10, 10]^2 x [6, 7] with m observation planes (both voxel-centred), the ten point sources of
    one experiment (the cross (0, 0), (+-8, 0), (0, +-8) on the planes z0 = 3 and z0 = 5: Q = 1, L = 10),
    A0 = 1 (g = exp(-t)), and the model solution (paper_model_xi).  Noise: i.i.d. Gaussian of relative
    level noise_level (the paper's data errors, about 1e-8, lie below the FP32 data's own precision)."""
    rng = np.random.default_rng(seed)
    h = 20.0 / n
    x0 = -10.0
    zr, nu = slab_depths(mp, 1.0, 2.0)
    zy, _ = slab_depths(m, 6.0, 7.0)
    cross = np.array([(0.0, 0.0), (-8.0, 0.0), (8.0, 0.0), (0.0, -8.0), (0.0, 8.0)])
    sources = np.zeros((1, 10, 3))
    for k, z0 in enumerate((3.0, 5.0)):
        sources[0, 5 * k:5 * k + 5, :2] = cross
        sources[0, 5 * k:5 * k + 5, 2] = z0
    xi = paper_model_xi(n, x0, h, zr)
    noise = rng.standard_normal((1, m, n, n))
    alphas = np.logspace(-8.0, -1.0, n_alpha)
    return Workload(n=n, x0=x0, h=h, zr=zr, nu=nu, zy=zy, sources=sources, xi_true=xi,
                    noise=noise, noise_level=noise_level, alphas=alphas, seed=seed)


# The five workload shapes (sizes, counts and ranges) of the benchmark suite.
def config_workload(k: int, seed: int | None = None, instance: int = 0):
    """k = 1: 32^2 x 16, single source, 2 Gaussians, 1 % noise, 16 alphas.
    k = 2: 128^2 x 32, single source, 5 Gaussian/ellipsoid inclusions, 2 % noise, 32 alphas.
    k = 3: 256^2 x 64, 8 source parameters, 10 inclusions, 1 % noise, 64 alphas."""
    s = 1000 * k + instance if seed is None else seed
    if k == 1:
        return make_workload(32, 16, q=1, n_incl=2, noise_level=0.01, n_alpha=16, seed=s)
    if k == 2:
        return make_workload(128, 32, q=1, n_incl=5, kinds=("gauss", "ellipsoid"), noise_level=0.02,
                             n_alpha=32, seed=s)
    if k == 3:
        return make_workload(256, 64, q=8, n_incl=10, kinds=("gauss", "ellipsoid"), noise_level=0.01,
                             n_alpha=64, seed=s)
    raise ValueError(k)


def batch_workloads(count: int = 64, seed: int = 4000):
    """Uneven batch: n from {64, 96, 128, 192, 256}, M' from {16, 32, 48, 64}, 1-8 sources,
    1-10 Gaussian inclusions, 0.5-5 % noise (one seeded draw per instance)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([64, 96, 128, 192, 256]))
        mp = int(rng.choice([16, 32, 48, 64]))
        q = int(rng.integers(1, 9))
        ni = int(rng.integers(1, 11))
        nl = float(rng.uniform(0.005, 0.05))
        out.append(make_workload(n, mp, q=q, n_incl=ni, noise_level=nl, n_alpha=32, seed=seed + 1 + i))
    return out
