"""Training and use of the learned post-corrector (fr3d_unet): a 3D U-Net that maps the plain
discrepancy-principle reconstruction (fr3d_invert) to a corrected xi.

Every step that computes runs in libfr3d's kernels: the forward operator that makes the training pairs
(fr3d_zeta_from_xi, fr3d_fwd_apply), the plain inversion that makes the network's input (fr3d_invert,
alpha by the discrepancy principle), and the network's forward pass, gradient and Adam update on the
tensor cores (fr3d_unet_*).  Torch supplies device buffers, the phantom volumes of the synthetic data
(synth.PhantomSampler) and the seeded noise draws.

Pairs follow the learned configuration of the benchmark suite: 1-12 Gaussian or ellipsoidal inclusions
with amplitudes in [-0.5, 0.5] (modulated in depth like the paper's model solution, Sec. 6), one
observation plane, one point-source parameter, 0.5-5 % relative Gaussian noise, generated on the fly
(not stored) from seeds: sample i of a stream uses NumPy seed ``seed + i`` for the phantom and the noise
level and a torch generator seeded the same way for the noise.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fr3d
from .synth import PhantomSampler


@dataclass
class PairStream:
    """One geometry's pair generator: a handle, the sources, the alpha grid and reusable buffers."""

    H: object
    n: int
    zr: np.ndarray
    points: np.ndarray
    alphas: np.ndarray
    sampler: object
    device: object
    n_incl: tuple = (1, 12)
    noise: tuple = (0.005, 0.05)

    @classmethod
    def create(cls, w, device, n_incl=(1, 12), noise=(0.005, 0.05)):
        """From a workload description (inputs.Workload: grid, depths, sources, alpha grid)."""
        H = fr3d.kernel_transform(w.n, w.x0, w.h, w.zr, w.zy, w.nu)
        samp = PhantomSampler(w.n, w.x0, w.h, w.zr, device, kinds=("gauss", "ellipsoid"))
        return cls(H, w.n, np.asarray(w.zr), np.asarray(w.sources), np.asarray(w.alphas), samp, device, n_incl, noise)

    def batch(self, seed: int, count: int, x_out, t_out, info=None):
        """Fill x_out [count, M', n, n] with plain reconstructions and t_out with the true xi of samples
        seed .. seed + count - 1."""
        import torch
        Q = self.points.shape[0]
        Mp, n = self.zr.size, self.n
        zeta = torch.empty((Q, Mp, n, n), device=self.device)
        U = torch.empty((Q, 1, n, n), device=self.device)
        gen = torch.Generator(device=self.device)
        for i in range(count):
            s = seed + i
            rng = np.random.default_rng(s)
            xi = self.sampler.draw(rng, int(rng.integers(self.n_incl[0], self.n_incl[1] + 1)))
            level = float(rng.uniform(*self.noise))
            t_out[i].copy_(xi)
            fr3d.zeta_from_xi(self.H, xi, self.points, zeta)
            fr3d.fwd_apply(self.H, zeta, Q, U)
            gen.manual_seed(s)
            nz = torch.randn(U.shape, generator=gen, device=self.device)
            nz *= level * U.norm() / nz.norm()
            delta = float(nz.norm())
            U += nz
            fr3d.invert(self.H, U, Q, x_out[i],
                        fr3d.Opts(alphas=self.alphas, delta=delta, tau=1.1, points=self.points, info=info))


def rel_l2_per_sample(a, b):
    """||a_i - b_i|| / ||b_i|| for every sample i (host numpy)."""
    d = (a.double() - b.double()).flatten(1).norm(dim=1)
    return (d / b.double().flatten(1).norm(dim=1)).cpu().numpy()


def train(net: fr3d.Unet, stream: PairStream, pairs: int, batch: int, seed: int, lr: float = 1e-3,
          lr_final: float = 1e-4, log_every: int = 50):
    """Adam on fresh pairs: ``pairs`` samples in batches of ``batch`` (seeds seed, seed + 1, ...);
    returns the loss history (every ``log_every`` steps, host floats) and the wall time spent in the
    pair generation and in the network's steps."""
    import time

    import torch
    d, hgt, wid = net.shape
    x = torch.empty((batch, d, hgt, wid), device=stream.device)
    t = torch.empty_like(x)
    loss = torch.zeros(1, device=stream.device)
    steps = max(1, pairs // batch)
    hist, t_gen, t_net = [], 0.0, 0.0
    for k in range(steps):
        a = time.perf_counter()
        stream.batch(seed + k * batch, batch, x, t)
        torch.cuda.synchronize()
        b = time.perf_counter()
        rate = lr * (lr_final / lr) ** (k / max(steps - 1, 1))
        net.train_step(x, t, rate, loss)
        if k % log_every == 0 or k == steps - 1:
            hist.append(float(loss))
        torch.cuda.synchronize()
        c = time.perf_counter()
        t_gen += b - a
        t_net += c - b
    return hist, t_gen, t_net


def evaluate(net: fr3d.Unet, stream: PairStream, count: int, seed: int, batch: int):
    """Plain and post-corrected relative L2 errors against the true xi on ``count`` held-out samples."""
    import torch
    d, hgt, wid = net.shape
    x = torch.empty((batch, d, hgt, wid), device=stream.device)
    t = torch.empty_like(x)
    y = torch.empty_like(x)
    plain, learned = [], []
    for k in range(0, count, batch):
        m = min(batch, count - k)
        stream.batch(seed + k, m, x, t)
        net.forward(x[:m], y[:m])
        plain.append(rel_l2_per_sample(x[:m], t[:m]))
        learned.append(rel_l2_per_sample(y[:m], t[:m]))
    return np.concatenate(plain), np.concatenate(learned)
