"""The learned post-corrector (fr3d_unet) against its FP64 oracle (oracle/unet_oracle.py): the forward pass,
the loss, every layer's gradient and the Adam step through the C ABI, and a small training run showing
what the trained network gains over the plain discrepancy-principle inversion.

Parity: the oracle rounds to BF16 (round to nearest even) every tensor the kernels store -- weights, the
input, each activation and each activation gradient -- so the two sides differ only by FP32 against FP64
accumulation and the BF16 roundings that this flips (each a change of 2^-8 in one stored element):
forward 1e-3 and loss 1e-4 (relative); each layer's weight and bias gradient 3e-2 (relative L2), because a
gradient is a sum over thousands of voxels whose terms largely cancel (its size is about sqrt(N) of its
terms'), which magnifies the few flipped terms (measured on GB300: forward 5.1e-4, loss 2.7e-5, layer
gradients 1.8e-3 to 1.4e-2, the largest at the first layer, the longest chain); the Adam step is FP32 on
both sides given the same gradient (1e-6).
"""

import numpy as np
import pytest

from oracle import learned_oracle as LO
from oracle import unet_oracle as UO
from paper_1703_01216_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    from paper_1703_01216_gb300 import build, fr3d
    assert torch.cuda.is_available()
    build.build()
    fr3d.load()
    return fr3d


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _params(seed=11):
    rng = np.random.default_rng(seed)
    p = UO.init_params(seed=seed)
    p[-1] = (rng.standard_normal((1, 16)) * 0.3, rng.standard_normal(1) * 0.05)
    p = [(w, b + 0.02 * rng.standard_normal(b.shape)) for w, b in p]
    return p


def test_unet_forward_loss_and_gradient_match_the_oracle(F):
    D, Hh, W, B = 8, 16, 16, 2
    rng = np.random.default_rng(12)
    x = rng.standard_normal((B, 1, D, Hh, W)) * 0.5
    t = x + 0.2 * rng.standard_normal(x.shape)
    p = _params()
    net = F.Unet(D, Hh, W, B, in_scale=1.0, seed=1)
    assert net.n_params == UO.param_count() == 1902081
    net.set_params(UO.pack(p).astype(np.float32))
    p32 = UO.unpack(UO.pack(p).astype(np.float32).astype(np.float64))       # what the GPU holds
    r = LO.bf16_round
    y_ref, cache = UO.forward(p32, x, rnd=r)
    loss_ref, dy = UO.loss_and_grad(y_ref, t)
    g_ref = UO.backward(p32, cache, dy, rnd=r)
    xd = torch.tensor(x[:, 0], dtype=torch.float32, device="cuda")
    td = torch.tensor(t[:, 0], dtype=torch.float32, device="cuda")
    y = torch.empty_like(xd)
    net.forward(xd, y)
    grad = torch.empty(net.n_params, device="cuda")
    loss = torch.zeros(1, device="cuda")
    net.gradient(xd, td, grad, loss)
    torch.cuda.synchronize()
    e_fwd = rel(y.cpu().numpy(), y_ref[:, 0])
    e_loss = abs(float(loss) - loss_ref) / loss_ref
    gl = UO.unpack(grad.double().cpu().numpy())
    e_layers = [(rel(gw, rw), rel(gb, rb)) for (gw, gb), (rw, rb) in zip(gl, g_ref)]
    print(f"unet parity: forward {e_fwd:.2e}, loss {e_loss:.2e}, layers (w, b): "
          + ", ".join(f"({a:.1e}, {b:.1e})" for a, b in e_layers))
    assert e_fwd <= 1e-3, e_fwd
    assert e_loss <= 1e-4, e_loss
    for k, (ew, eb) in enumerate(e_layers):
        assert ew <= 3e-2 and eb <= 3e-2, (k, ew, eb)
    assert net.error_flags() == 0


def test_unet_adam_step_matches_the_oracle(F):
    D, Hh, W, B = 8, 16, 16, 1
    rng = np.random.default_rng(13)
    x = torch.tensor(rng.standard_normal((B, D, Hh, W)) * 0.5, dtype=torch.float32, device="cuda")
    t = x + 0.2 * torch.tensor(rng.standard_normal((B, D, Hh, W)), dtype=torch.float32, device="cuda")
    net = F.Unet(D, Hh, W, B, seed=3)
    p0 = net.get_params().astype(np.float64)
    grad = torch.empty(net.n_params, device="cuda")
    net.gradient(x, t, grad)
    g = grad.double().cpu().numpy()
    loss = torch.zeros(1, device="cuda")
    net.train_step(x, t, 1e-3, loss)
    p1 = net.get_params().astype(np.float64)
    ref, _, _ = LO.adam_step(p0, np.zeros_like(p0), np.zeros_like(p0), g, 1, 1e-3)
    assert rel(p1, ref) <= 1e-6, rel(p1, ref)
    assert not np.array_equal(p1, p0)


def test_trained_post_corrector_beats_the_plain_inversion(F):
    """A small run of the learned configuration (64 x 64 x 16 grid instead of 128 x 128 x 32, 768 fresh
    pairs, 96 held-out seeds): the post-corrected error against the true xi is below the plain
    discrepancy-principle inversion's on average and on most samples."""
    from paper_1703_01216_gb300 import postcorrect as PC
    w = I.make_workload(64, 16, q=1, n_alpha=24, seed=5000)
    dev = torch.device("cuda")
    stream = PC.PairStream.create(w, dev)
    net = F.Unet(16, 64, 64, 8, in_scale=2.0, seed=21)
    hist, t_gen, t_net = PC.train(net, stream, pairs=768, batch=8, seed=100000, lr=1e-3, lr_final=2e-4)
    plain, learned = PC.evaluate(net, stream, 96, seed=900000, batch=8)
    gain = float(np.median(plain) - np.median(learned))
    print(f"unet gain test: loss {hist}; pairs {t_gen:.1f} s, network {t_net:.1f} s; rel L2 plain median "
          f"{np.median(plain):.4f} mean {np.mean(plain):.4f}, learned median {np.median(learned):.4f} mean "
          f"{np.mean(learned):.4f}; better on {np.mean(learned < plain):.2f} of the samples")
    # the median (a sample with a tiny true xi can have a large relative error either way)
    assert gain >= 0.05, gain
    assert np.mean(learned < plain) >= 0.8
    assert net.error_flags() == 0
