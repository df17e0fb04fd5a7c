"""Pins of the U-Net post-corrector's FP64 oracle (oracle/unet_oracle.py) against things other than
itself: scipy's n-dimensional correlation, adjoint identities, central finite differences of the whole
network's loss, and hand-counted sizes.  CPU only."""

import numpy as np
import pytest

from oracle import unet_oracle as UO

ndimage = pytest.importorskip("scipy.ndimage")


def test_conv3_is_scipys_zero_padded_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = UO.conv3(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(ndimage.correlate(x[bi, c], w[o, c], mode="constant", cval=0.0) for c in range(3))
            assert np.max(np.abs(y[bi, o] - ref)) < 1e-12


def test_conv3_backward_is_the_adjoint_and_the_weight_derivative():
    """<conv3(x, w, 0), dy> is bilinear in (x, w): its gradients are <x, dx> and <w, dw>, and db = sum dy."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 4, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    dy = rng.standard_normal((2, 2, 4, 5, 6))
    dx, dw, db = UO.conv3_backward(x, w, dy)
    s = np.sum(UO.conv3(x, w, np.zeros(2)) * dy)
    assert abs(np.sum(x * dx) - s) < 1e-10 * abs(s)
    assert abs(np.sum(w * dw) - s) < 1e-10 * abs(s)
    assert np.allclose(db, dy.sum(axis=(0, 2, 3, 4)))


def test_pool_and_upsample_adjoints_and_round_trip():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 2, 4, 6, 8))
    y = rng.standard_normal((1, 2, 2, 3, 4))
    assert abs(np.sum(UO.pool2(x) * y) - np.sum(x * UO.pool2_backward(y))) < 1e-12
    assert abs(np.sum(UO.up2(y) * x) - np.sum(y * UO.up2_backward(x))) < 1e-12
    assert np.allclose(UO.pool2(UO.up2(y)), y)
    assert np.allclose(UO.pool2(x)[0, 1, 1, 2, 3], x[0, 1, 2:4, 4:6, 6:8].mean())


def test_leaky_and_its_derivative():
    x = np.array([-2.0, -0.5, 0.0, 0.3, 4.0])
    assert np.allclose(UO.leaky(x), [-0.02, -0.005, 0.0, 0.3, 4.0])
    assert np.allclose(UO.leaky_backward(UO.leaky(x), np.ones(5)), [0.01, 0.01, 0.01, 1.0, 1.0])


def test_parameter_count_of_the_configured_network():
    """4 levels, base width 16: hand count 1 902 081 (the learned configuration's ~2M)."""
    assert UO.param_count() == 1902081
    assert UO.pack(UO.init_params()).size == 1902081
    assert [s for s in UO.layer_shapes()][:3] == [(16, 1), (16, 16), (32, 16)]


def test_initial_network_is_the_identity():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 1, 8, 8, 8))
    p = UO.init_params((2, 3, 4), seed=5)
    assert np.array_equal(UO.predict(p, x, (2, 3, 4)), x)


def _tiny(seed=6, widths=(2, 3, 4)):
    rng = np.random.default_rng(seed)
    p = UO.init_params(widths, seed=seed)
    p[-1] = (rng.standard_normal((1, widths[0])) * 0.5, rng.standard_normal(1) * 0.1)   # a non-trivial head
    p = [(w, b + 0.05 * rng.standard_normal(b.shape)) for w, b in p]                    # non-zero biases
    x = rng.standard_normal((2, 1, 8, 8, 8))
    t = x + 0.3 * rng.standard_normal(x.shape)
    return p, x, t, widths


def _loss(flat, x, t, widths):
    y = UO.predict(UO.unpack(flat, widths), x, widths)
    return UO.loss_and_grad(y, t)[0]


def test_network_gradient_matches_central_differences():
    """The chain rule of ``backward`` (through the head, every conv3 and leaky, the concatenations, the
    skip connections, pooling and upsampling) against central differences of the loss, in FP64: along
    random directions and on single parameters of every layer."""
    p, x, t, widths = _tiny()
    y, cache = UO.forward(p, x, widths)
    loss, dy = UO.loss_and_grad(y, t)
    g = UO.pack(UO.backward(p, cache, dy, widths))
    flat = UO.pack(p)
    rng = np.random.default_rng(7)
    eps = 1e-6          # small enough that no pre-activation crosses leaky's kink
    # a random direction within every layer's parameters
    o = 0
    for w, b in p:
        v = np.zeros(flat.size)
        v[o:o + w.size + b.size] = rng.standard_normal(w.size + b.size)
        fd = (_loss(flat + eps * v, x, t, widths) - _loss(flat - eps * v, x, t, widths)) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), 1e-12), (fd, g @ v)
        o += w.size + b.size
    # one coordinate in every layer's weights and biases
    o = 0
    for w, b in p:
        for idx in (o + w.size // 2, o + w.size):          # a weight, the first bias
            e = np.zeros(flat.size)
            e[idx] = 1.0
            fd = (_loss(flat + eps * e, x, t, widths) - _loss(flat - eps * e, x, t, widths)) / (2 * eps)
            # absolute floor: the rounding of a loss of order one divided by 2 eps
            assert abs(fd - g[idx]) <= 1e-6 * abs(fd) + 1e-10, (idx, fd, g[idx])
        o += w.size + b.size


def test_loss_is_the_mean_squared_relative_error():
    rng = np.random.default_rng(8)
    t = rng.standard_normal((3, 1, 2, 2, 2))
    y = t * np.array([1.1, 0.8, 1.0])[:, None, None, None, None]
    loss, _ = UO.loss_and_grad(y, t)
    assert abs(loss - np.mean([0.01, 0.04, 0.0])) < 1e-14
