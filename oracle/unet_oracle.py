"""Plain FP64 CPU oracle of the learned post-corrector: a small 3D U-Net that maps the Tikhonov
reconstruction xi_alpha (Algorithm 1's output) to a corrected xi.

TEST INFRASTRUCTURE ONLY, like fr3d_oracle: imported by ``tests/`` and by nothing on the product path;
it shares no code with the CUDA path and only consumes plain numpy arrays.

The paper has no network.  The learned part of the benchmark suite asks for a 4-level 3D U-Net of base
width 16 that post-corrects the reconstruction; its task is the part of xi that Algorithm 1 cannot see:
with one observation plane every frequency's system has rank one, so the normal solution (Assumption U,
Sec. 4) drops M' - 1 depth directions per frequency and a prior learnt from examples has to put them
back.  Everything below is written out from the definitions:

* conv3(x, w, b): 3 x 3 x 3 cross-correlation with zero padding 1 and a bias,
      y[o, d, h, w] = b[o] + sum_{c, a, e, f} w[o, c, a, e, f] x[c, d + a - 1, h + e - 1, w + f - 1];
* leaky(x) = x for x > 0, SLOPE x otherwise;
* pool2: the mean of each 2 x 2 x 2 block; up2: nearest-neighbour upsampling by 2 per axis;
* the network (widths w_0 .. w_{L-1}, L levels): at level 0 conv3(1 -> w_0), conv3(w_0 -> w_0); at
  levels 1 .. L-2 pool2 then conv3(w_{l-1} -> w_l), conv3(w_l -> w_l); at the bottom level pool2 then three
  conv3 (w_{L-2} -> w_{L-1} -> w_{L-1} -> w_{L-1}); going up, for l = L-2 .. 0, up2 of the level below,
  concatenated (channels first) with level l's encoder output, conv3(w_{l+1} + w_l -> w_l), conv3(w_l -> w_l);
  every conv3 followed by leaky; the head is a 1 x 1 x 1 convolution w_0 -> 1 and the input is added back:
      y = x + head(...)   (the network learns the correction);
* the loss: per sample ||y - t||^2 / ||t||^2, averaged over the batch (the relative L2 error squared);
* its gradient by the chain rule (conv3's adjoint is the correlation of the output gradient with the
  flipped weights, its weight gradient the correlation of the output gradient with the input), and
  the Adam step of ``learned_oracle.adam_step``.

Arrays are [batch, channels, depth, height, width].  Parameters are a list of (w, b) per layer in the
order above (3D layers w [co, ci, 3, 3, 3], the head w [1, w_0]); ``rnd`` (optional) is applied to every
tensor the GPU kernels store (weights, activations, activation gradients) so that a test can reproduce
their BF16 storage exactly.
"""

from __future__ import annotations

import numpy as np

SLOPE = 0.01
WIDTHS = (16, 32, 64, 128)


# --------------------------------------------------------------------------- the layers
def conv3(x, w, b):
    """3 x 3 x 3 cross-correlation, zero padding 1, plus bias.  x [B, ci, D, H, W], w [co, ci, 3, 3, 3]."""
    x = np.asarray(x, np.float64)
    B, ci, D, H, W = x.shape
    xp = np.zeros((B, ci, D + 2, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    y = np.zeros((B, w.shape[0], D, H, W)) + np.asarray(b, np.float64)[None, :, None, None, None]
    for a in range(3):
        for e in range(3):
            for f in range(3):
                y += np.einsum("oc,bcdhw->bodhw", w[:, :, a, e, f], xp[:, :, a:a + D, e:e + H, f:f + W])
    return y


def conv3_backward(x, w, dy):
    """Gradients of conv3 with respect to x, w and b for the output gradient dy."""
    x = np.asarray(x, np.float64)
    dy = np.asarray(dy, np.float64)
    B, ci, D, H, W = x.shape
    xp = np.zeros((B, ci, D + 2, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w, dtype=np.float64)
    for a in range(3):
        for e in range(3):
            for f in range(3):
                dxp[:, :, a:a + D, e:e + H, f:f + W] += np.einsum("oc,bodhw->bcdhw", w[:, :, a, e, f], dy)
                dw[:, :, a, e, f] = np.einsum("bodhw,bcdhw->oc", dy, xp[:, :, a:a + D, e:e + H, f:f + W])
    return dxp[:, :, 1:-1, 1:-1, 1:-1], dw, dy.sum(axis=(0, 2, 3, 4))


def leaky(x):
    x = np.asarray(x, np.float64)
    return np.where(x > 0, x, SLOPE * x)


def leaky_backward(y, dy):
    """Gradient through leaky given its OUTPUT y (the sign of y is the sign of the input)."""
    return np.where(np.asarray(y) > 0, dy, SLOPE * np.asarray(dy, np.float64))


def pool2(x):
    B, C, D, H, W = x.shape
    return np.asarray(x, np.float64).reshape(B, C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(3, 5, 7))


def pool2_backward(dy):
    return up2(dy) / 8.0


def up2(x):
    x = np.asarray(x, np.float64)
    return x.repeat(2, axis=2).repeat(2, axis=3).repeat(2, axis=4)


def up2_backward(dy):
    B, C, D, H, W = dy.shape
    return np.asarray(dy, np.float64).reshape(B, C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(3, 5, 7))


# --------------------------------------------------------------------------- the network
def layer_shapes(widths=WIDTHS):
    """(co, ci) of every conv3 in network order, then the head (1, w_0)."""
    L = len(widths)
    s = [(widths[0], 1), (widths[0], widths[0])]
    for l in range(1, L - 1):
        s += [(widths[l], widths[l - 1]), (widths[l], widths[l])]
    s += [(widths[-1], widths[-2]), (widths[-1], widths[-1]), (widths[-1], widths[-1])]
    for l in range(L - 2, -1, -1):
        s += [(widths[l], widths[l + 1] + widths[l]), (widths[l], widths[l])]
    return s


def param_count(widths=WIDTHS):
    return sum(co * ci * 27 + co for co, ci in layer_shapes(widths)) + widths[0] + 1


def init_params(widths=WIDTHS, seed=0):
    """He-normal 3D weights (std sqrt(2 / (27 ci))), zero biases; the head starts at zero (identity map)."""
    rng = np.random.default_rng(seed)
    ps = [(rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci)), np.zeros(co))
          for co, ci in layer_shapes(widths)]
    ps.append((np.zeros((1, widths[0])), np.zeros(1)))
    return ps


def pack(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unpack(flat, widths=WIDTHS):
    flat = np.asarray(flat, np.float64)
    out, o = [], 0
    for co, ci in layer_shapes(widths):
        n = co * ci * 27
        out.append((flat[o:o + n].reshape(co, ci, 3, 3, 3), flat[o + n:o + n + co]))
        o += n + co
    out.append((flat[o:o + widths[0]].reshape(1, widths[0]), flat[o + widths[0]:o + widths[0] + 1]))
    assert o + widths[0] + 1 == flat.size
    return out


def _ident(a):
    return a


def forward(params, x, widths=WIDTHS, rnd=None):
    """y = x + head(U-Net(x)); returns y and the cache for ``backward``."""
    r = rnd or _ident
    L = len(widths)
    P = [(r(w), b) for w, b in params]
    x = r(np.asarray(x, np.float64))
    cache = {"x": x, "acts": [], "skips": [], "pools": [], "ups": []}
    acts = cache["acts"]
    k = 0

    def cv(inp):
        nonlocal k
        w, b = P[k]
        out = r(leaky(conv3(inp, w, b)))
        acts.append((inp, out))
        k += 1
        return out

    h = cv(cv(x))
    cache["skips"].append(h)
    for l in range(1, L):
        p = r(pool2(h))
        cache["pools"].append(p)
        h = cv(cv(p))
        if l == L - 1:
            h = cv(h)
        else:
            cache["skips"].append(h)
    for l in range(L - 2, -1, -1):
        u = r(up2(h))
        cache["ups"].append(u)
        h = cv(cv(np.concatenate([u, cache["skips"][l]], axis=1)))
    wh, bh = P[k]
    y = x + np.einsum("oc,bcdhw->bodhw", wh, h) + bh[None, :, None, None, None]
    cache["last"] = h
    return y, cache


def loss_and_grad(y, t):
    """mean over the batch of ||y_b - t_b||^2 / ||t_b||^2, and its gradient with respect to y."""
    y = np.asarray(y, np.float64)
    t = np.asarray(t, np.float64)
    B = y.shape[0]
    nt = np.sum(t.reshape(B, -1) ** 2, axis=1)
    d = y - t
    loss = float(np.mean(np.sum(d.reshape(B, -1) ** 2, axis=1) / nt))
    return loss, 2.0 * d / (B * nt[:, None, None, None, None])


def backward(params, cache, dy, widths=WIDTHS, rnd=None):
    """Gradients of every parameter (same structure as params) for the output gradient dy."""
    r = rnd or _ident
    L = len(widths)
    P = [(r(w), b) for w, b in params]
    acts = cache["acts"]
    grads = [None] * len(P)
    wh, _ = P[-1]
    dy = np.asarray(dy, np.float64)
    h = cache["last"]
    grads[-1] = (np.einsum("bodhw,bcdhw->oc", dy, h), dy.sum(axis=(0, 2, 3, 4)))
    g = r(np.einsum("oc,bodhw->bcdhw", wh, dy))          # gradient of the last activation
    k = len(acts) - 1

    def cv_back(g_out):
        """through leaky and conv3 number k: the layer input's gradient (stored) and the parameter grads"""
        nonlocal k
        inp, out = acts[k]
        g_pre = r(leaky_backward(out, g_out))
        dx, dw, db = conv3_backward(inp, P[k][0], g_pre)
        grads[k] = (dw, db)
        k -= 1
        return dx

    skip_grads = [None] * (L - 1)
    for l in range(0, L - 1):
        g = r(cv_back(g))
        dcat = r(cv_back(g))
        cu = widths[l + 1]
        skip_grads[l] = dcat[:, cu:]
        g = r(up2_backward(dcat[:, :cu]))
    g = r(cv_back(r(cv_back(g))))
    g = r(cv_back(g))                                   # the bottom level's three conv3
    for l in range(L - 2, -1, -1):
        g = r(pool2_backward(g)) + skip_grads[l]
        g = r(cv_back(g))
        if l > 0:
            g = r(cv_back(g))
        else:
            cv_back(g)                                   # the input's gradient is not needed
    return grads


def predict(params, x, widths=WIDTHS, rnd=None):
    return forward(params, x, widths, rnd)[0]
