"""FP64 reference of the warm-start surrogate network (plain numpy).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: tests compare the CUDA
surrogate kernels with these functions; the product path never imports them.

The paper has no network: the surrogate is an addition of this project that
maps a cavity's obstacle mask, Rayleigh and Prandtl numbers to an initial
state for the LBM-FVM iteration, which then runs to the same residual as from
rest.  Nothing here is therefore pinned by the paper ("parity unpinned" in the
paper's sense); the functions are pinned instead by a library routine
(scipy's 2-D correlation for the convolution), by central finite differences
of the loss for every gradient, and by the closed-form first step of Adam.

Conventions (shared by value with the CUDA path, not by code):
* activations are NHWC arrays [B, H, W, C];
* a 3x3 convolution is a cross-correlation with zero padding 1 and weights
  [Co, 3, 3, Ci] (tap (ky, kx) reads the input at (y + ky - 1, x + kx - 1));
* the activation is the leaky ReLU with slope 1/16 for negative inputs;
* down-sampling is 2x2 average pooling, up-sampling nearest-neighbour 2x;
* a decoder level concatenates the up-sampled coarse features (first) with
  the encoder features of its resolution (second);
* the loss is the mean squared error over the fluid nodes and the three
  output channels (u/U0, v/U0, T).
"""

from __future__ import annotations

import numpy as np

LEAK = 1.0 / 16.0


def conv3x3(x, w, b):
    """y[b, y, x, o] = b[o] + sum_{ky, kx, c} w[o, ky, kx, c] x[b, y + ky - 1, x + kx - 1, c]."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, W, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W, :], w[:, ky, kx, :])
    return y + b


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 with respect to x, w and b, given dL/dy."""
    B, H, W, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W, :] += np.einsum("bhwo,oc->bhwc", dy, w[:, ky, kx, :])
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dy, xp[:, ky:ky + H, kx:kx + W, :])
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum(axis=(0, 1, 2))


def conv1x1(x, w, b):
    """y[b, y, x, o] = b[o] + sum_c w[o, c] x[b, y, x, c]."""
    return np.einsum("bhwc,oc->bhwo", x, w) + b


def conv1x1_backward(x, w, dy):
    return np.einsum("bhwo,oc->bhwc", dy, w), np.einsum("bhwo,bhwc->oc", dy, x), dy.sum(axis=(0, 1, 2))


def leaky(x):
    return np.where(x > 0, x, LEAK * x)


def leaky_backward(y, dy):
    """dL/d(pre-activation) from the activation's output y (same sign as its input)."""
    return np.where(y > 0, dy, LEAK * dy)


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def masked_mse(pred, target, fluid):
    """Mean of (pred - target)^2 over fluid nodes and channels; and its gradient."""
    m = fluid[..., None].astype(np.float64)
    n = m.sum() * pred.shape[-1]
    d = (pred - target) * m
    return float((d * d).sum() / n), 2.0 * d / n


def param_shapes(widths, cin=3, cout=3):
    """Parameters in order: per encoder level two 3x3 convolutions, per decoder
    level (coarse to fine) two 3x3 convolutions, then the 1x1 output layer."""
    shapes = []
    c = cin
    for w in widths:
        shapes += [("w", (w, 3, 3, c)), ("b", (w,)), ("w", (w, 3, 3, w)), ("b", (w,))]
        c = w
    for lvl in range(len(widths) - 2, -1, -1):
        w = widths[lvl]
        shapes += [("w", (w, 3, 3, widths[lvl + 1] + w)), ("b", (w,)), ("w", (w, 3, 3, w)), ("b", (w,))]
    shapes += [("w", (cout, widths[0])), ("b", (cout,))]
    return shapes


def forward(params, x, widths):
    """Network output and the activations the backward pass needs."""
    L = len(widths)
    p = iter(params)
    acts = {"x": x}
    h = x
    enc = []
    for lvl in range(L):
        w1, b1, w2, b2 = next(p), next(p), next(p), next(p)
        a1 = leaky(conv3x3(h, w1, b1))
        a2 = leaky(conv3x3(a1, w2, b2))
        acts[("enc", lvl)] = (h, a1, a2)
        enc.append(a2)
        if lvl < L - 1:
            h = avgpool2(a2)
    d = enc[-1]
    for lvl in range(L - 2, -1, -1):
        w1, b1, w2, b2 = next(p), next(p), next(p), next(p)
        cat = np.concatenate([upsample2(d), enc[lvl]], axis=-1)
        a1 = leaky(conv3x3(cat, w1, b1))
        a2 = leaky(conv3x3(a1, w2, b2))
        acts[("dec", lvl)] = (cat, a1, a2)
        d = a2
    wo, bo = next(p), next(p)
    acts["last"] = d
    return conv1x1(d, wo, bo), acts


def backward(params, acts, dout, widths):
    """Gradients of the loss with respect to every parameter (same order as
    param_shapes) and to the input, given dL/d(output)."""
    L = len(widths)
    grads = [None] * len(params)
    wo = params[-2]
    dd, grads[-2], grads[-1] = conv1x1_backward(acts["last"], wo, dout)
    denc = [None] * L  # gradient reaching each encoder output through its skip
    k = len(params) - 2
    for lvl in range(0, L - 1):
        k -= 4
        w1, w2 = params[k], params[k + 2]
        cat, a1, a2 = acts[("dec", lvl)]
        g = leaky_backward(a2, dd)
        da1, grads[k + 2], grads[k + 3] = conv3x3_backward(a1, w2, g)
        g = leaky_backward(a1, da1)
        dcat, grads[k], grads[k + 1] = conv3x3_backward(cat, w1, g)
        cu = dcat.shape[-1] - widths[lvl]
        denc[lvl] = dcat[..., cu:]
        dd = upsample2_backward(dcat[..., :cu])
    # dd now holds the gradient reaching the deepest encoder output
    dh = dd
    for lvl in range(L - 1, -1, -1):
        k = 4 * lvl
        w1, w2 = params[k], params[k + 2]
        h, a1, a2 = acts[("enc", lvl)]
        g = dh if lvl == L - 1 else dh + denc[lvl]
        g = leaky_backward(a2, g)
        da1, grads[k + 2], grads[k + 3] = conv3x3_backward(a1, w2, g)
        g = leaky_backward(a1, da1)
        dx, grads[k], grads[k + 1] = conv3x3_backward(h, w1, g)
        if lvl > 0:
            dh = avgpool2_backward(dx)
    return grads, dx


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of parameter p with gradient g;
    returns the new (p, m, v); t counts updates from 1."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
