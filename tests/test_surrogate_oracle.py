"""The FP64 surrogate reference against a library routine, finite differences
and closed forms (CPU only)."""

import numpy as np
import pytest

from oracle import surrogate_ref as R


def test_conv3x3_is_scipy_correlation_with_zero_padding():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(11)
    x = rng.standard_normal((2, 9, 7, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = R.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same", boundary="fill")
                             for c in range(3))
            assert np.abs(y[n, :, :, o] - ref).max() <= 1e-12


def test_conv1x1_is_the_centre_tap_of_conv3x3():
    rng = np.random.default_rng(12)
    x = rng.standard_normal((1, 5, 6, 4))
    w = rng.standard_normal((3, 4))
    b = rng.standard_normal(3)
    w3 = np.zeros((3, 3, 3, 4))
    w3[:, 1, 1, :] = w
    assert np.abs(R.conv1x1(x, w, b) - R.conv3x3(x, w3, b)).max() <= 1e-13


def test_pool_and_upsample_backward_are_adjoints():
    rng = np.random.default_rng(13)
    x = rng.standard_normal((2, 8, 6, 3))
    y = rng.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(R.avgpool2(x) * y), np.sum(x * R.avgpool2_backward(y)), rtol=1e-13)
    assert np.isclose(np.sum(R.upsample2(y) * x), np.sum(y * R.upsample2_backward(x)), rtol=1e-13)


def toy(seed=5, widths=(4, 6, 8), H=16):
    rng = np.random.default_rng(seed)
    params = [rng.standard_normal(s) * (0.5 if k == "w" else 0.1) for k, s in R.param_shapes(widths)]
    x = rng.standard_normal((2, H, H, 3))
    target = rng.standard_normal((2, H, H, 3))
    fluid = rng.random((2, H, H)) > 0.3
    return params, x, target, fluid


def loss_of(params, x, target, fluid, widths):
    out, _ = R.forward(params, x, widths)
    return R.masked_mse(out, target, fluid)[0]


def test_backward_matches_central_differences_on_a_16x16_toy():
    widths = (4, 6, 8)
    params, x, target, fluid = toy(widths=widths)
    out, acts = R.forward(params, x, widths)
    _, dout = R.masked_mse(out, target, fluid)
    grads, dx = R.backward(params, acts, dout, widths)
    rng = np.random.default_rng(6)
    h = 1e-6
    worst = 0.0
    for i, p in enumerate(params):
        for _ in range(4):
            idx = tuple(rng.integers(0, n) for n in p.shape)
            keep = p[idx]
            p[idx] = keep + h
            lp = loss_of(params, x, target, fluid, widths)
            p[idx] = keep - h
            lm = loss_of(params, x, target, fluid, widths)
            p[idx] = keep
            fd = (lp - lm) / (2 * h)
            worst = max(worst, abs(fd - grads[i][idx]) / max(abs(fd), 1e-3))
    for _ in range(8):
        idx = tuple(rng.integers(0, n) for n in x.shape)
        keep = x[idx]
        x[idx] = keep + h
        lp = loss_of(params, x, target, fluid, widths)
        x[idx] = keep - h
        lm = loss_of(params, x, target, fluid, widths)
        x[idx] = keep
        fd = (lp - lm) / (2 * h)
        worst = max(worst, abs(fd - dx[idx]) / max(abs(fd), 1e-3))
    assert worst <= 1e-5, worst


def test_adam_first_step_moves_by_lr_against_the_gradient_sign():
    # with m0 = v0 = 0 the bias-corrected moments are g and g^2, so the first
    # step is lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = R.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_the_warm_start_network_has_about_a_million_parameters():
    n = sum(int(np.prod(s)) for _, s in R.param_shapes((32, 64, 96, 160)))
    assert 0.9e6 <= n <= 1.1e6, n
