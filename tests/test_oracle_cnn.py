"""Pins for the oracle's CNN post-equaliser (CPU only)."""

import numpy as np
import pytest

from oracle import cnn


def test_conv1d_by_direct_summation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 11))
    W = rng.normal(size=(5, 3, 9))
    b = rng.normal(size=5)
    y = cnn.conv1d(x, W, b)
    for o in range(5):
        for t in range(11):
            ref = b[o] + sum(W[o, i, k] * x[i, t + k - 4] for i in range(3) for k in range(9) if 0 <= t + k - 4 < 11)
            assert abs(y[o, t] - ref) < 1e-12


def test_conv1d_single_channel_matches_numpy_correlate():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 40))
    W = rng.normal(size=(1, 1, 9))
    y = cnn.conv1d(x, W, np.zeros(1))
    ref = np.correlate(np.pad(x[0], 4), W[0, 0], mode="valid")
    assert np.allclose(y[0], ref, atol=1e-13)


def test_gradients_against_finite_differences():
    rng = np.random.default_rng(2)
    C, K, T = 6, 9, 24
    params = cnn.init_params(C, K, seed=3, out_scale=1.0)
    for layer in params:
        layer[1] = rng.normal(0, 0.1, size=layer[1].shape)
    z = rng.normal(size=(4, T))
    tgt = rng.normal(size=(4, T))
    out, acts = cnn.forward(params, z)
    grads = cnn.backward(params, acts, out, tgt)
    vec = cnn.flatten(params)
    gvec = cnn.flatten(grads)
    h = 1e-6
    idx = rng.choice(vec.size, size=60, replace=False)
    for i in idx:
        vp, vm = vec.copy(), vec.copy()
        vp[i] += h
        vm[i] -= h
        lp = cnn.mse(cnn.forward(cnn.unflatten(vp, C, K), z)[0], tgt)
        lm = cnn.mse(cnn.forward(cnn.unflatten(vm, C, K), z)[0], tgt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gvec[i]) <= 1e-6 * max(1e-3, abs(gvec[i])) + 1e-9, (i, fd, gvec[i])


def test_zero_last_layer_is_the_identity():
    params = cnn.init_params(8, 9, seed=1)
    params[-1][0][:] = 0.0
    z = np.random.default_rng(4).normal(size=(4, 50))
    out, _ = cnn.forward(params, z)
    assert np.array_equal(out, z)


def test_adam_first_step_is_lr_times_sign():
    params = [[np.array([1.0, -2.0]), np.array([0.5])]] + [[np.zeros(1), np.zeros(1)] for _ in range(3)]
    grads = [[np.array([0.3, -7.0]), np.array([1e-3])]] + [[np.zeros(1), np.zeros(1)] for _ in range(3)]
    opt = cnn.Adam(params, lr=1e-2)
    new = opt.step([[p.copy() for p in layer] for layer in params], grads)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> update = lr * g / (|g| + eps)
    assert new[0][0] == pytest.approx([1.0 - 1e-2, -2.0 + 1e-2], abs=1e-9)
    assert new[0][1] == pytest.approx([0.5 - 1e-2], abs=1e-6)


def test_training_reduces_the_loss_on_a_learnable_distortion():
    rng = np.random.default_rng(5)
    T = 400
    s = (rng.integers(0, 2, size=(4, T)) * 2 - 1) / np.sqrt(2)
    z = s + 0.2 * np.roll(s, 1, axis=1) ** 3              # a memory-1 nonlinearity the CNN can undo
    params = cnn.init_params(8, 9, seed=0)
    opt = cnn.Adam(params, lr=3e-3)
    first = cnn.mse(cnn.forward(params, z)[0], s)
    for _ in range(150):
        out, acts = cnn.forward(params, z)
        params = opt.step(params, cnn.backward(params, acts, out, s))
    assert cnn.mse(cnn.forward(params, z)[0], s) < 0.3 * first
