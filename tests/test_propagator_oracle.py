"""Pins of the propagator oracle (closed forms, brute force, finite differences)."""
import itertools

import numpy as np
import pytest

from oracle import propagator as P


def test_delta_kernel_is_a_periodic_shift():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 4, 5, 6))
    for k, d in enumerate(P.OFFSETS):
        W = np.zeros((27, 2, 3))
        W[k, 1, 2] = 1.0
        y = P.conv(x, W)
        assert np.all(y[:2] == 0.0)
        dz, dy, dx = d
        for z, yy, xx in itertools.product(range(4), range(5), range(6)):
            assert y[2, z, yy, xx] == x[1, (z + dz) % 4, (yy + dy) % 5, (xx + dx) % 6]


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 3, 4, 5))
    W = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=2)
    y = P.conv(x, W, b)
    ref = np.zeros_like(y)
    for co in range(2):
        for z, yy, xx in itertools.product(range(3), range(4), range(5)):
            s = b[co]
            for k, (dz, dy, dx) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
                for ci in range(3):
                    s += W[k, ci, co] * x[ci, (z + dz) % 3, (yy + dy) % 4, (xx + dx) % 5]
            ref[co, z, yy, xx] = s
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_constant_input_gives_summed_kernel():
    W = np.random.default_rng(2).normal(size=(27, 2, 4))
    y = P.conv(np.full((2, 3, 3, 3), 1.5), W)
    np.testing.assert_allclose(y[:, 1, 2, 0], 1.5 * W.sum(axis=(0, 1)), rtol=1e-12)


def test_silu_closed_form():
    assert P.silu(np.array(0.0)) == 0.0
    assert P.silu_grad(np.array(0.0)) == pytest.approx(0.5)
    z = np.linspace(-6, 6, 41)
    h = 1e-6
    np.testing.assert_allclose(P.silu_grad(z), (P.silu(z + h) - P.silu(z - h)) / (2 * h),
                               rtol=1e-7, atol=1e-9)
    assert P.silu(np.array(40.0)) == pytest.approx(40.0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    params = P.init_params(seed=4)
    params = [(W * 3.0, rng.normal(scale=0.1, size=b.shape)) for W, b in params]
    x = rng.normal(size=(4, 4, 3, 5))
    t = rng.normal(scale=0.1, size=(2, 4, 3, 5))
    L, grads = P.backward(params, x, t)
    assert L == pytest.approx(P.loss(params, x, t), rel=1e-14)
    h = 1e-6
    for li in range(3):
        W, b = params[li]
        for idx in [(0, 0, 0), (13, W.shape[1] - 1, W.shape[2] - 1), (26, 1, 0), (5, 2, 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params); pp[li] = (Wp, b)
            pm = list(params); pm[li] = (Wm, b)
            fd = (P.loss(pp, x, t) - P.loss(pm, x, t)) / (2 * h)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        for j in (0, b.shape[0] - 1):
            bp, bm = b.copy(), b.copy()
            bp[j] += h
            bm[j] -= h
            pp = list(params); pp[li] = (W, bp)
            pm = list(params); pm[li] = (W, bm)
            fd = (P.loss(pp, x, t) - P.loss(pm, x, t)) / (2 * h)
            assert grads[li][1][j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_first_adam_step_closed_form():
    params = [(np.array([[[0.5]]]), np.array([1.0]))]
    grads = [(np.array([[[2.0]]]), np.array([-3.0]))]
    new, state = P.adam_step(params, grads, P.adam_state(params), lr=0.01)
    # after one step m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    assert new[0][0][0, 0, 0] == pytest.approx(0.5 - 0.01 * 2.0 / (2.0 + 1e-8))
    assert new[0][1][0] == pytest.approx(1.0 + 0.01 * 3.0 / (3.0 + 1e-8))
    assert state[0] == 1
