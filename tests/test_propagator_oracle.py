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


@pytest.mark.parametrize("scale", [1.0, 37.0])
def test_backward_matches_finite_differences(scale):
    rng = np.random.default_rng(3)
    params = P.init_params(seed=4)
    params = [(W * 3.0, rng.normal(scale=0.1, size=b.shape)) for W, b in params]
    x = rng.normal(size=(4, 4, 3, 5))
    x[:2] = x[2:] - rng.normal(scale=1.0 / scale, size=(2, 4, 3, 5))
    t = rng.normal(scale=0.1 / scale, size=(2, 4, 3, 5))
    L, grads = P.backward(params, x, t, scale)
    assert L == pytest.approx(P.loss(params, x, t, scale), rel=1e-14)
    h = 1e-6
    for li in range(3):
        W, b = params[li]
        for idx in [(0, 0, 0), (13, W.shape[1] - 1, W.shape[2] - 1), (26, 1, 0), (5, 2, 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params); pp[li] = (Wp, b)
            pm = list(params); pm[li] = (Wm, b)
            fd = (P.loss(pp, x, t, scale) - P.loss(pm, x, t, scale)) / (2 * h)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        for j in (0, b.shape[0] - 1):
            bp, bm = b.copy(), b.copy()
            bp[j] += h
            bm[j] -= h
            pp = list(params); pp[li] = (W, bp)
            pm = list(params); pm[li] = (W, bm)
            fd = (P.loss(pp, x, t, scale) - P.loss(pm, x, t, scale)) / (2 * h)
            assert grads[li][1][j] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_first_adam_step_closed_form():
    params = [(np.array([[[0.5]]]), np.array([1.0]))]
    grads = [(np.array([[[2.0]]]), np.array([-3.0]))]
    new, state = P.adam_step(params, grads, P.adam_state(params), lr=0.01)
    # after one step m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    assert new[0][0][0, 0, 0] == pytest.approx(0.5 - 0.01 * 2.0 / (2.0 + 1e-8))
    assert new[0][1][0] == pytest.approx(1.0 + 0.01 * 3.0 / (3.0 + 1e-8))
    assert state[0] == 1


def test_features_are_the_change_and_the_current_density():
    rng = np.random.default_rng(9)
    x = rng.uniform(size=(4, 3, 4, 5))
    f = P.features(x)
    np.testing.assert_array_equal(f[0], x[2] - x[0])
    np.testing.assert_array_equal(f[1], x[3] - x[1])
    np.testing.assert_array_equal(f[2:], x[2:])
    # the forward pass starts from the features: a first layer that copies the
    # change channel of species A into every output shows it
    params = P.init_params(1)
    W1 = np.zeros((27, 4, 16))
    W1[13, 0, :] = 1.0  # centre offset, channel 0
    y, cache = P.forward([(W1, np.zeros(16))] + params[1:], x)
    np.testing.assert_array_equal(cache[0][0], f)
    np.testing.assert_allclose(cache[0][1][5], x[2] - x[0], rtol=1e-15)


def test_change_scale_enters_the_change_channels_and_the_output_only():
    """Scaling the change channels by s and dividing the output by s is a
    reparametrisation: dividing the first layer's change-channel weights by s
    and multiplying the last layer by s gives the same predictions at s as
    the original weights at s = 1; the loss is s^2 times the mean squared error."""
    rng = np.random.default_rng(11)
    params = P.init_params(5)
    params = [(W * 2.0, rng.normal(scale=0.1, size=b.shape)) for W, b in params]
    x = rng.uniform(0.2, 1.0, size=(4, 5, 4, 3))
    t = rng.normal(scale=0.05, size=(2, 5, 4, 3))
    s = 23.0
    (W1, b1), mid, (W3, b3) = params
    W1s = W1.copy()
    W1s[:, :2, :] /= s
    rep = [(W1s, b1), mid, (W3 * s, b3 * s)]
    y1, _ = P.forward(params, x)
    ys, _ = P.forward(rep, x, s)
    np.testing.assert_allclose(ys, y1, rtol=1e-12, atol=1e-14)
    assert P.loss(rep, x, t, s) == pytest.approx(s * s * np.mean((ys - t) ** 2), rel=1e-12)
    # the phi(t) channels are not scaled: a first layer reading only them
    # gives predictions that scale as 1 / s
    W1p = W1.copy()
    W1p[:, :2, :] = 0.0
    yp1, _ = P.forward([(W1p, b1), mid, (W3, b3)], x)
    yps, _ = P.forward([(W1p, b1), mid, (W3, b3)], x, s)
    np.testing.assert_allclose(yps * s, yp1, rtol=1e-12, atol=1e-14)


# ---- the binomial filter of the smoothed-density variant

def test_smooth_keeps_constants_and_the_total():
    rng = np.random.default_rng(7)
    c = np.full((2, 6, 5, 7), 0.37)
    np.testing.assert_allclose(P.smooth(c, 3), c, rtol=0, atol=1e-15)
    a = rng.uniform(0.0, 1.0, size=(2, 6, 5, 7))
    np.testing.assert_allclose(P.smooth(a, 4).sum(axis=(1, 2, 3)), a.sum(axis=(1, 2, 3)),
                               rtol=1e-13)


def test_smooth_spike_is_the_binomial_distribution():
    """A unit spike on a mesh wider than the filter's reach becomes, per axis,
    C(2p, k) / 4^p at offsets k - p (p passes), the product over the axes."""
    from math import comb
    p, M = 3, 15
    a = np.zeros((1, M, M, M))
    a[0, 7, 7, 7] = 1.0
    got = P.smooth(a, p)
    w = np.zeros(M)
    for k in range(2 * p + 1):
        w[7 - p + k] = comb(2 * p, k) / 4.0 ** p
    np.testing.assert_allclose(got[0], np.einsum("i,j,k->ijk", w, w, w), rtol=0, atol=1e-15)


def test_smooth_attenuates_a_sinusoid_by_the_closed_form():
    """sin(2 pi m x / M) along x: each pass multiplies it by cos^2(pi m / M)."""
    M, m, p = 16, 3, 5
    x = np.arange(M)
    a = np.broadcast_to(np.sin(2 * np.pi * m * x / M), (1, 4, 3, M)).copy()
    f = np.cos(np.pi * m / M) ** (2 * p)
    np.testing.assert_allclose(P.smooth(a, p), f * a, rtol=0, atol=1e-13)
