"""Pins of the oracle's harmonic angle form (section "Bonded forces": the
alternative U = k (theta - theta0)^2 to the cosine form), theta the angle at
the middle bead of every pair of bond partners, in radians.

Closed forms fix the energy at known angles and the force on an end bead at a
right angle (along the other arm, magnitude 2k |theta - theta0| / |u|);
forces are minus the numerical derivative of the energy; they sum to zero
with no net torque; a straight chain at theta0 = pi is force-free; close to
theta0 the two forms agree to first order once the cosine form's constant is
k / sin^2 theta0; and a chain with harmonic angles conserves energy.
"""
import numpy as np
import pytest

import oracle as orc
from paper_1310_2041_gb300 import workloads as W


def params(k=1.3, th0=1.9, **kw):
    return orc.make_params(1, 4, 10.0, angle_k=k, angle_form=1, angle_theta0=th0, **kw)


def triangle(theta, ru=1.1, rw=0.8):
    j = np.array([4.0, 5.0, 6.0])
    a = j + ru * np.array([1.0, 0.0, 0.0])
    b = j + rw * np.array([np.cos(theta), np.sin(theta), 0.0])
    return np.stack([a, j, b]), np.array([[0, 1], [1, 2]], np.int32)


def chain(n, seed=0):
    rng = np.random.default_rng(seed)
    steps = rng.normal(size=(n - 1, 3))
    steps *= 0.7 / np.linalg.norm(steps, axis=1)[:, None]
    pos = np.vstack([np.zeros(3), np.cumsum(steps, axis=0)]) + 3.0
    bonds = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    return pos, bonds


@pytest.mark.parametrize("theta", [np.pi / 2, np.pi / 3, 2.6, 0.2, np.pi - 1e-3])
def test_closed_form_energy(theta):
    p = params(k=1.3, th0=1.9)
    pos, bonds = triangle(theta)
    assert orc.angle_energy(p, pos, bonds) == pytest.approx(1.3 * (theta - 1.9) ** 2, rel=1e-12)


def test_right_angle_end_force():
    k, th0, ru = 1.3, 1.9, 1.1
    pos, bonds = triangle(np.pi / 2, ru=ru)
    F = orc.angle_force(params(k, th0), pos, bonds)
    # theta < theta0: the end bead a is pushed away from the other arm (+y)
    want = -2.0 * k * (np.pi / 2 - th0) / ru * np.array([0.0, -1.0, 0.0])
    np.testing.assert_allclose(F[0], want, atol=1e-12)


@pytest.mark.parametrize("n", [3, 4, 12])
def test_forces_are_minus_the_energy_derivative(n):
    p = params(k=2.1, th0=2.0)
    pos, bonds = chain(n, seed=n)
    F = orc.angle_force(p, pos, bonds)
    h = 1e-6
    for i in range(n):
        for a in range(3):
            xp, xm = pos.copy(), pos.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(orc.angle_energy(p, xp, bonds) - orc.angle_energy(p, xm, bonds)) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_no_net_force_or_torque():
    pos, bonds = chain(15, seed=3)
    F = orc.angle_force(params(k=1.7, th0=1.7), pos, bonds)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(pos, F).sum(axis=0), 0.0, atol=1e-11)


def test_straight_chain_at_pi_is_force_free():
    pos = np.array([[1.0, 2.0, 3.0]]) + np.arange(6)[:, None] * np.array([[0.7, 0.0, 0.0]])
    bonds = np.array([[i, i + 1] for i in range(5)], np.int32)
    p = params(k=3.0, th0=np.pi)
    assert orc.angle_energy(p, pos, bonds) == 0.0
    assert np.all(orc.angle_force(p, pos, bonds) == 0.0)


def test_first_order_agreement_with_the_cosine_form():
    """(cos t - cos t0)^2 = sin^2 t0 (t - t0)^2 + O((t - t0)^3): near theta0
    the harmonic form with k equals the cosine form with k / sin^2 theta0."""
    th0, k = 1.9, 1.3
    pos, bonds = triangle(th0 + 1e-4)
    Fh = orc.angle_force(params(k, th0), pos, bonds)
    Fc = orc.angle_force(orc.make_params(1, 4, 10.0, angle_k=k / np.sin(th0) ** 2,
                                         angle_cos0=np.cos(th0)), pos, bonds)
    assert np.max(np.abs(Fh)) > 1e-5
    np.testing.assert_allclose(Fh, Fc, rtol=2e-4, atol=1e-12)


def test_nve_conservation_with_harmonic_angles():
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    d = W.with_bond_angles(w, W.generate(w))
    pp = dict(w.params(), gamma=0.0, dt=0.0025, chi=np.zeros((2, 2)), inv_kappa=0.0,
              angle_k=4.0, angle_form=1, angle_theta0=2.0)
    p = orc.make_params(**pp)
    _, _, E = orc.run(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 800, energies=True)
    assert np.ptp(E[:, 1]) / w.n_beads > 0.05
    assert np.max(np.abs(E[:, 3] - E[0, 3])) / w.n_beads < 1e-3
