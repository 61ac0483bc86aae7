"""Pins of the oracle's angle potential (section "Bonded forces", cosine form):
U = k (cos theta - cos theta0)^2 for every pair of bond partners of a bead,
theta the angle at that bead.  Closed forms, finite differences of the
energy, momentum and angular-momentum conservation, and a straight chain."""
import numpy as np
import pytest

import oracle as orc


def params(k=1.7, cos0=-0.3, **kw):
    return orc.make_params(1, 4, 10.0, angle_k=k, angle_cos0=cos0, **kw)


def chain(n, seed=0):
    rng = np.random.default_rng(seed)
    steps = rng.normal(size=(n - 1, 3))
    steps *= 0.7 / np.linalg.norm(steps, axis=1)[:, None]
    pos = np.vstack([np.zeros(3), np.cumsum(steps, axis=0)]) + 3.0
    bonds = np.array([[i, i + 1] for i in range(n - 1)], np.int32)
    return pos, bonds


def test_right_angle_closed_form():
    # theta = 90 deg: cos = 0, U = k cos0^2; the end bead a is pushed along -w/|w|
    # with magnitude 2 k (0 - cos0) / |u|
    k, cos0 = 1.7, -0.3
    pos = np.array([[1.3, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 2.0, 0.0]]) + 5.0
    bonds = np.array([[0, 1], [1, 2]], np.int32)
    p = params(k, cos0)
    assert orc.angle_energy(p, pos, bonds) == pytest.approx(k * cos0 ** 2, rel=1e-15)
    F = orc.angle_force(p, pos, bonds)
    g = -2.0 * k * (0.0 - cos0)
    np.testing.assert_allclose(F[0], [0.0, g / 1.3, 0.0], atol=1e-15)
    np.testing.assert_allclose(F[2], [g / 2.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(F[1], -(F[0] + F[2]), atol=1e-15)


def test_straight_chain_at_cos0_minus_one_is_force_free():
    pos = np.array([[0.0, 0.0, 0.0], [0.7, 0.0, 0.0], [1.4, 0.0, 0.0], [2.1, 0.0, 0.0]]) + 1.0
    bonds = np.array([[0, 1], [1, 2], [2, 3]], np.int32)
    p = params(3.0, -1.0)
    assert orc.angle_energy(p, pos, bonds) == pytest.approx(0.0, abs=1e-28)
    assert np.max(np.abs(orc.angle_force(p, pos, bonds))) < 1e-12


@pytest.mark.parametrize("n", [3, 4, 12])
def test_force_is_minus_the_energy_gradient(n):
    pos, bonds = chain(n, seed=n)
    p = params()
    F = orc.angle_force(p, pos, bonds)
    h = 1e-6
    for i in range(n):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            fd = -(orc.angle_energy(p, pp, bonds) - orc.angle_energy(p, pm, bonds)) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_total_force_and_torque_vanish():
    pos, bonds = chain(15, seed=3)
    F = orc.angle_force(params(), pos, bonds)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(pos, F).sum(axis=0), 0.0, atol=1e-11)


def test_one_angle_per_interior_bead_of_a_chain():
    pos, bonds = chain(9, seed=4)
    p = params()
    e = orc.angle_energy(p, pos, bonds)
    want = 0.0
    for j in range(1, 8):
        u, w = pos[j - 1] - pos[j], pos[j + 1] - pos[j]
        c = u @ w / np.sqrt((u @ u) * (w @ w))
        want += 1.7 * (c + 0.3) ** 2
    assert e == pytest.approx(want, rel=1e-13)


def test_energy_includes_angles_in_the_bonded_entry():
    pos, bonds = chain(10, seed=5)
    p = orc.make_params(1, 4, 10.0, angle_k=2.0, angle_cos0=-0.5, gamma=0.0)
    types = np.zeros(10, np.int32)
    D = orc.scatter(p, pos, types)
    V, G = orc.field(p, D)
    E = orc.energy(p, pos, np.zeros_like(pos), types, bonds, V, G, 0)
    assert E[1] == pytest.approx(orc.bond_energy(p, pos, bonds) + orc.angle_energy(p, pos, bonds),
                                 rel=1e-14)


def test_nve_with_angles_conserves_energy_in_the_exact_force_mode():
    """gamma = 0, exact field force: the integrator's energy error stays at the
    O(dt^2) level with angles included (bonds-only and angles-only melts)."""
    pos, bonds = chain(20, seed=6)
    types = np.zeros(20, np.int32)
    p = orc.make_params(1, 4, 10.0, angle_k=2.0, angle_cos0=-0.5, gamma=0.0, dt=0.002,
                        force_mode=1)
    vel = np.random.default_rng(7).normal(scale=0.5, size=pos.shape)
    vel -= vel.mean(axis=0)
    D = orc.scatter(p, pos, types)
    V, G = orc.field(p, D)
    e0 = orc.energy(p, pos, vel, types, bonds, V, G, 0)[3]
    po, vo, _ = orc.run(p, pos, vel, types, bonds, 0, 500)
    D = orc.scatter(p, po, types)
    V, G = orc.field(p, D)
    e1 = orc.energy(p, po, vo, types, bonds, V, G, 500)[3]
    assert abs(e1 - e0) / 20 < 1e-4
