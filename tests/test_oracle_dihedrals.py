"""Pins of the oracle's dihedral potential (section "Bonded forces":
U = k [1 + cos(n phi - delta)] per bonded quadruplet, phi the angle between
the planes (i, j, k) and (j, k, l)).

Closed forms fix the convention: a quadruplet built with x_l = x_k +
(cos phi0, sin phi0, 0) around the bond j -> k along +z and x_i - x_j along
+x has phi = phi0 (trans pi, cis 0), so U = k [1 + cos(n phi0 - delta)] for
any n and delta, including signs that distinguish phi from -phi.  Forces are
minus the numerical derivative of the energy on random chains; they sum to
zero and exert no net torque; a chain has one dihedral per consecutive
quadruplet (the energy of a longer chain against a sum of closed forms with
phi from an independent route: the angle between the bond projections on
the plane perpendicular to the middle bond).
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W


def params(orc, k=1.7, n=2, delta=0.4, **over):
    return orc.make_params(1, 8, 10.0, chi=np.zeros((1, 1)), bond_k=0.0, dihedral_k=k,
                           dihedral_n=n, dihedral_delta=delta, **over)


def chain_bonds(n):
    return np.array([[i, i + 1] for i in range(n - 1)], np.int32)


def quad(phi0, r=(1.0, 1.3, 0.9)):
    j = np.array([2.0, 3.0, 4.0])
    k = j + np.array([0.0, 0.0, r[1]])
    i = j + np.array([r[0], 0.0, 0.0])
    l = k + r[2] * np.array([np.cos(phi0), np.sin(phi0), 0.0])
    return np.stack([i, j, k, l])


@pytest.mark.parametrize("n,delta", [(1, 0.0), (2, 0.4), (3, -1.1)])
def test_closed_form_energy(orc, n, delta):
    p = params(orc, k=1.7, n=n, delta=delta)
    for phi0 in (np.pi, 0.0, np.pi / 2, -np.pi / 2, 2.1, -0.7):
        U = orc.dihedral_energy(p, quad(phi0), chain_bonds(4))
        assert U == pytest.approx(1.7 * (1.0 + np.cos(n * phi0 - delta)), abs=1e-12)


def random_chain(rng, n, step=0.8):
    pos = [np.zeros(3)]
    for _ in range(n - 1):
        v = rng.normal(size=3)
        pos.append(pos[-1] + step * v / np.linalg.norm(v))
    return np.array(pos) + 4.0


@pytest.mark.parametrize("length,n,delta", [(4, 1, 0.3), (6, 2, -0.5), (12, 3, 1.2)])
def test_forces_are_minus_the_energy_derivative(orc, length, n, delta):
    rng = np.random.default_rng(length)
    p = params(orc, n=n, delta=delta)
    x = random_chain(rng, length)
    bonds = chain_bonds(length)
    F = orc.dihedral_force(p, x, bonds)
    h = 1e-6
    for i in range(length):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, a] += h
            xm[i, a] -= h
            fd = -(orc.dihedral_energy(p, xp, bonds) - orc.dihedral_energy(p, xm, bonds)) / (2 * h)
            assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_no_net_force_or_torque(orc):
    rng = np.random.default_rng(5)
    p = params(orc, n=3, delta=0.8)
    x = random_chain(rng, 15)
    F = orc.dihedral_force(p, x, chain_bonds(15))
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.cross(x, F).sum(axis=0), 0.0, atol=1e-11)


def test_one_dihedral_per_consecutive_quadruplet(orc):
    """delta = 0 makes U even in phi, so |phi| from the bond projections on
    the plane perpendicular to the middle bond suffices."""
    rng = np.random.default_rng(9)
    p = params(orc, k=0.9, n=2, delta=0.0)
    x = random_chain(rng, 10)
    want = 0.0
    for s in range(7):
        i, j, k, l = x[s:s + 4]
        b = (k - j) / np.linalg.norm(k - j)
        v = (i - j) - np.dot(i - j, b) * b
        w = (l - k) - np.dot(l - k, b) * b
        phi = np.arccos(np.clip(np.dot(v, w) / np.linalg.norm(v) / np.linalg.norm(w), -1, 1))
        want += 0.9 * (1 + np.cos(2 * phi))
    assert orc.dihedral_energy(p, x, chain_bonds(10)) == pytest.approx(want, rel=1e-10)


def test_bonded_energy_entry_includes_dihedrals(orc):
    w = W.diblock(20, 3, 3, 5.0, 5, 1.0)
    d = W.generate(w)
    base = dict(w.params(), dihedral_k=0.0)
    p0 = orc.make_params(**base)
    p1 = orc.make_params(**dict(base, dihedral_k=1.3, dihedral_n=2, dihedral_delta=0.2))
    V, G = orc.field(p0, orc.scatter(p0, d["pos"], d["type"]))
    e0 = orc.energy(p0, d["pos"], d["vel"], d["type"], d["bonds"], V, G, 0)
    e1 = orc.energy(p1, d["pos"], d["vel"], d["type"], d["bonds"], V, G, 0)
    ud = orc.dihedral_energy(p1, d["pos"], d["bonds"])
    assert ud > 0
    assert e1[1] == pytest.approx(e0[1] + ud, rel=1e-12)


def test_nve_conservation_with_dihedrals(orc):
    """Bonds, a stiff angle term and dihedrals, no field and no thermostat, on
    chains whose bond angles start in 100..140 degrees: the total energy is
    conserved (dihedral forces grow without bound as three beads become
    collinear, which the angle term keeps them away from: with angle_k 8
    some seeded chains come close enough in 1600 steps to drift by 1e-3 per
    bead; with 16, five seeds drift by 2e-5 to 6e-5)."""
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    d = W.with_bond_angles(w, W.generate(w))
    pp = dict(w.params(), gamma=0.0, dt=0.00125, chi=np.zeros((2, 2)), inv_kappa=0.0,
              angle_k=16.0, angle_cos0=-0.5, dihedral_k=0.5, dihedral_n=3, dihedral_delta=0.0)
    p = orc.make_params(**pp)
    _, _, E = orc.run(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 1600, energies=True)
    assert np.ptp(E[:, 1]) / w.n_beads > 0.05      # the bonded energy moves
    assert np.max(np.abs(E[:, 3] - E[0, 3])) / w.n_beads < 5e-4
