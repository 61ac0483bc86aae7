"""Pins of the oracle's Andersen thermostat (orc_run with thermostat 2).

The section "MD methods and algorithms" names the Andersen thermostat for the
canonical ensemble.  Reading: a bead collides at step n with probability
nu dt (the Philox uniform of counter (tag, n lo, n hi, 1) below fl32(nu dt)),
and a colliding bead's on-step velocity is redrawn from the Maxwell
distribution, sqrt(kT/m) xi with xi the Box-Muller normals of counter
(tag, n lo, n hi, 0).  Pins: nu = 0 is velocity-Verlet bit for bit; for
force-free beads every velocity is either its start value (no collision yet)
or exactly the draw of its last collision, recomputed here from the counters
by brute force, and the surviving fraction follows (1 - nu dt)^n; the
collision rate is nu dt; the mean temperature relaxes to kT.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W


def small_melt(n_chains=200, **over):
    w = W.diblock(n_chains, 5, 5, (10.0 * n_chains / 3.0) ** (1.0 / 3.0), 8, 1.0,
                  name="andersen_melt")
    d = W.generate(w)
    pp = w.params()
    pp.update(over)
    return w, d, pp


def test_zero_frequency_is_velocity_verlet(orc):
    w, d, pp = small_melt(field_every=2)
    nve = orc.make_params(**dict(pp, gamma=0.0))
    an = orc.make_params(**dict(pp, thermostat=2, andersen_nu=0.0, gamma=3.0))
    p1, v1, E1 = orc.run(nve, d["pos"], d["vel"], d["type"], d["bonds"], 3, 15, energies=True)
    p2, v2, E2 = orc.run(an, d["pos"], d["vel"], d["type"], d["bonds"], 3, 15, energies=True)
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(E1, E2)


def test_collision_rate(orc):
    p = orc.make_params(1, 8, 8.0, thermostat=2, andersen_nu=5.0, dt=0.01, seed=7)
    hits = sum(orc.andersen_collides(p, tag, step) for tag in range(2000) for step in range(50))
    n = 2000 * 50
    q = float(np.float32(5.0 * 0.01))
    assert abs(hits / n - q) < 4.0 * np.sqrt(q * (1 - q) / n)


def test_force_free_velocities_are_the_last_draw(orc):
    rng = np.random.default_rng(3)
    n, steps, nu, dt, kT = 400, 30, 3.0, 0.02, 1.7
    pos = rng.uniform(0.0, 8.0, size=(n, 3))
    vel = rng.normal(scale=1.3, size=(n, 3))
    p = orc.make_params(1, 8, 8.0, chi=np.zeros((1, 1)), inv_kappa=0.0, bond_k=0.0, dt=dt,
                        thermostat=2, andersen_nu=nu, kT=kT, seed=99)
    _, v, E = orc.run(p, pos, vel, np.zeros(n, np.int32), np.zeros((0, 2), np.int32), 0, steps,
                      energies=True)
    survived = 0
    for i in range(n):
        last = None
        for k in range(steps):
            if orc.andersen_collides(p, i, k):
                last = k
        if last is None:
            survived += 1
            assert np.array_equal(v[i], vel[i])
        else:
            want = np.sqrt(kT) * orc.gauss3(p.seed, i, last)
            np.testing.assert_allclose(v[i], want, rtol=1e-14, atol=1e-14)
    q = float(np.float32(nu * dt))
    expect = n * (1 - q) ** steps
    assert abs(survived - expect) < 4.0 * np.sqrt(expect * (1 - (1 - q) ** steps))
    # the record of step k holds the on-step velocities after that step's collisions
    ke = 0.0
    for i in range(n):
        if orc.andersen_collides(p, i, 0):
            ke += 0.5 * kT * np.sum(orc.gauss3(p.seed, i, 0) ** 2)
        else:
            ke += 0.5 * np.sum(vel[i] ** 2)
    assert E[0, 0] == pytest.approx(ke, rel=1e-12)


def test_temperature_relaxes_to_kT(orc):
    w, d, pp = small_melt(n_chains=300, field_every=1, thermostat=2, andersen_nu=10.0)
    p = orc.make_params(**pp)
    _, _, E = orc.run(p, d["pos"], 1.5 * d["vel"], d["type"], d["bonds"], 0, 800, energies=True)
    T = E[:, 5]
    assert T[0] > 1.8
    assert abs(np.mean(T[300:]) - 1.0) < 0.03


def test_bad_frequency_is_rejected(orc):
    w, d, pp = small_melt(thermostat=2, andersen_nu=-1.0)
    with pytest.raises(ValueError):
        orc.run(orc.make_params(**pp), d["pos"], d["vel"], d["type"], d["bonds"], 0, 1)


def test_every_bead_colliding_takes_the_half_kick(orc):
    """nu dt = 1: every bead collides every step, so one step from (x0, v) gives
    v1 = sqrt(kT/m) xi(tag, 0) + dt/(2m) F0 and x1 = x0 + dt v1 with F0 the
    conservative force at x0 (field refreshed at the first step)."""
    w, d, pp = small_melt(n_chains=40, thermostat=2, kT=1.3, mass=1.5)
    pp["andersen_nu"] = 1.0 / pp["dt"]
    p = orc.make_params(**pp)
    x1, v1, _ = orc.run(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 1)
    x0 = d["pos"].astype(np.float64)
    V, G = orc.field(p, orc.scatter(p, x0, d["type"]))
    F0 = orc.field_force(p, x0, d["type"], G) + orc.bond_force(p, x0, d["bonds"])
    xi = np.array([orc.gauss3(p.seed, i, 0) for i in range(len(x0))])
    want_v = np.sqrt(1.3 / 1.5) * xi + 0.5 * pp["dt"] / 1.5 * F0
    np.testing.assert_allclose(v1, want_v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(x1, x0 + pp["dt"] * want_v, rtol=1e-12, atol=1e-12)
