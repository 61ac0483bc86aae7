"""Pins of the oracle's Nose-Hoover thermostat (orc_run_nh).

The section "MD methods and algorithms" names the Nose-Hoover thermostat for
the canonical ensemble; its equations are Hoover's: dv/dt = F/m - xi v,
dxi/dt = (2K/(g kT) - 1)/tau^2, deta/dt = xi, with the extended energy
E + g kT (tau^2 xi^2 / 2 + eta) conserved.  Pins: the limit tau -> infinity is
velocity-Verlet (NVE); for force-free beads the kinetic energy and xi follow
the thermostat's ODE pair, which the scheme must reproduce to second order in
dt; the extended energy is conserved by the exact-gradient force; the mean
kinetic temperature relaxes to kT.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W


def small_melt(n_chains=200, **over):
    w = W.diblock(n_chains, 5, 5, (10.0 * n_chains / 3.0) ** (1.0 / 3.0), 8, 1.0,
                  name="nh_melt")
    d = W.generate(w)
    pp = w.params()
    pp.update(over)
    return w, d, pp


def test_infinite_tau_is_velocity_verlet(orc):
    w, d, pp = small_melt(gamma=0.0, field_every=3)
    nve = orc.make_params(**pp)
    nh = orc.make_params(**dict(pp, thermostat=1, nh_tau=1e30))
    p1, v1, _ = orc.run(nve, d["pos"], d["vel"], d["type"], d["bonds"], 4, 20)
    p2, v2, xe, _ = orc.run_nh(nh, d["pos"], d["vel"], d["type"], d["bonds"], 4, 20)
    assert np.max(np.abs(p2 - p1)) < 1e-12 and np.max(np.abs(v2 - v1)) < 1e-12
    assert abs(xe[0]) < 1e-50 and abs(xe[1]) < 1e-50


def thermostat_ode(K0, xi0, eta0, dof, kT, tau, t):
    from scipy.integrate import solve_ivp

    def rhs(_, y):
        K, xi, _eta = y
        return [-2.0 * xi * K, (2.0 * K / (dof * kT) - 1.0) / tau ** 2, xi]

    sol = solve_ivp(rhs, (0.0, t), [K0, xi0, eta0], rtol=1e-12, atol=1e-14, method="DOP853")
    return sol.y[:, -1]


@pytest.mark.parametrize("tau", [0.3, 1.0])
def test_free_beads_follow_the_thermostat_equations(orc, tau):
    """No forces at all (no bonds, chi = 0, 1/kappa = 0): every velocity is
    scaled by the same factor, and (K, xi, eta) after N steps must match the
    ODE solution over N dt (the state's thermostat sits at mid-step, so the
    elapsed time is N dt), with an error that falls as dt^2."""
    rng = np.random.default_rng(5)
    n = 300
    pos = rng.uniform(0.0, 8.0, size=(n, 3))
    vel = rng.normal(scale=1.7, size=(n, 3))
    types = np.zeros(n, dtype=np.int32)
    bonds = np.zeros((0, 2), dtype=np.int32)
    T_end = 3.0
    dof = 3.0 * (n - 1)
    errs = []
    for dt in (0.02, 0.01):
        p = orc.make_params(1, 8, 8.0, chi=np.zeros((1, 1)), inv_kappa=0.0, bond_k=0.0,
                            dt=dt, thermostat=1, nh_tau=tau, kT=1.3)
        N = int(round(T_end / dt))
        p2, v2, (xi, eta), _ = orc.run_nh(p, pos, vel, types, bonds, 0, N, xe=(0.4, 0.1))
        K = 0.5 * np.sum(v2 ** 2)
        K0 = 0.5 * np.sum(vel ** 2)
        Kr, xir, etar = thermostat_ode(K0, 0.4, 0.1, dof, 1.3, tau, N * dt)
        errs.append(max(abs(K - Kr) / Kr, abs(xi - xir), abs(eta - etar)))
        # one common scale for every velocity
        ratio = v2 / vel
        assert np.allclose(ratio, ratio[0, 0], rtol=1e-12)
    assert errs[1] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0  # second order


def test_extended_energy_is_conserved(orc):
    """Exact-gradient field force refreshed every step, bonds, Nose-Hoover with
    a short tau: the physical energy moves by many kT while the extended
    energy stays put."""
    w, d, pp = small_melt(dt=0.005, force_mode=1, field_every=1, thermostat=1, nh_tau=0.2)
    p = orc.make_params(**pp)
    vel = 1.6 * d["vel"]  # start hot so the thermostat works
    _, _, xe, E = orc.run_nh(p, d["pos"], vel, d["type"], d["bonds"], 0, 600, energies=True)
    n = w.n_beads
    assert np.ptp(E[:, 3]) / n > 0.3             # the thermostat moves energy
    assert np.max(np.abs(E[:, 6] - E[0, 6])) / n < 2e-4
    assert xe[0] != 0.0 and xe[1] != 0.0


def test_temperature_relaxes_to_kT(orc):
    w, d, pp = small_melt(n_chains=300, field_every=1, thermostat=1, nh_tau=0.2, kT=1.0)
    p = orc.make_params(**pp)
    vel = 1.5 * d["vel"]
    _, _, _, E = orc.run_nh(p, d["pos"], vel, d["type"], d["bonds"], 0, 1500, energies=True)
    n = w.n_beads
    T = 2.0 * E[:, 0] / (3.0 * (n - 1))
    assert T[0] > 1.8
    assert abs(np.mean(T[500:]) - 1.0) < 0.03


def test_energy_record_matches_the_state(orc):
    """The record of step k is taken from the state at k: its kinetic energy is
    that of the on-step velocity s1 (v + dt/(2m) F), consistent with a run
    that stops at k and restarts (bit-identical continuation)."""
    w, d, pp = small_melt(field_every=1, thermostat=1, nh_tau=0.5)
    p = orc.make_params(**pp)
    pa, va, xa, Ea = orc.run_nh(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 12,
                                energies=True)
    pb, vb, xb, Eb = orc.run_nh(p, d["pos"], d["vel"], d["type"], d["bonds"], 0, 7,
                                energies=True)
    pc, vc, xc, Ec = orc.run_nh(p, pb, vb, d["type"], d["bonds"], 7, 5, xe=xb, energies=True)
    assert np.array_equal(pa, pc) and np.array_equal(va, vc) and xa == xc
    np.testing.assert_allclose(Ea[7:], Ec, rtol=1e-12)
    np.testing.assert_allclose(Ea[:8], Eb, rtol=1e-15)


def test_bad_tau_is_rejected(orc):
    w, d, pp = small_melt(thermostat=1, nh_tau=0.0)
    with pytest.raises(ValueError):
        orc.run_nh(orc.make_params(**pp), d["pos"], d["vel"], d["type"], d["bonds"], 0, 1)
