"""Nose-Hoover NVT on the GPU against the oracle's orc_run_nh, through the C ABI.

Bars as for the Langevin path: 10-step positions and velocities within 1e-4
of the FP64 oracle (the thermostat variables xi, eta within 1e-5, their only
difference being the FP32 velocities inside the kinetic-energy sum); the
observables within 2e-6 relative (1e-5 for the potential energies, whose
positions have drifted by FP32 rounding); the extended energy conserved to FP32
rounding on the GPU.  How the steps are split into calls does not change a
bit, and a checkpoint (state + xi, eta) resumes the run bit for bit.
Chains of any length (one thread per bead; neighbours' drifts recomputed).
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def hot(data, factor=1.5):
    d = dict(data)
    d["vel"] = (data["vel"] * factor).astype(np.float32)
    return d


def make(hpf, w, data, **over):
    pp = w.params()
    pp.update(thermostat=1, nh_tau=0.3)
    pp.update(over)
    s = hpf.System(hpf.make_params(**pp))
    s.set_state(data["pos"], data["vel"], data["type"], data["bonds"], over.get("step", 0))
    return s, pp


CASES = [
    (W.diblock(60, 4, 6, 9.3, 8, 1.0, name="ragged_600"), {}),
    (W.diblock(80, 5, 5, 8.0, 8, 1.0, name="melt_800"), {"field_every": 3}),
    (W.Workload("aniso", [(40, [0, 1, 2, 1]), (90, [2])], 7.0, 7, 3,
                [[0, 1.2, 0.3], [1.2, 0, 0.8], [0.3, 0.8, 0]], 0.05, 3, 10), {}),
    (W.diblock(80, 5, 5, 8.0, 8, 1.0, name="exact_angles"),
     {"force_mode": 1, "angle_k": 2.0, "angle_cos0": -0.5, "field_every": 2}),
]


@pytest.mark.parametrize("w,over", CASES, ids=lambda c: getattr(c, "name", "") or "")
def test_ten_step_trajectory_matches_oracle(hpf_gpu, orc, w, over):
    d = hot(W.generate(w))
    s, pp = make(hpf_gpu, w, d, **over)
    s.set_thermostat(0.2, -0.1)
    s.step(10)
    pos, vel, step = s.get_state()
    xi, eta = s.get_thermostat()
    po, vo, (xo, eo), _ = orc.run_nh(orc.make_params(**pp), d["pos"], d["vel"], d["type"],
                                     d["bonds"], 0, 10, xe=(0.2, -0.1))
    assert step == 10
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4
    assert abs(xi - xo) <= 1e-5 and abs(eta - eo) <= 1e-5
    assert abs(xi - 0.2) > 1e-3  # the thermostat acted


def test_thermostat_moves_temperature_toward_kT(hpf_gpu):
    w = W.a5b5_10k()
    d = hot(W.generate(w), 1.6)
    s, pp = make(hpf_gpu, w, d, nh_tau=0.2)
    T0 = s.energy()[5]
    s.step(300)
    Ts = []
    for _ in range(10):
        s.step(20)
        Ts.append(s.energy()[5])
    assert T0 > 2.0 and abs(np.mean(Ts) - 1.0) < 0.1


@pytest.mark.parametrize("fe", [1, 4, 10])
def test_calls_do_not_change_a_bit(hpf_gpu, fe):
    w = W.diblock(120, 5, 5, 8.5, 8, 1.0)
    d = hot(W.generate(w))
    a, _ = make(hpf_gpu, w, d, field_every=fe)
    b, _ = make(hpf_gpu, w, d, field_every=fe)
    a.step(12)
    for c in (1, 4, 7):
        b.step(c)
    pa, va, sa = a.get_state()
    pb, vb, sb = b.get_state()
    assert sa == sb == 12
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert a.get_thermostat() == b.get_thermostat()


def test_observables_match_oracle(hpf_gpu, orc):
    w = W.diblock(60, 4, 6, 9.3, 8, 1.0, name="ragged_600")
    d = hot(W.generate(w))
    s, pp = make(hpf_gpu, w, d, field_every=2)
    s.set_thermostat(0.1, 0.05)
    got = []
    for k in range(4):
        got.append(np.append(s.energy(), s.nh_conserved()))
        s.step(2)
    _, _, _, E = orc.run_nh(orc.make_params(**pp), d["pos"], d["vel"], d["type"], d["bonds"],
                            0, 6, xe=(0.1, 0.05), energies=True)
    for k in range(4):
        e, o = got[k], E[2 * k]
        for j in (0, 3, 5, 6):
            assert e[j] == pytest.approx(o[j], rel=2e-6), (k, j)
        assert e[1] == pytest.approx(o[1], rel=1e-5) and e[2] == pytest.approx(o[2], rel=1e-5)
        assert abs(e[4] - o[4]) <= 1e-4 * max(1.0, o[4])


def test_extended_energy_is_conserved(hpf_gpu):
    """Exact-gradient field force refreshed every step: the extended energy
    stays put while the thermostat moves the physical energy by many kT."""
    w = W.a5b5_10k()
    d = hot(W.generate(w), 1.5)
    s, pp = make(hpf_gpu, w, d, dt=0.005, force_mode=1, field_every=1, nh_tau=0.2)
    H0, E0 = s.nh_conserved(), s.energy()[3]
    Hs, Es = [], []
    for _ in range(8):
        s.step(50)
        Hs.append(s.nh_conserved())
        Es.append(s.energy()[3])
    n = w.n_beads
    assert max(abs(e - E0) for e in Es) / n > 0.3
    assert max(abs(h - H0) for h in Hs) / n < 5e-4


def test_checkpoint_resumes_bit_for_bit(hpf_gpu):
    """State and (xi, eta) saved at step 12 and loaded into a new context
    continue exactly: step 12 is a refresh step for both runs and both sort
    there (the bead order, which fixes the kinetic-energy summation order,
    depends only on the positions at the sort)."""
    w = W.diblock(120, 5, 5, 8.5, 8, 1.0)
    d = hot(W.generate(w))
    a, pp = make(hpf_gpu, w, d, field_every=4, sort_every=4)
    a.step(12)
    pos, vel, step = a.get_state()
    xe = a.get_thermostat()
    b = hpf_gpu.System(hpf_gpu.make_params(**pp))
    b.set_state(pos, vel, d["type"], d["bonds"], step)
    b.set_thermostat(*xe)
    a.step(9)
    b.step(9)
    pa, va, _ = a.get_state()
    pb, vb, _ = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert a.get_thermostat() == b.get_thermostat()


def test_set_state_resets_and_invalid_uses_fail(hpf_gpu):
    w = W.diblock(30, 4, 4, 5.0, 5, 1.0)
    d = W.generate(w)
    s, pp = make(hpf_gpu, w, d)
    s.set_thermostat(0.5, 0.25)
    assert s.get_thermostat() == (0.5, 0.25)
    s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    assert s.get_thermostat() == (0.0, 0.0)
    with pytest.raises(hpf_gpu.HPFError):
        s.set_thermostat(float("nan"), 0.0)
    # Langevin contexts have no thermostat state
    lv = hpf_gpu.System(hpf_gpu.make_params(**dict(pp, thermostat=0)))
    for call in (lv.get_thermostat, lambda: lv.set_thermostat(0.0, 0.0), lv.nh_conserved):
        with pytest.raises(hpf_gpu.HPFError):
            call()
    # bad tau, and batches (Langevin only)
    for bad in (0.0, -1.0, float("inf")):
        with pytest.raises(hpf_gpu.HPFError):
            hpf_gpu.System(hpf_gpu.make_params(**dict(pp, nh_tau=bad)))
    with pytest.raises(hpf_gpu.HPFError):
        hpf_gpu.Batch([hpf_gpu.make_params(**pp)] * 2)


def test_long_chains_with_angles_match_oracle(hpf_gpu, orc):
    """Chains of 80 beads (longer than a warp segment) with angles."""
    w = W.diblock(8, 40, 40, 6.0, 6, 1.0, name="long_640")
    d = hot(W.generate(w))
    s, pp = make(hpf_gpu, w, d, angle_k=1.5, angle_cos0=-0.8, field_every=3)
    s.step(10)
    pos, vel, _ = s.get_state()
    xi, eta = s.get_thermostat()
    po, vo, (xo, eo), _ = orc.run_nh(orc.make_params(**pp), d["pos"], d["vel"], d["type"],
                                     d["bonds"], 0, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4 and np.max(np.abs(vel - vo)) <= 1e-4
    assert abs(xi - xo) <= 1e-5 and abs(eta - eo) <= 1e-5


def test_empty_system_steps(hpf_gpu):
    w = W.diblock(1, 1, 1, 5.0, 5, 1.0)
    pp = dict(w.params(), n_beads=0, thermostat=1, nh_tau=0.5)
    s = hpf_gpu.System(hpf_gpu.make_params(**pp))
    z = np.zeros((0, 3), np.float32)
    s.set_state(z, z, np.zeros(0, np.int32), np.zeros((0, 2), np.int32))
    s.step(5)
    assert s.get_state()[2] == 5
