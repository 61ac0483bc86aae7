"""The Andersen thermostat on the GPU against the oracle, through the C ABI.

Collisions are decided by the same Philox counters on both sides and compared
in FP32 on both (the uniform and fl32(nu dt) are exact there), so every bead
collides at the same steps; trajectories then agree to the Langevin bars
(1e-4 over 10 steps), in the warp-segment kernel, the halo kernel for long
chains, with angles and the exact-gradient force, and in batches (bit for
bit with independent contexts).
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NU = 5.0  # 5 % of the beads per step at dt = 0.01


def make(hpf, w, data, **over):
    pp = w.params()
    pp.update(thermostat=2, andersen_nu=NU)
    pp.update(over)
    s = hpf.System(hpf.make_params(**pp))
    s.set_state(data["pos"], data["vel"], data["type"], data["bonds"], over.get("step", 0))
    return s, pp


CASES = [
    (W.diblock(60, 4, 6, 9.3, 8, 1.0, name="ragged_600"), {}),
    (W.diblock(80, 5, 5, 8.0, 8, 1.0, name="melt_800"), {"field_every": 3, "step": 4}),
    (W.diblock(8, 40, 40, 6.0, 6, 1.0, name="long_640"), {"field_every": 2}),
    (W.diblock(80, 5, 5, 8.0, 8, 1.0, name="exact_angles"),
     {"force_mode": 1, "angle_k": 2.0, "angle_cos0": -0.5, "field_every": 2}),
]


@pytest.mark.parametrize("w,over", CASES, ids=lambda c: getattr(c, "name", "") or "")
def test_ten_step_trajectory_matches_oracle(hpf_gpu, orc, w, over):
    d = W.generate(w)
    s, pp = make(hpf_gpu, w, d, **over)
    step0 = over.get("step", 0)
    s.step(4)
    s.step(6)
    pos, vel, step = s.get_state()
    op = orc.make_params(**pp)
    po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], step0, 10)
    assert step == step0 + 10
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4
    # collisions happened, and they matter: the NVE run is elsewhere
    hits = sum(orc.andersen_collides(op, i, step0 + k) for i in range(w.n_beads)
               for k in range(10))
    assert hits > 0
    pn, vn, _ = orc.run(orc.make_params(**dict(pp, andersen_nu=0.0)), d["pos"], d["vel"],
                        d["type"], d["bonds"], step0, 10)
    assert np.max(np.abs(vel - vn)) > 0.1


def test_observables_match_oracle(hpf_gpu, orc):
    w = W.diblock(60, 4, 6, 9.3, 8, 1.0, name="ragged_600")
    d = W.generate(w)
    s, pp = make(hpf_gpu, w, d, andersen_nu=20.0)
    E = s.energy()
    op = orc.make_params(**pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    assert E[0] == pytest.approx(Eo[0], rel=1e-6)
    assert E[1] == pytest.approx(Eo[1], rel=1e-12)
    assert E[2] == pytest.approx(Eo[2], rel=1e-12)
    assert E[5] == pytest.approx(Eo[5], rel=1e-6)
    # the redrawn velocities enter: the count of collisions at step 0 is not zero
    assert sum(orc.andersen_collides(op, i, 0) for i in range(w.n_beads)) > 0


def test_temperature_relaxes_to_kT(hpf_gpu):
    w = W.a5b5_10k()
    d = W.generate(w)
    d["vel"] = (1.6 * d["vel"]).astype(np.float32)
    s, pp = make(hpf_gpu, w, d, andersen_nu=10.0)
    T0 = s.energy()[5]
    s.step(300)
    Ts = []
    for _ in range(10):
        s.step(20)
        Ts.append(s.energy()[5])
    assert T0 > 2.0 and abs(np.mean(Ts) - 1.0) < 0.05


def test_batch_is_bitwise_the_independent_runs(hpf_gpu):
    import torch
    ws = [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=5, seed=11),
          W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5, seed=12)]
    stream = torch.cuda.Stream()
    params = [hpf_gpu.make_params(**dict(w.params(), thermostat=2, andersen_nu=NU)) for w in ws]
    data = [W.generate(w) for w in ws]
    with hpf_gpu.Batch(params, stream=stream) as b:
        for r, d in enumerate(data):
            b.replica(r).set_state(d["pos"], d["vel"], d["type"], d["bonds"])
        b.step(23)
        stream.synchronize()
        for r, (w, d) in enumerate(zip(ws, data)):
            pos, vel, _ = b.replica(r).get_state()
            s, _ = make(hpf_gpu, w, d)
            s.step(23)
            pi, vi, _ = s.get_state()
            assert np.array_equal(pos, pi) and np.array_equal(vel, vi)


def test_invalid_settings_are_rejected(hpf_gpu):
    w = W.diblock(30, 4, 4, 5.0, 5, 1.0)
    pp = dict(w.params(), thermostat=2)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(hpf_gpu.HPFError):
            hpf_gpu.System(hpf_gpu.make_params(**dict(pp, andersen_nu=bad)))
    with pytest.raises(hpf_gpu.HPFError):
        hpf_gpu.System(hpf_gpu.make_params(**dict(pp, thermostat=3)))
    # a batch runs one thermostat kind
    with pytest.raises(hpf_gpu.HPFError):
        hpf_gpu.Batch([hpf_gpu.make_params(**dict(pp, andersen_nu=1.0)),
                       hpf_gpu.make_params(**dict(pp, thermostat=0))])
