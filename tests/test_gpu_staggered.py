"""Algorithm 1's staggered field force (force_mode = 2) against the oracle.

force_mode 2 is kernels 3-4 of Algorithm 1 read literally: per axis, the
backward and forward differences of V at the bead's nearest vertex blended by
linear fraction ratios (orc_field_force_staggered, pinned in
tests/test_oracle_staggered.py).  Both sides pick the vertex from the same
FP32 mesh coordinate, so they always use the same vertex.  Bars as for the
default force: per-bead force within 1e-5 (|F| + F_rms), 10-step trajectories
within 1e-4, in the warp-segment kernel, the halo kernel for long chains,
with angles, under the Nose-Hoover and Andersen thermostats, in batches (bit
for bit with contexts) and in the observables.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

from test_gpu_parity import SMALL, force_ok, make, oparams, run_both, thermal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_staggered_field_force_matches_oracle(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), force_mode=2)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Fo = orc.field_force_staggered(op, d["pos"], d["type"], Vo)
    ok, worst = force_ok(s.forces(1), Fo)
    assert ok, worst
    # not the interpolated central difference: the two differ by far more than the bar
    assert np.max(np.abs(Fo - orc.field_force(op, d["pos"], d["type"], Go))) > 1e-3


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_staggered_ten_step_trajectory(hpf_gpu, orc, w):
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, force_mode=2)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_staggered_long_chains_with_angles(hpf_gpu, orc):
    """The halo kernel (chains longer than a warp segment) has the variant too."""
    w = W.diblock(30, 50, 50, 10.0, 10, 1.0, field_every=5)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, force_mode=2, angle_k=1.0,
                                angle_cos0=-0.7)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("thermostat", [1, 2])
def test_staggered_under_other_thermostats(hpf_gpu, orc, thermostat):
    w = W.diblock(80, 5, 5, 8.0, 8, 1.0, field_every=3)
    d = W.generate(w)
    pp = dict(w.params(), force_mode=2, thermostat=thermostat, nh_tau=0.4, andersen_nu=5.0)
    s = hpf_gpu.System(hpf_gpu.make_params(**pp))
    s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    s.step(10)
    pos, vel, _ = s.get_state()
    op = orc.make_params(**pp)
    if thermostat == 1:
        po, vo, _, _ = orc.run_nh(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, 10)
    else:
        po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, 10)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_staggered_energy_matches_oracle(hpf_gpu, orc):
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), force_mode=2)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    E = s.energy()
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)  # kinetic: the staggered force enters
    assert E[2] == pytest.approx(Eo[2], rel=1e-12)


def test_staggered_batch_is_bitwise_the_contexts(hpf_gpu):
    import torch
    ws = [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=5, seed=11),
          W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5, seed=12)]
    stream = torch.cuda.Stream()
    params = [hpf_gpu.make_params(**dict(w.params(), force_mode=2)) for w in ws]
    data = [W.generate(w) for w in ws]
    with hpf_gpu.Batch(params, stream=stream) as b:
        for r, d in enumerate(data):
            b.replica(r).set_state(d["pos"], d["vel"], d["type"], d["bonds"])
        b.step(23)
        stream.synchronize()
        for r, (w, d) in enumerate(zip(ws, data)):
            pos, vel, _ = b.replica(r).get_state()
            s = hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), force_mode=2)))
            s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
            s.step(23)
            pi, vi, _ = s.get_state()
            assert np.array_equal(pos, pi) and np.array_equal(vel, vi)


def test_force_mode_out_of_range_is_rejected(hpf_gpu):
    w = W.diblock(30, 4, 4, 5.0, 5, 1.0)
    for bad in (-1, 3):
        with pytest.raises(hpf_gpu.HPFError):
            hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), force_mode=bad)))
