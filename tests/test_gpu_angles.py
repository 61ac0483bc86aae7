"""Angle potential (section "Bonded forces", cosine form) on the GPU against
the oracle: bonded forces, 10-step trajectories in the warp-segment and the
halo kernel, the bonded energy, batches (bit for bit against contexts, also
with replicas without angles), and energy conservation with the exact field
force.  Bars as for the other forces: per-bead force within
1e-5 (|F| + F_rms), trajectories within 1e-4, FP64 energies within 1e-12."""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

from test_gpu_parity import SMALL, force_ok, make, oparams, run_both, thermal

pytestmark = pytest.mark.gpu

ANG = dict(angle_k=1.5, angle_cos0=-0.4)


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_bonded_forces_with_angles_match_oracle(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), **ANG)
    op = oparams(orc, pp)
    Fo = orc.bond_force(op, d["pos"], d["bonds"]) + orc.angle_force(op, d["pos"], d["bonds"])
    ok, worst = force_ok(s.forces(2), Fo)
    assert ok, worst
    assert np.max(np.abs(orc.angle_force(op, d["pos"], d["bonds"]))) > 1e-2


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_ten_step_trajectory_with_angles(hpf_gpu, orc, w):
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, **ANG)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("fe", [1, 5, 10])
def test_long_chains_with_angles_in_the_halo_kernel(hpf_gpu, orc, fe):
    w = W.diblock(30, 50, 50, 10.0, 10, 1.0, field_every=fe)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, **ANG)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_bonded_energy_includes_angles(hpf_gpu, orc):
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), **ANG)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    E = s.energy()
    assert E[1] == pytest.approx(Eo[1], rel=1e-12)
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)


def test_batch_with_angles_is_bitwise_the_contexts(hpf_gpu):
    import torch
    ws = [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=5, seed=11),
          W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5, seed=12)]
    over = [ANG, dict(angle_k=0.7, angle_cos0=0.1)]  # each replica its own angle constants
    stream = torch.cuda.Stream()
    params = [hpf_gpu.make_params(**dict(w.params(), **o)) for w, o in zip(ws, over)]
    b = hpf_gpu.Batch(params, stream=stream)
    data = [W.generate(w) for w in ws]
    for r, d in enumerate(data):
        b.replica(r).set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    b.step(23)
    stream.synchronize()
    for r, d in enumerate(data):
        s = hpf_gpu.System(params[r])
        s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
        s.step(23)
        pa, va, _ = b.replica(r).get_state()
        pi, vi, _ = s.get_state()
        np.testing.assert_array_equal(pa, pi)
        np.testing.assert_array_equal(va, vi)
    b.close()


def test_batch_rejects_replicas_with_and_without_angles(hpf_gpu):
    w = W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5)
    params = [hpf_gpu.make_params(**dict(w.params(), **o)) for o in (ANG, {})]
    with pytest.raises(hpf_gpu.HPFError):
        hpf_gpu.Batch(params)


def test_exact_force_with_angles_conserves_energy(hpf_gpu):
    w = W.a5b5_10k()
    s, d, pp = make(hpf_gpu, w, gamma=0.0, dt=0.005, field_every=1, force_mode=1, **ANG)
    e0 = s.energy()[3]
    s.step(1000)
    assert abs(s.energy()[3] - e0) / w.n_beads < 1e-4


def test_invalid_angle_parameters_are_rejected(hpf_gpu):
    w = W.diblock(10, 5, 5, 5.0, 5, 1.0)
    for bad in (dict(angle_k=float("nan")), dict(angle_k=1.0, angle_cos0=1.5)):
        with pytest.raises(hpf_gpu.HPFError):
            hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), **bad)))
