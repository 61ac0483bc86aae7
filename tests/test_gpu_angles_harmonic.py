"""The harmonic angle form (section "Bonded forces": U = k (theta - theta0)^2)
on the GPU against the oracle: bonded forces, 10-step trajectories in the
warp-segment and the halo kernel, under Nose-Hoover, with dihedrals, the FP64
bonded energy, a batch mixing both angle forms (bit for bit against
contexts), and parameter checks.  Chains start with bond angles in
100..140 degrees (workloads.with_bond_angles): the form's force changes
direction abruptly where a chain passes through straight, and on random-walk
chains the oracle itself, fed positions perturbed at the FP32 rounding level,
moves by 2.3e-4 in ten steps on the 10k melt, against at most 3.8e-5 on the
chains used here.  Bars as for the cosine form."""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

from test_gpu_parity import SMALL, force_ok, make, oparams, thermal

pytestmark = pytest.mark.gpu

HARM = dict(angle_k=4.0, angle_form=1, angle_theta0=2.0)


def chains(w):
    return W.with_bond_angles(w, W.generate(w))


def run_both(hpf, orc, w, n_steps, **over):
    d = chains(w)
    s, d, pp = make(hpf, w, data=d, **over)
    s.step(n_steps)
    pos, vel, step = s.get_state()
    op = oparams(orc, pp)
    if pp.get("thermostat", 0) == 1:
        po, vo, _, _ = orc.run_nh(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, n_steps)
    else:
        po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, n_steps)
    assert step == n_steps
    return pos, vel, po, vo


@pytest.mark.parametrize("th0", [2.0, np.pi, 1.2])
@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_bonded_forces_with_harmonic_angles_match_oracle(hpf_gpu, orc, w, th0):
    s, d, pp = make(hpf_gpu, w, data=thermal(chains(w)), **dict(HARM, angle_theta0=th0))
    op = oparams(orc, pp)
    Fa = orc.angle_force(op, d["pos"], d["bonds"])
    Fo = orc.bond_force(op, d["pos"], d["bonds"]) + Fa
    ok, worst = force_ok(s.forces(2), Fo)
    assert ok, worst
    assert np.max(np.abs(Fa)) > 1e-2
    # not the cosine form with the same constants
    Fc = orc.angle_force(oparams(orc, dict(pp, angle_form=0, angle_cos0=np.cos(th0))),
                         d["pos"], d["bonds"])
    assert np.max(np.abs(Fa - Fc)) > 1e-2


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_ten_step_trajectory_with_harmonic_angles(hpf_gpu, orc, w):
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, **HARM)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("fe,steps", [(1, 4), (5, 10), (16, 16)])
def test_long_chains_with_harmonic_angles_in_the_halo_kernel(hpf_gpu, orc, fe, steps):
    w = W.diblock(30, 50, 50, 10.0, 10, 1.0, field_every=fe)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, steps, **HARM)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_harmonic_angles_under_nose_hoover_and_with_dihedrals(hpf_gpu, orc):
    w = W.diblock(80, 5, 5, 8.0, 8, 1.0, field_every=3)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, thermostat=1, nh_tau=0.4, **HARM)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, dt=0.005, dihedral_k=0.8, dihedral_n=3,
                                dihedral_delta=0.3, **dict(HARM, angle_k=8.0))
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_bonded_energy_with_harmonic_angles(hpf_gpu, orc):
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    s, d, pp = make(hpf_gpu, w, data=thermal(chains(w)), **HARM)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    E = s.energy()
    assert E[1] == pytest.approx(Eo[1], rel=1e-12)
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)


def test_batch_mixing_angle_forms_is_bitwise_the_contexts(hpf_gpu):
    import torch
    ws = [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=5, seed=11),
          W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5, seed=12)]
    over = [HARM, dict(angle_k=1.5, angle_cos0=-0.4)]
    stream = torch.cuda.Stream()
    params = [hpf_gpu.make_params(**dict(w.params(), **o)) for w, o in zip(ws, over)]
    data = [chains(w) for w in ws]
    with hpf_gpu.Batch(params, stream=stream) as b:
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


def test_invalid_harmonic_angle_parameters_are_rejected(hpf_gpu):
    w = W.diblock(10, 5, 5, 5.0, 5, 1.0)
    for bad in (dict(HARM, angle_form=2), dict(HARM, angle_form=-1), dict(HARM, angle_theta0=3.5),
                dict(HARM, angle_theta0=-0.1), dict(HARM, angle_theta0=float("nan"))):
        with pytest.raises(hpf_gpu.HPFError):
            hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), **bad)))
