"""Dihedral potential (section "Bonded forces": k [1 + cos(n phi - delta)] per
run of three consecutive bonds) on the GPU against the oracle: bonded forces
with and without angles, 10-step trajectories in the warp-segment and the
halo kernel, under the Nose-Hoover and Andersen thermostats, the bonded
energy, batches (bit for bit against contexts), energy conservation, and
parameter checks.  Chains start with bond angles in 100..140 degrees
(workloads.with_bond_angles): a dihedral is undefined where three beads are
collinear, and both sides lose digits near there.  Bars as for the other
forces: per-bead force within 1e-5 (|F| + F_rms), trajectories within 1e-4,
the FP64 bonded energy within 1e-12, the kinetic energy within 1e-7.

Trajectories run at dt = 0.005 with a stiffer angle term (TRAJ).  Dihedral
forces grow as 1 / sin(theta) as a bond angle opens towards 180 degrees, and
with the soft angle term of DIH at dt = 0.01 some angles reach 170 degrees
within ten steps: there the oracle itself, fed positions perturbed at the
FP32 rounding level before each field period, moves by 3e-3 (1e-2 on the 10k
melt), so no FP32 path can meet a fixed bar.  Under TRAJ the same
perturbation moves the oracle by at most 3.6e-5 on every trajectory below.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

from test_gpu_parity import SMALL, force_ok, make, oparams, thermal

pytestmark = pytest.mark.gpu

DIH = dict(angle_k=1.5, angle_cos0=-0.4, dihedral_k=0.8, dihedral_n=3, dihedral_delta=0.3)
TRAJ = dict(DIH, angle_k=8.0, angle_cos0=-0.5, dt=0.005)


def chains(w):
    return W.with_bond_angles(w, W.generate(w))


def run_both(hpf, orc, w, n_steps, chunks=None, **over):
    d = chains(w)
    s, d, pp = make(hpf, w, data=d, **over)
    for c in (chunks or [n_steps]):
        s.step(c)
    pos, vel, step = s.get_state()
    op = oparams(orc, pp)
    if pp.get("thermostat", 0) == 1:
        po, vo, _, _ = orc.run_nh(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, n_steps)
    else:
        po, vo, _ = orc.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, n_steps)
    assert step == n_steps
    return pos, vel, po, vo


def oracle_bonded(orc, op, pos, bonds):
    return (orc.bond_force(op, pos, bonds) + orc.angle_force(op, pos, bonds) +
            orc.dihedral_force(op, pos, bonds))


@pytest.mark.parametrize("over", [DIH, dict(DIH, angle_k=0.0), dict(DIH, dihedral_n=1,
                                                                    dihedral_delta=-2.0)],
                         ids=["with_angles", "without_angles", "n1"])
@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_bonded_forces_with_dihedrals_match_oracle(hpf_gpu, orc, w, over):
    s, d, pp = make(hpf_gpu, w, data=thermal(chains(w)), **over)
    op = oparams(orc, pp)
    Fo = oracle_bonded(orc, op, d["pos"], d["bonds"])
    ok, worst = force_ok(s.forces(2), Fo)
    assert ok, worst
    Fd = orc.dihedral_force(op, d["pos"], d["bonds"])
    assert np.max(np.abs(Fd)) > 1e-2  # the dihedral term is really there
    # the whole conservative force too (field + bonded)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Fall = Fo + orc.field_force(op, d["pos"], d["type"], Go)
    ok, worst = force_ok(s.forces(3), Fall)
    assert ok, worst


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_ten_step_trajectory_with_dihedrals(hpf_gpu, orc, w):
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, **TRAJ)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("fe,steps", [(1, 4), (5, 10), (10, 10), (16, 16)])
def test_long_chains_with_dihedrals_in_the_halo_kernel(hpf_gpu, orc, fe, steps):
    """Chains of 100 beads: the halo kernel, whose halo is 3 beads per fused
    step (48 at 16 steps per launch, the most one launch fuses)."""
    w = W.diblock(30, 50, 50, 10.0, 10, 1.0, field_every=fe)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, steps, **TRAJ)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("form", [0, 1])
def test_dihedrals_do_not_depend_on_sorting(hpf_gpu, orc, form):
    """Re-sorting at every launch moves chains between warp segments and
    lanes (a bead's dihedral shares then add up in another order): the
    trajectory is still the oracle's, with either angle form."""
    w = W.diblock(150, 5, 5, 8.0, 8, 1.0, field_every=2)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, chunks=[3, 3, 4], sort_every=1,
                                **dict(TRAJ, angle_form=form, angle_theta0=2.0))
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("thermostat", [1, 2])
@pytest.mark.parametrize("force_mode", [0, 2])
def test_dihedrals_under_other_thermostats(hpf_gpu, orc, thermostat, force_mode):
    w = W.diblock(80, 5, 5, 8.0, 8, 1.0, field_every=3)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, thermostat=thermostat, nh_tau=0.4,
                                andersen_nu=5.0, force_mode=force_mode, **TRAJ)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_nose_hoover_long_chains_with_dihedrals(hpf_gpu, orc):
    w = W.diblock(20, 40, 40, 9.0, 9, 1.0, field_every=4)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 8, thermostat=1, nh_tau=0.5, **TRAJ)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


@pytest.mark.parametrize("over", [DIH, dict(DIH, dihedral_n=6, dihedral_delta=1.1)],
                         ids=["n3", "n6"])
def test_bonded_energy_includes_dihedrals(hpf_gpu, orc, over):
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    s, d, pp = make(hpf_gpu, w, data=thermal(chains(w)), **over)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    E = s.energy()
    assert E[1] == pytest.approx(Eo[1], rel=1e-12)
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)
    assert orc.dihedral_energy(op, d["pos"], d["bonds"]) > 1.0


def test_batch_with_dihedrals_is_bitwise_the_contexts(hpf_gpu):
    import torch
    ws = [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=5, seed=11),
          W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5, seed=12)]
    over = [DIH, dict(angle_k=0.7, angle_cos0=0.1, dihedral_k=0.4, dihedral_n=2,
                      dihedral_delta=-0.6)]
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


def test_batch_rejects_replicas_with_and_without_dihedrals(hpf_gpu):
    w = W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5)
    params = [hpf_gpu.make_params(**dict(w.params(), **o))
              for o in (DIH, dict(DIH, dihedral_k=0.0))]
    with pytest.raises(hpf_gpu.HPFError):
        hpf_gpu.Batch(params)


def test_nve_with_dihedrals_conserves_energy(hpf_gpu):
    """The oracle's NVE pin on the GPU: bonds, a stiff angle term (angle_k
    16) and dihedrals, no field, no thermostat, dt = 0.00125, 1600 steps."""
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    s, d, pp = make(hpf_gpu, w, data=chains(w), gamma=0.0, dt=0.00125, chi=np.zeros((2, 2)),
                    inv_kappa=0.0, angle_k=16.0, angle_cos0=-0.5, dihedral_k=0.5, dihedral_n=3,
                    dihedral_delta=0.0)
    E = [s.energy()]
    for _ in range(8):
        s.step(200)
        E.append(s.energy())
    E = np.array(E)
    assert np.ptp(E[:, 1]) / w.n_beads > 0.02  # energy moves between the terms
    assert np.max(np.abs(E[:, 3] - E[0, 3])) / w.n_beads < 2e-3


def test_invalid_dihedral_parameters_are_rejected(hpf_gpu):
    w = W.diblock(10, 5, 5, 5.0, 5, 1.0)
    for bad in (dict(dihedral_k=1.0, dihedral_n=0), dict(dihedral_k=1.0, dihedral_n=7),
                dict(dihedral_k=float("nan")), dict(dihedral_k=1.0, dihedral_delta=float("inf"))):
        with pytest.raises(hpf_gpu.HPFError):
            hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), **bad)))
    # the multiplicity is not checked without dihedrals
    hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), dihedral_k=0.0, dihedral_n=0))).close()
