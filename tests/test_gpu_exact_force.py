"""The exact-energy-gradient field force (force_mode = 1) against the oracle.

force_mode 1 replaces the paper's interpolated central-difference gradient
by the exact derivative of the CIC field energy: minus the gradient of the
trilinear interpolant of V_T at the bead.  The oracle's variant
(orc_field_force_exact, pinned there by energy conservation) is the
reference; the bars are those of the default force (per-bead force within
1e-5 (|F| + F_rms), 10-step trajectories within 1e-4).  On the GPU the
variant must conserve energy as the oracle's does: with gamma = 0 and the
field refreshed every step, the total energy drifts below 1e-4 kT per bead
over 1000 steps at dt = 0.005, where the default force drifts by an order of
magnitude more.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

from test_gpu_parity import SMALL, force_ok, make, oparams, run_both, thermal

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_exact_field_force_matches_oracle(hpf_gpu, orc, w):
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), force_mode=1)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Fo = orc.field_force_exact(op, d["pos"], d["type"], Vo)
    ok, worst = force_ok(s.forces(1), Fo)
    assert ok, worst
    # not the default force: the two differ by far more than the bar
    assert np.max(np.abs(Fo - orc.field_force(op, d["pos"], d["type"], Go))) > 1e-3


@pytest.mark.parametrize("w", SMALL + [W.a5b5_10k()], ids=lambda w: w.name)
def test_exact_force_ten_step_trajectory(hpf_gpu, orc, w):
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, force_mode=1)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_exact_force_long_chains(hpf_gpu, orc):
    """The CTA kernel (chains longer than a warp segment) has the variant too."""
    w = W.diblock(30, 50, 50, 10.0, 10, 1.0, field_every=5)
    pos, vel, po, vo = run_both(hpf_gpu, orc, w, 10, force_mode=1)
    assert np.max(np.abs(pos - po)) <= 1e-4
    assert np.max(np.abs(vel - vo)) <= 1e-4


def test_exact_force_energy_matches_oracle(hpf_gpu, orc):
    w = W.diblock(100, 5, 5, 7.0, 7, 1.0)
    s, d, pp = make(hpf_gpu, w, data=thermal(W.generate(w)), force_mode=1)
    op = oparams(orc, pp)
    Vo, Go = orc.field(op, orc.scatter(op, d["pos"], d["type"]))
    Eo = orc.energy(op, d["pos"], d["vel"], d["type"], d["bonds"], Vo, Go, 0)
    E = s.energy()
    assert E[0] == pytest.approx(Eo[0], rel=1e-7)  # kinetic: the exact-gradient force enters
    assert E[2] == pytest.approx(Eo[2], rel=1e-12)


def test_exact_force_batch_is_bitwise_the_contexts(hpf_gpu):
    import torch
    ws = [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=5, seed=11),
          W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5, seed=12)]
    stream = torch.cuda.Stream()
    params = [hpf_gpu.make_params(**dict(w.params(), force_mode=1)) for w in ws]
    b = hpf_gpu.Batch(params, stream=stream)
    data = [W.generate(w) for w in ws]
    for r, d in enumerate(data):
        b.replica(r).set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    b.step(23)
    stream.synchronize()
    for r, (w, d) in enumerate(zip(ws, data)):
        s = hpf_gpu.System(params[r])
        s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
        s.step(23)
        pa, va, _ = b.replica(r).get_state()
        pi, vi, _ = s.get_state()
        np.testing.assert_array_equal(pa, pi)
        np.testing.assert_array_equal(va, vi)
    b.close()


def test_batch_rejects_mixed_force_modes(hpf_gpu):
    w = W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=5)
    params = [hpf_gpu.make_params(**dict(w.params(), force_mode=m)) for m in (0, 1)]
    with pytest.raises(hpf_gpu.HPFError):
        hpf_gpu.Batch(params)


def drift_per_bead(hpf, force_mode, steps=1000):
    w = W.a5b5_10k()
    s, d, pp = make(hpf, w, gamma=0.0, dt=0.005, field_every=1, force_mode=force_mode)
    e0 = s.energy()[3]
    s.step(steps)
    return abs(s.energy()[3] - e0) / w.n_beads


def test_exact_force_conserves_energy(hpf_gpu):
    exact = drift_per_bead(hpf_gpu, 1)
    default = drift_per_bead(hpf_gpu, 0)
    assert exact < 1e-4
    assert default > 3 * exact
