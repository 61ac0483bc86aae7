"""Pipelined state upload and split observables against the serial calls.

hpf_upload_state copies a new state into one of two staging slots on the
context's copy stream while the previous step still runs; hpf_apply_state
makes the step wait for it.  hpf_energy_start / hpf_energy_finish split
hpf_energy, and hpf_energy_finish waits only for the work enqueued up to
its start.  A pipelined loop (the upload of step k + 1 issued before the
observables of step k are read), and a deeper one (step k + 1's permutation
and step and step k + 2's upload also enqueued before they are read), must
give, bit for bit, the observables and final state of the serial loop
(hpf_update_state, hpf_step, hpf_energy), with a different input array
every step, so that a wrong slot or an unfinished copy would show.  Misuse
is an error, not a race.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def inputs(w, k_steps, seed=3):
    rng = np.random.default_rng(seed)
    d = W.generate(w)
    out = []
    for _ in range(k_steps):
        out.append(((d["pos"] + rng.normal(0, 0.05, d["pos"].shape)).astype(np.float32),
                    (d["vel"] + rng.normal(0, 0.1, d["vel"].shape)).astype(np.float32)))
    return d, out


@pytest.mark.parametrize("device_inputs", [False, True])
def test_pipelined_loop_equals_the_serial_loop(hpf_gpu, device_inputs):
    import torch
    w = W.diblock(2000, 8, 12, 23.7, 24, 1.0, field_every=5)
    d, steps = inputs(w, 7)
    if device_inputs:
        host = [(torch.from_numpy(p).cuda(), torch.from_numpy(v).cuda()) for p, v in steps]
    else:
        host = [(torch.from_numpy(p).pin_memory(), torch.from_numpy(v).pin_memory())
                for p, v in steps]
    pp = w.params()
    a = hpf_gpu.System(hpf_gpu.make_params(**pp))
    a.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    Ea = []
    for k, (p, v) in enumerate(host):
        a.update_state(p, v, 3 * k)
        a.step(2)
        Ea.append(a.energy())
    pa, va, sa = a.get_state()
    b = hpf_gpu.System(hpf_gpu.make_params(**pp))
    b.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    Eb = []
    b.upload_state(*host[0])
    for k in range(len(host)):
        b.apply_state(3 * k)
        b.step(2)
        b.energy_start()
        if k + 1 < len(host):
            b.upload_state(*host[k + 1])
        Eb.append(b.energy_finish())
    pb, vb, sb = b.get_state()
    assert sa == sb
    np.testing.assert_array_equal(np.array(Ea), np.array(Eb))
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)
    # deeper: step k + 1's permutation and step, and step k + 2's upload,
    # enqueued before step k's observables are read (hpf_energy_finish waits
    # for its own copies only)
    c = hpf_gpu.System(hpf_gpu.make_params(**pp))
    c.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    Ec = []
    c.upload_state(*host[0])
    c.apply_state(0)
    c.step(2)
    c.energy_start()
    c.upload_state(*host[1])
    for k in range(len(host)):
        if k + 1 < len(host):
            c.apply_state(3 * (k + 1))
            c.step(2)
            if k + 2 < len(host):
                c.upload_state(*host[k + 2])
        Ec.append(c.energy_finish())
        if k + 1 < len(host):
            c.energy_start()
    pc, vc, sc = c.get_state()
    assert sa == sc
    np.testing.assert_array_equal(np.array(Ea), np.array(Ec))
    np.testing.assert_array_equal(pa, pc)
    np.testing.assert_array_equal(va, vc)
    a.close()
    b.close()
    c.close()


def test_pipeline_misuse_is_an_error(hpf_gpu):
    w = W.diblock(50, 4, 4, 5.0, 5, 1.0)
    d = W.generate(w)
    s = hpf_gpu.System(hpf_gpu.make_params(**w.params()))
    s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    with pytest.raises(hpf_gpu.HPFError):
        s.apply_state(0)                       # nothing uploaded
    s.upload_state(d["pos"], d["vel"])
    with pytest.raises(hpf_gpu.HPFError):
        s.upload_state(d["pos"], d["vel"])     # one upload at a time
    s.apply_state(0)
    with pytest.raises(hpf_gpu.HPFError):
        s.energy_finish()                      # no start
    s.energy_start()
    with pytest.raises(hpf_gpu.HPFError):
        s.energy()                             # the mirror is in use
    with pytest.raises(hpf_gpu.HPFError):
        s.energy_start()
    e1 = s.energy_finish()
    np.testing.assert_array_equal(e1, s.energy())
    s.close()


def test_nose_hoover_observables_survive_thermostat_calls_while_pending(hpf_gpu):
    """hpf_energy_finish applies the pending Nose-Hoover half step with the
    thermostat state in the pinned mirror that hpf_get_thermostat and
    hpf_set_thermostat write: both are refused while a start is pending, so
    the split observables equal hpf_energy's even after such a call."""
    w = W.diblock(300, 5, 5, 9.4, 9, 1.0, field_every=2)
    d = W.generate(w)
    pp = dict(w.params(), thermostat=1, nh_tau=0.5)
    s = hpf_gpu.System(hpf_gpu.make_params(**pp))
    s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    s.step(3)
    ref = s.energy()
    s.energy_start()
    s.step(2)                                   # moves xi, eta on the device
    with pytest.raises(hpf_gpu.HPFError):
        s.get_thermostat()
    with pytest.raises(hpf_gpu.HPFError):
        s.set_thermostat(0.3, 0.1)
    np.testing.assert_array_equal(s.energy_finish(), ref)
    s.close()
