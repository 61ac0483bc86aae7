"""Batched replicas (hpf_batch_*) against independent contexts and the oracle.

A batch advances every replica with one batched field launch and one
persistent step launch per field period (plus CUDA graph replays in the steady
state).  Each replica must follow exactly the trajectory an independent
context would, bit for bit: the batched kernels run the same arithmetic with
the replica's own constants.
"""
import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def replica_workloads(fe=5):
    return [W.diblock(90, 8, 12, 8.7, 9, 0.3, field_every=fe, seed=11),
            W.diblock(40, 8, 12, 6.4, 6, 1.1, field_every=fe, seed=12),
            W.diblock(150, 8, 12, 10.3, 10, 1.7, field_every=fe, seed=13),
            W.diblock(65, 8, 12, 7.6, 8, 2.0, field_every=fe, seed=14)]


def make_batch(hpf, ws, sort_every=0, graphs=True):
    import torch
    stream = torch.cuda.Stream()
    params = []
    for w in ws:
        p = w.params()
        p["sort_every"] = sort_every
        params.append(hpf.make_params(**p))
    b = hpf.Batch(params, stream=stream)
    b.use_graphs(graphs)
    data = [W.generate(w) for w in ws]
    for r, d in enumerate(data):
        b.replica(r).set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    return b, data, params, stream


def independent(hpf, w, d, n, sort_every=0):
    p = w.params()
    p["sort_every"] = sort_every
    s = hpf.System(hpf.make_params(**p))
    s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
    s.step(n)
    return s.get_state()


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("n", [23, 40])
def test_batch_is_bitwise_the_independent_runs(hpf_gpu, graphs, n):
    ws = replica_workloads()
    b, data, _, stream = make_batch(hpf_gpu, ws, graphs=graphs)
    b.step(n)
    stream.synchronize()
    for r, (w, d) in enumerate(zip(ws, data)):
        pos, vel, step = b.replica(r).get_state()
        pi, vi, _ = independent(hpf_gpu, w, d, n)
        assert step == n
        np.testing.assert_array_equal(pos, pi)
        np.testing.assert_array_equal(vel, vi)
    b.close()


def test_batch_with_resorting(hpf_gpu):
    ws = replica_workloads()
    b, data, _, stream = make_batch(hpf_gpu, ws, sort_every=10)
    b.step(35)
    stream.synchronize()
    for r, (w, d) in enumerate(zip(ws, data)):
        pos, vel, _ = b.replica(r).get_state()
        pi, vi, _ = independent(hpf_gpu, w, d, 35, sort_every=10)
        np.testing.assert_array_equal(pos, pi)
        np.testing.assert_array_equal(vel, vi)
    b.close()


def test_batch_replica_matches_the_oracle(hpf_gpu, orc):
    ws = replica_workloads(fe=2)
    b, data, _, stream = make_batch(hpf_gpu, ws)
    b.step(10)
    stream.synchronize()
    for r in (1, 3):
        pos, vel, _ = b.replica(r).get_state()
        po, vo, _ = orc.run(orc.make_params(**ws[r].params()), data[r]["pos"], data[r]["vel"],
                            data[r]["type"], data[r]["bonds"], 0, 10)
        assert np.max(np.abs(pos - po)) <= 1e-4
        assert np.max(np.abs(vel - vo)) <= 1e-4
    # per-replica calls still work on a batch member
    E = b.replica(0).energy()
    assert np.all(np.isfinite(E))
    b.close()


def test_batch_with_long_chains_falls_back(hpf_gpu):
    ws = [W.diblock(10, 40, 40, 7.0, 7, 1.0, field_every=5, seed=3),
          W.diblock(20, 8, 12, 6.0, 6, 0.5, field_every=5, seed=4)]
    b, data, _, stream = make_batch(hpf_gpu, ws)
    b.step(12)
    stream.synchronize()
    for r, (w, d) in enumerate(zip(ws, data)):
        pos, vel, _ = b.replica(r).get_state()
        pi, vi, _ = independent(hpf_gpu, w, d, 12)
        np.testing.assert_array_equal(pos, pi)
        np.testing.assert_array_equal(vel, vi)
    b.close()


def test_batch_energy_is_every_replicas_energy(hpf_gpu, orc):
    """hpf_batch_energy gives each replica's hpf_energy bit for bit (one
    synchronisation for all), and each agrees with the oracle's observables."""
    ws = replica_workloads()
    b, data, params, stream = make_batch(hpf_gpu, ws)
    b.step(7)
    E = b.energy()
    assert E.shape == (len(ws), 6)
    for r, (w, d) in enumerate(zip(ws, data)):
        assert np.array_equal(E[r], b.replica(r).energy())
        pos, vel, _ = b.replica(r).get_state()
        op = orc.make_params(**w.params())
        # the field in force at step 7 is the one refreshed at step 5
        pos5, vel5, _ = independent(hpf_gpu, w, d, 5)
        V5, G5 = orc.field(op, orc.scatter(op, pos5, d["type"]))
        eo = orc.energy(op, pos, vel, d["type"], d["bonds"], V5, G5, 7)
        assert E[r][1] == pytest.approx(eo[1], rel=1e-12)
        assert E[r][2] == pytest.approx(eo[2], rel=1e-12)
        assert E[r][0] == pytest.approx(eo[0], rel=1e-6)
    b.close()
