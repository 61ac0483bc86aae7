"""Two-rank (gloo, CPU) check of the chain-partitioned density exchange.

Splitting the system by whole chains and summing the per-rank int64 meshes
with one all-reduce must give the single-rank mesh bit for bit: integer
addition is associative, so the exchange is deterministic.  Runs on CPU with
the oracle's scatter; no GPU is involved.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1310_2041_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.diblock(301, 6, 4, 9.1, 9, 1.0)
    d = W.generate(w)
    p = oracle.make_params(**w.params())
    clen = 10
    chains = np.arange(301)
    mine = chains[chains % world == rank]                      # whole chains per rank
    idx = (mine[:, None] * clen + np.arange(clen)[None, :]).reshape(-1)
    part = oracle.scatter(p, d["pos"][idx], d["type"][idx])
    t = torch.from_numpy(part.copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_mesh_allreduce_is_bit_exact(tmp_path):
    import oracle
    oracle.build()
    out = str(tmp_path / "mesh.npy")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = W.diblock(301, 6, 4, 9.1, 9, 1.0)
    d = W.generate(w)
    full = oracle.scatter(oracle.make_params(**w.params()), d["pos"], d["type"])
    np.testing.assert_array_equal(np.load(out), full)


class _FrozenPart:
    """Stands in for a library context in the protocol test: its beads do not
    move, and step_partial follows hpf_step_partial's contract (stop where a
    refresh is due and hand out the part's own density, as a CPU tensor;
    the next call takes the mesh as it then stands)."""

    def __init__(self, op, pd, field_every):
        import oracle
        self.mine = torch.from_numpy(oracle.scatter(op, pd["pos"], pd["type"]).copy())
        self.fe, self.step, self.field_step, self.part_step = field_every, 0, -1, -1
        self.meshes_used = []

    def step_partial(self, n):
        done = 0
        while True:
            if self.step % self.fe == 0 and self.field_step != self.step:
                if self.part_step != self.step:
                    self.part_step = self.step
                    self.mesh = self.mine.clone()
                    return done, self.mesh
                self.meshes_used.append(self.mesh.clone())   # the field's source
                self.field_step = self.step
            if n == done:
                return done, None
            k = min(self.fe - self.step % self.fe, n - done)
            self.step += k
            done += k


def _protocol_rank(rank, world, port, out_path):
    import oracle
    from paper_1310_2041_gb300 import partition as PT
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.diblock(203, 6, 4, 8.1, 8, 1.0)
    d = W.generate(w)
    op = oracle.make_params(**w.params())
    base, pd = PT.split_chains(d, world)[rank]
    part = _FrozenPart(op, pd, field_every=3)
    ex = PT.step_part(part, 10, lambda m: dist.all_reduce(m, op=dist.ReduceOp.SUM))
    full = oracle.scatter(op, d["pos"], d["type"])
    ok = ex == 4 and len(part.meshes_used) == 4 and \
        all(np.array_equal(m.numpy(), full) for m in part.meshes_used)
    flag = torch.tensor([1 if ok else 0])
    dist.all_reduce(flag, op=dist.ReduceOp.MIN)
    if rank == 0:
        np.save(out_path, flag.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_step_protocol_on_two_ranks(tmp_path):
    """partition.step_part on two gloo ranks: every field refresh of a 10-step
    run (field every 3: steps 0, 3, 6, 9) is fed the all-reduced mesh, which
    is the whole system's density bit for bit."""
    import oracle
    oracle.build()
    out = str(tmp_path / "ok.npy")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_protocol_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.load(out)[0] == 1


def test_split_chains_keeps_whole_chains():
    from paper_1310_2041_gb300 import partition as PT
    w = W.diblock(97, 7, 3, 8.0, 8, 1.0)
    d = W.generate(w)
    for parts in (1, 2, 3, 5):
        split = PT.split_chains(d, parts)
        assert len(split) == parts
        bases = [b for b, _ in split]
        sizes = [len(pd["type"]) for _, pd in split]
        assert bases[0] == 0 and sum(sizes) == w.n_beads
        assert all(b % 10 == 0 for b in bases)               # cuts at chain starts
        assert max(sizes) - min(sizes) <= 10
        for b, pd in split:
            n = len(pd["type"])
            np.testing.assert_array_equal(pd["pos"], d["pos"][b:b + n])
            bonds = pd["bonds"]
            assert bonds.min() >= 0 and bonds.max() < n
            assert len(bonds) == (n // 10) * 9
