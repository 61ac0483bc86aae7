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
