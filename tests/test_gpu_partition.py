"""Chain-partitioned stepping through the C ABI (hpf_set_tag_base, hpf_step_partial).

One system split by whole chains into parts, each part a context on the same
GPU.  At every field refresh the parts' partial int64 meshes are summed (here
with device adds, in a multi-GPU run an all-reduce) and every part computes the
field from the total.  Because the integer sum is exact, the field identical on
every part, bonds never cross parts and the noise is keyed by the global tag,
the parts must reproduce a single context holding every chain bit for bit,
through sorts, fused deposits and refreshes.
"""
import numpy as np
import pytest

import oracle
from paper_1310_2041_gb300 import partition as PT
from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run_single(hpf, w, d, pp, n_steps):
    with hpf.System(hpf.make_params(**pp)) as s:
        s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
        s.step(n_steps)
        return s.get_state()


def run_parts(hpf, w, d, pp, n_steps, n_parts):
    systems, parts = [], PT.split_chains(d, n_parts)
    for base, pd in parts:
        q = dict(pp, n_beads=len(pd["type"]))
        s = hpf.System(hpf.make_params(**q))
        s.set_tag_base(base)
        s.set_state(pd["pos"], pd["vel"], pd["type"], pd["bonds"])
        systems.append(s)
    ex = PT.step_parts_local(systems, n_steps)
    out = [s.get_state() for s in systems]
    for s in systems:
        s.close()
    pos = np.concatenate([o[0] for o in out])
    vel = np.concatenate([o[1] for o in out])
    return pos, vel, {o[2] for o in out}, ex


CASES = {
    # warp-segment kernel, sorts inside the run, refresh every 3 steps
    "langevin": (W.diblock(700, 5, 5, 13.3, 13, 1.0, field_every=3), dict(sort_every=4)),
    "andersen": (W.diblock(500, 4, 6, 11.9, 12, 0.6, field_every=2),
                 dict(thermostat=2, andersen_nu=3.0)),
    # chains longer than a warp segment: the halo kernel
    "long_chains": (W.diblock(60, 40, 40, 11.7, 12, 0.8, field_every=4), dict(sort_every=5)),
    "angles": (W.diblock(600, 6, 6, 13.9, 14, 0.9, field_every=3),
               dict(angle_k=2.0, angle_cos0=-0.5)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n_parts", [2, 3])
def test_parts_reproduce_one_context(hpf_gpu, case, n_parts):
    w, extra = CASES[case]
    d = W.generate(w)
    pp = dict(w.params(), **extra)
    n_steps = 11
    ps, vs, ss = run_single(hpf_gpu, w, d, pp, n_steps)
    pp_, vp_, sp_, ex = run_parts(hpf_gpu, w, d, pp, n_steps, n_parts)
    fe = pp["field_every"]
    assert ex == (n_steps + fe - 1) // fe + (1 if n_steps % fe == 0 else 0)
    assert sp_ == {ss}
    np.testing.assert_array_equal(pp_, ps)
    np.testing.assert_array_equal(vp_, vs)


def test_first_partial_mesh_is_the_parts_density(hpf_gpu):
    """Right after set_state the call returns at once with the part's own
    density, which equals the oracle's scatter of that part's beads."""
    w = W.diblock(300, 5, 5, 10.0, 10, 1.0, field_every=2)
    d = W.generate(w)
    pp = w.params()
    op = oracle.make_params(**pp)
    for base, pd in PT.split_chains(d, 2):
        with hpf_gpu.System(hpf_gpu.make_params(**dict(pp, n_beads=len(pd["type"])))) as s:
            s.set_tag_base(base)
            s.set_state(pd["pos"], pd["vel"], pd["type"], pd["bonds"])
            done, mesh = s.step_partial(4)
            assert done == 0 and mesh is not None
            np.testing.assert_array_equal(mesh.cpu().numpy(),
                                          oracle.scatter(op, pd["pos"], pd["type"]))


def test_partial_steps_of_one_part_equal_hpf_step(hpf_gpu):
    """A single part (nothing to sum) through hpf_step_partial is hpf_step."""
    w, extra = CASES["langevin"]
    d = W.generate(w)
    pp = dict(w.params(), **extra)
    ps, vs, _ = run_single(hpf_gpu, w, d, pp, 9)
    pp_, vp_, _, _ = run_parts(hpf_gpu, w, d, pp, 9, 1)
    np.testing.assert_array_equal(pp_, ps)
    np.testing.assert_array_equal(vp_, vs)


def test_partial_stepping_refusals(hpf_gpu):
    w = W.diblock(40, 4, 4, 5.0, 5, 1.0)
    d = W.generate(w)
    with hpf_gpu.System(hpf_gpu.make_params(**dict(w.params(), thermostat=1, nh_tau=1.0))) as s:
        s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
        with pytest.raises(hpf_gpu.HPFError):
            s.step_partial(2)
    with hpf_gpu.System(hpf_gpu.make_params(**w.params())) as s:
        with pytest.raises(hpf_gpu.HPFError):
            s.set_tag_base(-1)
        with pytest.raises(hpf_gpu.HPFError):
            s.set_tag_base((1 << 24) - w.n_beads + 1)
        s.set_tag_base((1 << 24) - w.n_beads)


def _gloo_rank(rank, world, port, out_path):
    """One rank: its part as a library context on cuda:0; the mesh sum by a
    gloo all-reduce of a host copy (the GPU machine has one GPU; on several GPUs
    bench.py sums with NCCL in place)."""
    import os
    import torch
    import torch.distributed as dist
    from paper_1310_2041_gb300 import hpf
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    w, extra = CASES["langevin"]
    d = W.generate(w)
    base, pd = PT.split_chains(d, world)[rank]
    pp = dict(w.params(), **extra, n_beads=len(pd["type"]))

    def reduce(mesh):
        host = mesh.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.SUM)
        mesh.copy_(host)

    with hpf.System(hpf.make_params(**pp)) as s:
        s.set_tag_base(base)
        s.set_state(pd["pos"], pd["vel"], pd["type"], pd["bonds"])
        PT.step_part(s, 11, reduce)
        pos, vel, step = s.get_state()
    np.savez(f"{out_path}.{rank}.npz", pos=pos, vel=vel, step=step)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_context(hpf_gpu, tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    out = str(tmp_path / "part")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    w, extra = CASES["langevin"]
    d = W.generate(w)
    ps, vs, ss = run_single(hpf_gpu, w, d, dict(w.params(), **extra), 11)
    got = [np.load(f"{out}.{r}.npz") for r in range(2)]
    assert all(int(g["step"]) == ss for g in got)
    np.testing.assert_array_equal(np.concatenate([g["pos"] for g in got]), ps)
    np.testing.assert_array_equal(np.concatenate([g["vel"] for g in got]), vs)
