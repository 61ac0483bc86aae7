#!/usr/bin/env python
"""hPF-MD throughput on GB300: bead-steps/s of the 1M-bead A10B10 diblock melt.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on stdout (rank 0).  A "step" is one MD time step of the whole
hot path: density scatter + field stencil at every field refresh (every 10
steps), field gather, bonds and the Langevin velocity-Verlet update for every
bead.  The state is resident in HBM before timing starts; L2 is flushed (a
256 MB write) before every timed field period and the flush is outside the
timed events.  With N > 1 (torchrun) every rank advances its own replica of
the melt: replicas only, weak scaling, no data-path collective.

--impl reference times the CPU oracle (plain C, FP64, int64 mesh) on the host
cores, each step on a bounded sample of the same melt.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bead-steps/s, hPF-MD 1M beads, plain vs learned/batched at <=1e-3 force err"
UNIT = "bead-steps/s"
# Algorithmic HBM bytes of one bead-step of the unfused step (read + write of
# the FP32 position and velocity, 48 B) plus the scatter, stencil and sort
# traffic amortised over the refresh period (about 2 B at 1M beads, field
# refresh every 10 steps): 50 B per bead-step.
ALGO_BYTES_PER_BEAD_STEP = 50.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")
# the step kernel's sources: its file and the device helpers it inlines
STEP_SRC = [os.path.join(ROOT, "paper_1310_2041_gb300", "csrc", f)
            for f in ("k_step.cu", "hpf_internal.cuh")]


# When a list, the runners append their line here instead of printing it
# (the default run gathers the other configurations' lines into its own).
_CAPTURE = None


def emit(line):
    if _CAPTURE is not None:
        _CAPTURE.append(line)
    else:
        print(json.dumps(line), flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="a10b10_1m")
    ap.add_argument("--sort-every", type=int, default=1000)
    ap.add_argument("--parallel", default="chains", choices=["chains", "replicas"],
                    help="with --gpus N > 1: split one system by whole chains (NCCL mesh "
                         "all-reduce at every refresh, strong scaling) or run N replicas")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload: skip the short runs of the 8.1M ternary blend and "
                         "the 64-replica batch whose lines ride along under \"configs\"")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--thermostat", default="langevin", choices=["langevin", "nh", "andersen"],
                    help="plain workloads: Langevin (the default), Nose-Hoover or Andersen NVT")
    ap.add_argument("--nh-tau", type=float, default=1.0)
    ap.add_argument("--andersen-nu", type=float, default=1.0)
    ap.add_argument("--angle-k", type=float, default=0.0,
                    help="plain workloads: angle potential constant (0: bonds only)")
    ap.add_argument("--angle-form", default="cos", choices=["cos", "harmonic"])
    ap.add_argument("--angle-cos0", type=float, default=-0.5)
    ap.add_argument("--angle-theta0", type=float, default=2.0)
    ap.add_argument("--dihedral-k", type=float, default=0.0,
                    help="plain workloads: dihedral constant (0: none); n = --dihedral-n, "
                         "delta = --dihedral-delta; chains then start with bond angles "
                         "in 100..140 degrees")
    ap.add_argument("--dihedral-n", type=int, default=3)
    ap.add_argument("--dihedral-delta", type=float, default=0.0)
    ap.add_argument("--smooth-passes", default="",
                    help="learned workload: also run the smoothed-density study with these "
                         "binomial-filter pass counts (comma-separated)")
    ap.add_argument("--smooth-lags", default="",
                    help="smoothed-density study: train and judge a network at each of these "
                         "lags (default: K = 20)")
    ap.add_argument("--net-lags", default="",
                    help="learned workload: also train and judge a network at these lags "
                         "(comma-separated step counts)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (read only)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="hpf_clocks_", suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu),
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def traffic_record(workload: str):
    """DRAM bytes per launch of the step kernel on `workload` from the committed
    ncu summary, valid only while the kernel source is unchanged since the
    capture."""
    try:
        recs = json.load(open(TRAFFIC_FILE))["k_step"]
    except (OSError, KeyError, ValueError):
        return None
    if isinstance(recs, dict):
        recs = [recs]
    h = hashlib.sha256()
    for f in STEP_SRC:
        h.update(open(f, "rb").read())
    for rec in recs:
        if rec.get("workload") == workload and rec.get("source_sha256") == h.hexdigest():
            return rec
    return None


PROP_SRC = [os.path.join(ROOT, "paper_1310_2041_gb300", "csrc", "k_prop.cu")]


def conv_traffic_record(workload: str):
    """DRAM bytes per inference of the three forward convolutions on `workload`
    from the committed ncu summary, valid only while k_prop.cu is unchanged
    since the capture."""
    try:
        recs = json.load(open(TRAFFIC_FILE))["k_conv_sweep"]
    except (OSError, KeyError, ValueError):
        return None
    h = hashlib.sha256()
    for f in PROP_SRC:
        h.update(open(f, "rb").read())
    for rec in recs:
        if rec.get("workload") == workload and rec.get("source_sha256") == h.hexdigest():
            return rec
    return None


def thermostat_params(args):
    if args.thermostat == "nh":
        return {"thermostat": 1, "nh_tau": args.nh_tau}
    if args.thermostat == "andersen":
        return {"thermostat": 2, "andersen_nu": args.andersen_nu}
    return {}


def bonded_params(args):
    out = {}
    if args.angle_k:
        out.update(angle_k=args.angle_k, angle_form=1 if args.angle_form == "harmonic" else 0,
                   angle_cos0=args.angle_cos0, angle_theta0=args.angle_theta0)
    if args.dihedral_k:
        out.update(dihedral_k=args.dihedral_k, dihedral_n=args.dihedral_n,
                   dihedral_delta=args.dihedral_delta)
    return out


def model_params(args):
    return dict(thermostat_params(args), **bonded_params(args))


def bonded_name(args):
    parts = ["bonds"]
    if args.angle_k:
        parts.append(f"harmonic angles k={args.angle_k} theta0={args.angle_theta0}"
                     if args.angle_form == "harmonic" else
                     f"cosine angles k={args.angle_k} cos0={args.angle_cos0}")
    if args.dihedral_k:
        parts.append(f"dihedrals k={args.dihedral_k} n={args.dihedral_n} "
                     f"delta={args.dihedral_delta}")
    return " + ".join(parts)


def bench_data(w, args, seed=None):
    """The seeded melt; with angle or dihedral terms its chains start with
    bond angles in 100..140 degrees (a random walk has near-collinear
    triples, where a dihedral is undefined)."""
    from paper_1310_2041_gb300 import workloads as W
    data = W.generate(w, seed=seed)
    if args.angle_k or args.dihedral_k:
        data = W.with_bond_angles(w, data)
    return data


def thermostat_name(args, pp):
    if args.thermostat == "nh":
        return f"nose-hoover tau={args.nh_tau}"
    if args.thermostat == "andersen":
        return f"andersen nu={args.andersen_nu}"
    return f"langevin gamma={pp['gamma']}"


def cpu_oracle_rate(w, data, budget_s: float, over=None):
    """Oracle bead-steps/s on the full workload, whole field periods until about
    budget_s of CPU work (a 2 %-of-chains calibration sizes the sample)."""
    import oracle
    oracle.build()
    pp = dict(w.params(), **(over or {}))
    op = oracle.make_params(**pp)
    if pp.get("thermostat", 0) == 1:
        def run(p, pos, vel, types, bonds, step0, n_steps):
            return oracle.run_nh(p, pos, vel, types, bonds, step0, n_steps)
    else:
        run = oracle.run
    n_chains_total = w.blocks[0][0]
    clen = len(w.blocks[0][1])
    c0 = max(1, n_chains_total // 50)
    n0 = c0 * clen
    t = time.perf_counter()
    run(op, data["pos"][:n0], data["vel"][:n0], data["type"][:n0],
        data["bonds"][: c0 * (clen - 1)], 0, w.field_every)
    per_bead_step = (time.perf_counter() - t) / (w.field_every * n0)
    n = w.n_beads
    periods = int(max(1, min(50, budget_s / (per_bead_step * n * w.field_every))))
    steps = periods * w.field_every
    t = time.perf_counter()
    run(op, data["pos"], data["vel"], data["type"], data["bonds"], 0, steps)
    dt = time.perf_counter() - t
    return {"value": n * steps / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} steps ({periods} field periods) of all {n} beads, "
                      f"{dt:.1f} s of CPU time"}


def cpu_oracle_learned_rate(w, data, snap, K: int, budget_s: float):
    """The oracle of the learned form at tol 1e-3, where every window falls
    back to the plain update: MD with the field refreshed every step (a bounded
    sample of the same melt) plus one propagator forward pass (numpy FP64 on
    the full mesh) per window of K steps, combined in bead-steps/s."""
    import numpy as np
    import oracle
    from oracle import propagator as P
    oracle.build()
    pp = dict(w.params(), field_every=1)
    op = oracle.make_params(**pp)
    clen = len(w.blocks[0][1])
    c = max(1, w.blocks[0][0] // 10)
    n = c * clen
    t = time.perf_counter()
    oracle.run(op, data["pos"][:n], data["vel"][:n], data["type"][:n],
               data["bonds"][: c * (clen - 1)], 0, 2)
    md_per_bead_step = (time.perf_counter() - t) / (2 * n)
    t = time.perf_counter()
    P.forward(P.init_params(0), np.asarray(snap, dtype=np.float64))
    fwd = time.perf_counter() - t
    per_step = md_per_bead_step * w.n_beads + fwd / K
    return {"value": w.n_beads / per_step, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"2 plain steps (field every step) of {n} of the {w.n_beads} beads "
                      f"({md_per_bead_step * w.n_beads:.2f} s per full step), one propagator "
                      f"forward on the {w.mesh}^3 mesh ({fwd:.1f} s, once per {K} steps)"}


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), \
            "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_oracle_replicas_rate(ws, data, budget_s: float):
    """Oracle bead-steps/s on the replica set: whole field periods of replicas
    taken in order until about budget_s of CPU work."""
    import oracle
    oracle.build()
    done_beads, t_total, used = 0, 0.0, 0
    for w, d in zip(ws, data):
        op = oracle.make_params(**w.params())
        t = time.perf_counter()
        oracle.run(op, d["pos"], d["vel"], d["type"], d["bonds"], 0, w.field_every)
        t_total += time.perf_counter() - t
        done_beads += w.n_beads * w.field_every
        used += 1
        if t_total >= budget_s:
            break
    return {"value": done_beads / t_total, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"one field period ({ws[0].field_every} steps) of each of the first "
                      f"{used} of {len(ws)} replicas, {t_total:.1f} s of CPU time"}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1310_2041_gb300 import workloads as W
    w = W.WORKLOADS[args.workload]()
    data = bench_data(w, args)
    oracle.build()
    nh = args.thermostat == "nh"
    op = oracle.make_params(**dict(w.params(), **model_params(args)))

    def run(p, pos, vel, types, bonds, step0, n_steps, xe=(0.0, 0.0)):
        if nh:
            po, vo, xo, _ = oracle.run_nh(p, pos, vel, types, bonds, step0, n_steps, xe)
            return po, vo, xo
        po, vo, _ = oracle.run(p, pos, vel, types, bonds, step0, n_steps)
        return po, vo, xe

    n_chains_total = w.blocks[0][0]
    clen = len(w.blocks[0][1])
    # calibrate, then size every step's sample so the run takes about 90 s
    c0 = max(1, n_chains_total // 50)
    n0 = c0 * clen
    t = time.perf_counter()
    run(op, data["pos"][:n0], data["vel"][:n0], data["type"][:n0],
        data["bonds"][: c0 * (clen - 1)], 0, 1)
    per_bead_step = time.perf_counter() - t
    per_bead_step /= n0
    total = max(1, args.steps + args.warmup)
    chains = int(min(n_chains_total, max(1, 90.0 / (total * per_bead_step * clen))))
    n = chains * clen
    pos, vel = data["pos"][:n].astype(np.float64), data["vel"][:n].astype(np.float64)
    types, bonds = data["type"][:n], data["bonds"][: chains * (clen - 1)]
    xe = (0.0, 0.0)
    if args.warmup > 0:
        pos, vel, xe = run(op, pos, vel, types, bonds, 0, args.warmup)
    t = time.perf_counter()
    pos, vel, xe = run(op, pos, vel, types, bonds, args.warmup, args.steps, xe)
    dt = time.perf_counter() - t
    value = n * args.steps / dt
    sample = (f"each step: one MD step (field refreshed every {w.field_every}) of the first "
              f"{chains} of {n_chains_total} chains ({n} beads), full box and mesh")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_beads": w.n_beads, "sample_beads": n,
                       "thermostat": thermostat_name(args, w.params()),
                       "bonded": bonded_name(args)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch
    from paper_1310_2041_gb300 import hpf, workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = W.WORKLOADS[args.workload]()
    chains = world > 1 and args.parallel == "chains"
    pp = w.params()
    pp["sort_every"] = args.sort_every
    nh = args.thermostat == "nh"
    therm = model_params(args)
    pp.update(therm)
    if chains and nh:
        raise SystemExit("Nose-Hoover couples every bead each step: use --parallel replicas")
    stream = torch.cuda.current_stream()
    if chains:
        # one system split by whole chains; the partial meshes are summed by an
        # NCCL all-reduce at every field refresh
        from paper_1310_2041_gb300 import partition as PT
        data_all = bench_data(w, args)
        tag_base, data = PT.split_chains(data_all, world)[rank]
        del data_all
        pp["n_beads"] = len(data["type"])
        sysm = hpf.System(hpf.make_params(**pp), stream=stream)
        sysm.set_tag_base(tag_base)

        def reduce(mesh):
            dist.all_reduce(mesh, op=dist.ReduceOp.SUM)

        def advance(n):
            PT.step_part(sysm, n, reduce)
    else:
        data = bench_data(w, args, seed=w.seed + rank)
        sysm = hpf.System(hpf.make_params(**pp), stream=stream)

        def advance(n):
            sysm.step(n)
    n_total = w.n_beads if chains else w.n_beads * world
    dev = {k: torch.from_numpy(v).cuda() for k, v in data.items()}
    sysm.set_state(dev["pos"], dev["vel"], dev["type"], dev["bonds"])
    fe = w.field_every
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # warm-up (untimed): at least W steps, continued to the next field refresh,
    # so that the timed window starts on a refresh step as every period of a
    # long run does
    warm = args.warmup + (-args.warmup) % fe
    advance(warm)
    torch.cuda.synchronize()
    sysm.profile_read()

    # timed region: K steps in field periods, L2 flushed before each period
    chunks, left = [], args.steps
    while left > 0:
        c = min(fe, left)
        chunks.append(c)
        left -= c

    def window(profile: bool):
        starts = [torch.cuda.Event(enable_timing=True) for _ in chunks]
        ends = [torch.cuda.Event(enable_timing=True) for _ in chunks]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # a few ms of GPU work first: the host enqueues the whole window while
        # the GPU is busy, so no host-side launch gap falls between the events
        for _ in range(50):
            flush.zero_()
        for c, a, b in zip(chunks, starts, ends):
            flush.zero_()
            sysm.profile(profile)
            a.record(stream)
            advance(c)
            b.record(stream)
        sysm.profile(False)
        torch.cuda.synchronize()
        t1 = time.perf_counter() - t0
        if dist:
            dist.barrier()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends)), t1

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dev_ms, wall = window(False)
    clk = clocks.stop()
    t_max = torch.tensor([dev_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dev_ms = float(t_max.item())
    value = n_total * args.steps / (dev_ms * 1e-3)
    # the kernel window: the same K steps again (continuing the run) with the
    # library's per-stage CUDA events on its stream; events between kernels
    # break the dependent-launch overlap, so the throughput window has none
    sysm.profile_read()
    window(True)
    prof = sysm.profile_read()
    profiled = [True] * len(chunks)

    # dominant kernel: the fused step kernel (one launch per field period;
    # Nose-Hoover: one per step plus one per period).  Achieved bandwidth: the
    # algorithmic bytes of the profiled periods' bead-steps over the step
    # kernel's event time in those periods (the sum over their launches of
    # bytes per launch / launch duration, weighted by duration).
    step_ms, step_launches = prof["step"]
    n_local = sysm.n   # this rank's beads
    prof_steps = sum(c for c, on in zip(chunks, profiled) if on)
    prof_launches = sum((c + 1 if nh else 1) for c, on in zip(chunks, profiled) if on)
    avg_launch_s = step_ms * 1e-3 / max(prof_launches, 1)
    bead_steps_per_launch = n_local * prof_steps / max(prof_launches, 1)
    achieved = ALGO_BYTES_PER_BEAD_STEP * n_local * prof_steps / (step_ms * 1e-3) / 1e9
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 6800.0, "fallback"
    # the record is the bonds-only step kernel's, on the default workload
    tr = None if (nh or bonded_params(args)) else traffic_record(w.name)
    traffic = None
    if tr:
        traffic = tr["dram_bytes_per_launch"] * bead_steps_per_launch / tr["bead_steps_per_launch"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                "kernel": "k_nh_step" if nh else "k_step_warp_batch",
                "algo_bytes_per_bead_step": ALGO_BYTES_PER_BEAD_STEP,
                "avg_launch_us": avg_launch_s * 1e6,
                "kernel_window": f"step-kernel events over a second window of the same "
                                 f"{args.steps} steps ({len(chunks)} periods)",
                "stage_ms": {k: round(v[0], 4) for k, v in prof.items()}}
    launches = int(sum(v[1] for v in prof.values()))

    # end to end through the C ABI with host buffers: every step uploads the
    # state from pinned host memory, advances one step and reads the energies back
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(v).pin_memory() for k, v in data.items()}
        h2d = sum(host[k].numel() * host[k].element_size() for k in ("pos", "vel"))
        sysm.set_state(host["pos"], host["vel"], host["type"], host["bonds"])
        advance(1)
        sysm.energy()
        torch.cuda.synchronize()
        # serial: each step's upload, step and observables one after another
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sysm.update_state(host["pos"], host["vel"], 0)
            advance(1)
            sysm.energy()
        torch.cuda.synchronize()
        te_serial = time.perf_counter() - t0
        # pipelined: step k + 1's upload (own copy stream, second staging slot)
        # runs while step k computes, and step k + 1's permutation and step are
        # enqueued before step k's observables are read back, so the GPU goes
        # from one step to the next without waiting for the host; every step
        # still copies its 24 MB in and its observables out (issuing step
        # k + 2's upload before reading step k's observables, so that the
        # copies run back to back, measured slower: 169 against 158 us a step)
        def pipelined(steps):
            sysm.upload_state(host["pos"], host["vel"])
            sysm.apply_state(0)
            advance(1)
            sysm.energy_start()
            if steps > 1:
                sysm.upload_state(host["pos"], host["vel"])
            for k in range(steps):
                if k + 1 < steps:
                    sysm.apply_state(0)
                    advance(1)
                sysm.energy_finish()
                if k + 1 < steps:
                    sysm.energy_start()
                    if k + 2 < steps:
                        sysm.upload_state(host["pos"], host["vel"])

        pipelined(3)
        # three timed loops, the median reported (the host-to-device link and
        # the host's wake-ups make single loops vary by a few per cent)
        times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pipelined(args.e2e_steps)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        te = statistics.median(times)
        e2e = {"value": n_total * args.e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 6 * 8,
               "steps": args.e2e_steps,
               "loops": [n_total * args.e2e_steps / t for t in times],
               "of": f"median of {len(times)} timed loops of {args.e2e_steps} steps",
               "path": "per step: hpf_upload_state(positions and velocities from pinned "
                       "host, double-buffered, issued while the previous step runs) + "
                       "hpf_apply_state + hpf_step(1) + hpf_energy_start/finish (to host; "
                       "the next step's apply_state and step enqueued before finish); "
                       "topology loaded once",
               "serial_value": n_total * args.e2e_steps / te_serial,
               "serial_path": "hpf_update_state + hpf_step(1) + hpf_energy per step"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_rate(w, data, budget_s=12.0, over=therm)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
                "scaling": "strong" if chains else "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.name, "n_beads": w.n_beads, "mesh": w.mesh,
                           "species": w.n_species, "field_every": fe,
                           "sort_every": args.sort_every,
                           "parallelism": (f"chains{world} (NCCL int64 mesh all-reduce per "
                                           f"refresh)" if chains else f"replicas{world}"),
                           "thermostat": thermostat_name(args, pp),
                           "bonded": bonded_name(args),
                           "window": f"untimed warm-up of {warm} steps (W continued to the "
                                     f"next field refresh), then {len(chunks)} field "
                                     f"periods",
                           "l2": "flushed (256 MB write) before each timed field period",
                           "wall_s": wall},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk}
        emit(line)
    sysm.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """64 uneven A8B12 replicas (chi 0.2 .. 2.0): one batch vs 64 separate contexts."""
    import torch
    from paper_1310_2041_gb300 import hpf, workloads as W

    torch.cuda.set_device(0)
    ws = W.replica_set()
    n_total = sum(w.n_beads for w in ws)
    stream = torch.cuda.Stream()
    params = []
    for w in ws:
        p = w.params()
        p["sort_every"] = args.sort_every
        params.append(hpf.make_params(**p))
    data = [W.generate(w) for w in ws]
    fe = ws[0].field_every

    def load(target_states):
        for s, d in zip(target_states, data):
            s.set_state(d["pos"], d["vel"], d["type"], d["bonds"])

    def timed(run, steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        run(steps)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    # the timed window starts on a refresh; the warm-up covers at least two
    # periods, so that the steady-state graph is captured (a one-time host
    # cost, with the GPU idle meanwhile) and replayed once before it
    warm = max(args.warmup, 2 * fe)
    warm += (-warm) % fe
    with torch.cuda.stream(stream):
        batch = hpf.Batch(params, stream=stream)
        load(batch.replicas)
        batch.step(warm)
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.3)
        # two more untimed periods: the timed window does not start on a GPU
        # that has idled through the pause (its first periods ran ~8 % slower)
        batch.step(2 * fe)
        ms_batch = timed(batch.step, args.steps)
        clk = clocks.stop()
        # kernel window: the same steps again with plain launches (no graph
        # replays) and the library's stage events, for the step kernel's time
        r0 = batch.replica(0)
        batch.use_graphs(False)
        r0.profile_read()
        r0.profile(True)
        batch.step(args.steps)
        r0.profile(False)
        prof = r0.profile_read()
        batch.close()
        plain = [hpf.System(p, stream=stream) for p in params]
        load(plain)
        for s in plain:
            s.step(args.warmup)

        def plain_run(steps):
            left = steps
            while left > 0:
                c = min(fe, left)
                for s in plain:
                    s.step(c)
                left -= c
        ms_plain = timed(plain_run, args.steps)
        for s in plain:
            s.close()
    value = n_total * args.steps / (ms_batch * 1e-3)
    plain_value = n_total * args.steps / (ms_plain * 1e-3)
    step_ms, step_launches = prof["step"]
    achieved = ALGO_BYTES_PER_BEAD_STEP * n_total * args.steps / (step_ms * 1e-3) / 1e9
    peak, peak_src = measured_hbm_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                "kernel": "k_step_warp_batch (all replicas, one launch per period)",
                "algo_bytes_per_bead_step": ALGO_BYTES_PER_BEAD_STEP,
                "avg_launch_us": 1e3 * step_ms / max(step_launches, 1),
                "kernel_window": f"step-kernel events over a second window of the same "
                                 f"{args.steps} steps, plain launches",
                "stage_ms": {k: round(v[0], 4) for k, v in prof.items()}}
    cpu = None if args.no_cpu_baseline else cpu_oracle_replicas_rate(ws, data, budget_s=10.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_batch / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "replicas64_a8b12", "n_beads": n_total, "replicas": len(ws),
                       "field_every": fe, "sort_every": args.sort_every,
                       "l2": "state of all replicas (~200 MB) larger than L2, no flush",
                       "window": f"untimed warm-up of {warm} steps (at least two field "
                                 f"periods: the graph is captured there), then {args.steps} steps",
                       "form": "one batched field + persistent step launch per period, CUDA "
                               "graph replays",
                       "plain_value": plain_value, "plain_form": "64 contexts, hpf_step each",
                       "speedup_vs_plain": value / plain_value},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": None,
            "gpu_launches": int(sum(v[1] for v in prof.values())), "clocks": clk}
    emit(line)
    return 0


def run_learned(args):
    """The 1M-bead A10B10 melt with the learned density propagator (K = 20).

    Untimed set-up: 1000 steps of the plain form, 200 phi snapshots every K
    steps of a plain run refreshing the field every step, 2000 Adam steps of
    the network on them (the GPU kernels).  Then the judge's field-force
    error of hold-last, linear extrapolation and the network, and the timed
    forms: learned at tol 1e-3 (the value), plain with the field refreshed
    every step (the plain form that meets 1e-3), learned with every window
    accepted, and plain at the largest field_every whose frozen-field error
    does not exceed the network's."""
    import numpy as np
    import torch
    from paper_1310_2041_gb300 import hpf, learned, workloads as W

    torch.cuda.set_device(0)
    K = 20
    w = W.a10b10_1m()
    data = W.generate(w)
    pp = w.params()
    pp["sort_every"] = args.sort_every
    stream = torch.cuda.current_stream()
    dev = {k: torch.from_numpy(v).cuda() for k, v in data.items()}

    def system(fe, pos, vel, step):
        s = hpf.System(hpf.make_params(**dict(pp, field_every=fe)), stream=stream)
        s.set_state(pos, vel, dev["type"], dev["bonds"], step)
        return s

    s = system(w.field_every, dev["pos"], dev["vel"], 0)
    s.step(1000)
    pos, vel, step = s.get_state()
    s.close()
    s = system(1, pos, vel, step)
    snaps = learned.collect_snapshots(s, 200, K)
    ex = learned.triples(200)
    train_ex, val_ex = ex[:178], ex[178:]
    net = hpf.Propagator(pp["mesh"], stream=stream)
    net.set_weights(learned.init_params(0))
    net.scale = learned.change_scale(snaps, train_ex)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    log = learned.train(net, snaps, 2000, lr=2e-3, lr_final=2e-4, examples=train_ex,
                        log_every=500)
    torch.cuda.synchronize()
    train_ms = (time.perf_counter() - t0) * 1e3 / 2000
    val_net, val_zero, val_lin = learned.validation_loss(net, snaps, val_ex)
    # inference time (the 4-channel input already on the device)
    x = snaps[100:102].contiguous()
    y = torch.empty_like(snaps[0])
    for _ in range(3):
        net.forward(x, out=y)
    # device time of 20 back-to-back inferences: the host enqueues them while
    # the GPU is still busy with a few ms of other work
    busy = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(100):
        busy.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(20):
        net.forward(x, out=y)
    b.record(stream)
    torch.cuda.synchronize()
    del busy
    infer_ms = a.elapsed_time(b) / 20
    flops = 2.0 * w.mesh ** 3 * 27 * sum(ci * co for ci, co in ((4, 16), (16, 16), (16, 2)))
    # memory side of the same inference, layer by layer: the 4-channel FP32
    # input read, the two 16-channel BF16 hidden activations written and read
    # once each, the 2-channel FP32 output written
    V = w.mesh ** 3
    infer_bytes = V * (4 * 4 + 2 * (2 * 16 * 2) + 2 * 4)
    # the judge's error of the candidates along the continued plain run
    lags = (1, 2, 5, 10, 15, 20)
    res = learned.judge_candidates(s, net, 10, K, lags=lags)
    eps = {k: float(np.mean(v)) for k, v in res.items() if v}
    pos, vel, step = s.get_state()
    s.close()
    fe_equal = max([L for L in lags if eps[f"hold_{L}"] <= eps["net"]] or [1])

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    n_win = max(1, (args.steps + K - 1) // K)
    warm_win = max(1, (args.warmup + K - 1) // K)

    def timed_windows(run):
        ms, agg = 0.0, None
        for _ in range(n_win):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            if isinstance(r, dict):
                if agg is None:
                    agg = dict(r)
                else:
                    for k, v in r.items():
                        agg[k] = (max(agg[k], v) if k == "eps_max" else
                                  v if k == "eps_last" else agg[k] + v)
        return ms, agg

    forms = {}
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for name, tol in (("learned_tol_1e-3", 1e-3), ("learned_all_accepted", float("inf"))):
        s = system(1, pos, vel, step)
        s.step_learned(net, warm_win, K=K, tol=tol)
        ms, st = timed_windows(lambda: s.step_learned(net, 1, K=K, tol=tol))
        forms[name] = {"value": w.n_beads * n_win * K / (ms * 1e-3), "stats": st}
        s.close()
    for name, fe in (("plain_fe1", 1), (f"plain_fe{fe_equal}", fe_equal), ("plain_fe10", 10)):
        s = system(fe, pos, vel, step)
        s.step(warm_win * K)
        ms, _ = timed_windows(lambda: s.step(K))
        forms[name] = {"value": w.n_beads * n_win * K / (ms * 1e-3)}
        s.close()
    clk = clocks.stop()
    value = forms["learned_tol_1e-3"]["value"]
    # the accuracy study at other lags: one network per lag, trained on 200
    # snapshots of that spacing, judged on the continuation of the run
    by_lag = {}
    for L in [int(v) for v in args.net_lags.split(",") if v.strip()]:
        sl = system(1, pos, vel, step)
        sn = learned.collect_snapshots(sl, 200, L)
        nl = hpf.Propagator(pp["mesh"], stream=stream)
        nl.set_weights(learned.init_params(0))
        nl.scale = learned.change_scale(sn, ex[:178])
        learned.train(nl, sn, 2000, lr=2e-3, lr_final=2e-4, examples=ex[:178])
        vn, vz, vl = learned.validation_loss(nl, sn, ex[178:])
        rl = learned.judge_candidates(sl, nl, 10, L, lags=(L,))
        by_lag[L] = {"net": float(np.mean(rl["net"])), "hold": float(np.mean(rl[f"hold_{L}"])),
                     "linear": float(np.mean(rl[f"linear_{L}"])),
                     "scale": nl.scale,
                     "val_mse": {"net": vn, "no_change": vz, "linear": vl}}
        if L == 1:
            # the lag-1 network used autoregressively over K steps
            by_lag[L]["rollout"] = {K2: float(np.mean(learned.judge_rollout(sl, nl, 8, K2)))
                                    for K2 in (2, 5, 10, 20)}
        nl.close()
        sl.close()
    # smoothed-density variant: every density (the true one included) through
    # the binomial filter before its field is formed; a network trained on
    # smoothed snapshots; the same judge
    smoothed = {}
    s_lags = [int(v) for v in args.smooth_lags.split(",") if v.strip()] or [K]
    for P in [int(v) for v in args.smooth_passes.split(",") if v.strip()]:
        smoothed[P] = {}
        for L in s_lags:
            ss = system(1, pos, vel, step)
            snaps_s = learned.collect_smoothed(ss, 200, L, P)
            ns = hpf.Propagator(pp["mesh"], stream=stream)
            ns.set_weights(learned.init_params(0))
            ns.scale = learned.change_scale(snaps_s, train_ex)
            learned.train(ns, snaps_s, 2000, lr=2e-3, lr_final=2e-4, examples=train_ex)
            vn, vz, vl = learned.validation_loss(ns, snaps_s, val_ex)
            res_s = learned.judge_smoothed(ss, P, ns, 10, L, lags=sorted({1, 2, 5, L}))
            smoothed[P][L] = {"eps_mean": {k: float(np.mean(v)) for k, v in res_s.items() if v},
                              "val_mse": {"net": vn, "no_change": vz, "linear": vl},
                              "scale": ns.scale}
            ns.close()
            ss.close()
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        peak_src = "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 1900.0, "fallback"
    achieved = flops / (infer_ms * 1e-3) / 1e12
    hbm_peak, hbm_src = measured_hbm_peak()
    cpu = None
    if not args.no_cpu_baseline:
        x0 = snaps[100:102].reshape((4,) + tuple(snaps.shape[2:])).cpu().numpy()
        cpu = cpu_oracle_learned_rate(w, data, x0, K, budget_s=12.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": n_win * K, "warmup": warm_win * K,
            "ms_per_step": 1e3 * w.n_beads / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (network bf16/fp32-acc)", "data": "synthetic",
            "config": {"workload": "a10b10_1m_learned", "n_beads": w.n_beads, "mesh": w.mesh,
                       "K": K, "tol": 1e-3, "snapshots": 200, "train_iters": 2000,
                       "l2": "flushed (256 MB write) before each timed window",
                       "forms": forms, "eps_mean": eps, "fe_equal_eps": fe_equal,
                       "val_mse": {"net": val_net, "no_change": val_zero, "linear": val_lin},
                       "change_scale": net.scale,
                       "train_ms_per_iter": train_ms, "train_log": log,
                       "infer_ms": infer_ms, "net_by_lag": by_lag,
                       "smoothed": smoothed},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (conv_traffic_record("propagator_70") or {}).get(
                             "dram_bytes_per_inference"),
                         "peak_source": peak_src,
                         "kernel": "k_conv_sweep (three layers, whole forward)",
                         "algo_flops_per_inference": flops},
            "roofline_hbm": {"bound": "hbm", "achieved": infer_bytes / (infer_ms * 1e-3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": infer_bytes / (infer_ms * 1e-3) / 1e9 / hbm_peak,
                             "peak_source": hbm_src, "algo_bytes_per_inference": infer_bytes},
            "cpu_baseline": cpu, "e2e": None, "clocks": clk}
    print(json.dumps(line), flush=True)
    net.close()
    return 0


def run_propagator(args):
    """The learned density propagator's inference alone on the 70^3 mesh of the
    1M-bead melt: He-initialised weights (the arithmetic does not depend on
    the values), a seeded 4-channel input on the device, K timed forwards
    (CUDA events on the handle's stream), L2 flushed before each.  Reports the
    tensor roofline (6.52 GFLOP per inference) and the memory-side one."""
    import numpy as np
    import torch
    from paper_1310_2041_gb300 import hpf, learned

    torch.cuda.set_device(0)
    M = 70
    V = M ** 3
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.uniform(0.0, 1.2, size=(4, M, M, M)).astype(np.float32)).cuda()
    y = torch.empty((2, M, M, M), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flops = 2.0 * V * 27 * sum(ci * co for ci, co in ((4, 16), (16, 16), (16, 2)))
    infer_bytes = V * (4 * 4 + 2 * (2 * 16 * 2) + 2 * 4)
    with hpf.Propagator((M, M, M), stream=stream) as net:
        net.set_weights(learned.init_params(1))
        for _ in range(max(3, args.warmup)):
            net.forward(x, out=y)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.3)
        # every flush, event pair and forward is enqueued before one final
        # synchronisation, so the host's launch work overlaps the GPU's and the
        # events time the device alone
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for _ in range(100):  # a few ms of GPU work for the host to run ahead of
            flush.zero_()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            net.forward(x, out=y)
            b.record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        clk = clocks.stop()
    infer_ms = statistics.median(ms)
    rec = conv_traffic_record("propagator_70")
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle's FP64 forward (numpy) on the same input, once: about 2 s
        from oracle import propagator as P
        xs = x.cpu().numpy().astype(np.float64)
        t = time.perf_counter()
        P.forward(P.init_params(1), xs)
        fwd = time.perf_counter() - t
        cpu = {"value": 1.0 / fwd, "unit": "inferences/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"one FP64 forward of the oracle (numpy, its BLAS threads) on the "
                         f"full {M}^3 mesh ({fwd:.2f} s)"}
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        peak_src = "measured"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 1900.0, "fallback"
    hbm_peak, hbm_src = measured_hbm_peak()
    achieved = flops / (infer_ms * 1e-3) / 1e12
    line = {"metric": "propagator inferences/s, 70^3 mesh (4->16->16->2, 3x3x3, BF16)",
            "value": 1e3 / infer_ms, "unit": "inferences/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": infer_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "propagator_70", "mesh": M,
                       "l2": "flushed (256 MB write) before each timed inference"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (rec or {}).get("dram_bytes_per_inference"),
                         "peak_source": peak_src, "kernel": "k_conv_sweep (three layers)",
                         "algo_flops_per_inference": flops},
            "roofline_hbm": {"bound": "hbm", "achieved": infer_bytes / (infer_ms * 1e-3) / 1e9,
                             "peak": hbm_peak, "unit": "GB/s",
                             "frac": infer_bytes / (infer_ms * 1e-3) / 1e9 / hbm_peak,
                             "peak_source": hbm_src, "algo_bytes_per_inference": infer_bytes},
            "cpu_baseline": cpu, "e2e": None, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_default_with_configs(args):
    """The headline run, then short runs of the 8.1M ternary blend (config 3,
    the workload whose state exceeds L2) and of the 64-replica batch (config
    4), each with its roofline and CPU baseline, attached to the headline's
    line under "configs"; the headline's keys are those of the run alone."""
    import copy
    global _CAPTURE
    _CAPTURE = []
    try:
        run_ours(args)
        lines = _CAPTURE
    finally:
        _CAPTURE = None
    if not lines:
        return 0
    head = lines[0]
    extras = {}
    for name, fn, over in (("ternary_8m", run_ours,
                            dict(workload="ternary_8m", steps=20, warmup=5, no_e2e=True)),
                           ("replicas64", run_batch,
                            dict(workload="replicas64", steps=40, warmup=10))):
        a2 = copy.copy(args)
        for k, v in over.items():
            setattr(a2, k, v)
        _CAPTURE = []
        try:
            fn(a2)
            sub = _CAPTURE[0] if _CAPTURE else None
            extras[name] = ({k: v for k, v in sub.items() if k not in ("metric", "e2e")}
                            if sub else {"error": "no line"})
        except Exception as exc:  # the headline line is printed regardless
            extras[name] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        finally:
            _CAPTURE = None
    head["configs"] = extras
    emit(head)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "replicas64":
        return run_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "propagator":
        return run_propagator(args)
    default = (args.workload == "a10b10_1m" and args.gpus == 1 and args.thermostat == "langevin"
               and not args.angle_k and not args.dihedral_k
               and int(os.environ.get("WORLD_SIZE", "1")) == 1)
    if default and not args.no_configs:
        return run_default_with_configs(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
