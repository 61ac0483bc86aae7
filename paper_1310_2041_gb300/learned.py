"""Training and evaluation driver of the learned density propagator.

Marshalling and bookkeeping only: densities come from the library's CIC
scatter (``System.density_phi``), the network runs and trains in the
library's BF16 tensor-core kernels (``Propagator``), and field-force errors
are the library's judge (``System.judge_density``).  Snapshot meshes stay in
device memory (torch tensors) between calls.
"""
from __future__ import annotations

import numpy as np

from . import hpf


CHANNELS = ((4, 16), (16, 16), (16, 2))


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded He-uniform initial weights (bound sqrt(6 / fan_in), fan_in = 27 C_in;
    the last layer scaled by 0.1, biases zero) as the flat FP32 parameter vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for k, (ci, co) in enumerate(CHANNELS):
        bound = np.sqrt(6.0 / (27 * ci)) * (0.1 if k == len(CHANNELS) - 1 else 1.0)
        parts.append(rng.uniform(-bound, bound, size=27 * ci * co))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def collect_snapshots(system: hpf.System, n_snap: int, K: int, out=None):
    """phi of the current positions, then K steps, n_snap times.

    ``out``: optional preallocated float32 tensor [n_snap, S, Mz, My, Mx] (CUDA
    for device-resident snapshots).  Returns it."""
    import torch
    shape = (n_snap,) + system.mesh_shape
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device="cuda")
    for k in range(n_snap):
        system.density_phi(out[k])
        if k + 1 < n_snap:
            system.step(K)
    return out


def triples(n_snap: int):
    """Indices k with a training example (phi[k-1], phi[k]) -> phi[k+1]."""
    return list(range(1, n_snap - 1))


def change_scale(snaps, examples=None) -> float:
    """The change scale s for a network trained on ``snaps``: the inverse RMS
    of the input changes phi[k] - phi[k - 1] over the examples, so that the
    network reads and writes changes of order one."""
    ex = triples(snaps.shape[0]) if examples is None else list(examples)
    ms = [float(((snaps[k] - snaps[k - 1]).double() ** 2).mean()) for k in ex]
    rms = float(np.sqrt(np.mean(ms)))
    return 1.0 / rms if rms > 0.0 else 1.0


def train(prop: hpf.Propagator, snaps, iters: int, lr: float = 2e-3, lr_final: float = 2e-4,
          examples=None, seed: int = 0, log_every: int = 0):
    """Adam on the mean squared error of the predicted change, one example per
    step in a seeded random order, learning rate decayed geometrically from lr
    to lr_final.  Returns the loss log [(iteration, loss)]."""
    ex = triples(snaps.shape[0]) if examples is None else list(examples)
    rng = np.random.default_rng(seed)
    order = []
    log = []
    decay = (lr_final / lr) ** (1.0 / max(iters - 1, 1))
    for it in range(iters):
        if not order:
            order = list(rng.permutation(ex))
        k = int(order.pop())
        x = snaps[k - 1:k + 1]  # phi(t - K), phi(t): 4 contiguous channels
        want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
        loss = prop.train_step(x, snaps[k + 1], lr * decay ** it, want_loss=want)
        if want:
            log.append((it, loss))
    return log


def validation_loss(prop: hpf.Propagator, snaps, examples):
    """Mean squared error of the predicted change over examples: of the
    network, of predicting no change, and of linear extrapolation
    (phi[k] - phi[k - 1])."""
    net, zero, lin = [], [], []
    s2 = prop.scale ** 2
    for k in examples:
        x = snaps[k - 1:k + 1]
        net.append(prop.backward(x, snaps[k + 1])[0] / s2)
        d = (snaps[k + 1] - snaps[k]).double()
        zero.append(float((d * d).mean()))
        e = d - (snaps[k] - snaps[k - 1]).double()
        lin.append(float((e * e).mean()))
    return float(np.mean(net)), float(np.mean(zero)), float(np.mean(lin))


def judge_candidates(system: hpf.System, prop: hpf.Propagator | None, n_windows: int, K: int,
                     lags=(1, 2, 5, 10, 20)):
    """Field-force errors (the judge's eps) of density candidates along a plain
    trajectory of ``system`` (which should refresh its field every step).

    For every lag L in ``lags``: hold-last phi(t) and linear extrapolation
    2 phi(t) - phi(t - L), judged at t + L.  With a network (trained for lag
    K): phi(t) + net(phi(t - K), phi(t)) judged at t + K.  Returns
    {name: [eps per judged point]}."""
    import torch
    H = 2 * max(max(lags), K)
    hist = torch.empty((H + 1,) + system.mesh_shape, dtype=torch.float32, device="cuda")
    res = {f"hold_{L}": [] for L in lags}
    res.update({f"linear_{L}": [] for L in lags})
    res["net"] = []
    res["hold_net"] = []
    n_steps = n_windows * K + H
    for s in range(n_steps + 1):
        cur = hist[s % (H + 1)]
        system.density_phi(cur)
        if s >= H:
            for L in lags:
                if (s - H) % L == 0:
                    prev = hist[(s - L) % (H + 1)]
                    prev2 = hist[(s - 2 * L) % (H + 1)]
                    res[f"hold_{L}"].append(system.judge_density(prev))
                    res[f"linear_{L}"].append(system.judge_density(2 * prev - prev2))
            if prop is not None and (s - H) % K == 0:
                a, b = hist[(s - 2 * K) % (H + 1)], hist[(s - K) % (H + 1)]
                x = torch.cat([a, b]).contiguous()
                pred = prop.rollout(x, 1, out=torch.empty_like(b))   # phi(t) + net(...)
                res["net"].append(system.judge_density(pred))
                res["hold_net"].append(system.judge_density(b))
        if s < n_steps:
            system.step(1)
    return res


def rollout(prop: hpf.Propagator, prev, cur, K: int):
    """Autoregressive use of a network trained at lag 1: from phi(t - 1) = prev
    and phi(t) = cur, predict phi(t + 1) = phi(t) + net(phi(t - 1), phi(t)),
    then feed the prediction back, K times (hpf_prop_rollout).  Returns the
    predicted phi(t + K)."""
    import torch
    x = torch.cat([prev, cur]).contiguous()
    return prop.rollout(x, K, out=torch.empty_like(cur))


def judge_rollout(system: hpf.System, prop: hpf.Propagator, n_windows: int, K: int):
    """The judge's eps of K-step autoregressive rollouts of a lag-1 network
    along a plain trajectory of ``system`` (which should refresh its field
    every step): each window starts from the true phi(t - 1), phi(t) and is
    judged at t + K.  Returns [eps per window]."""
    import torch
    shape = system.mesh_shape
    prev = torch.empty(shape, dtype=torch.float32, device="cuda")
    cur = torch.empty_like(prev)
    system.density_phi(prev)
    system.step(1)
    system.density_phi(cur)
    res = []
    for _ in range(n_windows):
        pred = rollout(prop, prev, cur, K)
        system.step(K - 1)
        system.density_phi(prev)
        system.step(1)
        system.density_phi(cur)
        res.append(system.judge_density(pred))
    return res


def collect_smoothed(system: hpf.System, n_snap: int, K: int, passes: int):
    """collect_snapshots with every phi passed through the binomial filter
    (hpf_smooth_phi) in place."""
    snaps = collect_snapshots(system, n_snap, K)
    for k in range(n_snap):
        system.smooth_phi(snaps[k], passes, out=snaps[k])
    return snaps


def judge_smoothed(system: hpf.System, passes: int, prop: hpf.Propagator | None,
                   n_windows: int, K: int, lags=(1, 2, 5, 10, 20)):
    """The smoothed-density variant of judge_candidates: every density, the
    true one included, passes through the binomial filter before its field is
    formed (hpf_smooth_phi), and eps compares a candidate's field force with
    that of the smoothed true density at the same positions
    (hpf_judge_density_pair).  Candidates: hold-last s(t - L), linear
    extrapolation 2 s(t - L) - s(t - 2 L), and with a network trained on
    smoothed snapshots at lag K its prediction from (s(t - 2K), s(t - K)).
    ``system`` should refresh its field every step.  Returns {name: [eps]}."""
    import torch
    H = 2 * max(max(lags), K)
    hist = torch.empty((H + 1,) + system.mesh_shape, dtype=torch.float32, device="cuda")
    res = {f"hold_{L}": [] for L in lags}
    res.update({f"linear_{L}": [] for L in lags})
    res["net"] = []
    n_steps = n_windows * K + H
    for s in range(n_steps + 1):
        cur = hist[s % (H + 1)]
        system.density_phi(cur)
        system.smooth_phi(cur, passes, out=cur)
        if s >= H:
            for L in lags:
                if (s - H) % L == 0:
                    prev = hist[(s - L) % (H + 1)]
                    prev2 = hist[(s - 2 * L) % (H + 1)]
                    res[f"hold_{L}"].append(system.judge_density_pair(prev, cur))
                    res[f"linear_{L}"].append(system.judge_density_pair(2 * prev - prev2, cur))
            if prop is not None and (s - H) % K == 0:
                a, b = hist[(s - 2 * K) % (H + 1)], hist[(s - K) % (H + 1)]
                pred = prop.rollout(torch.cat([a, b]).contiguous(), 1, out=torch.empty_like(b))
                res["net"].append(system.judge_density_pair(pred, cur))
        if s < n_steps:
            system.step(1)
    return res
