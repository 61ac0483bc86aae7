"""Chain-partitioned hPF-MD: one system split into parts by whole chains.

The MD-SCF section drives every bead by one field, computed from the density
of all beads.  Split by whole chains, the parts (one context each, e.g. one
per GPU) share nothing between field refreshes: bonds stay inside a part and
the field is frozen.  At a refresh each part's partial int64 density mesh is
summed over the parts (exact and order-independent) and every part computes
the same field from the total.  The library does the stepping, the scatter
and the field (hpf_step_partial); this module only splits the input and
drives the calls, with the sum left to the caller's collective.
"""
from __future__ import annotations

import numpy as np


def chain_starts(n_beads: int, bonds) -> np.ndarray:
    """Tags of the first bead of every chain (bonds join i and i + 1)."""
    has_prev = np.zeros(n_beads, dtype=bool)
    b = np.asarray(bonds).reshape(-1, 2)
    if b.size:
        has_prev[np.maximum(b[:, 0], b[:, 1])] = True
    return np.flatnonzero(~has_prev)


def split_chains(data: dict, parts: int) -> list[tuple[int, dict]]:
    """Split a tag-ordered system into `parts` contiguous runs of whole chains
    of about equal bead counts: [(tag_base, part_data)], part_data holding the
    part's pos, vel, type and bonds (re-indexed from 0)."""
    n = len(data["type"])
    starts = chain_starts(n, data["bonds"])
    cuts = [0]
    for k in range(1, parts):
        j = int(np.searchsorted(starts, round(k * n / parts)))
        cut = int(starts[j]) if j < len(starts) else n
        cuts.append(max(cut, cuts[-1]))
    cuts.append(n)
    bonds = np.asarray(data["bonds"]).reshape(-1, 2)
    out = []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        keep = (bonds[:, 0] >= lo) & (bonds[:, 0] < hi)
        out.append((lo, dict(pos=np.ascontiguousarray(data["pos"][lo:hi]),
                             vel=np.ascontiguousarray(data["vel"][lo:hi]),
                             type=np.ascontiguousarray(data["type"][lo:hi]),
                             bonds=np.ascontiguousarray((bonds[keep] - lo).astype(np.int32)))))
    return out


def step_part(system, n_steps: int, reduce) -> int:
    """Advance one part by n_steps through hpf_step_partial; at every field
    refresh `reduce(mesh)` must leave in `mesh` (this part's int64 mesh, a
    device tensor) the sum over all parts, e.g. an all-reduce.  Every part
    makes the same calls, so the collectives match up.  Returns the number of
    exchanges."""
    left, exchanges = int(n_steps), 0
    while True:
        done, mesh = system.step_partial(left)
        left -= done
        if mesh is None:
            return exchanges
        reduce(mesh)
        exchanges += 1


def step_parts_local(systems, n_steps: int) -> int:
    """All parts in this process (on one device): the meshes are summed with
    device adds, in place in every part's mesh."""
    left = [int(n_steps)] * len(systems)
    exchanges = 0
    while True:
        out = [s.step_partial(k) for s, k in zip(systems, left)]
        left = [k - d for k, (d, _) in zip(left, out)]
        meshes = [m for _, m in out]
        if meshes[0] is None:
            if any(m is not None for m in meshes):
                raise RuntimeError("parts disagree on the refresh schedule")
            return exchanges
        if any(m is None for m in meshes):
            raise RuntimeError("parts disagree on the refresh schedule")
        total = meshes[0].clone()
        for m in meshes[1:]:
            total += m
        for m in meshes:
            m.copy_(total)
        exchanges += 1
