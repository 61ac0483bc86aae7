"""Seeded synthetic workloads for the hPF-MD step.

This module only builds inputs: bead positions, velocities, species and bonds
for the polymer systems the step is run on, plus the physical parameters that
go with them.  It holds none of the method's arithmetic (no density, field,
force or integrator code), so both the CUDA path and the CPU oracle can be fed
from it without sharing any of the method.

The paper's own hPF benchmarks (DPPC/water, section "Simulating phospholipids
in water with MD-SCF") need a coarse-grained lipid model that is not available,
so the systems here are generic block-copolymer and blend melts at the same
reduced density (rho0 = 3) and mesh spacing (about 1 sigma) used for MD-SCF
melts.  Chains are random walks of fixed step length from uniform random
starts; positions are kept unwrapped (the periodic box is applied in mesh-index
space only).  Velocities are Maxwell-Boltzmann at kT/m with the centre-of-mass
velocity removed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

MAX_SPECIES = 8


@dataclass
class Workload:
    """One synthetic hPF-MD system.

    ``blocks`` lists the chain families: ``(n_chains, species_sequence)``; a
    sequence of length 1 is an unbonded solvent bead.  Beads are numbered
    family by family, chain by chain, bead by bead; that numbering is the bead
    tag used everywhere (outputs are returned in tag order).
    """

    name: str
    blocks: list
    box: float
    mesh: int
    n_species: int
    chi: list  # [S][S] in kT units, symmetric, zero diagonal
    inv_kappa: float
    field_every: int
    steps: int
    rho0: float = 3.0
    kT: float = 1.0
    bond_k: float = 4.0
    bond_r0: float = 0.7
    mass: float = 1.0
    dt: float = 0.01
    gamma: float = 1.0
    seed: int = 42
    walk_step: float = 0.7
    extra: dict = field(default_factory=dict)

    @property
    def n_beads(self) -> int:
        return sum(n * len(seq) for n, seq in self.blocks)

    def params(self) -> dict:
        """Physical parameters as plain Python values (for both sides)."""
        S = self.n_species
        chi = np.zeros((MAX_SPECIES, MAX_SPECIES))
        chi[:S, :S] = np.asarray(self.chi, dtype=np.float64)
        return dict(
            n_beads=self.n_beads,
            n_species=S,
            mesh=(self.mesh, self.mesh, self.mesh),
            box=(self.box, self.box, self.box),
            kT=self.kT,
            rho0=self.rho0,
            inv_kappa=self.inv_kappa,
            chi=chi,
            bond_k=self.bond_k,
            bond_r0=self.bond_r0,
            mass=self.mass,
            dt=self.dt,
            gamma=self.gamma,
            seed=self.seed,
            field_every=self.field_every,
        )


def _chi2(chi_ab: float) -> list:
    return [[0.0, chi_ab], [chi_ab, 0.0]]


def a5b5_10k() -> Workload:
    """1,000 A5B5 diblocks = 10,000 beads, L = 14.94, mesh 15^3, field every step."""
    return Workload("a5b5_10k", [(1000, [0] * 5 + [1] * 5)], 14.94, 15, 2,
                    _chi2(1.0), 0.1, field_every=1, steps=100)


def a10b10_1m() -> Workload:
    """50,000 A10B10 diblocks = 1,000,000 beads, L = 69.3, mesh 70^3, field every 10 steps."""
    return Workload("a10b10_1m", [(50000, [0] * 10 + [1] * 10)], 69.3, 70, 2,
                    _chi2(0.5), 0.1, field_every=10, steps=10000)


def ternary_8m() -> Workload:
    """A20 + B20 homopolymers (45 % + 45 % of beads) + 10 % solvent S = 8,100,000 beads."""
    chi = [[0.0, 1.2, 0.3], [1.2, 0.0, 0.8], [0.3, 0.8, 0.0]]
    return Workload("ternary_8m", [(182250, [0] * 20), (182250, [1] * 20), (810000, [2])],
                    139.2, 140, 3, chi, 0.05, field_every=5, steps=200)


def diblock(n_chains: int, n_a: int, n_b: int, box: float, mesh: int, chi_ab: float,
            inv_kappa: float = 0.1, field_every: int = 1, seed: int = 42, name: str = "diblock",
            **kw) -> Workload:
    """A small AnBm melt for tests (any size, any mesh)."""
    return Workload(name, [(n_chains, [0] * n_a + [1] * n_b)], box, mesh, 2, _chi2(chi_ab),
                    inv_kappa, field_every=field_every, steps=10, seed=seed, **kw)


def replica_set(n_replicas: int = 64, seed: int = 42) -> list:
    """64 A8B12 melts of uneven size: N_r = 20 (1000 + floor(u_r * 4001)) in [20k, 100k],
    L_r = (N_r / 3)^(1/3), mesh M_r = round(L_r), chi_r = 0.2 + 1.8 r / 63."""
    rng = np.random.Generator(np.random.Philox(key=seed + 1))
    out = []
    for r in range(n_replicas):
        n_chains = 1000 + int(math.floor(rng.random() * 4001))
        n = 20 * n_chains
        L = (n / 3.0) ** (1.0 / 3.0)
        chi_ab = 0.2 + 1.8 * r / max(n_replicas - 1, 1)
        out.append(Workload(f"replica{r:02d}", [(n_chains, [0] * 8 + [1] * 12)], L, int(round(L)),
                            2, _chi2(chi_ab), 0.1, field_every=10, steps=5000, seed=seed + r))
    return out


WORKLOADS = {
    "a5b5_10k": a5b5_10k,
    "a10b10_1m": a10b10_1m,
    "ternary_8m": ternary_8m,
}


def _unit_vectors(rng: np.random.Generator, shape) -> np.ndarray:
    """Uniform directions on the sphere (z uniform in [-1,1], azimuth uniform)."""
    z = rng.uniform(-1.0, 1.0, size=shape)
    a = rng.uniform(0.0, 2.0 * np.pi, size=shape)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(a), r * np.sin(a), z], axis=-1)


def generate(w: Workload, seed: int | None = None) -> dict:
    """Build the bead state of ``w``.

    Returns a dict of numpy arrays in tag order:
      pos   float32 [N,3]  unwrapped positions (chain starts uniform in [0,L)^3)
      vel   float32 [N,3]  Maxwell velocities at kT/m, total momentum removed
      type  int32   [N]    species index
      bonds int32   [B,2]  bonded bead pairs (i, i+1) along each chain
    """
    seed = w.seed if seed is None else seed
    rng = np.random.Generator(np.random.Philox(key=seed))
    pos_parts, type_parts, bond_parts = [], [], []
    base = 0
    for n_chains, seq in w.blocks:
        clen = len(seq)
        start = rng.uniform(0.0, w.box, size=(n_chains, 1, 3))
        if clen > 1:
            steps = w.walk_step * _unit_vectors(rng, (n_chains, clen - 1))
            walk = np.concatenate([np.zeros((n_chains, 1, 3)), np.cumsum(steps, axis=1)], axis=1)
        else:
            walk = np.zeros((n_chains, 1, 3))
        pos_parts.append((start + walk).reshape(-1, 3))
        type_parts.append(np.tile(np.asarray(seq, dtype=np.int32), n_chains))
        if clen > 1:
            first = base + clen * np.arange(n_chains, dtype=np.int64)[:, None]
            i = (first + np.arange(clen - 1, dtype=np.int64)[None, :]).reshape(-1)
            bond_parts.append(np.stack([i, i + 1], axis=1))
        base += n_chains * clen
    pos = np.concatenate(pos_parts).astype(np.float32)
    types = np.concatenate(type_parts).astype(np.int32)
    n = pos.shape[0]
    vel = rng.normal(0.0, math.sqrt(w.kT / w.mass), size=(n, 3))
    vel -= vel.mean(axis=0, keepdims=True)
    bonds = (np.concatenate(bond_parts).astype(np.int32) if bond_parts
             else np.zeros((0, 2), dtype=np.int32))
    return dict(pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel.astype(np.float32)),
                type=types, bonds=np.ascontiguousarray(bonds))


def with_bond_angles(w: Workload, data: dict, theta_deg=(100.0, 140.0), seed: int = 0) -> dict:
    """The same melt with every chain rebuilt bead by bead from its first
    bead: bond length walk_step, each bond angle drawn uniformly in
    theta_deg (degrees) and each torsion uniformly, so no three consecutive
    beads start near collinear (where a dihedral is undefined).  Types,
    bonds and velocities are kept."""
    rng = np.random.Generator(np.random.Philox(key=seed + 7))
    pos = data["pos"].astype(np.float64).copy()
    b = w.walk_step
    base = 0

    def unit(v):
        return v / np.linalg.norm(v, axis=-1, keepdims=True)

    for n_chains, seq in w.blocks:
        clen = len(seq)
        if clen >= 2:
            x = pos[base:base + n_chains * clen].reshape(n_chains, clen, 3)
            v = _unit_vectors(rng, (n_chains,))
            x[:, 1] = x[:, 0] + b * v
            u = _unit_vectors(rng, (n_chains,))
            u = unit(u - np.sum(u * v, axis=1, keepdims=True) * v)
            for k in range(2, clen):
                th = np.radians(rng.uniform(theta_deg[0], theta_deg[1], size=(n_chains, 1)))
                ph = rng.uniform(-np.pi, np.pi, size=(n_chains, 1))
                t = unit(x[:, k - 1] - x[:, k - 2])
                n1 = unit(np.cross(t, u))
                m1 = np.cross(n1, t)
                d = -np.cos(th) * t + np.sin(th) * (np.cos(ph) * m1 + np.sin(ph) * n1)
                x[:, k] = x[:, k - 1] + b * d
                u = t
            pos[base:base + n_chains * clen] = x.reshape(-1, 3)
        base += n_chains * clen
    out = dict(data)
    out["pos"] = np.ascontiguousarray(pos.astype(np.float32))
    return out
