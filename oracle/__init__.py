"""CPU oracle of the hPF-MD step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``hpf_oracle.c`` (plain C,
FP64 with an int64 fixed-point density mesh) through ctypes and shares no code
with the CUDA library.  Parity status per function:

  scatter        pinned (mass conservation, single-bead closed forms, brute force)
  field          pinned (uniform melt -> zero gradient, sinusoid closed form, linearity)
  field_force    pinned (weights sum to one, linear field reproduced, node values)
  bond_force     pinned (two-bead closed form, minus the numerical energy derivative)
  run            pinned (harmonic-oscillator closed form of the discrete scheme,
                 exact velocity decay and stationary variance of the thermostat,
                 NVE energy drift)
  philox/gauss3  pinned against an independent Philox4x32-10 implementation and
                 by moments of the normals
  energy         pinned (kinetic energy of known velocities, bond closed form,
                 field energy derivative equals the potential)
  run (Andersen) pinned (nu = 0 is NVE, force-free velocity autocorrelation
                 (1 - nu dt)^n, collision rate, mean temperature)
  field_force_staggered  pinned (quadratic fields exact, central difference on
                 a vertex, continuity between vertices, sinusoid closed form)
  dihedral_force / dihedral_energy  pinned (closed forms in phi, minus the
                 numerical energy derivative, zero net force and torque)
  run_nh         pinned (NVE limit, free-particle thermostat ODE, extended-energy
                 conservation, mean temperature)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpf_oracle.c")
_LIB = os.path.join(_HERE, "libhpf_oracle.so")
_lock = threading.Lock()
_lib = None

MAX_SPECIES = 8
FRAC_BITS = 13


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast math, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hpf_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int32),
        ("mesh", ctypes.c_int32 * 3),
        ("box", ctypes.c_float * 3),
        ("kT", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("inv_kappa", ctypes.c_double),
        ("chi", ctypes.c_double * (MAX_SPECIES * MAX_SPECIES)),
        ("bond_k", ctypes.c_double),
        ("bond_r0", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("field_every", ctypes.c_int32),
        ("force_mode", ctypes.c_int32),
        ("angle_k", ctypes.c_double),
        ("angle_cos0", ctypes.c_double),
        ("thermostat", ctypes.c_int32),
        ("nh_tau", ctypes.c_double),
        ("andersen_nu", ctypes.c_double),
        ("dihedral_k", ctypes.c_double),
        ("dihedral_n", ctypes.c_int32),
        ("dihedral_delta", ctypes.c_double),
        ("angle_form", ctypes.c_int32),
        ("angle_theta0", ctypes.c_double),
    ]


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER
            i64, i32, u32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double
            pp = P(Params)
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_philox4x32_10.argtypes = [P(u32), P(u32), P(u32)]
            L.orc_gauss3.argtypes = [ctypes.c_uint64, u32, i64, P(f64)]
            L.orc_inv_h.argtypes = [pp, ctypes.c_int]
            L.orc_inv_h.restype = ctypes.c_float
            L.orc_scatter.argtypes = [pp, i64, P(f64), P(i32), P(i64)]
            L.orc_field.argtypes = [pp, P(i64), P(f64), P(f64)]
            L.orc_field_force.argtypes = [pp, i64, P(f64), P(i32), P(f64), P(f64)]
            L.orc_bond_table.argtypes = [i64, i64, P(i32), P(i32), P(i32)]
            L.orc_bond_table.restype = ctypes.c_int
            L.orc_bond_force.argtypes = [pp, i64, P(f64), P(i32), P(i32), P(f64)]
            L.orc_bond_energy.argtypes = [pp, i64, P(f64), P(i32), P(i32)]
            L.orc_bond_energy.restype = f64
            L.orc_angle_force.argtypes = [pp, i64, P(f64), P(i32), P(i32), P(f64)]
            L.orc_angle_energy.argtypes = [pp, i64, P(f64), P(i32), P(i32)]
            L.orc_angle_energy.restype = f64
            L.orc_dihedral_force.argtypes = [pp, i64, P(f64), P(i32), P(i32), P(f64)]
            L.orc_dihedral_energy.argtypes = [pp, i64, P(f64), P(i32), P(i32)]
            L.orc_dihedral_energy.restype = f64
            L.orc_field_energy.argtypes = [pp, P(i64)]
            L.orc_field_energy.restype = f64
            L.orc_field_force_exact.argtypes = [pp, i64, P(f64), P(i32), P(f64), P(f64)]
            L.orc_field_force_staggered.argtypes = [pp, i64, P(f64), P(i32), P(f64), P(f64)]
            L.orc_energy.argtypes = [pp, i64, P(f64), P(f64), P(i32), P(i32), P(i32), P(f64),
                                     P(f64), i64, P(f64)]
            L.orc_run.argtypes = [pp, i64, P(f64), P(f64), P(i32), i64, P(i32), i64, i32, P(f64)]
            L.orc_run.restype = ctypes.c_int
            L.orc_run_nh.argtypes = [pp, i64, P(f64), P(f64), P(i32), i64, P(i32), i64, i32,
                                     P(f64), P(f64)]
            L.orc_run_nh.restype = ctypes.c_int
            L.orc_andersen_collides.argtypes = [pp, u32, i64]
            L.orc_andersen_collides.restype = ctypes.c_int
            L.orc_cell_key.argtypes = [pp, P(f64), i32]
            L.orc_cell_key.restype = i64
            _lib = L
    return _lib


def make_params(n_species, mesh, box, kT=1.0, rho0=3.0, inv_kappa=0.1, chi=None, bond_k=4.0,
                bond_r0=0.7, mass=1.0, dt=0.01, gamma=1.0, seed=42, field_every=1, force_mode=0,
                angle_k=0.0, angle_cos0=-1.0, thermostat=0, nh_tau=1.0, andersen_nu=0.0,
                dihedral_k=0.0, dihedral_n=1, dihedral_delta=0.0, angle_form=0,
                angle_theta0=np.pi, **_ignored):
    p = Params()
    p.n_species = int(n_species)
    m = (mesh,) * 3 if np.isscalar(mesh) else tuple(mesh)
    b = (box,) * 3 if np.isscalar(box) else tuple(box)
    for a in range(3):
        p.mesh[a] = int(m[a])
        p.box[a] = float(b[a])
    p.kT, p.rho0, p.inv_kappa = float(kT), float(rho0), float(inv_kappa)
    c = np.zeros((MAX_SPECIES, MAX_SPECIES))
    if chi is not None:
        chi = np.asarray(chi, dtype=np.float64)
        c[:chi.shape[0], :chi.shape[1]] = chi
    for k in range(MAX_SPECIES * MAX_SPECIES):
        p.chi[k] = float(c.reshape(-1)[k])
    p.bond_k, p.bond_r0, p.mass, p.dt, p.gamma = (float(bond_k), float(bond_r0), float(mass),
                                                  float(dt), float(gamma))
    p.seed = int(seed)
    p.field_every = int(field_every)
    p.force_mode = int(force_mode)
    p.angle_k, p.angle_cos0 = float(angle_k), float(angle_cos0)
    p.thermostat, p.nh_tau = int(thermostat), float(nh_tau)
    p.andersen_nu = float(andersen_nu)
    p.dihedral_k, p.dihedral_n, p.dihedral_delta = (float(dihedral_k), int(dihedral_n),
                                                    float(dihedral_delta))
    p.angle_form, p.angle_theta0 = int(angle_form), float(angle_theta0)
    return p


def num_threads() -> int:
    return lib().orc_num_threads()


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                            _p(out, ctypes.c_uint32))
    return out


def gauss3(seed, tag, step) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_gauss3(int(seed), int(tag), int(step), _p(out, ctypes.c_double))
    return out


def inv_h(p: Params, axis: int) -> float:
    return lib().orc_inv_h(ctypes.byref(p), axis)


def n_nodes(p: Params) -> int:
    return int(p.mesh[0]) * int(p.mesh[1]) * int(p.mesh[2])


def mesh_shape(p: Params):
    return (p.n_species, int(p.mesh[2]), int(p.mesh[1]), int(p.mesh[0]))


def scatter(p: Params, pos, types) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    D = np.zeros(mesh_shape(p), dtype=np.int64)
    lib().orc_scatter(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                      _p(types, ctypes.c_int32), _p(D, ctypes.c_int64))
    return D


def field(p: Params, D):
    D = np.ascontiguousarray(D, dtype=np.int64)
    V = np.zeros(mesh_shape(p))
    G = np.zeros(mesh_shape(p) + (3,))
    lib().orc_field(ctypes.byref(p), _p(D, ctypes.c_int64), _p(V, ctypes.c_double),
                    _p(G, ctypes.c_double))
    return V, G


def field_force(p: Params, pos, types, G) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    G = _f64(G)
    F = np.zeros_like(pos)
    lib().orc_field_force(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                          _p(types, ctypes.c_int32), _p(G, ctypes.c_double),
                          _p(F, ctypes.c_double))
    return F


def bond_table(n, bonds):
    bonds = _i32(np.asarray(bonds).reshape(-1, 2))
    BL = np.zeros((8, max(n, 1)), dtype=np.int32)
    BN = np.zeros(max(n, 1), dtype=np.int32)
    rc = lib().orc_bond_table(n, bonds.shape[0], _p(bonds, ctypes.c_int32),
                              _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32))
    if rc != 0:
        raise ValueError("bad bond list")
    return BL, BN


def bond_force(p: Params, pos, bonds) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    BL, BN = bond_table(pos.shape[0], bonds)
    F = np.zeros_like(pos)
    lib().orc_bond_force(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                         _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32), _p(F, ctypes.c_double))
    return F


def angle_force(p: Params, pos, bonds) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    BL, BN = bond_table(pos.shape[0], bonds)
    F = np.zeros_like(pos)
    lib().orc_angle_force(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                          _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32), _p(F, ctypes.c_double))
    return F


def angle_energy(p: Params, pos, bonds) -> float:
    pos = _f64(pos, (-1, 3))
    BL, BN = bond_table(pos.shape[0], bonds)
    return lib().orc_angle_energy(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                                  _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32))


def bond_energy(p: Params, pos, bonds) -> float:
    pos = _f64(pos, (-1, 3))
    BL, BN = bond_table(pos.shape[0], bonds)
    return lib().orc_bond_energy(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                                 _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32))


def field_energy(p: Params, D) -> float:
    D = np.ascontiguousarray(D, dtype=np.int64)
    return lib().orc_field_energy(ctypes.byref(p), _p(D, ctypes.c_int64))


def field_force_exact(p: Params, pos, types, V) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    V = _f64(V)
    F = np.zeros_like(pos)
    lib().orc_field_force_exact(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                                _p(types, ctypes.c_int32), _p(V, ctypes.c_double),
                                _p(F, ctypes.c_double))
    return F


def field_force_staggered(p: Params, pos, types, V) -> np.ndarray:
    """Algorithm 1's staggered field force (force_mode 2) from the potential V."""
    pos = _f64(pos, (-1, 3))
    types = _i32(types)
    V = _f64(V)
    F = np.zeros_like(pos)
    lib().orc_field_force_staggered(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                                    _p(types, ctypes.c_int32), _p(V, ctypes.c_double),
                                    _p(F, ctypes.c_double))
    return F


def dihedral_force(p: Params, pos, bonds) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    BL, BN = bond_table(pos.shape[0], bonds)
    F = np.zeros_like(pos)
    lib().orc_dihedral_force(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                             _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32), _p(F, ctypes.c_double))
    return F


def dihedral_energy(p: Params, pos, bonds) -> float:
    pos = _f64(pos, (-1, 3))
    BL, BN = bond_table(pos.shape[0], bonds)
    return lib().orc_dihedral_energy(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                                     _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32))


def energy(p: Params, pos, vel, types, bonds, V, G, step) -> np.ndarray:
    pos = _f64(pos, (-1, 3))
    vel = _f64(vel, (-1, 3))
    types = _i32(types)
    BL, BN = bond_table(pos.shape[0], bonds)
    V = _f64(V)
    G = _f64(G)
    out = np.zeros(6)
    lib().orc_energy(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                     _p(vel, ctypes.c_double), _p(types, ctypes.c_int32),
                     _p(BL, ctypes.c_int32), _p(BN, ctypes.c_int32), _p(V, ctypes.c_double),
                     _p(G, ctypes.c_double), int(step), _p(out, ctypes.c_double))
    return out


def run(p: Params, pos, vel, types, bonds, step0, n_steps, energies=False):
    """Advance the state; returns (pos, vel, energies or None).  vel is v_{n-1/2}."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    types = _i32(types)
    bonds = _i32(np.asarray(bonds).reshape(-1, 2))
    E = np.zeros((n_steps + 1, 6)) if energies else None
    rc = lib().orc_run(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                       _p(vel, ctypes.c_double), _p(types, ctypes.c_int32), bonds.shape[0],
                       _p(bonds, ctypes.c_int32), int(step0), int(n_steps),
                       _p(E, ctypes.c_double) if E is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the input")
    return pos, vel, E


def run_nh(p: Params, pos, vel, types, bonds, step0, n_steps, xe=(0.0, 0.0), energies=False):
    """Nose-Hoover NVT (``orc_run_nh``).  Returns (pos, vel, (xi, eta), energies
    or None); vel is v_{n-1/2}, (xi, eta) the thermostat at the middle of the
    last step, energies [n_steps + 1][7] (kinetic, bonded, field, total, |P|,
    T, extended energy)."""
    pos = _f64(pos, (-1, 3)).copy()
    vel = _f64(vel, (-1, 3)).copy()
    types = _i32(types)
    bonds = _i32(np.asarray(bonds).reshape(-1, 2))
    x = np.array(xe, dtype=np.float64)
    E = np.zeros((n_steps + 1, 7)) if energies else None
    rc = lib().orc_run_nh(ctypes.byref(p), pos.shape[0], _p(pos, ctypes.c_double),
                          _p(vel, ctypes.c_double), _p(types, ctypes.c_int32), bonds.shape[0],
                          _p(bonds, ctypes.c_int32), int(step0), int(n_steps),
                          _p(x, ctypes.c_double), _p(E, ctypes.c_double) if E is not None else None)
    if rc != 0:
        raise ValueError("oracle rejected the input")
    return pos, vel, (float(x[0]), float(x[1])), E


def andersen_collides(p: Params, tag: int, step: int) -> bool:
    return bool(lib().orc_andersen_collides(ctypes.byref(p), int(tag), int(step)))


def cell_key(p: Params, x, brick: int) -> int:
    x = _f64(x, (3,))
    return lib().orc_cell_key(ctypes.byref(p), _p(x, ctypes.c_double), int(brick))


def chain_order(p: Params, pos, first_beads, brick: int) -> np.ndarray:
    """Chain order of the bead sort: by (cell key of the first bead, first-bead tag)."""
    keys = [cell_key(p, pos[i], brick) for i in first_beads]
    return np.array(sorted(range(len(first_beads)), key=lambda c: (keys[c], first_beads[c])),
                    dtype=np.int64)
