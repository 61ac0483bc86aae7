"""Thin Python binding of libhpf.so (the C ABI of include/hpf.h).

Argument marshalling only: every step of the hPF-MD path runs in the CUDA
library.  Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA); the library copies through the pointer with cudaMemcpyDefault.  The
library must have been built (``python -m paper_1310_2041_gb300.build``);
there is no fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

MAX_SPECIES = 8
FORCE_FIELD = 1
FORCE_BOND = 2
STAGES = ("scatter", "field", "step", "sort", "energy", "other")

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhpf.so")
_lib = None
_lock = threading.Lock()

STATUS = {0: "HPF_OK", 1: "HPF_ERR_INVALID", 2: "HPF_ERR_CUDA", 3: "HPF_ERR_NOMEM",
          4: "HPF_ERR_OVERFLOW", 5: "HPF_ERR_NONFINITE", 6: "HPF_ERR_TIMEOUT",
          7: "HPF_ERR_STATE"}


class HPFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of hpf_params."""
    _fields_ = [
        ("n_beads", ctypes.c_int32),
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
        ("sort_every", ctypes.c_int32),
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


class LearnedStats(ctypes.Structure):
    """Mirror of hpf_learned_stats."""
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("windows", ctypes.c_int32),
        ("learned", ctypes.c_int32),
        ("rejected", ctypes.c_int32),
        ("plain", ctypes.c_int32),
        ("judged", ctypes.c_int32),
        ("eps_last", ctypes.c_double),
        ("eps_max", ctypes.c_double),
        ("eps_sum", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def load():
    """Load libhpf.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_1310_2041_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.hpf_status_string.restype = ctypes.c_char_p
        L.hpf_status_string.argtypes = [ctypes.c_int]
        L.hpf_last_error.restype = ctypes.c_char_p
        L.hpf_last_error.argtypes = [vp]
        L.hpf_init.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
        L.hpf_destroy.argtypes = [vp]
        L.hpf_set_state.argtypes = [vp, vp, vp, vp, vp, i64, i64]
        L.hpf_get_state.argtypes = [vp, vp, vp, ctypes.POINTER(i64)]
        L.hpf_update_state.argtypes = [vp, vp, vp, i64]
        L.hpf_upload_state.argtypes = [vp, vp, vp]
        L.hpf_apply_state.argtypes = [vp, i64]
        L.hpf_energy_start.argtypes = [vp]
        L.hpf_energy_finish.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_get_order.argtypes = [vp, vp]
        L.hpf_field_tile.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.hpf_set_field_tile.argtypes = [vp, i32]
        L.hpf_scatter_density.argtypes = [vp, vp]
        L.hpf_field.argtypes = [vp, vp, vp]
        L.hpf_forces.argtypes = [vp, vp, i32]
        L.hpf_step.argtypes = [vp, i32]
        L.hpf_set_tag_base.argtypes = [vp, i64]
        L.hpf_step_partial.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(vp)]
        L.hpf_energy.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_get_thermostat.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_set_thermostat.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_nh_conserved.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_selftest_timeout.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_selftest_timeout.restype = ctypes.c_int
        L.hpf_batch_init.argtypes = [ctypes.POINTER(Params), i32, vp, ctypes.POINTER(vp)]
        L.hpf_batch_replica.argtypes = [vp, i32]
        L.hpf_batch_replica.restype = vp
        L.hpf_batch_step.argtypes = [vp, i32]
        L.hpf_batch_use_graphs.argtypes = [vp, i32]
        L.hpf_batch_energy.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        L.hpf_batch_destroy.argtypes = [vp]
        for name in ("hpf_batch_init", "hpf_batch_step", "hpf_batch_use_graphs",
                     "hpf_batch_destroy", "hpf_batch_energy"):
            getattr(L, name).restype = ctypes.c_int
        L.hpf_profile.argtypes = [vp, i32]
        L.hpf_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]
        fp, dp = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
        L.hpf_prop_init.argtypes = [ctypes.POINTER(i32), vp, ctypes.POINTER(vp)]
        L.hpf_prop_destroy.argtypes = [vp]
        L.hpf_prop_param_count.restype = i32
        L.hpf_prop_param_count.argtypes = []
        L.hpf_prop_set_weights.argtypes = [vp, vp]
        L.hpf_prop_get_weights.argtypes = [vp, vp]
        L.hpf_prop_set_scale.argtypes = [vp, ctypes.c_float]
        L.hpf_prop_get_scale.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.hpf_prop_set_ctas.argtypes = [vp, i32]
        L.hpf_prop_selftest_timeout.argtypes = [vp, dp]
        L.hpf_prop_forward.argtypes = [vp, vp, vp]
        L.hpf_prop_rollout.argtypes = [vp, vp, i32, vp]
        L.hpf_prop_backward.argtypes = [vp, vp, vp, vp, dp]
        L.hpf_prop_adam_step.argtypes = [vp, vp, ctypes.c_float]
        L.hpf_prop_train_step.argtypes = [vp, vp, vp, ctypes.c_float, dp]
        L.hpf_density_phi.argtypes = [vp, vp]
        L.hpf_judge_density.argtypes = [vp, vp, dp]
        L.hpf_smooth_phi.argtypes = [vp, vp, vp, i32]
        L.hpf_learned_mode.argtypes = [vp, i32]
        L.hpf_judge_density_pair.argtypes = [vp, vp, vp, dp]
        L.hpf_step_learned.argtypes = [vp, vp, i32, i32, ctypes.c_double,
                                       ctypes.POINTER(LearnedStats)]
        for name in ("hpf_prop_init", "hpf_prop_destroy", "hpf_prop_set_weights",
                     "hpf_prop_set_scale", "hpf_prop_get_scale", "hpf_prop_set_ctas",
                     "hpf_prop_selftest_timeout",
                     "hpf_prop_get_weights", "hpf_prop_forward", "hpf_prop_rollout",
                     "hpf_prop_backward",
                     "hpf_prop_adam_step", "hpf_prop_train_step", "hpf_density_phi",
                     "hpf_judge_density", "hpf_step_learned", "hpf_smooth_phi", "hpf_learned_mode",
                     "hpf_judge_density_pair"):
            getattr(L, name).restype = ctypes.c_int
        del fp
        for name in ("hpf_init", "hpf_destroy", "hpf_set_state", "hpf_get_state", "hpf_update_state",
                     "hpf_scatter_density", "hpf_field", "hpf_forces", "hpf_step", "hpf_energy",
                     "hpf_profile", "hpf_profile_read", "hpf_get_order", "hpf_field_tile",
                     "hpf_set_field_tile", "hpf_get_thermostat", "hpf_set_thermostat",
                     "hpf_nh_conserved", "hpf_set_tag_base", "hpf_step_partial"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return _lib


def make_params(n_beads, n_species, mesh, box, kT=1.0, rho0=3.0, inv_kappa=0.1, chi=None,
                bond_k=4.0, bond_r0=0.7, mass=1.0, dt=0.01, gamma=1.0, seed=42, field_every=1,
                sort_every=0, force_mode=0, angle_k=0.0, angle_cos0=-1.0, thermostat=0, nh_tau=1.0,
                andersen_nu=0.0, dihedral_k=0.0, dihedral_n=1, dihedral_delta=0.0,
                angle_form=0, angle_theta0=np.pi, **_ignored) -> Params:
    p = Params()
    p.n_beads, p.n_species = int(n_beads), int(n_species)
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
    for k, v in enumerate(c.reshape(-1)):
        p.chi[k] = float(v)
    p.bond_k, p.bond_r0, p.mass, p.dt, p.gamma = (float(bond_k), float(bond_r0), float(mass),
                                                  float(dt), float(gamma))
    p.seed = int(seed)
    p.field_every, p.sort_every = int(field_every), int(sort_every)
    p.force_mode = int(force_mode)
    p.angle_k, p.angle_cos0 = float(angle_k), float(angle_cos0)
    p.thermostat, p.nh_tau = int(thermostat), float(nh_tau)
    p.andersen_nu = float(andersen_nu)
    p.dihedral_k, p.dihedral_n = float(dihedral_k), int(dihedral_n)
    p.dihedral_delta = float(dihedral_delta)
    p.angle_form, p.angle_theta0 = int(angle_form), float(angle_theta0)
    return p


def _ptr(a, dtype, shape=None, name="array"):
    """Raw pointer of a numpy array or torch tensor after dtype / layout checks."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            a = np.ascontiguousarray(a, dtype=dtype)
        if shape is not None and a.size != int(np.prod(shape)):
            raise ValueError(f"{name}: expected {shape}, got {a.shape}")
        return a.ctypes.data, a
    import torch  # tensors only
    tdt = {np.float32: torch.float32, np.int32: torch.int32, np.int64: torch.int64,
           np.float64: torch.float64}[np.dtype(dtype).type]
    if a.dtype != tdt or not a.is_contiguous():
        raise ValueError(f"{name}: needs a contiguous {tdt} tensor")
    if shape is not None and a.numel() != int(np.prod(shape)):
        raise ValueError(f"{name}: expected {shape}, got {tuple(a.shape)}")
    return a.data_ptr(), a


class _CudaArray:
    """A device buffer described by __cuda_array_interface__ (version 3)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape),
                                         "typestr": typestr, "data": (int(ptr), False),
                                         "strides": None, "version": 3}


def device_view(ptr, shape, typestr):
    """A torch tensor over library-owned device memory (no copy; the library
    keeps ownership)."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


def current_stream_handle():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class System:
    """One hPF-MD context (hpf_init ... hpf_destroy)."""

    @classmethod
    def _borrow(cls, lib, handle, params):
        """A non-owning view of a context that a batch owns."""
        s = cls.__new__(cls)
        s.lib, s.p, s.h, s._owned = lib, params, ctypes.c_void_p(handle), False
        s.stream = 0
        s.n, s.S = params.n_beads, params.n_species
        s.mesh_shape = (s.S, params.mesh[2], params.mesh[1], params.mesh[0])
        return s

    def __init__(self, params: Params | dict, stream=None):
        self._owned = True
        self.lib = load()
        self.p = params if isinstance(params, Params) else make_params(**params)
        if stream is None:
            stream = current_stream_handle()
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        h = ctypes.c_void_p()
        self._check(self.lib.hpf_init(ctypes.byref(self.p), ctypes.c_void_p(self.stream),
                                      ctypes.byref(h)), None)
        self.h = h
        self.n = self.p.n_beads
        self.S = self.p.n_species
        self.mesh_shape = (self.S, self.p.mesh[2], self.p.mesh[1], self.p.mesh[0])

    def _check(self, status, h=...):
        if status != 0:
            handle = self.h if h is ... else h
            msg = self.lib.hpf_last_error(handle).decode() if handle else ""
            raise HPFError(status, msg or self.lib.hpf_status_string(status).decode())

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                self.lib.hpf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- state
    def set_state(self, pos, vel, types, bonds, step=0):
        n = self.n
        pp, _a = _ptr(pos, np.float32, (n, 3), "pos")
        vp, _b = _ptr(vel, np.float32, (n, 3), "vel")
        tp, _c = _ptr(types, np.int32, (n,), "type")
        nb = 0 if bonds is None else (bonds.shape[0] if hasattr(bonds, "shape") else len(bonds))
        if bonds is not None and isinstance(bonds, (list, tuple)):
            bonds = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
        bp, _d = _ptr(bonds, np.int32, (nb, 2), "bonds") if nb else (None, None)
        self._check(self.lib.hpf_set_state(self.h, pp, vp, tp, bp, nb, int(step)))

    def update_state(self, pos, vel, step):
        """New positions and velocities (tag order), same topology and bead order."""
        pp, _a = _ptr(pos, np.float32, (self.n, 3), "pos")
        vp, _b = _ptr(vel, np.float32, (self.n, 3), "vel")
        self._check(self.lib.hpf_update_state(self.h, pp, vp, int(step)))

    # ---- pipelined state upload (double-buffered staging, own copy stream)
    def upload_state(self, pos, vel):
        """Start copying new positions and velocities (tag order); returns at
        once.  The copy is not ordered after other GPU work: device arrays
        must be complete when this is called.  The arrays are kept referenced
        here until a synchronising call has covered the apply_state that
        consumes them (energy or get_state after it, or energy_finish of an
        energy_start issued after it)."""
        pp, a = _ptr(pos, np.float32, (self.n, 3), "pos")
        vp, b = _ptr(vel, np.float32, (self.n, 3), "vel")
        self._check(self.lib.hpf_upload_state(self.h, pp, vp))
        self._uploads().append([(pos, vel, a, b), False])

    def apply_state(self, step):
        """Replace the state with the pending upload (the stream waits for its copy)."""
        self._check(self.lib.hpf_apply_state(self.h, int(step)))
        for u in self._uploads():
            u[1] = True

    def _uploads(self):
        if not hasattr(self, "_up"):
            self._up = []
        return self._up

    def _synced(self, applied=None):
        # uploads applied before a synchronising point have been copied
        # (applied: the uploads that had been applied at that point)
        done = applied if applied is not None else [u for u in self._uploads() if u[1]]
        self._up = [u for u in self._uploads() if not any(u is d for d in done)]

    def energy_start(self):
        """Enqueue the observables of the current step (see energy_finish)."""
        self._check(self.lib.hpf_energy_start(self.h))
        self._energy_applied = [u for u in self._uploads() if u[1]]

    def energy_finish(self):
        """The six observables of the step energy_start was called at; waits
        only for the work enqueued up to energy_start (later work, such as the
        next step's apply_state and step, may still be running)."""
        out = (ctypes.c_double * 6)()
        self._check(self.lib.hpf_energy_finish(self.h, out))
        self._synced(getattr(self, "_energy_applied", []))
        self._energy_applied = []
        return np.array(list(out))

    def get_state(self, pos=None, vel=None):
        if pos is None:
            pos = np.empty((self.n, 3), dtype=np.float32)
        if vel is None:
            vel = np.empty((self.n, 3), dtype=np.float32)
        step = ctypes.c_int64()
        pp, _a = _ptr(pos, np.float32, (self.n, 3), "pos")
        vp, _b = _ptr(vel, np.float32, (self.n, 3), "vel")
        self._check(self.lib.hpf_get_state(self.h, pp, vp, ctypes.byref(step)))
        self._synced()
        return pos, vel, step.value

    def order(self, out=None):
        """Tags in the library's storage order (the locality sort's permutation)."""
        if out is None:
            out = np.empty(self.n, dtype=np.int32)
        op, _a = _ptr(out, np.int32, (self.n,), "order")
        self._check(self.lib.hpf_get_order(self.h, op))
        return out

    def field_tile(self):
        """(tile shape (x, y, z), staged by TMA) chosen for this mesh; zeros before the first field."""
        shape = (ctypes.c_int32 * 3)()
        tma = ctypes.c_int32()
        self._check(self.lib.hpf_field_tile(self.h, shape, ctypes.byref(tma)))
        return tuple(shape), bool(tma.value)

    def force_field_tile(self, tile):
        """Pin the stencil to candidate `tile` (0..7), or -1 to autotune again."""
        self._check(self.lib.hpf_set_field_tile(self.h, int(tile)))

    # ---- the path
    def scatter_density(self, out=None):
        if out is None:
            out = np.empty(self.mesh_shape, dtype=np.int64)
        op, _a = _ptr(out, np.int64, self.mesh_shape, "D_out")
        self._check(self.lib.hpf_scatter_density(self.h, op))
        return out

    def field(self, D_in=None, out=None):
        if out is None:
            out = np.empty(self.mesh_shape + (4,), dtype=np.float32)
        dp, _a = _ptr(D_in, np.int64, self.mesh_shape, "D_in")
        op, _b = _ptr(out, np.float32, self.mesh_shape + (4,), "field_out")
        self._check(self.lib.hpf_field(self.h, dp, op))
        return out

    def forces(self, which=FORCE_FIELD | FORCE_BOND, out=None):
        if out is None:
            out = np.empty((self.n, 3), dtype=np.float32)
        op, _a = _ptr(out, np.float32, (self.n, 3), "F_out")
        self._check(self.lib.hpf_forces(self.h, op, int(which)))
        return out

    def step(self, n_steps=1):
        self._check(self.lib.hpf_step(self.h, int(n_steps)))

    # ---- chain-partitioned runs
    def set_tag_base(self, tag_base):
        """This part's beads are tags tag_base .. tag_base + n - 1 of the system."""
        self._check(self.lib.hpf_set_tag_base(self.h, int(tag_base)))

    def step_partial(self, n_steps):
        """hpf_step_partial: (steps run, mesh) with mesh None, or a torch int64
        tensor [S][Mz][My][Mx] viewing the library's mesh (no copy) that holds
        this part's density; sum the other parts into it before the next call."""
        done, mesh = ctypes.c_int32(0), ctypes.c_void_p(0)
        self._check(self.lib.hpf_step_partial(self.h, int(n_steps), ctypes.byref(done),
                                              ctypes.byref(mesh)))
        if not mesh.value:
            return done.value, None
        return done.value, device_view(mesh.value, self.mesh_shape, "<i8")

    def energy(self):
        out = (ctypes.c_double * 6)()
        self._check(self.lib.hpf_energy(self.h, out))
        self._synced()
        return np.array(list(out))

    # ---- Nose-Hoover thermostat (thermostat == 1)
    def get_thermostat(self):
        """(xi, eta) of the state, at the middle of the last step."""
        out = (ctypes.c_double * 2)()
        self._check(self.lib.hpf_get_thermostat(self.h, out))
        return float(out[0]), float(out[1])

    def set_thermostat(self, xi, eta):
        arr = (ctypes.c_double * 2)(float(xi), float(eta))
        self._check(self.lib.hpf_set_thermostat(self.h, arr))

    def selftest_timeout(self):
        """Run the bounded-wait self-test: (status, seconds); status 6
        (HPF_ERR_TIMEOUT) when the wait gave up as designed."""
        t = ctypes.c_double()
        st = self.lib.hpf_selftest_timeout(self.h, ctypes.byref(t))
        return int(st), t.value

    def nh_conserved(self):
        """The extended energy conserved by the Nose-Hoover equations."""
        v = ctypes.c_double()
        self._check(self.lib.hpf_nh_conserved(self.h, ctypes.byref(v)))
        return v.value

    # ---- learned propagator
    def density_phi(self, out=None):
        """Volume fractions phi [S][Mz][My][Mx] (FP32) of the current positions."""
        if out is None:
            out = np.empty(self.mesh_shape, dtype=np.float32)
        op, _a = _ptr(out, np.float32, self.mesh_shape, "phi")
        self._check(self.lib.hpf_density_phi(self.h, op))
        return out

    def judge_density(self, phi):
        """Field-force error of candidate volume fractions against the true scatter."""
        pp, _a = _ptr(phi, np.float32, self.mesh_shape, "phi")
        eps = ctypes.c_double()
        self._check(self.lib.hpf_judge_density(self.h, pp, ctypes.byref(eps)))
        return eps.value

    def learned_mode(self, in_launch=True):
        """hpf_learned_mode: learned windows in one launch (True) or per step."""
        self._check(self.lib.hpf_learned_mode(self.h, 1 if in_launch else 0))

    def smooth_phi(self, phi, passes, out=None):
        """hpf_smooth_phi: the periodic binomial filter, passes times per axis."""
        if out is None:
            out = np.empty(self.mesh_shape, dtype=np.float32)
        ip, _a = _ptr(phi, np.float32, self.mesh_shape, "phi_in")
        op, _b = _ptr(out, np.float32, self.mesh_shape, "phi_out")
        self._check(self.lib.hpf_smooth_phi(self.h, ip, op, int(passes)))
        return out

    def judge_density_pair(self, phi_cand, phi_ref):
        """hpf_judge_density_pair: eps of the candidate's field force against
        the reference density's, at the current positions."""
        cp, _a = _ptr(phi_cand, np.float32, self.mesh_shape, "phi_cand")
        rp, _b = _ptr(phi_ref, np.float32, self.mesh_shape, "phi_ref")
        eps = ctypes.c_double()
        self._check(self.lib.hpf_judge_density_pair(self.h, cp, rp, ctypes.byref(eps)))
        return float(eps.value)

    def step_learned(self, prop, n_windows, K=20, tol=1e-3):
        """n_windows windows of K steps with the learned propagator; returns the stats dict."""
        st = LearnedStats()
        self._check(self.lib.hpf_step_learned(self.h, prop.h, int(n_windows), int(K),
                                              float(tol), ctypes.byref(st)))
        return st.as_dict()

    # ---- profiling
    def profile(self, enable=True):
        self._check(self.lib.hpf_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{stage: (device ms, kernel launches)} since the last read (synchronises)."""
        ms = (ctypes.c_double * len(STAGES))()
        ln = (ctypes.c_int64 * len(STAGES))()
        self._check(self.lib.hpf_profile_read(self.h, ms, ln))
        return {s: (ms[k], ln[k]) for k, s in enumerate(STAGES)}


class Batch:
    """Replicas advanced together (hpf_batch_*); replica(r) gives each one's context."""

    def __init__(self, params_list, stream=None):
        self.lib = load()
        self.params = [p if isinstance(p, Params) else make_params(**p) for p in params_list]
        arr = (Params * len(self.params))(*self.params)
        if stream is None:
            stream = current_stream_handle()
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = ctypes.c_void_p()
        st = self.lib.hpf_batch_init(arr, len(self.params), ctypes.c_void_p(int(stream)),
                                     ctypes.byref(h))
        if st != 0:
            raise HPFError(st, self.lib.hpf_status_string(st).decode())
        self.h = h
        self.replicas = [System._borrow(self.lib, self.lib.hpf_batch_replica(h, r), p)
                         for r, p in enumerate(self.params)]

    def replica(self, r):
        return self.replicas[r]

    def step(self, n_steps=1):
        st = self.lib.hpf_batch_step(self.h, int(n_steps))
        if st != 0:
            msg = self.lib.hpf_last_error(self.replicas[0].h).decode()
            raise HPFError(st, msg or self.lib.hpf_status_string(st).decode())

    def energy(self):
        """hpf_energy's six observables of every replica, [R][6]."""
        out = (ctypes.c_double * (6 * len(self.params)))()
        st = self.lib.hpf_batch_energy(self.h, out)
        if st != 0:
            raise HPFError(st, self.lib.hpf_status_string(st).decode())
        return np.array(list(out)).reshape(len(self.params), 6)

    def use_graphs(self, enable=True):
        self.lib.hpf_batch_use_graphs(self.h, 1 if enable else 0)

    def close(self):
        if getattr(self, "h", None):
            for r in self.replicas:
                r.h = None
            self.lib.hpf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Propagator:
    """The learned density propagator network (hpf_prop_init ... hpf_prop_destroy).

    Mesh arrays are planar FP32: inputs x [4][Mz][My][Mx] = (phi_A, phi_B at
    t - K, phi_A, phi_B at t); outputs and targets [2][Mz][My][Mx].  ``scale``
    is the change scale s (input change channels times s, output divided by
    s; the training loss is s^2 times the mean squared error)."""

    def __init__(self, mesh, stream=None):
        self.lib = load()
        m = (mesh,) * 3 if np.isscalar(mesh) else tuple(mesh)
        self.mesh = tuple(int(v) for v in m)
        if stream is None:
            stream = current_stream_handle()
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        arr = (ctypes.c_int32 * 3)(*self.mesh)
        h = ctypes.c_void_p()
        st = self.lib.hpf_prop_init(arr, ctypes.c_void_p(self.stream), ctypes.byref(h))
        if st != 0:
            raise HPFError(st, self.lib.hpf_status_string(st).decode())
        self.h = h
        self.n_params = int(self.lib.hpf_prop_param_count())
        self.V = self.mesh[0] * self.mesh[1] * self.mesh[2]
        self.grid = (self.mesh[2], self.mesh[1], self.mesh[0])

    def _check(self, st):
        if st != 0:
            raise HPFError(st, self.lib.hpf_status_string(st).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.hpf_prop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def scale(self) -> float:
        v = ctypes.c_float()
        self._check(self.lib.hpf_prop_get_scale(self.h, ctypes.byref(v)))
        return float(v.value)

    @scale.setter
    def scale(self, value: float):
        self._check(self.lib.hpf_prop_set_scale(self.h, float(value)))

    def set_ctas(self, ctas: int):
        """At most ctas CTAs for the persistent forward convolutions (0: the
        default, two per SM); results do not depend on it."""
        self._check(self.lib.hpf_prop_set_ctas(self.h, int(ctas)))

    def selftest_timeout(self):
        """Run the forward convolutions' wait self-test; returns (status code,
        seconds): HPF_ERR_TIMEOUT (6) when the bounded waits gave up as designed."""
        secs = ctypes.c_double()
        st = self.lib.hpf_prop_selftest_timeout(self.h, ctypes.byref(secs))
        return int(st), float(secs.value)

    def set_weights(self, params):
        pp, _a = _ptr(params, np.float32, (self.n_params,), "params")
        self._check(self.lib.hpf_prop_set_weights(self.h, pp))

    def get_weights(self, out=None):
        if out is None:
            out = np.empty(self.n_params, dtype=np.float32)
        op, _a = _ptr(out, np.float32, (self.n_params,), "params")
        self._check(self.lib.hpf_prop_get_weights(self.h, op))
        return out

    def forward(self, x, out=None):
        if out is None:
            out = np.empty((2,) + self.grid, dtype=np.float32)
        xp, _a = _ptr(x, np.float32, (4,) + self.grid, "x")
        op, _b = _ptr(out, np.float32, (2,) + self.grid, "dphi")
        self._check(self.lib.hpf_prop_forward(self.h, xp, op))
        return out

    def rollout(self, x, steps, out=None):
        """hpf_prop_rollout: phi(t + steps) from x = (phi(t - 1), phi(t)), each
        prediction phi + network(phi_prev, phi) fed back as the next input."""
        if out is None:
            out = np.empty((2,) + self.grid, dtype=np.float32)
        xp, _a = _ptr(x, np.float32, (4,) + self.grid, "x")
        op, _b = _ptr(out, np.float32, (2,) + self.grid, "phi_out")
        self._check(self.lib.hpf_prop_rollout(self.h, xp, int(steps), op))
        return out

    def backward(self, x, phi_next, grads=None):
        """(loss, gradient vector) of the mean squared error against phi_next - x[2:4]."""
        if grads is None:
            grads = np.empty(self.n_params, dtype=np.float32)
        xp, _a = _ptr(x, np.float32, (4,) + self.grid, "x")
        tp, _b = _ptr(phi_next, np.float32, (2,) + self.grid, "phi_next")
        gp, _c = _ptr(grads, np.float32, (self.n_params,), "grads")
        loss = ctypes.c_double()
        self._check(self.lib.hpf_prop_backward(self.h, xp, tp, gp, ctypes.byref(loss)))
        return loss.value, grads

    def adam_step(self, grads, lr):
        gp, _a = _ptr(grads, np.float32, (self.n_params,), "grads")
        self._check(self.lib.hpf_prop_adam_step(self.h, gp, float(lr)))

    def train_step(self, x, phi_next, lr, want_loss=False):
        xp, _a = _ptr(x, np.float32, (4,) + self.grid, "x")
        tp, _b = _ptr(phi_next, np.float32, (2,) + self.grid, "phi_next")
        loss = ctypes.c_double()
        self._check(self.lib.hpf_prop_train_step(self.h, xp, tp, float(lr),
                                                 ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def pack_params(layers):
    """[(W [27][Ci][Co], b [Co]) per layer] -> the flat FP32 parameter vector."""
    return np.concatenate([np.concatenate([np.asarray(W, dtype=np.float32).reshape(-1),
                                           np.asarray(b, dtype=np.float32).reshape(-1)])
                           for W, b in layers])


def unpack_params(vec, channels=((4, 16), (16, 16), (16, 2))):
    """Inverse of pack_params."""
    out, k = [], 0
    vec = np.asarray(vec)
    for ci, co in channels:
        W = vec[k:k + 27 * ci * co].reshape(27, ci, co)
        k += 27 * ci * co
        b = vec[k:k + co]
        k += co
        out.append((W, b))
    return out
