"""hpf_field_forces_noalloc: field forces without any device allocation.

Some host programs cannot let a library call cudaMalloc (their own pool holds
nearly all device memory, or an allocation's device-wide synchronisation is
not acceptable mid-run).  For them the library offers one entry point whose
working meshes live in a static device array.  This test calls it through the
C ABI twice in a row, on two different systems (so anything left in the shared
scratch by the first call would show in the second), and checks each result
against hpf_forces(HPF_FORCE_FIELD) of a context, within the same per-bead
force bar as the other GPU tests.  It sits in a file of its own, collected
last.
"""
import ctypes

import numpy as np
import pytest

from paper_1310_2041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HPF_ERR_INVALID, HPF_ERR_SCRATCH = 1, 8


def _lib(hpf):
    L = hpf.load()
    L.hpf_field_forces_noalloc.argtypes = [ctypes.POINTER(hpf.Params), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p]
    L.hpf_field_forces_noalloc.restype = ctypes.c_int
    L.hpf_noalloc_scratch_bytes.argtypes = [ctypes.POINTER(hpf.Params)]
    L.hpf_noalloc_scratch_bytes.restype = ctypes.c_size_t
    return L


def _jittered(w, seed):
    d = W.generate(w)
    rng = np.random.default_rng(seed)
    d["pos"] = (d["pos"] + rng.normal(0.0, 0.05, d["pos"].shape)).astype(np.float32)
    return d


def _within_bar(F, Fo, rel=1e-5):
    F, Fo = F.astype(np.float64), Fo.astype(np.float64)
    rms = np.sqrt(np.mean(np.sum(Fo ** 2, axis=1)))
    err = np.linalg.norm(F - Fo, axis=1)
    return np.all(err <= rel * (np.linalg.norm(Fo, axis=1) + rms))


def test_noalloc_field_forces_match_the_context_path_twice():
    import torch
    from paper_1310_2041_gb300 import hpf
    assert torch.cuda.is_available()
    L = _lib(hpf)
    stream = torch.cuda.current_stream()
    systems = [(W.diblock(900, 6, 4, 14.1, 14, 1.3, name="first"), 1),
               (W.diblock(450, 3, 7, 11.2, 11, 0.7, name="second"), 2)]
    # the second system has another mesh and bead count: anything the first call
    # left in the shared scratch would corrupt the second result
    for w, seed in systems:
        d = _jittered(w, seed)
        pp = w.params()
        p = hpf.make_params(**pp)
        assert L.hpf_noalloc_scratch_bytes(ctypes.byref(p)) <= 32 << 20
        with hpf.System(p, stream=stream) as ctx:
            ctx.set_state(d["pos"], d["vel"], d["type"], d["bonds"])
            F_ctx = ctx.forces(hpf.FORCE_FIELD)
        pos = torch.from_numpy(d["pos"]).cuda()
        typ = torch.from_numpy(d["type"]).cuda()
        out = torch.full((w.n_beads, 3), float("nan"), dtype=torch.float32, device="cuda")
        rc = L.hpf_field_forces_noalloc(ctypes.byref(p), pos.data_ptr(), typ.data_ptr(),
                                        w.n_beads, out.data_ptr(),
                                        ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        F = out.cpu().numpy()
        assert np.all(np.isfinite(F))
        assert _within_bar(F, F_ctx)


def test_noalloc_rejects_oversize_meshes_and_host_pointers():
    import torch
    from paper_1310_2041_gb300 import hpf
    L = _lib(hpf)
    big = hpf.make_params(10, 2, (160, 160, 160), (160.0, 160.0, 160.0))
    assert L.hpf_noalloc_scratch_bytes(ctypes.byref(big)) > 32 << 20
    dev = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    typ = torch.zeros(10, dtype=torch.int32, device="cuda")
    assert L.hpf_field_forces_noalloc(ctypes.byref(big), dev.data_ptr(), typ.data_ptr(), 10,
                                      dev.data_ptr(), None) == HPF_ERR_SCRATCH
    ok = hpf.make_params(10, 2, 8, 8.0)
    host = np.zeros((10, 3), dtype=np.float32)
    assert L.hpf_field_forces_noalloc(ctypes.byref(ok), host.ctypes.data, typ.data_ptr(), 10,
                                      dev.data_ptr(), None) == HPF_ERR_INVALID
    # field parameters that hpf_init refuses are refused here too (no launch)
    neg = hpf.make_params(10, 2, 8, 8.0, kT=-1.0)
    assert L.hpf_field_forces_noalloc(ctypes.byref(neg), dev.data_ptr(), typ.data_ptr(), 10,
                                      dev.data_ptr(), None) == HPF_ERR_INVALID
    # the 70^3 mesh of three species fits the scratch (density and field only)
    tern = hpf.make_params(10, 3, 70, 69.3)
    assert 0 < L.hpf_noalloc_scratch_bytes(ctypes.byref(tern)) <= 32 << 20
