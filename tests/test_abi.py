"""The C-ABI library builds for sm_103a, loads, and exports every declared entry point.

No compute call is made here (no GPU on this machine); the GPU tests cover them.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1310_2041_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(hpf_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hpf_init", "hpf_scatter_density", "hpf_field", "hpf_forces", "hpf_step",
                     "hpf_energy", "hpf_set_state", "hpf_get_state", "hpf_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(hpf_[a-z0-9_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_without_a_gpu(lib_path):
    L = ctypes.CDLL(lib_path)
    L.hpf_status_string.restype = ctypes.c_char_p
    assert L.hpf_status_string(0) == b"ok"
    assert L.hpf_status_string(4).startswith(b"fixed-point")
    # argument validation happens before any CUDA call
    from paper_1310_2041_gb300 import hpf
    p = hpf.make_params(10, 2, 4, 4.0)
    L.hpf_init.argtypes = [ctypes.POINTER(hpf.Params), ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert L.hpf_init(ctypes.byref(p), None, None) == 1
    p.n_beads = 1 << 24
    assert L.hpf_init(ctypes.byref(p), None, ctypes.byref(h)) == 4   # overflow guard
    p.n_beads = 10
    p.chi[1] = 0.5                                                    # asymmetric chi
    assert L.hpf_init(ctypes.byref(p), None, ctypes.byref(h)) == 1
    p.chi[1] = 0.0
    p.field_every = 0
    assert L.hpf_init(ctypes.byref(p), None, ctypes.byref(h)) == 1


@pytest.mark.parametrize("mirror,cname", [("Params", "hpf_params"),
                                           ("LearnedStats", "hpf_learned_stats")])
def test_struct_layout_matches_header(tmp_path, mirror, cname):
    """Field offsets of the ctypes mirrors equal offsetof() of the C header."""
    from paper_1310_2041_gb300 import hpf
    cls = getattr(hpf, mirror)
    fields = [f for f, _ in cls._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu\\n", offsetof({cname}, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hpf.h"\n'
                   f'int main(void){{ {body} printf("%zu\\n", sizeof({cname})); return 0; }}')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [getattr(cls, f).offset for f in fields] + [ctypes.sizeof(cls)]
    assert got == want
