"""The C-ABI library builds, loads and exports every symbol include/mg.h declares (no GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_0805_3041_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*\s+)+\*?\s*(mg_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    assert sorted(binding.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(build.build())
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_invalid_parameters_are_rejected_without_a_gpu():
    lib = binding.load()
    p = binding.Params()
    k = binding.Coeffs()
    p.dim, p.levels, p.smoother, p.nu1, p.nu2, p.omega, p.max_cycles = 2, 3, binding.RBGS, 2, 2, 1.0, 10
    p.n = (C.c_int * 3)(17, 17, 1)
    k.kind = binding.CONST
    k.c = (C.c_double * 3)(1.0, 1.0, 0.0)
    assert lib.mg_workspace_bytes(C.byref(p), C.byref(k)) > 0
    for field, bad in [("dim", 4), ("levels", 0), ("levels", 6), ("smoother", 9), ("nu1", -1)]:
        q = binding.Params.from_buffer_copy(p)
        setattr(q, field, bad)
        assert lib.mg_workspace_bytes(C.byref(q), C.byref(k)) == 0, field
    q = binding.Params.from_buffer_copy(p)
    q.n = (C.c_int * 3)(18, 17, 1)        # not 2^m + 1 for 3 levels
    assert lib.mg_workspace_bytes(C.byref(q), C.byref(k)) == 0
    q = binding.Params.from_buffer_copy(p)
    q.periodic_y, q.smoother = 1, binding.ZEBRA_Y   # lines across a periodic direction: cyclic systems
    q.n = (C.c_int * 3)(17, 16, 1)
    assert lib.mg_workspace_bytes(C.byref(q), C.byref(k)) > 0
    ke = binding.Coeffs.from_buffer_copy(k)
    ke.kind = binding.EDGE   # edge weights without their arrays
    assert lib.mg_workspace_bytes(C.byref(p), C.byref(ke)) == 0
    ctx = C.c_void_p()
    assert lib.mg_setup(C.byref(p), C.byref(k), None, 0, C.byref(ctx)) == binding.EINVAL
    assert lib.mg_status_str(binding.ENOCONV) == b"maximum number of cycles reached"
