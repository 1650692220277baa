"""The C-ABI library builds, loads and exports every symbol include/mg.h declares (no GPU)."""
import ctypes as C
import os
import re
import shutil
import subprocess

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


def _header_text():
    src = open(os.path.join(ROOT, "include", "mg.h")).read()
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)


def test_binding_constants_match_the_header():
    """Every flag, status, smoother, coefficient kind, precision and batch form the binding passes
    across the ABI has the header's value, and every flag the header defines is in the binding."""
    src = _header_text()
    flags = dict((k, int(v)) for k, v in re.findall(r"#define\s+MG_FLAG_(\w+)\s+(\d+)u", src))
    assert flags, "no flags parsed"
    for name, v in flags.items():
        assert getattr(binding, "FLAG_" + name) == v, name
    for name in dir(binding):
        if name.startswith("FLAG_"):
            assert name[5:] in flags, name
    for name, v in re.findall(r"#define\s+MG_BATCH_(\w+)\s+(\d+)", src):
        assert getattr(binding, "BATCH_" + name) == int(v), name
    enums = {m.group(2): m.group(1) for m in re.finditer(r"typedef\s+enum\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S)}
    entries = {k: [(n, int(v)) for n, v in re.findall(r"MG_(\w+)\s*=\s*(\d+)", body)] for k, body in enums.items()}
    for n, v in entries["mg_status"]:
        assert binding.STATUS[v] == "MG_" + n and getattr(binding, n) == v, n
    assert len(binding.STATUS) == len(entries["mg_status"])
    for n, v in entries["mg_smoother"]:
        assert getattr(binding, n) == v, n
    assert sorted(binding.SMOOTHERS.values()) == sorted(v for _, v in entries["mg_smoother"])
    for n, v in entries["mg_coef_kind"]:
        assert getattr(binding, n.replace("COEF_", "")) == v, n
    for n, v in entries["mg_precision"]:
        assert getattr(binding, n) == v, n


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures the binding fills have the C structures' field offsets, field sizes and
    total sizes, as the host compiler lays out include/mg.h."""
    gcc = shutil.which("gcc") or shutil.which("cc")
    if not gcc:
        pytest.skip("no host C compiler")
    structs = {"mg_params": binding.Params, "mg_coeffs": binding.Coeffs, "mg_report": binding.Report}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mg.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} . %zu %zu\\n", (size_t)0, sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f"sizeof((({cname} *)0)->{fname}));")
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line.strip():
            continue
        cname, fname, off, size = line.split()
        cls = structs[cname]
        if fname == ".":
            assert C.sizeof(cls) == int(size), cname
        else:
            f = getattr(cls, fname)
            assert (f.offset, f.size) == (int(off), int(size)), (cname, fname)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_every_header_function_is_documented():
    """Each entry point of include/mg.h follows a comment block (a group of declarations, or the
    constants that belong to it, may share one)."""
    lines = open(os.path.join(ROOT, "include", "mg.h")).read().split("\n")
    decl = re.compile(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*\s+)+\*?\s*(mg_[a-z_0-9]+)\s*\(")
    found = 0
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        found += 1
        j = i - 1
        while j >= 0:
            t = lines[j].strip()
            cont = lines[j].startswith(" ") and t.endswith((",", ");"))   # a declaration's later lines
            if not t or decl.match(lines[j]) or cont or t.startswith(("#define", "typedef")):
                j -= 1   # blank lines and the group's declarations, constants and types
                continue
            break
        assert j >= 0 and lines[j].strip().endswith("*/"), m.group(1)
    assert found == len(declared_functions())
