"""Guard words around the caller's workspace (a stand-in for a memory checker): after set-up and
several solves of every smoother family, coefficient kind and precision, the bytes just before
and after the workspace the library was given are untouched."""
import ctypes as C

import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300 import binding  # noqa: E402
from paper_0805_3041_gb300.binding import Solver, FLAG_NO_GRAPH, FLAG_ADAPTIVE_CORR, FLAG_FMG_START  # noqa: E402
from test_gpu_parity import spec_of  # noqa: E402

GUARD = 1 << 20   # bytes on each side


class GuardedSolver(Solver):
    """A Solver whose workspace sits between two guard regions filled with a known pattern."""

    def guard(self):
        lib = self.lib
        nbytes = lib.mg_workspace_bytes(C.byref(self.params), C.byref(self.coeffs))
        lib.mg_destroy(self.ctx)
        buf = torch.empty(nbytes + 2 * GUARD + 256, dtype=torch.uint8, device=self.device)
        buf.fill_(0xA5)
        base = (buf.data_ptr() + GUARD + 255) & ~255
        ctx = C.c_void_p()
        assert lib.mg_setup(C.byref(self.params), C.byref(self.coeffs), C.c_void_p(base), nbytes, C.byref(ctx)) == 0
        self.ctx = ctx
        self.workspace = buf
        self.lo = base - buf.data_ptr()
        self.hi = self.lo + nbytes
        return self

    def intact(self):
        torch.cuda.synchronize()
        h = self.workspace.cpu().numpy()
        return bool(np.all(h[: self.lo] == 0xA5) and np.all(h[self.hi:] == 0xA5))


CASES = [
    # dim, n, periodic, kind, levels, smoother, precision, flags
    (2, (257, 129), False, inputs.CONST, 6, "rbgs", "mixed", 0),
    (2, (257, 129), False, inputs.CONST, 6, "rbgs", "fp64", FLAG_NO_GRAPH | FLAG_ADAPTIVE_CORR),
    (2, (129, 128), True, inputs.SEPARABLE, 5, "gsadi", "mixed", FLAG_FMG_START),
    (2, (129, 129), False, inputs.CELL, 5, "zebra_y", "fp64", 0),
    (3, (33, 33, 33), False, inputs.CONST, 3, "zebra_x", "mixed", 0),
    (2, (257, 129), False, inputs.CONST, 2, "rbgs", "mixed", 0),   # coarsest by conjugate gradients
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}d-{c[1]}-k{c[3]}-{c[5]}-{c[6]}-f{c[7]}")
def test_workspace_guards_stay_intact(case):
    dim, n, per, kind, L, sm, prec, fl = case
    sp = spec_of(dim, n, per, kind, np.random.default_rng(21))
    s = GuardedSolver(sp, levels=L, smoother=sm, omega=1.0, precision=prec, max_cycles=60, flags=fl).guard()
    for _ in range(2):
        x, info = s.solve(sp.b, tol=1e-10)
        assert info["status"] == "MG_OK"
    s.solve_adjoint(sp.b, tol=1e-8)
    assert s.intact()
