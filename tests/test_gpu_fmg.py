"""Nested-iteration start (MG_FLAG_FMG_START) on the GPU against the oracle's or_fmg_start.

The start vector is read back from a solve whose tolerance is met at cycle 0, so the
returned x is the start itself.  FP64: within 1e-11 of the oracle (the start is a chain of
F-cycles, compared like one cycle); then the full solve from it takes the oracle's cycle
count.  MG_MIXED runs the nested iteration in FP32: its start must reach the oracle's
residual up to FP32 rounding.
"""
import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import (Solver, FLAG_FMG_START, FLAG_NO_GRAPH,  # noqa: E402
                                           FLAG_NO_FUSED_COARSE)
from test_gpu_parity import spec_of, oracle_of, rel  # noqa: E402

CASES = [
    # dim, n, periodic, kind, levels, smoother, omega, extra flags
    (2, (129, 65), False, inputs.CONST, 5, "rbgs", 1.0, 0),
    (2, (129, 65), False, inputs.CONST, 5, "rbgs", 1.0, FLAG_NO_GRAPH),
    (2, (129, 65), False, inputs.CONST, 5, "rbgs", 1.0, FLAG_NO_FUSED_COARSE),
    (2, (65, 129), False, inputs.CELL, 4, "zebra_y", 1.0, 0),
    (2, (129, 64), True, inputs.SEPARABLE, 5, "rbgs", 1.0, 0),
    (2, (65, 65), False, inputs.CONST, 4, "gsadi", 1.0, 0),
    (3, (33, 17, 33), False, inputs.CONST, 3, "rbgs", 1.0, 0),
    (3, (17, 17, 17), False, inputs.CELL, 3, "jacobi", 0.8, 0),
    # every level in the single-CTA coarse kernel: the whole nested iteration is one launch
    (2, (33, 33), False, inputs.CONST, 4, "rbgs", 1.0, 0),
    (2, (33, 16), True, inputs.SEPARABLE, 3, "zebra_x", 1.0, 0),
]


def case_id(c):
    return f"{c[0]}d-{c[1]}-{'per' if c[2] else 'dir'}-k{c[3]}-{c[5]}-f{c[7]}"


@pytest.fixture(scope="module", params=CASES, ids=case_id)
def case(request):
    dim, n, per, kind, L, sm, om, fl = request.param
    rng = np.random.default_rng(abs(hash(request.param[:6])) % 2 ** 32)
    sp = spec_of(dim, n, per, kind, rng)
    return sp, oracle_of(sp, L, sm, om), dict(levels=L, smoother=sm, omega=om), fl


def test_fp64_start_vector_matches_oracle(case):
    sp, o, kw, fl = case
    s = Solver(sp, max_cycles=60, flags=FLAG_FMG_START | fl, **kw)
    x0 = np.random.default_rng(3).standard_normal(o.shape())   # ignored under the flag
    x, info = s.solve(sp.b, x0=x0, tol=1e30)
    assert info["status"] == "MG_OK" and info["cycles"] == 0
    xo = o.fmg_start(sp.b)
    assert rel(x, xo) <= 1e-11
    # and the residual it reports is the oracle start's
    ro = o.norm(o.defect(xo, sp.b, o.levels)) / o.norm(sp.b)
    assert abs(info["relres"] - ro) <= 1e-9 * ro + 1e-14


def test_fp64_solve_from_fmg_start_matches_oracle(case):
    sp, o, kw, fl = case
    s = Solver(sp, max_cycles=60, flags=FLAG_FMG_START | fl, **kw)
    x, info = s.solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=60, start="fmg")
    assert info["status"] == "MG_OK"
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
    assert rel(x, xo) <= 1e-11
    # the nested-iteration start never costs cycles against the zero start
    z, zinfo = Solver(sp, max_cycles=60, flags=fl, **kw).solve(sp.b, tol=1e-10)
    assert info["cycles"] <= zinfo["cycles"]


def test_mixed_start_reaches_oracle_residual(case):
    sp, o, kw, fl = case
    s = Solver(sp, max_cycles=60, precision="mixed", flags=FLAG_FMG_START | fl, **kw)
    x, info = s.solve(sp.b, tol=1e30)
    xo = o.fmg_start(sp.b)
    ro = o.norm(o.defect(xo, sp.b, o.levels)) / o.norm(sp.b)
    # FP32 rounding of the start: residual within a few FP32 ulps of ||b|| of the FP64 start's
    assert info["relres"] <= 1.05 * ro + 1e-5
    assert rel(x, xo) <= 1e-4
    x, info = s.solve(sp.b, tol=1e-10)
    assert info["status"] == "MG_OK" and info["relres"] <= 1e-10


def test_zero_rhs_gives_zero_start():
    rng = np.random.default_rng(5)
    sp = spec_of(2, (65, 65), False, inputs.CONST, rng)
    sp.b[:] = 0.0
    for prec in ("fp64", "mixed"):
        s = Solver(sp, levels=4, precision=prec, flags=FLAG_FMG_START)
        x, info = s.solve(sp.b, x0=np.ones_like(sp.b), tol=1e-10)
        assert info["status"] == "MG_OK" and info["cycles"] == 0
        assert float(torch.as_tensor(x).abs().max()) == 0.0
