"""Adaptive correction weight (MG_FLAG_ADAPTIVE_CORR) on the GPU against the oracle.

FP64: one cycle (plain and transposed) within 1e-11 of the oracle's cycle with
adaptive_corr, and the solve takes the oracle's cycle count.  Cases cover the per-level
kernels, the single-CTA coarse kernel (whose program carries the weight step) and the whole
cycle in that kernel.  MG_MIXED computes the weight in FP32 arithmetic (FP64 sums): its
solve must converge like the oracle's.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import (Solver, FLAG_ADAPTIVE_CORR, FLAG_FMG_START,  # noqa: E402
                                           FLAG_NO_FUSED_COARSE, FLAG_NO_GRAPH)
from test_gpu_parity import spec_of, rel  # noqa: E402

CASES = [
    # dim, n, periodic, kind, levels, smoother, omega, extra flags
    (2, (129, 65), False, inputs.CONST, 5, "rbgs", 1.0, 0),
    (2, (129, 65), False, inputs.CONST, 5, "rbgs", 1.0, FLAG_NO_FUSED_COARSE),
    (2, (129, 65), False, inputs.CONST, 5, "jacobi", 0.8, FLAG_NO_GRAPH),
    (2, (65, 129), False, inputs.CELL, 4, "zebra_y", 1.0, 0),
    (2, (129, 64), True, inputs.SEPARABLE, 5, "rbgs", 1.0, 0),
    (2, (65, 65), False, inputs.CELL, 4, "gsadi", 1.0, 0),
    (3, (33, 17, 33), False, inputs.CONST, 3, "rbgs", 1.0, 0),
    (3, (17, 16, 17), True, inputs.CELL, 3, "jacobi", 0.8, 0),
    # the whole F-cycle in the single-CTA coarse kernel
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
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c,
                    sx=sp.sx, sy=sp.sy, sz=sp.sz, k=sp.k)
    # omega_corr 0.5 is ignored by both sides under the adaptive rule
    o = orc.Oracle(p, levels=L, smoother=sm, omega=om, omega_corr=0.5, adaptive_corr=True, dense_max=4096)
    kw = dict(levels=L, smoother=sm, omega=om, omega_corr=0.5)
    return sp, o, kw, fl, rng


@pytest.mark.parametrize("transposed", [False, True])
def test_one_adaptive_cycle_matches_oracle(case, transposed):
    sp, o, kw, fl, rng = case
    s = Solver(sp, max_cycles=60, flags=FLAG_ADAPTIVE_CORR | fl, **kw)
    x = rng.standard_normal(o.shape()) * o.unknown_mask()
    assert rel(s.cycle(x, sp.b, transposed), o.cycle(x, sp.b, transposed=transposed)) <= 1e-11


def test_adaptive_solve_matches_oracle(case):
    sp, o, kw, fl, rng = case
    s = Solver(sp, max_cycles=60, flags=FLAG_ADAPTIVE_CORR | fl, **kw)
    x, info = s.solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=60)
    assert info["status"] == "MG_OK" and sto == orc.OK
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
        assert np.allclose(info["history"], ho, rtol=1e-8, atol=1e-14)
    assert rel(x, xo) <= 1e-11


def test_adaptive_with_fmg_start_matches_oracle(case):
    sp, o, kw, fl, rng = case
    s = Solver(sp, max_cycles=60, flags=FLAG_ADAPTIVE_CORR | FLAG_FMG_START | fl, **kw)
    x, info = s.solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=60, start="fmg")
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
    assert rel(x, xo) <= 1e-11


def test_mixed_adaptive_solve_converges(case):
    sp, o, kw, fl, rng = case
    s = Solver(sp, max_cycles=60, precision="mixed", flags=FLAG_ADAPTIVE_CORR | fl, **kw)
    x, info = s.solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=60)
    assert info["status"] == "MG_OK" and info["relres"] <= 1e-10
    assert info["cycles"] <= co + 2
    assert rel(x, xo) <= 1e-6
