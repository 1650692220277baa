"""Galerkin coarse operators (MG_FLAG_GALERKIN) on the GPU against the oracle.

Every level below the finest holds R A P of the next finer one: a 9-point stencil, built on
the device from the finest operator of any coefficient kind.  Damped Jacobi and Gauss-Seidel
run on those levels (the latter in four colours).  Checked element by element against the
oracle's Galerkin hierarchy: the operator on every level, sweeps, the two halves of a level
visit, the coarsest solve, one cycle plain and transposed, whole solves (same cycle counts),
adjoint solves, and the mixed-precision form to 1e-10 in the oracle's residual.
Bars as for the rediscretised operators: 1e-12 for single steps, 1e-11 for cycles and solves.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300 import binding  # noqa: E402
from paper_0805_3041_gb300.binding import Solver, FLAG_GALERKIN  # noqa: E402
from test_gpu_parity import spec_of, rel  # noqa: E402
from test_gpu_edge import random_edges  # noqa: E402

TOL64 = 1e-12


def galerkin_oracle(sp, levels, smoother, omega):
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c, sx=sp.sx, sy=sp.sy,
                    sz=sp.sz, k=sp.k, ex=sp.ex, ey=sp.ey, ez=sp.ez)
    return orc.Oracle(p, levels=levels, smoother=smoother, omega=omega, nu1=2, nu2=2, dense_max=4096, galerkin=True)


def _spec(kind, n, seed, eps=1.0):
    if kind == inputs.EDGE:
        return random_edges(2, n, False, seed)
    return spec_of(2, n, False, kind, np.random.default_rng(seed), eps=eps)


CASES = [
    # kind, n, levels, smoother, omega
    (inputs.CONST, (129, 65), 5, "rbgs", 1.0),
    (inputs.CONST, (257, 257), 7, "jacobi", 0.8),
    (inputs.SEPARABLE, (65, 129), 5, "rbgs", 1.0),
    (inputs.CELL, (129, 129), 6, "rbgs", 1.0),
    (inputs.CELL, (65, 33), 4, "jacobi", 0.8),
    (inputs.EDGE, (65, 65), 5, "rbgs", 1.0),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"k{c[0]}-{c[1][0]}x{c[1][1]}-{c[3]}")
def pair(request):
    kind, n, L, sm, om = request.param
    sp = _spec(kind, n, seed=sum(n) + kind)
    o = galerkin_oracle(sp, L, sm, om)
    s = Solver(sp, levels=L, smoother=sm, omega=om, max_cycles=60, flags=FLAG_GALERKIN)
    return sp, o, s, np.random.default_rng(hash(request.param) % 2 ** 32)


def test_operator_on_every_level(pair):
    sp, o, s, rng = pair
    for l in range(1, o.levels + 1):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        assert rel(s.apply(u, l), o.apply(u, l)) <= TOL64, l


@pytest.mark.parametrize("order", [0, 1])
def test_sweeps_on_galerkin_levels(pair, order):
    sp, o, s, rng = pair
    for l in sorted({o.levels - 1, 2}):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        g = rng.standard_normal(o.shape(l))
        for sweeps in (1, 2):
            assert rel(s.smooth(u, g, sweeps, order, l), o.smooth(u, g, sweeps, order, l)) <= TOL64, (l, sweeps)
        assert rel(s.defect(u, g, l), o.defect(u, g, l)) <= TOL64


@pytest.mark.parametrize("transposed", [False, True])
def test_visit_halves(pair, transposed):
    sp, o, s, rng = pair
    order = 1 if transposed else 0
    for l in sorted({o.levels, o.levels - 1, 2}):
        m = o.unknown_mask(l)
        u = rng.standard_normal(o.shape(l)) * m
        g = rng.standard_normal(o.shape(l))
        for start in ("u", "zero"):
            uo, gc = s.descend(u if start == "u" else None, g, l, transposed=transposed)
            ref = o.smooth(u if start == "u" else o.zeros(l), g, 2, order, l)
            assert rel(uo, ref) <= TOL64, (l, start)
            assert rel(gc, o.restrict(o.defect(ref, g, l), l)) <= TOL64, (l, start)
        ec = rng.standard_normal(o.shape(l - 1)) * o.unknown_mask(l - 1)
        ref = o.smooth(o.prolong_add(ec, u, 1.0, l), g, 2, order, l)
        assert rel(s.ascend(ec, u, g, l, transposed=transposed), ref) <= TOL64, l


def test_coarse_solve(pair):
    sp, o, s, rng = pair
    g = rng.standard_normal(o.shape(1)) * o.unknown_mask(1)
    assert rel(s.coarse_solve(g), o.coarse_solve(g)) <= 1e-11


@pytest.mark.parametrize("transposed", [False, True])
def test_one_cycle(pair, transposed):
    sp, o, s, rng = pair
    x = rng.standard_normal(o.shape()) * o.unknown_mask()
    assert rel(s.cycle(x, sp.b, transposed), o.cycle(x, sp.b, transposed=transposed)) <= 1e-11


def test_solve_and_adjoint_solve(pair):
    sp, o, s, rng = pair
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=60)
    xg, info = s.solve(sp.b, tol=1e-10)
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
    assert info["status"] == "MG_OK" and rel(xg, xo) <= 1e-11
    g = rng.uniform(-1, 1, o.shape()) * o.unknown_mask()
    lo = o.solve(g, tol=1e-10, maxit=60, transposed=True)[0]
    lg, _ = s.solve_adjoint(g, tol=1e-10)
    assert rel(lg, lo) <= 1e-11


@pytest.mark.parametrize("kind,n,L", [(inputs.CONST, (1025, 1025), 9), (inputs.CELL, (257, 257), 7),
                                      (inputs.EDGE, (129, 129), 6)])
def test_mixed_precision_reaches_the_fp64_residual(kind, n, L):
    """FP32 cycles on the Galerkin levels (the finest grid's fused FP32 kernels included), FP64
    refinement: 1e-10 in the oracle's FP64 residual, in about as many steps as FP64 cycles."""
    sp = _spec(kind, n, seed=3, eps=0.5)
    o = galerkin_oracle(sp, L, "rbgs", 1.0)
    s = Solver(sp, levels=L, smoother="rbgs", precision="mixed", max_cycles=40, flags=FLAG_GALERKIN)
    x, info = s.solve(sp.b, tol=1e-10)
    rr = o.norm(o.defect(x.cpu().numpy(), sp.b)) / o.norm(sp.b)
    _, _, co, _, _ = o.solve(sp.b, tol=1e-10, maxit=60)
    print(f"Galerkin mixed {n}: {info['cycles']} steps (FP64 oracle {co} cycles), oracle relres {rr:.2e}")
    assert info["status"] == "MG_OK" and rr <= 1e-10
    assert info["cycles"] <= co + 2


def test_galerkin_rejects_what_it_does_not_cover():
    rng = np.random.default_rng(9)
    for sp, sm, L in ((spec_of(3, (17, 17, 17), False, inputs.CONST, rng), "rbgs", 3),
                      (spec_of(2, (33, 32), True, inputs.CONST, rng), "rbgs", 3),
                      (spec_of(2, (33, 33), False, inputs.CONST, rng), "zebra_x", 3),
                      (spec_of(2, (257, 257), False, inputs.CONST, rng), "rbgs", 2)):   # coarsest > 4096 unknowns
        with pytest.raises(binding.MGError):
            Solver(sp, levels=L, smoother=sm, flags=FLAG_GALERKIN)
