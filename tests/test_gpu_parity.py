"""GPU (CUDA, through the C ABI) against the FP64 CPU oracle, element by element.

Bar: FP64 results within 1e-12 relative (max-norm over the array, relative to
the array's max) after the same fixed number of steps; the same cycle count to
the tolerance.  Shapes are chosen to span several 32-wide tiles with ragged
tails (n0 = 129: 127 unknowns per row), rectangular grids, periodic y, 3-D.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver, ENOCONV  # noqa: E402

TOL64 = 1e-12


def spec_of(dim, n, periodic_y, kind, rng, eps=1.0):
    """A small problem of the requested kind (inputs.ProblemSpec)."""
    n = tuple(n) + (1,) * (3 - len(n))
    if dim == 2:
        n = (n[0], n[1], 1)
    h = (1.0 / (n[0] - 1), (1.0 / n[1]) if periodic_y else 1.0 / (n[1] - 1), 1.0 / max(n[2] - 1, 1))
    shape = (n[1], n[0]) if dim == 2 else (n[2], n[1], n[0])
    b = rng.uniform(-1, 1, shape)
    sp = inputs.ProblemSpec(name="t", dim=dim, n=n, periodic_y=periodic_y, kind=kind, h=h, b=b)
    if kind == inputs.CONST:
        sp.c = (eps / h[0] ** 2, 1.0 / h[1] ** 2, (1.0 / h[2] ** 2) if dim == 3 else 0.0)
    elif kind == inputs.SEPARABLE:
        sp.sx = rng.uniform(0.5, 2, n[0] - 1) / h[0] ** 2
        sp.sy = rng.uniform(0.5, 2, n[0]) / h[1] ** 2
        sp.sz = rng.uniform(0.5, 2, n[0]) / h[2] ** 2
    else:
        cy = n[1] if periodic_y else n[1] - 1
        ks = (cy, n[0] - 1) if dim == 2 else (n[2] - 1, cy, n[0] - 1)
        sp.k = np.exp(0.7 * rng.standard_normal(ks))
    return sp


def oracle_of(sp, levels, smoother, omega, nu1=2, nu2=2):
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c,
                    sx=sp.sx, sy=sp.sy, sz=sp.sz, k=sp.k)
    return orc.Oracle(p, levels=levels, smoother=smoother, omega=omega, nu1=nu1, nu2=nu2, dense_max=4096)


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() / scale


CASES = [
    # dim, n, periodic, kind, levels, smoother, omega
    (2, (129, 65), False, inputs.CONST, 5, "rbgs", 1.0),
    (2, (129, 65), False, inputs.CONST, 5, "jacobi", 0.8),
    (2, (65, 129), False, inputs.CELL, 4, "rbgs", 1.15),
    (2, (129, 64), True, inputs.SEPARABLE, 5, "rbgs", 1.0),
    (2, (65, 33), False, inputs.SEPARABLE, 4, "zebra_y", 1.0),
    (2, (129, 64), True, inputs.CONST, 4, "zebra_x", 1.0),
    (2, (65, 65), False, inputs.CELL, 4, "line_y", 0.7),
    (2, (33, 65), False, inputs.CONST, 3, "line_x", 0.7),
    (3, (33, 17, 33), False, inputs.CONST, 3, "rbgs", 1.0),
    (3, (33, 16, 17), True, inputs.SEPARABLE, 3, "jacobi", 0.8),
    (3, (17, 17, 17), False, inputs.CELL, 3, "zebra_x", 1.0),
    # alternating-direction line smoothers (x lines then y lines)
    (2, (65, 65), False, inputs.CONST, 4, "adi", 0.8),
    (2, (129, 65), False, inputs.SEPARABLE, 5, "gsadi", 1.0),
    (2, (65, 33), False, inputs.CELL, 4, "gsadi", 1.0),
    (3, (17, 17, 17), False, inputs.CONST, 3, "adi", 0.8),
    # lines across the periodic direction (cyclic tridiagonal systems)
    (2, (129, 64), True, inputs.SEPARABLE, 5, "zebra_y", 1.0),
    (2, (65, 64), True, inputs.CELL, 4, "line_y", 0.7),
    (2, (129, 64), True, inputs.SEPARABLE, 5, "gsadi", 1.0),
    (3, (17, 16, 17), True, inputs.CONST, 3, "adi", 0.8),
    (3, (17, 64, 17), True, inputs.SEPARABLE, 3, "gsadi", 1.0),
    # every grid fits the single-CTA coarse cycle (the whole F-cycle runs in one launch)
    (2, (33, 33), False, inputs.CONST, 4, "rbgs", 1.0),
    (2, (17, 33), False, inputs.CELL, 3, "zebra_y", 1.0),
    (2, (33, 16), True, inputs.SEPARABLE, 3, "jacobi", 0.8),
    (2, (33, 33), False, inputs.CONST, 3, "gsadi", 1.0),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}d-{c[1]}-{'per' if c[2] else 'dir'}-k{c[3]}-{c[5]}")
def pair(request):
    dim, n, per, kind, L, sm, om = request.param
    rng = np.random.default_rng(hash(request.param) % 2 ** 32)
    sp = spec_of(dim, n, per, kind, rng)
    return sp, oracle_of(sp, L, sm, om), Solver(sp, levels=L, smoother=sm, omega=om, max_cycles=60), rng


def test_operator(pair):
    sp, o, s, rng = pair
    for l in range(1, o.levels + 1):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        assert rel(s.apply(u, l), o.apply(u, l)) <= TOL64


def test_defect(pair):
    sp, o, s, rng = pair
    for l in (o.levels, max(1, o.levels - 1)):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        g = rng.standard_normal(o.shape(l))
        assert rel(s.defect(u, g, l), o.defect(u, g, l)) <= TOL64


@pytest.mark.parametrize("order", [0, 1])
def test_smoother_sweeps(pair, order):
    sp, o, s, rng = pair
    for l in (o.levels, 2):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        g = rng.standard_normal(o.shape(l))
        for sweeps in (1, 3):
            assert rel(s.smooth(u, g, sweeps, order, l), o.smooth(u, g, sweeps, order, l)) <= TOL64


def test_transfers(pair):
    sp, o, s, rng = pair
    for lf in range(2, o.levels + 1):
        r = rng.standard_normal(o.shape(lf)) * o.unknown_mask(lf)
        assert rel(s.restrict(r, lf), o.restrict(r, lf)) <= TOL64
        e = rng.standard_normal(o.shape(lf - 1)) * o.unknown_mask(lf - 1)
        u = rng.standard_normal(o.shape(lf)) * o.unknown_mask(lf)
        assert rel(s.prolong_add(e, u, 0.9, lf), o.prolong_add(e, u, 0.9, lf)) <= TOL64


@pytest.mark.parametrize("transposed", [False, True])
def test_visit_halves(pair, transposed):
    """The two halves of a level visit as the cycle runs them (fused sweep + defect +
    restriction kernels included): pre-smoothing from u or from zero then R(g - A u);
    correction u + P ec then post-smoothing."""
    sp, o, s, rng = pair
    nu_pre = 2   # nu1 = nu2 = 2 in every case
    order = 1 if transposed else 0
    for l in sorted({o.levels, 2}):
        m = o.unknown_mask(l)
        u = rng.standard_normal(o.shape(l)) * m
        g = rng.standard_normal(o.shape(l))
        for start in ("u", "zero"):
            u0 = u if start == "u" else None
            uo, gc = s.descend(u0, g, l, transposed=transposed)
            ref = o.smooth(u if start == "u" else o.zeros(l), g, nu_pre, order, l)
            assert rel(uo, ref) <= TOL64, (l, start)
            assert rel(gc, o.restrict(o.defect(ref, g, l), l)) <= TOL64, (l, start)
        ec = rng.standard_normal(o.shape(l - 1)) * o.unknown_mask(l - 1)
        ref = o.smooth(o.prolong_add(ec, u, 1.0, l), g, nu_pre, order, l)
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


def test_fixed_cycles_and_cycle_count(pair):
    sp, o, s, rng = pair
    xo, sto, co, rro, ho = o.solve(sp.b, tol=0.0, maxit=4)
    # same iterate after the same number of cycles (max_cycles of the solver is 60: run to 4)
    s4 = Solver(sp, levels=o.levels, smoother=s.params.smoother, omega=s.params.omega, max_cycles=4)
    xg4, info4 = s4.solve(sp.b, tol=0.0)
    assert info4["status"] == "MG_ENOCONV" and info4["cycles"] == 4
    assert rel(xg4, xo) <= 1e-11
    # the computed residual carries a cancellation error ~ eps * || |A| |x| ||; relres differences
    # between two correct FP64 implementations are bounded by a small multiple of that over ||b||
    absAx = 2.0 * o.diag() * np.abs(xo)
    bound = 64 * 2.2e-16 * np.linalg.norm(absAx) / o.norm(sp.b)
    assert np.all(np.abs(info4["history"] - ho) <= 1e-12 * ho + bound)
    # same number of cycles to 1e-10 (unless a residual sits within 1e-3 of the tolerance)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=60)
    xg, info = s.solve(sp.b, tol=1e-10)
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
    assert info["relres"] <= 1e-10 or info["status"] == "MG_ENOCONV"
    assert rel(xg, xo) <= 1e-11


def test_adjoint_solve(pair):
    sp, o, s, rng = pair
    g = rng.uniform(-1, 1, o.shape()) * o.unknown_mask()
    lo, st, co, rro, ho = o.solve(g, tol=1e-10, maxit=60, transposed=True)
    lg, info = s.solve_adjoint(g, tol=1e-10)
    assert rel(lg, lo) <= 1e-11


# ---------------------------------------------------------------------------------------
# the plain-method case: 129^2 Poisson, sin sin right-hand side, 6 levels, Jacobi 0.8
# ---------------------------------------------------------------------------------------

def test_poisson_sin_closed_form():
    sp = inputs.poisson_sin(129)
    s = Solver(sp, levels=6, smoother="jacobi", omega=0.8, max_cycles=50)
    x, info = s.solve(sp.b, tol=1e-10)
    h = 1.0 / 128
    xs = np.arange(129) * h
    exact = 2 * math.pi ** 2 * h ** 2 / (8 * math.sin(math.pi * h / 2) ** 2) * np.outer(np.sin(math.pi * xs),
                                                                                        np.sin(math.pi * xs))
    exact[0, :] = exact[-1, :] = exact[:, 0] = exact[:, -1] = 0.0
    assert info["status"] == "MG_OK" and info["relres"] <= 1e-10
    assert np.linalg.norm(x.cpu().numpy() - exact) <= 2e-10 * np.linalg.norm(exact)
    o = oracle_of(sp, 6, "jacobi", 0.8)
    xo, st, co, rr, ho = o.solve(sp.b, tol=1e-10, maxit=50)
    assert info["cycles"] == co and rel(x, xo) <= TOL64


# ---------------------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------------------

def test_single_level_is_direct_solve():
    rng = np.random.default_rng(1)
    sp = spec_of(2, (9, 17), False, inputs.CELL, rng)
    o = oracle_of(sp, 1, "rbgs", 1.0)
    s = Solver(sp, levels=1, smoother="rbgs", max_cycles=3)
    x, info = s.solve(sp.b, tol=1e-12)
    assert info["cycles"] == 1 and rel(x, o.solve(sp.b, tol=1e-12)[0]) <= 1e-11


def test_zero_rhs_gives_zero():
    rng = np.random.default_rng(2)
    sp = spec_of(2, (33, 33), False, inputs.CONST, rng)
    s = Solver(sp, levels=4, smoother="rbgs")
    x, info = s.solve(np.zeros(sp.shape), x0=rng.standard_normal(sp.shape))
    assert info["status"] == "MG_OK" and info["cycles"] == 0 and float(x.abs().max()) == 0.0


def test_tiny_grid_and_boundary_values_ignored():
    rng = np.random.default_rng(3)
    sp = spec_of(2, (3, 3), False, inputs.CONST, rng)
    s = Solver(sp, levels=1, smoother="rbgs")
    b = rng.standard_normal((3, 3))
    x, info = s.solve(b, x0=rng.standard_normal((3, 3)), tol=1e-14)
    xn = x.cpu().numpy()
    assert xn[1, 1] == pytest.approx(b[1, 1] / (2 * sp.c[0] + 2 * sp.c[1]), rel=1e-14)
    assert np.all(xn[0, :] == 0) and np.all(xn[:, 0] == 0) and np.all(xn[-1, :] == 0) and np.all(xn[:, -1] == 0)


def test_no_convergence_status():
    rng = np.random.default_rng(4)
    sp = spec_of(2, (65, 65), False, inputs.CONST, rng, eps=1e-4)
    s = Solver(sp, levels=6, smoother="jacobi", omega=0.8, max_cycles=3)
    x, info = s.solve(sp.b, tol=1e-10)
    assert info["status"] == "MG_ENOCONV" and info["cycles"] == 3 and info["relres"] > 1e-10


def test_nonfinite_rhs_reports_divergence():
    rng = np.random.default_rng(5)
    sp = spec_of(2, (17, 17), False, inputs.CONST, rng)
    s = Solver(sp, levels=3, smoother="rbgs")
    b = sp.b.copy()
    b[5, 5] = np.nan
    x, info = s.solve(b, tol=1e-10)
    assert info["status"] == "MG_EDIVERGED"


# ---------------------------------------------------------------------------------------
# alternative kernel paths give the same iterates
# ---------------------------------------------------------------------------------------
from paper_0805_3041_gb300.binding import FLAG_NO_GRAPH  # noqa: E402

FLAG_NO_FUSED_COARSE, FLAG_NO_FUSED_SWEEP = 4, 8


@pytest.mark.parametrize("flags", [FLAG_NO_GRAPH, FLAG_NO_FUSED_COARSE, FLAG_NO_FUSED_SWEEP,
                                   FLAG_NO_FUSED_COARSE | FLAG_NO_FUSED_SWEEP | FLAG_NO_GRAPH])
@pytest.mark.parametrize("smoother", ["rbgs", "jacobi"])
def test_kernel_paths_agree(flags, smoother):
    rng = np.random.default_rng(11)
    sp = spec_of(2, (257, 129), False, inputs.CONST, rng, eps=0.5)
    om = 0.8 if smoother == "jacobi" else 1.0
    a = Solver(sp, levels=7, smoother=smoother, omega=om, max_cycles=3)
    b = Solver(sp, levels=7, smoother=smoother, omega=om, max_cycles=3, flags=flags)
    xa, ia = a.solve(sp.b, tol=0.0)
    xb, ib = b.solve(sp.b, tol=0.0)
    assert rel(xa, xb.cpu().numpy()) <= 1e-12


# ---------------------------------------------------------------------------------------
# mixed precision: FP32 cycles, FP64 defect / update / coarsest solve
# ---------------------------------------------------------------------------------------
MIXED = [
    (2, (257, 257), False, inputs.CONST, 8, "rbgs", 1.0, 1.0),
    (2, (257, 129), False, inputs.CONST, 7, "zebra_y", 1.0, 1e-3),
    (2, (129, 128), True, inputs.SEPARABLE, 7, "rbgs", 1.0, 1.0),
    (2, (129, 129), False, inputs.CELL, 7, "rbgs", 1.0, 1.0),
    (3, (33, 33, 33), False, inputs.CONST, 4, "rbgs", 1.0, 1.0),
    (2, (65, 65), False, inputs.CONST, 6, "jacobi", 0.8, 1.0),
]


@pytest.mark.parametrize("dim,n,per,kind,L,sm,om,eps", MIXED)
def test_mixed_precision_reaches_fp64_residual(dim, n, per, kind, L, sm, om, eps):
    """The refined solution meets the 1e-10 relative residual computed independently in FP64
    (by the oracle's operator); its distance to the FP64 oracle solution is reported."""
    rng = np.random.default_rng(12)
    sp = spec_of(dim, n, per, kind, rng, eps=eps)
    o = oracle_of(sp, L, sm, om)
    s = Solver(sp, levels=L, smoother=sm, omega=om, precision="mixed", max_cycles=40)
    x, info = s.solve(sp.b, tol=1e-10)
    xn = x.cpu().numpy()
    rr = o.norm(o.defect(xn, sp.b)) / o.norm(sp.b)
    assert info["status"] == "MG_OK" and rr <= 1e-10, (info, rr)
    assert abs(rr - info["relres"]) <= 1e-3 * rr + 1e-16
    xo, st, co, rro, ho = o.solve(sp.b, tol=1e-13, maxit=200)
    err = rel(xn, xo)
    print(f"mixed vs FP64 oracle: max rel err {err:.2e}, refinement steps {info['cycles']} (FP64 cycles to 1e-10: "
          f"{int(np.argmax(ho <= 1e-10))})")
    assert err <= 1e-6
