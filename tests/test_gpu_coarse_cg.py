"""Coarsest grids above the dense-inverse limit (4096 unknowns): FP64 conjugate gradients to a
relative residual of 1e-14 in one cooperative launch.

The coarse solve leaves a residual within 1e-12 of ||g|| (recomputed with the oracle's operator).
Against the oracle's own CG, and in the few-grid solves (the "Grid levels" study, where the
coarsest grid is large) against the oracle's F-cycles, the bar is what the two residuals allow:
u - u_o = A^{-1} (r_o - r) exactly, so

    ||u - u_o||_2 <= ||A^{-1}||_2 (||r - r_o||_2 + e_r),

with ||A^{-1}||_2 = 1 / lambda_min(A) estimated by power iteration on A^{-1} (the oracle's own
solve) and taken twice, and e_r the rounding of the two recomputed defects, 2 * 8 * 2^-53 times
the norm of |g| + |A||u|.  Few-grid solves also take the oracle's cycle count; single-level
solves are one CG solve.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver  # noqa: E402
from test_gpu_parity import spec_of, rel  # noqa: E402
from test_gpu_edge import random_edges  # noqa: E402


def oracle_for(sp, levels, smoother="rbgs", omega=1.0):
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c, sx=sp.sx, sy=sp.sy,
                    sz=sp.sz, k=sp.k, ex=sp.ex, ey=sp.ey, ez=sp.ez)
    return orc.Oracle(p, levels=levels, smoother=smoother, omega=omega, dense_max=4096)


CASES = [
    # name, spec factory, levels (coarsest unknowns)
    ("2d-257x129-const-L2", lambda r: spec_of(2, (257, 129), False, inputs.CONST, r), 2),        # 8001
    ("2d-257x128-per-sep-L2", lambda r: spec_of(2, (257, 128), True, inputs.SEPARABLE, r), 2),   # 8128
    ("2d-129x129-cell-L1", lambda r: spec_of(2, (129, 129), False, inputs.CELL, r), 1),          # 16129
    ("3d-33x33x33-const-L1", lambda r: spec_of(3, (33, 33, 33), False, inputs.CONST, r), 1),     # 29791
    ("2d-129x65-edge-L1", lambda r: random_edges(2, (129, 65), False, 11), 1),                   # 8001
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: c[0])
def case(request):
    name, make, L = request.param
    rng = np.random.default_rng(abs(hash(name)) % 2 ** 32)
    sp = make(rng)
    return sp, oracle_for(sp, L), L, rng


U64 = 2.0 ** -53


def inverse_norm(apply_inv, o, l, rng, iters=12):
    """||A_l^{-1}||_2 by power iteration on A_l^{-1} (A_l symmetric positive definite)."""
    v = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
    v /= o.norm(v, l)
    mu = 0.0
    for _ in range(iters):
        w = apply_inv(v)
        nu = o.norm(w, l)
        v = w / nu
        if abs(nu - mu) <= 1e-3 * nu:
            break
        mu = nu
    return nu


def residual_bar(o, l, u, uo, g, inv_norm):
    """2 ||A^{-1}|| (||r - r_o|| + e_r) for iterates u, uo of A_l u = g (2-norm over the unknowns)."""
    r, ro = o.defect(u, g, l), o.defect(uo, g, l)
    m = o.unknown_mask(l)
    terms = lambda v: (np.abs(g) + 2.0 * o.diag(l) * np.abs(v) - o.apply(np.abs(v), l)) * m   # |g| + |A||v|
    e_r = 8 * U64 * (o.norm(terms(u), l) + o.norm(terms(uo), l))
    return 2.0 * inv_norm * (o.norm(r - ro, l) + e_r)


def test_cg_coarse_solve_is_exact(case):
    sp, o, L, rng = case
    s = Solver(sp, levels=L, smoother="rbgs", max_cycles=50)
    g = rng.standard_normal(o.shape(1)) * o.unknown_mask(1)
    u = s.coarse_solve(g).cpu().numpy()
    r = o.defect(u, g, 1)
    # CG stops on its updated residual (1e-14); the recomputed one carries the rounding drift
    assert o.norm(r, 1) <= 1e-12 * o.norm(g, 1)
    uo = o.coarse_solve(g)
    inv = inverse_norm(o.coarse_solve, o, 1, rng)
    diff = o.norm((u - uo) * o.unknown_mask(1), 1)
    bar = residual_bar(o, 1, u, uo, g, inv)
    print(f"||u - u_o|| / ||u_o|| {diff / o.norm(uo, 1):.2e}, bar {bar / o.norm(uo, 1):.2e} "
          f"(||A^-1|| {inv:.3e})")
    assert diff <= bar


def test_few_grid_solve_matches_oracle(case):
    sp, o, L, rng = case
    x, info = Solver(sp, levels=L, smoother="rbgs", max_cycles=50).solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=50)
    assert info["status"] == "MG_OK" and sto == orc.OK
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-2):
        assert info["cycles"] == co
    if L == 1:
        assert info["cycles"] == 1   # one exact solve
        inv = inverse_norm(o.coarse_solve, o, 1, rng)
    else:
        inv = inverse_norm(lambda v: o.solve(v, tol=1e-12, maxit=100)[0], o, L, rng)
    xn = x.cpu().numpy()
    diff = o.norm((xn - xo) * o.unknown_mask(), L)
    bar = residual_bar(o, L, xn, xo, sp.b, inv)
    print(f"||x - x_o|| / ||x_o|| {diff / o.norm(xo, L):.2e}, bar {bar / o.norm(xo, L):.2e} (||A^-1|| {inv:.3e})")
    assert diff <= bar


def test_few_grid_mixed_solve(case):
    sp, o, L, rng = case
    x, info = Solver(sp, levels=L, smoother="rbgs", precision="mixed", max_cycles=50).solve(sp.b, tol=1e-10)
    assert info["status"] == "MG_OK" and info["relres"] <= 1e-10
