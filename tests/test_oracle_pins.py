"""Pins of the FP64 CPU oracle against facts fixed by the mathematics (no GPU).

Each test checks the oracle against something other than itself: closed-form
eigenpairs of the discrete operators, exact invariants of Gauss-Seidel-type
sweeps, the adjointness of restriction and prolongation, dense direct solves on
tiny grids (numpy), textbook two-grid rates, finite differences of the loss.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs


def const_problem(n, eps=1.0, dim=2, periodic_y=False):
    if dim == 2:
        n0, n1 = n if isinstance(n, tuple) else (n, n)
        hx = 1.0 / (n0 - 1)
        hy = 1.0 / n1 if periodic_y else 1.0 / (n1 - 1)
        return orc.Problem(dim=2, n=(n0, n1, 1), periodic_y=periodic_y, kind=orc.CONST, h=(hx, hy, 1.0),
                           c=(eps / hx ** 2, 1.0 / hy ** 2, 0.0))
    h = 1.0 / (n - 1)
    hy = 1.0 / (n - 1) if not periodic_y else 1.0 / (n - 1)
    return orc.Problem(dim=3, n=(n, n - 1 if periodic_y else n, n), periodic_y=periodic_y, kind=orc.CONST,
                       h=(h, hy, h), c=(eps / h ** 2, 1.0 / hy ** 2, 2.0 / h ** 2))


def rand_field(o, rng, l=None):
    return rng.standard_normal(o.shape(l)) * o.unknown_mask(l)


# --------------------------------------------------------------------------------------
# operator
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("n,eps", [(17, 1.0), (33, 0.01), (9, 1e-4)])
def test_eigenpairs_2d(n, eps):
    """A sin(p pi x) sin(q pi y) = (4/h^2)(eps sin^2(p pi h/2) + sin^2(q pi h/2)) sin sin."""
    o = orc.Oracle(const_problem(n, eps), levels=1)
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    for p, q in [(1, 1), (2, 5), (n - 2, 1), (3, n - 2)]:
        v = np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x))
        lam = 4.0 / h ** 2 * (eps * math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2)
        Av = o.apply(v)
        assert np.max(np.abs(Av - lam * v * o.unknown_mask())) <= 1e-12 * lam


def test_eigenpairs_3d():
    n = 9
    o = orc.Oracle(const_problem(n, 0.5, dim=3), levels=1)
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    cx, cy, cz = 0.5 / h ** 2, 1.0 / h ** 2, 2.0 / h ** 2
    for p, q, r in [(1, 1, 1), (2, 3, 7), (7, 1, 4)]:
        v = np.einsum("k,j,i->kji", np.sin(r * math.pi * x), np.sin(q * math.pi * x), np.sin(p * math.pi * x))
        lam = 4 * (cx * math.sin(p * math.pi * h / 2) ** 2 + cy * math.sin(q * math.pi * h / 2) ** 2
                   + cz * math.sin(r * math.pi * h / 2) ** 2)
        assert np.max(np.abs(o.apply(v) - lam * v * o.unknown_mask())) <= 1e-12 * lam


def test_eigenpairs_periodic_y():
    """Periodic y with n1 distinct nodes: mode sin(p pi x) cos(2 pi m j / n1)."""
    n0, n1 = 17, 16
    o = orc.Oracle(const_problem((n0, n1), 0.3, periodic_y=True), levels=1)
    hx = 1.0 / (n0 - 1)
    cx, cy = 0.3 / hx ** 2, float(n1) ** 2
    i = np.arange(n0)
    j = np.arange(n1)
    for p, m in [(1, 0), (3, 1), (15, 8), (2, 5)]:
        v = np.outer(np.cos(2 * math.pi * m * j / n1), np.sin(p * math.pi * i * hx))
        lam = 4 * cx * math.sin(p * math.pi * hx / 2) ** 2 + 4 * cy * math.sin(math.pi * m / n1) ** 2
        assert np.max(np.abs(o.apply(v) - lam * v * o.unknown_mask())) <= 1e-12 * max(lam, 1.0)


def _kinds(dim, periodic_y, rng):
    n = (17, 16 if periodic_y else 17, 9 if dim == 3 else 1)
    h = (1 / 16, 1 / 16, 1 / 8)
    out = [orc.Problem(dim=dim, n=n, periodic_y=periodic_y, kind=orc.CONST, h=h, c=(3.0, 1.5, 0.7))]
    out.append(orc.Problem(dim=dim, n=n, periodic_y=periodic_y, kind=orc.SEPARABLE, h=h,
                           sx=rng.uniform(0.5, 2, n[0] - 1), sy=rng.uniform(0.5, 2, n[0]),
                           sz=rng.uniform(0.5, 2, n[0])))
    cy = n[1] if periodic_y else n[1] - 1
    kshape = (cy, n[0] - 1) if dim == 2 else (n[2] - 1, cy, n[0] - 1)
    out.append(orc.Problem(dim=dim, n=n, periodic_y=periodic_y, kind=orc.CELL, h=h,
                           k=np.exp(rng.standard_normal(kshape))))
    out.append(_random_edge_problem(dim, n, periodic_y, h, rng))
    return out


def _random_edge_problem(dim, n, periodic_y, h, rng):
    """Edge weights log-normal and independent edge by edge (varying in every direction)."""
    shape = (n[1], n[0]) if dim == 2 else (n[2], n[1], n[0])
    w = [np.exp(0.5 * rng.standard_normal(shape)) for _ in range(3)]
    return orc.Problem(dim=dim, n=n, periodic_y=periodic_y, kind=orc.EDGE, h=h, ex=w[0], ey=w[1],
                       ez=w[2] if dim == 3 else None)


def _edge_of_separable(p):
    """The separable problem p written as per-edge weights (the same operator)."""
    shape = (p.n[1], p.n[0]) if p.dim == 2 else (p.n[2], p.n[1], p.n[0])
    ex, ey, ez = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    ex[..., :-1] = p.sx[: p.n[0] - 1]
    ey[...] = p.sy
    ez[...] = p.sz
    return orc.Problem(dim=p.dim, n=p.n, periodic_y=p.periodic_y, kind=orc.EDGE, h=p.h, ex=ex, ey=ey,
                       ez=ez if p.dim == 3 else None)


@pytest.mark.parametrize("dim,periodic_y", [(2, False), (2, True), (3, False), (3, True)])
def test_symmetry_all_kinds(dim, periodic_y):
    """<A u, v> = <u, A v> and <A u, u> > 0 for every coefficient kind on every level."""
    rng = np.random.default_rng(0)
    for prob in _kinds(dim, periodic_y, rng):
        o = orc.Oracle(prob, levels=3)
        for l in (1, 2, 3):
            u, v = rand_field(o, rng, l), rand_field(o, rng, l)
            a, b = np.vdot(o.apply(u, l), v), np.vdot(u, o.apply(v, l))
            assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
            assert np.vdot(o.apply(u, l), u) > 0


def test_energy_edge_sum_cell_kind():
    """u^T A u equals the edge sum sum_e w_e (u_p - u_q)^2 with w_e the mean of the
    cells touching the edge over h^2 (finite-volume weights), written out here by hand."""
    rng = np.random.default_rng(3)
    n = 9
    h = 1.0 / (n - 1)
    k = np.exp(rng.standard_normal((n - 1, n - 1)))
    o = orc.Oracle(orc.Problem(dim=2, n=(n, n, 1), kind=orc.CELL, h=(h, h, 1), k=k), levels=1)
    u = rand_field(o, rng)
    e = 0.0
    for j in range(n):
        for i in range(n):
            if i + 1 < n and 0 < j < n - 1:
                e += (k[j - 1, i] + k[j, i]) / (2 * h * h) * (u[j, i] - u[j, i + 1]) ** 2
            if j + 1 < n and 0 < i < n - 1:
                e += (k[j, i - 1] + k[j, i]) / (2 * h * h) * (u[j, i] - u[j + 1, i]) ** 2
    assert abs(np.vdot(u, o.apply(u)) - e) <= 1e-12 * e


def test_cell_kind_with_constant_k_is_laplacian():
    n = 17
    h = 1.0 / (n - 1)
    oc = orc.Oracle(orc.Problem(dim=2, n=(n, n, 1), kind=orc.CELL, h=(h, h, 1),
                                k=np.full((n - 1, n - 1), 2.5)), levels=3)
    ol = orc.Oracle(const_problem(n, 1.0), levels=3)
    u = rand_field(oc, np.random.default_rng(1))
    assert np.allclose(oc.apply(u), 2.5 * ol.apply(u), rtol=1e-13, atol=0)
    # the coarse cell fields average children: a constant stays constant, and h doubles
    assert np.allclose(oc.level_coeffs(2), 2.5)


def test_separable_coarsening_rule():
    """Coarse x-edge weight = 1/4 harmonic mean of the two fine edges; y-weights injected x 1/4;
    constant weights just scale by 1/4."""
    rng = np.random.default_rng(2)
    n = 17
    sx, sy = rng.uniform(1, 3, n - 1), rng.uniform(1, 3, n)
    o = orc.Oracle(orc.Problem(dim=2, n=(n, n, 1), kind=orc.SEPARABLE, sx=sx, sy=sy, sz=np.zeros(n)), levels=2)
    cc = o.level_coeffs(1)
    nc = 9
    a, b = sx[0::2], sx[1::2]
    assert np.allclose(cc[:nc - 1], 0.25 / (0.5 / a + 0.5 / b), rtol=1e-14)
    assert np.allclose(cc[nc:2 * nc], 0.25 * sy[0::2], rtol=1e-14)
    oc = orc.Oracle(const_problem(17, 0.3), levels=3)
    assert np.allclose(oc.level_coeffs(1)[:2], np.array([0.3, 1.0]) * 16 ** 2 / 16, rtol=1e-14)


def test_polar_weights_are_second_order():
    """The annulus weights discretise r * (-Laplace u) in polar coordinates: the
    truncation error on a smooth u falls 4x per halving of h."""
    errs = []
    for nr, nt in [(33, 32), (65, 64), (129, 128)]:
        sp = inputs.annulus_2d(nr=nr, nt=nt)
        o = orc.Oracle(orc.Problem(dim=2, n=sp.n, periodic_y=True, kind=orc.SEPARABLE, h=sp.h,
                                   sx=sp.sx, sy=sp.sy, sz=sp.sz), levels=1)
        r = 0.1 + sp.h[0] * np.arange(nr)
        t = sp.h[1] * np.arange(nt)
        R, T = np.meshgrid(r, t)
        s = (R - 0.1) / 0.9
        u = np.sin(math.pi * s) * (1 + 0.5 * np.cos(2 * T))     # zero at r = 0.1 and r = 1
        # -(1/r) d/dr(r u_r) - (1/r^2) u_tt, times r
        a = math.pi / 0.9
        ur = a * np.cos(math.pi * s) * (1 + 0.5 * np.cos(2 * T))
        urr = -a * a * np.sin(math.pi * s) * (1 + 0.5 * np.cos(2 * T))
        utt = np.sin(math.pi * s) * (-2.0 * np.cos(2 * T))
        exact = -(R * urr + ur) - utt / R
        m = o.unknown_mask()
        errs.append(np.max(np.abs((o.apply(u) - exact)[m])))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_diag_is_operator_diagonal():
    rng = np.random.default_rng(5)
    for prob in _kinds(2, True, rng) + _kinds(3, False, rng):
        o = orc.Oracle(prob, levels=1)
        D = o.diag()
        m = o.unknown_mask()
        idx = np.argwhere(m)[:: max(1, int(m.sum()) // 25)]
        for t in idx:
            e = np.zeros(o.shape())
            e[tuple(t)] = 1.0
            assert abs(o.apply(e)[tuple(t)] - D[tuple(t)]) <= 1e-13 * D[tuple(t)]


# --------------------------------------------------------------------------------------
# smoothers
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("omega", [0.8, 0.5])
def test_jacobi_mode_multiplier(omega):
    """One damped-Jacobi sweep multiplies a Dirichlet sine mode by 1 - omega lambda / D."""
    n, eps = 17, 0.25
    o = orc.Oracle(const_problem(n, eps), levels=1, smoother="jacobi", omega=omega)
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    D = 2 * eps / h ** 2 + 2 / h ** 2
    for p, q in [(1, 2), (9, 3), (15, 15)]:
        v = np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x))
        lam = 4.0 / h ** 2 * (eps * math.sin(p * math.pi * h / 2) ** 2 + math.sin(q * math.pi * h / 2) ** 2)
        out = o.smooth(v, np.zeros_like(v), 1)
        assert np.max(np.abs(out - (1 - omega * lam / D) * v * o.unknown_mask())) <= 1e-13


def test_jacobi_smoothing_factor():
    """Over the high modes (max(p,q) >= n/2) damped Jacobi with omega = 0.8 reduces
    every mode by at most mu = max(|1-2w|, |1-w/2|) = 0.6 (2-D Poisson)."""
    n = 33
    o = orc.Oracle(const_problem(n), levels=1, smoother="jacobi", omega=0.8)
    x = np.arange(n) / (n - 1)
    worst = 0.0
    for p in range(1, n - 1):
        for q in range(1, n - 1):
            if max(p, q) < (n - 1) // 2:
                continue
            v = np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x))
            out = o.smooth(v, np.zeros_like(v), 1)
            worst = max(worst, np.linalg.norm(out) / np.linalg.norm(v))
    assert 0.58 < worst <= 0.6 + 1e-12


@pytest.mark.parametrize("smoother,order,colour_of", [
    ("rbgs", orc.RED_FIRST, lambda i, j, k: (i + j + k) % 2 == 1),
    ("rbgs", orc.BLACK_FIRST, lambda i, j, k: (i + j + k) % 2 == 0),
    ("zebra_x", orc.RED_FIRST, lambda i, j, k: (j + k) % 2 == 1),
    ("zebra_y", orc.BLACK_FIRST, lambda i, j, k: (i + k) % 2 == 0),
])
@pytest.mark.parametrize("dim", [2, 3])
def test_gauss_seidel_invariant(smoother, order, colour_of, dim):
    """With omega = 1 the colour updated last has exactly zero residual afterwards."""
    rng = np.random.default_rng(7)
    prob = _kinds(dim, False, rng)[2]
    o = orc.Oracle(prob, levels=1, smoother=smoother, omega=1.0)
    u, g = rand_field(o, rng), rand_field(o, rng)
    r = o.defect(o.smooth(u, g, 1, order), g)
    m = o.unknown_mask()
    last = np.zeros_like(m)
    for idx in np.argwhere(m):
        if dim == 2:
            j, i = idx
            k = 0
        else:
            k, j, i = idx
        last[tuple(idx)] = colour_of(i, j, k)
    scale = np.max(np.abs(o.defect(u, g)))
    assert np.max(np.abs(r[last])) <= 1e-12 * scale
    assert np.max(np.abs(r[m & ~last])) > 1e-6 * scale


@pytest.mark.parametrize("direction", ["x", "y"])
def test_line_jacobi_mode_multiplier(direction):
    """Line Jacobi (C = tridiagonal part of A along the line) multiplies a sine mode by
    1 - omega lambda / c with c = 2 w_perp + 4 w_line sin^2(theta_line / 2)."""
    n, eps, omega = 17, 1e-3, 0.7
    o = orc.Oracle(const_problem(n, eps), levels=1, smoother="line_" + direction, omega=omega)
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    wx, wy = eps / h ** 2, 1 / h ** 2
    for p, q in [(1, 1), (4, 13), (15, 2)]:
        v = np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x))
        sx, sy = math.sin(p * math.pi * h / 2) ** 2, math.sin(q * math.pi * h / 2) ** 2
        lam = 4 * wx * sx + 4 * wy * sy
        c = 2 * wy + 4 * wx * sx if direction == "x" else 2 * wx + 4 * wy * sy
        out = o.smooth(v, np.zeros_like(v), 1)
        assert np.max(np.abs(out - (1 - omega * lam / c) * v * o.unknown_mask())) <= 1e-12


@pytest.mark.parametrize("eps", [1.0, 1e-3])
def test_adi_mode_multiplier_is_product_of_line_multipliers(eps):
    """One ADI sweep (x-line Jacobi, then y-line Jacobi) maps a sine mode of the constant
    operator to itself times (1 - omega lambda / c_x)(1 - omega lambda / c_y): each line
    sweep is diagonal in the sine basis with the multipliers of the line-Jacobi pin."""
    n, omega = 17, 0.7
    o = orc.Oracle(const_problem(n, eps), levels=1, smoother="adi", omega=omega)
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    wx, wy = eps / h ** 2, 1 / h ** 2
    for p, q in [(1, 1), (4, 13), (15, 2), (9, 9)]:
        v = np.outer(np.sin(q * math.pi * x), np.sin(p * math.pi * x))
        sx, sy = math.sin(p * math.pi * h / 2) ** 2, math.sin(q * math.pi * h / 2) ** 2
        lam = 4 * wx * sx + 4 * wy * sy
        cx, cy = 2 * wy + 4 * wx * sx, 2 * wx + 4 * wy * sy
        mult = (1 - omega * lam / cx) * (1 - omega * lam / cy)
        out = o.smooth(v, np.zeros_like(v), 1)
        assert np.max(np.abs(out - mult * v * o.unknown_mask())) <= 1e-12


def test_gsadi_is_zebra_x_then_zebra_y():
    """GSADI equals a zebra x-line sweep followed by a zebra y-line sweep (order matters:
    the reverse composition, which the transposed cycle uses, differs)."""
    rng = np.random.default_rng(17)
    prob = _small(2, False, 2, 17, rng)
    kw = dict(levels=1, omega=1.0)
    g = orc.Oracle(prob, smoother="gsadi", **kw)
    zx, zy = orc.Oracle(prob, smoother="zebra_x", **kw), orc.Oracle(prob, smoother="zebra_y", **kw)
    u = rand_field(g, rng)
    b = rand_field(g, rng)
    both = g.smooth(u, b, 1)
    assert np.array_equal(both, zy.smooth(zx.smooth(u, b, 1), b, 1))
    rev = zx.smooth(zy.smooth(u, b, 1, order=1), b, 1, order=1)
    assert np.array_equal(g.smooth(u, b, 1, order=1), rev)
    assert np.max(np.abs(rev - both)) > 1e-6 * np.max(np.abs(both))


def test_thomas_matches_dense():
    rng = np.random.default_rng(9)
    m = 37
    lo, up = -rng.uniform(0, 1, m), -rng.uniform(0, 1, m)
    di = 2.5 + rng.uniform(0, 1, m)
    d = rng.standard_normal(m)
    T = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    assert np.allclose(orc.thomas(lo, di, up, d), np.linalg.solve(T, d), rtol=0, atol=1e-13)


# --------------------------------------------------------------------------------------
# grid transfers
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,periodic_y", [(2, False), (2, True), (3, False), (3, True)])
def test_restriction_is_scaled_transpose_of_prolongation(dim, periodic_y):
    """<R r, e>_coarse = 2^-d <r, P e>_fine for all r, e (full weighting vs. (bi/tri)linear)."""
    rng = np.random.default_rng(4)
    o = orc.Oracle(_kinds(dim, periodic_y, rng)[0], levels=3)
    for lf in (2, 3):
        r, e = rand_field(o, rng, lf), rand_field(o, rng, lf - 1)
        lhs = np.vdot(o.restrict(r, lf), e)
        Pe = o.prolong_add(e, np.zeros(o.shape(lf)), 1.0, lf)
        assert abs(lhs - 2.0 ** -dim * np.vdot(r, Pe)) <= 1e-13 * np.abs(r).sum()


def test_prolongation_reproduces_bilinear():
    n = 33
    o = orc.Oracle(const_problem(n), levels=2)
    xc = np.arange(17) / 16
    X, Y = np.meshgrid(xc, xc)
    e = 0.3 + 1.7 * X - 0.9 * Y + 2.3 * X * Y
    u = o.prolong_add(e, np.zeros(o.shape()), 1.0)
    xf = np.arange(n) / (n - 1)
    Xf, Yf = np.meshgrid(xf, xf)
    ef = 0.3 + 1.7 * Xf - 0.9 * Yf + 2.3 * Xf * Yf
    # fine nodes whose interpolation stencil uses only coarse unknowns
    assert np.max(np.abs(u[2:-2, 2:-2] - ef[2:-2, 2:-2])) <= 1e-13
    # 3-D trilinear
    o3 = orc.Oracle(const_problem(17, dim=3), levels=2)
    xc = np.arange(9) / 8
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    e = 1 + X - 2 * Y + 3 * Z + X * Y * Z
    u = o3.prolong_add(e, np.zeros(o3.shape()), 1.0)
    xf = np.arange(17) / 16
    Z, Y, X = np.meshgrid(xf, xf, xf, indexing="ij")
    ef = 1 + X - 2 * Y + 3 * Z + X * Y * Z
    assert np.max(np.abs(u[2:-2, 2:-2, 2:-2] - ef[2:-2, 2:-2, 2:-2])) <= 1e-13


def test_restriction_of_constant():
    o = orc.Oracle(const_problem(33), levels=2)
    g = o.restrict(np.full(o.shape(), 1.0) * o.unknown_mask())
    assert np.allclose(g[1:-1, 1:-1][1:-1, 1:-1], 1.0, rtol=0, atol=1e-15)
    # periodic y: the constant is kept on every coarse row
    o = orc.Oracle(const_problem((17, 16), periodic_y=True), levels=2)
    g = o.restrict(np.full(o.shape(), 2.0) * o.unknown_mask())
    assert np.allclose(g[:, 2:-2], 2.0, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------------------
# coarsest solve, F-cycle
# --------------------------------------------------------------------------------------

def dense_matrix(o, l=None):
    m = o.unknown_mask(l)
    idx = np.argwhere(m)
    A = np.zeros((len(idx), len(idx)))
    for c, t in enumerate(idx):
        e = np.zeros(o.shape(l))
        e[tuple(t)] = 1.0
        A[:, c] = o.apply(e, l)[m]
    return A, m


@pytest.mark.parametrize("kind_idx", [0, 1, 2])
def test_coarse_solve_matches_dense(kind_idx):
    rng = np.random.default_rng(6)
    o = orc.Oracle(_kinds(2, True, rng)[kind_idx], levels=3)
    A, m = dense_matrix(o, 1)
    g = rand_field(o, rng, 1)
    u = o.coarse_solve(g)
    assert np.allclose(u[m], np.linalg.solve(A, g[m]), rtol=0, atol=1e-13 * np.abs(np.linalg.solve(A, g[m])).max())


def test_coarse_cg_matches_dense():
    rng = np.random.default_rng(6)
    o = orc.Oracle(_kinds(2, False, rng)[2], levels=2, dense_max=10)
    A, m = dense_matrix(o, 1)
    g = rand_field(o, rng, 1)
    ref = np.linalg.solve(A, g[m])
    assert np.max(np.abs(o.coarse_solve(g)[m] - ref)) <= 1e-11 * np.abs(ref).max()


CASES = [
    (2, False, 0, "rbgs", 5, 2), (2, False, 2, "jacobi", 9, 3), (2, True, 1, "zebra_x", 17, 4),
    (2, False, 2, "zebra_y", 17, 4), (2, False, 0, "line_y", 17, 3), (3, False, 0, "rbgs", 5, 2),
    (3, True, 1, "zebra_x", 9, 3), (3, False, 2, "jacobi", 9, 2),
    (2, False, 0, "adi", 17, 3), (2, False, 2, "gsadi", 17, 4), (3, False, 1, "adi", 9, 3),
    (3, False, 0, "gsadi", 9, 2),
    # edge weights varying in every direction
    (2, True, 3, "zebra_x", 17, 4), (2, False, 3, "gsadi", 17, 3), (3, False, 3, "rbgs", 9, 2),
    (3, True, 3, "jacobi", 9, 3),
    # lines across the periodic direction (cyclic tridiagonal systems)
    (2, True, 1, "zebra_y", 17, 3), (2, True, 2, "line_y", 17, 3), (2, True, 3, "gsadi", 17, 3),
    (3, True, 0, "adi", 9, 2),
]


def _small(dim, periodic_y, kind_idx, n, rng):
    probs = _kinds(dim, periodic_y, rng)
    p = probs[kind_idx]
    ny = n - 1 if periodic_y else n
    nn = (n, ny, n if dim == 3 else 1)
    h = p.h
    if p.kind == orc.CONST:
        return orc.Problem(dim=dim, n=nn, periodic_y=periodic_y, kind=orc.CONST, h=h, c=p.c)
    if p.kind == orc.SEPARABLE:
        return orc.Problem(dim=dim, n=nn, periodic_y=periodic_y, kind=orc.SEPARABLE, h=h,
                           sx=rng.uniform(0.5, 2, n - 1), sy=rng.uniform(0.5, 2, n), sz=rng.uniform(0.5, 2, n))
    if p.kind == orc.EDGE:
        return _random_edge_problem(dim, nn, periodic_y, h, rng)
    cy = ny if periodic_y else ny - 1
    ks = (cy, n - 1) if dim == 2 else (n - 1, cy, n - 1)
    return orc.Problem(dim=dim, n=nn, periodic_y=periodic_y, kind=orc.CELL, h=h, k=np.exp(rng.standard_normal(ks)))


@pytest.mark.parametrize("dim,per,kind_idx,smoother,n,levels", CASES)
def test_fcycle_converges_to_dense_solution(dim, per, kind_idx, smoother, n, levels):
    rng = np.random.default_rng(10)
    prob = _small(dim, per, kind_idx, n, rng)
    omega = 0.8 if smoother in ("jacobi", "line_y") else 1.0
    o = orc.Oracle(prob, levels=levels, smoother=smoother, omega=omega)
    A, m = dense_matrix(o)
    b = rand_field(o, rng)
    x, st, cyc, rr, hist = o.solve(b, tol=1e-13, maxit=200)
    assert st == orc.OK
    ref = np.linalg.solve(A, b[m])
    assert np.max(np.abs(x[m] - ref)) <= 1e-11 * np.abs(ref).max()
    assert np.all(x[~m] == 0.0)


@pytest.mark.parametrize("L", [2, 3, 5])
def test_fcycle_level_visits(L):
    """F(l) visits level l once and runs F(l-1) then V(l-1) (V skipped when l-1 is the
    coarsest grid): level k >= 2 is smoothed on 1 + (L - k) visits, the coarsest grid is
    solved L - 1 times per cycle."""
    n = 2 ** L + 1
    o = orc.Oracle(const_problem(n), levels=L, nu1=1, nu2=2)
    b = rand_field(o, np.random.default_rng(0))
    o.reset_counts()
    o.cycle(np.zeros_like(b), b)
    sweeps, coarse = o.counts()
    for k in range(2, L + 1):
        assert sweeps[k - 1] == (1 + L - k) * 3
    assert coarse == L - 1


def _rate(o, b, ncyc):
    """Asymptotic residual reduction per cycle, measured before the rounding floor."""
    x, st, cyc, rr, hist = o.solve(b, tol=0.0, maxit=ncyc)
    m = max(i for i in range(len(hist)) if hist[i] > 1e-11 * hist[0])
    s = max(1, m - 3) if m > 1 else 0
    return (hist[m] / hist[s]) ** (1.0 / max(1, m - s))


def test_two_grid_rate_rbgs_matches_lfa():
    """Two-grid method, red-black Gauss-Seidel nu1 = nu2 = 1, full weighting, bilinear
    interpolation, 2-D Poisson: local Fourier analysis gives rho = 0.074 (textbook value)."""
    o = orc.Oracle(const_problem(65), levels=2, smoother="rbgs", nu1=1, nu2=1)
    b = rand_field(o, np.random.default_rng(1))
    assert 0.055 <= _rate(o, b, 12) <= 0.085


def test_fcycle_rate_is_mesh_independent():
    rates = []
    for n, L in [(33, 5), (65, 6), (129, 7)]:
        o = orc.Oracle(const_problem(n), levels=L, smoother="rbgs", nu1=2, nu2=2)
        rates.append(_rate(o, rand_field(o, np.random.default_rng(2)), 10))
    assert max(rates) < 0.06
    assert max(rates) - min(rates) < 0.02


def test_line_smoother_is_robust_for_anisotropy_point_smoother_is_not():
    """Section "Anisotropies": point smoothers degrade for -eps u_xx - u_yy with eps << 1;
    y-line smoothing (lines along the strong coupling) does not."""
    eps = 1e-3
    o_pt = orc.Oracle(const_problem(65, eps), levels=6, smoother="rbgs")
    o_ln = orc.Oracle(const_problem(65, eps), levels=6, smoother="zebra_y")
    b = rand_field(o_pt, np.random.default_rng(3))
    assert _rate(o_pt, b, 10) > 0.5
    assert _rate(o_ln, b, 10) < 0.1


def test_manufactured_closed_form_solution():
    """f = 2 pi^2 sin(pi x) sin(pi y) is an eigenvector of the 5-point operator, so the
    discrete solution is u = [2 pi^2 h^2 / (8 sin^2(pi h / 2))] sin(pi x) sin(pi y)."""
    sp = inputs.poisson_sin(129)
    o = orc.Oracle(orc.Problem(dim=2, n=sp.n, kind=orc.CONST, h=sp.h, c=sp.c), levels=6,
                   smoother="jacobi", omega=0.8)
    x, st, cyc, rr, hist = o.solve(sp.b, tol=1e-10, maxit=50)
    h = 1.0 / 128
    xs = np.arange(129) * h
    exact = 2 * math.pi ** 2 * h ** 2 / (8 * math.sin(math.pi * h / 2) ** 2) * np.outer(
        np.sin(math.pi * xs), np.sin(math.pi * xs))
    exact[0, :] = exact[-1, :] = exact[:, 0] = exact[:, -1] = 0.0
    assert st == orc.OK and rr <= 1e-10
    assert np.linalg.norm(x - exact) <= 2e-10 * np.linalg.norm(exact)


def test_fmg_start_on_one_level_is_the_exact_solution():
    """With a single level the nested iteration is the coarsest (exact) solve."""
    rng = np.random.default_rng(30)
    o = orc.Oracle(_small(2, False, 2, 17, rng), levels=1)
    A, m = dense_matrix(o, 1)
    b = rand_field(o, rng)
    x = o.fmg_start(b)
    ref = np.linalg.solve(A, b[m])
    assert np.max(np.abs(x[m] - ref)) <= 1e-12 * np.abs(ref).max()


def test_fmg_start_reaches_the_discretisation_error():
    """Nested iteration (one F-cycle per level) lands within the discretisation error of the
    closed-form discrete solution of the 129^2 sin(pi x) sin(pi y) problem: its algebraic
    error is far below the O(h^2) difference between the discrete and continuous solutions,
    while one F-cycle from zero is not."""
    n = 129
    h = 1.0 / (n - 1)
    xs = np.arange(n) * h
    S = np.outer(np.sin(math.pi * xs), np.sin(math.pi * xs))
    b = 2 * math.pi ** 2 * S
    exact = (2 * math.pi ** 2 * h ** 2 / (8 * math.sin(math.pi * h / 2) ** 2)) * S
    exact[0, :] = exact[-1, :] = exact[:, 0] = exact[:, -1] = 0.0
    o = orc.Oracle(const_problem(n), levels=6, smoother="jacobi", omega=0.8)
    x = o.fmg_start(b)
    disc = np.linalg.norm(exact - S * o.unknown_mask()) / np.linalg.norm(exact)   # ~ pi^2 h^2 / 12
    err = np.linalg.norm(x - exact) / np.linalg.norm(exact)
    one = np.linalg.norm(o.cycle(o.zeros(), b) - exact) / np.linalg.norm(exact)
    assert err <= 0.5 * disc < one


@pytest.mark.parametrize("smoother,eps", [("rbgs", 1.0), ("zebra_y", 1e-3)])
def test_fmg_start_saves_outer_cycles(smoother, eps):
    rng = np.random.default_rng(31)
    o = orc.Oracle(const_problem(129, eps), levels=6, smoother=smoother)
    b = rand_field(o, rng)
    _, st0, c0, r0, _ = o.solve(b, tol=1e-10)
    _, st1, c1, r1, _ = o.solve(b, tol=1e-10, start="fmg")
    assert st0 == st1 == orc.OK and r1 <= 1e-10 and c1 < c0


def test_solve_reports_no_convergence():
    o = orc.Oracle(const_problem(33, 1e-4), levels=5, smoother="jacobi", omega=0.8)
    b = rand_field(o, np.random.default_rng(0))
    x, st, cyc, rr, hist = o.solve(b, tol=1e-10, maxit=5)
    assert st == orc.ENOCONV and cyc == 5 and rr > 1e-10 and len(hist) == 6


# --------------------------------------------------------------------------------------
# adjoint and gradient
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,per,kind_idx,smoother,n,levels", CASES)
@pytest.mark.parametrize("ncyc", [1, 2, 3])
def test_transposed_cycle_dot_product(dim, per, kind_idx, smoother, n, levels, ncyc):
    """<M b, c> = <b, M^T c>, M = ncyc F-cycles from zero, M^T = ncyc transposed cycles."""
    rng = np.random.default_rng(20)
    prob = _small(dim, per, kind_idx, n, rng)
    o = orc.Oracle(prob, levels=levels, smoother=smoother, omega=0.8, nu1=1, nu2=2)
    b, c = rand_field(o, rng), rand_field(o, rng)
    xb, xc = np.zeros_like(b), np.zeros_like(c)
    for _ in range(ncyc):
        xb = o.cycle(xb, b)
        xc = o.cycle(xc, c, transposed=True)
    lhs, rhs = np.vdot(xb, c), np.vdot(b, xc)
    assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(xb) * np.linalg.norm(c))


def _loss_and_grad(n, k, f, uobs, levels):
    h = 1.0 / (n - 1)
    o = orc.Oracle(orc.Problem(dim=2, n=(n, n, 1), kind=orc.CELL, h=(h, h, 1), k=k), levels=levels,
                   smoother="rbgs")
    u, st, *_ = o.solve(f, tol=1e-14, maxit=100)
    m = o.unknown_mask()
    L = float(np.sum(((u - uobs) * m) ** 2))
    lam, st2, *_ = o.solve(2 * (u - uobs) * m, tol=1e-14, maxit=100, transposed=True)
    return L, o.grad_k(u, lam), lam


def test_gradient_matches_central_differences():
    n = 17
    rng = np.random.default_rng(30)
    k = np.exp(0.5 * rng.standard_normal((n - 1, n - 1)))
    f = rng.uniform(-1, 1, (n, n))
    uobs = 0.01 * rng.standard_normal((n, n))
    L0, g, lam = _loss_and_grad(n, k, f, uobs, 3)
    for t in range(12):
        c = (int(rng.integers(0, n - 1)), int(rng.integers(0, n - 1)))
        d = 1e-6 * k[c]
        kp, km = k.copy(), k.copy()
        kp[c] += d
        km[c] -= d
        fd = (_loss_and_grad(n, kp, f, uobs, 3)[0] - _loss_and_grad(n, km, f, uobs, 3)[0]) / (2 * d)
        assert abs(fd - g[c]) <= 1e-5 * abs(g).max()


def test_adjoint_solution_matches_dense():
    rng = np.random.default_rng(31)
    prob = _small(2, False, 2, 17, rng)
    o = orc.Oracle(prob, levels=3, smoother="rbgs", nu1=1, nu2=2)
    A, m = dense_matrix(o)
    g = rand_field(o, rng)
    lam, st, *_ = o.solve(g, tol=1e-13, maxit=100, transposed=True)
    ref = np.linalg.solve(A.T, g[m])
    assert st == orc.OK and np.max(np.abs(lam[m] - ref)) <= 1e-11 * np.abs(ref).max()


# --------------------------------------------------------------------------------------
# adaptive correction weight omega_l (energy-norm optimal)
# --------------------------------------------------------------------------------------

def _interp_1d(nf, periodic):
    """Dense 1-D linear interpolation from the coarse to the fine nodes (numpy, independent
    of the oracle): even fine nodes copy, odd ones average their two coarse neighbours."""
    nc = nf // 2 if periodic else (nf - 1) // 2 + 1
    P = np.zeros((nf, nc))
    for i in range(nf):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, (i - 1) // 2] = 0.5
            P[i, ((i + 1) // 2) % nc] += 0.5
    return P


def _interp(o):
    """P of the finest level of `o` on full node arrays, rows of non-unknowns zero."""
    p = o.prob
    Px, Py = _interp_1d(p.n[0], False), _interp_1d(p.n[1], p.periodic_y)
    P = np.kron(Py, Px) if p.dim == 2 else np.kron(_interp_1d(p.n[2], False), np.kron(Py, Px))
    return P * o.unknown_mask().reshape(-1)[:, None]


ADAPT_CASES = [(2, False, 0), (2, False, 2), (2, True, 1), (3, False, 2)]


@pytest.mark.parametrize("dim,per,kind_idx", ADAPT_CASES)
def test_adaptive_omega_is_one_when_the_correction_is_the_error(dim, per, kind_idx):
    """If u = u* - P e0 with g = A u*, the correction P e0 removes the whole error, so the
    energy-optimal weight is exactly 1 (and 1/2 for 2 e0, -1 for -e0)."""
    rng = np.random.default_rng(40)
    o = orc.Oracle(_small(dim, per, kind_idx, 9, rng), levels=2)
    ustar = rand_field(o, rng)
    e0 = rand_field(o, rng, 1)
    u = ustar - (_interp(o) @ e0.reshape(-1)).reshape(o.shape())
    g = o.apply(ustar)
    for s, want in [(1.0, 1.0), (2.0, 0.5), (-1.0, -1.0)]:
        assert abs(o.adaptive_omega(u, g, s * e0) - want) <= 1e-11


@pytest.mark.parametrize("dim,per,kind_idx", ADAPT_CASES)
def test_adaptive_omega_minimises_the_energy_error(dim, per, kind_idx):
    """Brute force: with u* from a dense solve, the energy error E(w) = ||u* - u - w P e||_A^2
    is a parabola in w; its vertex from three samples is the oracle's weight."""
    rng = np.random.default_rng(41)
    o = orc.Oracle(_small(dim, per, kind_idx, 9, rng), levels=2)
    A, m = dense_matrix(o)
    u, g, e = rand_field(o, rng), rand_field(o, rng), rand_field(o, rng, 1)
    ustar = np.zeros(o.shape())
    ustar[m] = np.linalg.solve(A, g[m])
    pe = (_interp(o) @ e.reshape(-1)).reshape(o.shape())

    def energy(w):
        err = (ustar - u - w * pe)[m]
        return err @ A @ err

    e0, e1, e2 = energy(0.0), energy(1.0), energy(2.0)
    vertex = 0.5 * (3 * e0 - 4 * e1 + e2) / (e0 - 2 * e1 + e2)   # argmin of the parabola through w = 0, 1, 2
    w = o.adaptive_omega(u, g, e)
    assert abs(w - vertex) <= 1e-9 * max(1.0, abs(vertex))
    assert energy(w) <= min(e0, e1)


@pytest.mark.parametrize("dim,per,kind_idx,smoother,n,levels", CASES[:8])
def test_adaptive_fcycle_converges_to_dense_solution(dim, per, kind_idx, smoother, n, levels):
    rng = np.random.default_rng(42)
    prob = _small(dim, per, kind_idx, n, rng)
    omega = 0.8 if smoother in ("jacobi", "line_y") else 1.0
    o = orc.Oracle(prob, levels=levels, smoother=smoother, omega=omega, adaptive_corr=True, omega_corr=0.3)
    A, m = dense_matrix(o)
    b = rand_field(o, rng)
    x, st, cyc, rr, hist = o.solve(b, tol=1e-13, maxit=200)
    assert st == orc.OK
    ref = np.linalg.solve(A, b[m])
    assert np.max(np.abs(x[m] - ref)) <= 1e-11 * np.abs(ref).max()


def test_adaptive_weight_repairs_a_badly_damped_correction():
    """omega_corr is ignored under the adaptive rule: a correction damped to 0.3 converges
    slowly with the fixed weight and at the undamped rate (or better) with the adaptive one."""
    o_fix = orc.Oracle(const_problem(65), levels=5, smoother="rbgs", nu1=1, nu2=1, omega_corr=0.3)
    o_one = orc.Oracle(const_problem(65), levels=5, smoother="rbgs", nu1=1, nu2=1)
    o_ad = orc.Oracle(const_problem(65), levels=5, smoother="rbgs", nu1=1, nu2=1, omega_corr=0.3,
                      adaptive_corr=True)
    b = rand_field(o_one, np.random.default_rng(43))
    cyc = {k: o.solve(b, tol=1e-10)[2] for k, o in (("fix", o_fix), ("one", o_one), ("ad", o_ad))}
    assert cyc["ad"] <= cyc["one"] < cyc["fix"]


# --------------------------------------------------------------------------------------
# stretched grids (section "Anisotropies": refinement in one direction)
# --------------------------------------------------------------------------------------

def _stretched_oracle(sp, smoother="rbgs", omega=1.0, levels=None):
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=False, kind=orc.SEPARABLE, h=sp.h, sx=sp.sx, sy=sp.sy, sz=sp.sz)
    return orc.Oracle(p, levels=levels or inputs.max_levels(sp.n, dim=sp.dim), smoother=smoother, omega=omega)


@pytest.mark.parametrize("beta", [2.0, 4.0])
def test_stretched_grid_discretisation_is_second_order(beta):
    """Manufactured solution sin(pi x) sin(pi y) on x-stretched grids: the max-norm error of
    the discrete solution falls by ~4 per halving of the nominal spacing."""
    errs = []
    for n in (33, 65, 129):
        sp = inputs.stretched_x(n, beta=beta, manufactured=True)
        x, st, c, rr, h = _stretched_oracle(sp, "gsadi").solve(sp.b, tol=1e-11, maxit=100)
        assert st == orc.OK
        exact = np.outer(np.sin(math.pi * np.linspace(0, 1, n)), np.sin(math.pi * sp.x_nodes))
        errs.append(np.abs(x - exact).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.7 <= a / b <= 4.3


def test_stretched_grid_coarse_levels_are_the_coarse_stretched_grid():
    """The coarsening rule (harmonic mean along an edge, x1/4) reproduces the x-edge weights of
    the stretched grid built directly on the even nodes: series resistances add."""
    fine = inputs.stretched_x(129, beta=5.0)
    coarse = inputs.stretched_x(65, beta=5.0)
    o = _stretched_oracle(fine, levels=2)
    cc = o.level_coeffs(1)
    n = 65
    assert np.allclose(cc[:n - 1], coarse.sx, rtol=1e-13)


def test_stretched_grid_needs_alternating_lines():
    """Strong stretching makes the cells thin in x at one end and thin in y at the other: point
    Gauss-Seidel stalls, x-lines alone slow down, the alternating GSADI keeps its rate."""
    out = {}
    for n in (65, 129):
        sp = inputs.stretched_x(n, beta=6.0)
        for sm in ("rbgs", "zebra_x", "gsadi"):
            x, st, c, rr, h = _stretched_oracle(sp, sm).solve(sp.b, tol=1e-10, maxit=40)
            out[(n, sm)] = (st, c)
    for n in (65, 129):
        assert out[(n, "gsadi")][0] == orc.OK and out[(n, "gsadi")][1] <= 7
        assert out[(n, "rbgs")][0] == orc.ENOCONV
        assert out[(n, "zebra_x")][0] == orc.ENOCONV


# --------------------------------------------------------------------------------------
# edge-weight coefficients (per-edge weights varying in every direction)
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,periodic_y", [(2, False), (2, True), (3, False), (3, True)])
def test_edge_kind_reproduces_separable_on_every_level(dim, periodic_y):
    """Separable weights written edge by edge give the same operator on every level (the
    coarsening rule reduces to the separable one: the harmonic mean of two equal weights) and
    the same F-cycle, up to rounding: a transposed or shifted index in the edge arrays would
    break it, since sx and sy vary in x."""
    rng = np.random.default_rng(50)
    sep = _kinds(dim, periodic_y, rng)[1]
    edge = _edge_of_separable(sep)
    a = orc.Oracle(sep, levels=3, smoother="rbgs")
    b = orc.Oracle(edge, levels=3, smoother="rbgs")
    def close(p, q):
        return np.abs(p - q).max() <= 1e-14 * np.abs(q).max()

    for l in (1, 2, 3):
        u = rand_field(a, rng, l)
        assert close(b.apply(u, l), a.apply(u, l))
        assert close(b.diag(l), a.diag(l))
    f = rand_field(a, rng)
    x = a.zeros()
    y = b.zeros()
    for _ in range(3):
        x, y = a.cycle(x, f), b.cycle(y, f)
    assert np.abs(x - y).max() <= 1e-13 * np.abs(x).max()


def _second_order_errors(make, exact_of, sizes=(33, 65, 129)):
    errs = []
    for n in sizes:
        sp = make(n)
        p = orc.Problem(dim=2, n=sp.n, periodic_y=False, kind=orc.EDGE, h=sp.h, ex=sp.ex, ey=sp.ey)
        o = orc.Oracle(p, levels=inputs.max_levels(sp.n), smoother="gsadi")
        x, st, c, rr, h = o.solve(sp.b, tol=1e-11, maxit=100)
        assert st == orc.OK
        errs.append(np.abs(x - exact_of(sp)).max())
    return errs


def test_two_direction_stretched_grid_is_second_order():
    errs = _second_order_errors(lambda n: inputs.stretched_xy(n, beta_x=3.0, beta_y=-2.0, manufactured=True),
                                lambda sp: np.outer(np.sin(math.pi * sp.y_nodes), np.sin(math.pi * sp.x_nodes)))
    for a, b in zip(errs, errs[1:]):
        assert 3.7 <= a / b <= 4.3


def test_spherical_shell_is_second_order():
    """Manufactured axisymmetric solution on the spherical shell (r^2 sin(theta) weights):
    second-order convergence confirms the mapped weights and the right-hand-side factor."""
    def exact(sp):
        r, t = sp.r_nodes, sp.t_nodes
        a = np.sin(math.pi * (r - r[0]) / (r[-1] - r[0]))
        c = np.sin(math.pi * (t - t[0]) / (t[-1] - t[0]))
        return np.outer(c, a)
    errs = _second_order_errors(lambda n: inputs.spherical_shell(n, n, manufactured=True), exact)
    for a, b in zip(errs, errs[1:]):
        assert 3.7 <= a / b <= 4.3


# --------------------------------------------------------------------------------------
# lines across the periodic direction: cyclic tridiagonal systems
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("m", [3, 7, 16])
def test_cyclic_thomas_matches_dense(m):
    rng = np.random.default_rng(60 + m)
    lo, up = -rng.uniform(0.2, 1.0, m), -rng.uniform(0.2, 1.0, m)
    di = 2.0 + rng.uniform(0.0, 1.0, m)
    d = rng.standard_normal(m)
    A = np.diag(di)
    for t in range(m):
        A[t, (t - 1) % m] += lo[t]
        A[t, (t + 1) % m] += up[t]
    assert np.allclose(orc.cyclic_thomas(lo, di, up, d), np.linalg.solve(A, d), rtol=0, atol=1e-13)


def _thomas_ext(lo, di, up, d):
    """Thomas in numpy's extended precision (the reference for the forward-error pin)."""
    m = len(di)
    cp, dp = np.zeros(m, lo.dtype), np.zeros(m, lo.dtype)
    for s in range(m):
        den = di[s] - (lo[s] * cp[s - 1] if s else 0)
        cp[s] = up[s] / den
        dp[s] = (d[s] - (lo[s] * dp[s - 1] if s else 0)) / den
    x, xn = np.zeros(m, lo.dtype), lo.dtype.type(0)
    for s in range(m - 1, -1, -1):
        xn = dp[s] - cp[s] * xn
        x[s] = xn
    return x


def _cyclic_ext(lo, di, up, d):
    """The cyclic system in extended precision: the corner-free tridiagonal solve plus the rank-one
    (Sherman-Morrison) correction, written out independently of the oracle."""
    m = len(di)
    gamma, beta, alpha = -di[0], lo[0], up[m - 1]
    dd = di.copy()
    dd[0] -= gamma
    dd[m - 1] -= alpha * beta / gamma
    l2, u2 = lo.copy(), up.copy()
    l2[0] = 0
    u2[m - 1] = 0
    y = _thomas_ext(l2, dd, u2, d)
    e = np.zeros(m, lo.dtype)
    e[0], e[m - 1] = gamma, alpha
    z = _thomas_ext(l2, dd, u2, e)
    return y - (y[0] + beta / gamma * y[m - 1]) / (1 + z[0] + beta / gamma * z[m - 1]) * z


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 1e-18, reason="needs an extended-precision long double")
@pytest.mark.parametrize("m,per", [(1025, False), (2047, False), (2048, True)])
def test_line_solve_forward_error_on_anisotropic_lines(m, per):
    """A y-line of a strongly anisotropic grid (9 x m nodes on the unit square: y-couplings ~1e6 against
    an x margin ~1e2, Gershgorin condition bound kappa_G ~ 1e5).  The smoothed value u + C^{-1}(g - C u + s)
    from the oracle's Thomas (cyclic for a periodic line) lies within kappa_G u (u = 2^-53) of the
    same value in extended precision.  It also misses it by more than 1e-12 on the longest Dirichlet line.
    That is the rounding that any FP64 solve of these lines carries, so two FP64 orders of operations
    cannot agree to 1e-12 there."""
    LD = np.longdouble
    rng = np.random.default_rng(5 + m)
    hy, hx = 1.0 / (m + 1), 1.0 / 8
    wy = rng.uniform(0.5, 2, m + 1) / hy ** 2
    wx = rng.uniform(0.5, 2, (m, 2)) / hx ** 2
    lo, up = -wy[:-1].copy(), -wy[1:].copy()
    if per:
        lo[0] = up[-1] = -wy[0]
    di = -(lo + up) + wx.sum(1)
    if not per:
        lo[0] = up[-1] = 0.0
    u, g = rng.standard_normal(m), rng.standard_normal(m)
    Cu = di * u + np.r_[0.0, lo[1:] * u[:-1]] + np.r_[up[:-1] * u[1:], 0.0]
    if per:
        Cu[0] += lo[0] * u[-1]
        Cu[-1] += up[-1] * u[0]
    d = g - Cu + wx.sum(1) * rng.standard_normal(m)   # a defect like a sweep's: off-line terms included
    x = (orc.cyclic_thomas if per else orc.thomas)(lo, di, up, d)
    xe = (_cyclic_ext if per else _thomas_ext)(*(a.astype(LD) for a in (lo, di, up, d)))
    out, oute = u + x, u.astype(LD) + xe
    err = float(np.abs(out - oute).max() / np.abs(oute).max())
    kappa_g = 2.0 * di.max() / wx.sum(1).min()
    assert err <= kappa_g * 2.0 ** -53
    if m == 2047:
        assert err > 1e-12


def test_adi_is_robust_on_the_polar_map():
    """Section "Coordinate systems": on the annulus (r-weighted polar map, theta periodic) the
    alternating GSADI keeps its cycle count as the grid is refined, while point Gauss-Seidel and
    theta-lines alone (cyclic systems) degrade: the strong coupling is radial."""
    cyc = {}
    for n in (65, 129):
        sp = inputs.annulus_2d(nr=n, nt=n - 1)
        p = orc.Problem(dim=2, n=sp.n, periodic_y=True, kind=orc.SEPARABLE, h=sp.h, sx=sp.sx, sy=sp.sy, sz=sp.sz)
        for sm in ("gsadi", "zebra_y", "rbgs"):
            o = orc.Oracle(p, levels=inputs.max_levels(sp.n, periodic_y=True), smoother=sm)
            x, st, c, rr, h = o.solve(sp.b, tol=1e-10, maxit=100)
            cyc[(n, sm)] = c if st == orc.OK else 10 ** 6
    assert cyc[(65, "gsadi")] <= 7 and cyc[(129, "gsadi")] <= 7
    assert min(cyc[(n, s)] for n in (65, 129) for s in ("zebra_y", "rbgs")) > 5 * cyc[(129, "gsadi")]


# --------------------------------------------------------------------------------------
# qualitative claims of the paper
# --------------------------------------------------------------------------------------

def test_single_level_jacobi_rate_degrades_like_h_squared():
    """One level, damped Jacobi as the whole iteration: the slowest error mode decays by
    1 - omega (1 - cos(pi h)) per sweep, so 1 - rho falls by ~4 when h halves (the mesh
    dependence that multigrid removes).  Measured from the residual decay of the oracle's
    smoother on the lowest mode."""
    gaps = []
    for n in (17, 33, 65):
        o = orc.Oracle(const_problem(n), levels=2, smoother="jacobi", omega=0.8)
        x = np.linspace(0, 1, n)
        u = np.outer(np.sin(math.pi * x), np.sin(math.pi * x))   # the slowest mode, zero right-hand side
        g = o.zeros()
        u1 = o.smooth(u, g, 1, l=2)
        gaps.append(1.0 - np.linalg.norm(u1) / np.linalg.norm(u))
    for a, b in zip(gaps, gaps[1:]):
        assert 3.5 <= a / b <= 4.5


def test_more_smoothing_steps_give_better_rates():
    """Section "Smoothing": the F-cycle rate improves with nu1 = nu2 = 1, 2, 4 (RB-GS, 65^2)."""
    rates = []
    for nu in (1, 2, 4):
        o = orc.Oracle(const_problem(65), levels=5, smoother="rbgs", nu1=nu, nu2=nu)
        b = rand_field(o, np.random.default_rng(70))
        x, st, cyc, rr, hist = o.solve(b, tol=1e-10)
        rates.append((hist[-1] / hist[0]) ** (1.0 / cyc))
    assert rates[0] > rates[1] > rates[2]


# --------------------------------------------------------------------------------------
# coarsening rules written out by hand, on data that varies in every direction
# --------------------------------------------------------------------------------------

def _hand_apply(u, wx, wy, wz, periodic_y):
    """(A u)_p = sum over the edges e = (p, q) of w_e (u_p - u_q), at the unknowns only, from
    per-node weights of the +x, +y (+z) edges; Dirichlet nodes read as 0.  Plain loops."""
    dim = u.ndim
    U = u if dim == 3 else u[None]
    WX = wx if dim == 3 else wx[None]
    WY = wy if dim == 3 else wy[None]
    WZ = wz if dim == 3 else None
    n2, n1, n0 = U.shape
    out = np.zeros_like(U)

    def unknown(i, j, k):
        return 0 < i < n0 - 1 and (periodic_y or 0 < j < n1 - 1) and (dim == 2 or 0 < k < n2 - 1)

    def val(i, j, k):
        return U[k, j, i] if unknown(i, j, k) else 0.0

    edges = []
    for k in range(n2):
        for j in range(n1):
            for i in range(n0):
                if i + 1 < n0:
                    edges.append(((i, j, k), (i + 1, j, k), WX[k, j, i]))
                if j + 1 < n1 or periodic_y:
                    edges.append(((i, j, k), (i, (j + 1) % n1, k), WY[k, j, i]))
                if dim == 3 and k + 1 < n2:
                    edges.append(((i, j, k), (i, j, k + 1), WZ[k, j, i]))
    for p, q, w in edges:
        d = val(*p) - val(*q)
        if unknown(*p):
            out[p[2], p[1], p[0]] += w * d
        if unknown(*q):
            out[q[2], q[1], q[0]] -= w * d
    return out if dim == 3 else out[0]


def _cell_edges(k, h, dim, periodic_y, n):
    """Edge weights of -div(k grad u) from a cell field: an edge weighs the mean of the 2 (2-D)
    or 4 (3-D) cells that touch it, over h^2 of its direction.  Cells outside the grid do not
    exist (they touch only edges between Dirichlet nodes, which carry no unknown)."""
    n0, n1 = n[0], n[1]
    n2 = n[2] if dim == 3 else 1
    K = k if dim == 3 else k[None]
    ncy = n1 if periodic_y else n1 - 1
    ncz = n2 - 1 if dim == 3 else 1

    def cell(i, j, kk):
        if periodic_y:
            j %= n1
        if 0 <= i < n0 - 1 and 0 <= j < ncy and 0 <= kk < ncz:
            return K[kk, j, i]
        return None

    wx, wy, wz = (np.zeros((n2, n1, n0)) for _ in range(3))
    for kk in range(n2):
        for j in range(n1):
            for i in range(n0):
                for arr, d, around in (
                        (wx, 0, [(i, j - b, kk - c) for b in (0, 1) for c in ((0, 1) if dim == 3 else (0,))]),
                        (wy, 1, [(i - a, j, kk - c) for a in (0, 1) for c in ((0, 1) if dim == 3 else (0,))]),
                        (wz, 2, [(i - a, j - b, kk) for a in (0, 1) for b in (0, 1)] if dim == 3 else [])):
                    cs = [cell(*t) for t in around]
                    cs = [c for c in cs if c is not None]
                    if cs:
                        arr[kk, j, i] = sum(cs) / (len(around) * h[d] ** 2)
    if dim == 2:
        return wx[0], wy[0], None
    return wx, wy, wz


@pytest.mark.parametrize("dim,periodic_y", [(2, False), (2, True), (3, False)])
def test_cell_coarsening_by_hand_with_varying_k(dim, periodic_y):
    """Coarse cell coefficient = mean of the 2^d child cells (coarse cell (I, J[, K]) covers
    fine cells 2I..2I+1, 2J..2J+1[, 2K..2K+1]), edges formed from it with h doubled.  With k
    varying from cell to cell a wrong child offset or a missing child changes the coarse
    operator, which is compared on two coarser levels with one built here by hand."""
    rng = np.random.default_rng(61 + dim + periodic_y)
    n = (9, 8 if periodic_y else 9, 9 if dim == 3 else 1)
    h = (1.0 / 8, 1.0 / n[1] if periodic_y else 1.0 / 8, 1.0 / 8)
    ncy = n[1] if periodic_y else n[1] - 1
    ks = (ncy, n[0] - 1) if dim == 2 else (n[2] - 1, ncy, n[0] - 1)
    k = np.exp(rng.standard_normal(ks))
    o = orc.Oracle(orc.Problem(dim=dim, n=n, periodic_y=periodic_y, kind=orc.CELL, h=h, k=k), levels=3)
    kl, nl, hl = k, n, h
    for l in (3, 2, 1):
        if l < 3:
            # children of coarse cell I: fine cells 2I and 2I + 1 in each direction
            if dim == 2:
                kl = 0.25 * (kl[0::2, 0::2] + kl[0::2, 1::2] + kl[1::2, 0::2] + kl[1::2, 1::2])
            else:
                kl = 0.125 * sum(kl[c::2, b::2, a::2] for a in (0, 1) for b in (0, 1) for c in (0, 1))
            nl = ((nl[0] - 1) // 2 + 1, nl[1] // 2 if periodic_y else (nl[1] - 1) // 2 + 1,
                  (nl[2] - 1) // 2 + 1 if dim == 3 else 1)
            hl = tuple(2 * v for v in hl)
        assert o.dims(l) == nl
        wx, wy, wz = _cell_edges(kl, hl, dim, periodic_y, nl)
        for _ in range(2):
            u = rand_field(o, rng, l)
            want = _hand_apply(u, wx, wy, wz, periodic_y)
            assert np.abs(o.apply(u, l) - want).max() <= 1e-13 * np.abs(want).max(), l


@pytest.mark.parametrize("dim,periodic_y", [(2, False), (2, True), (3, False), (3, True)])
def test_edge_coarsening_by_hand_with_weights_varying_everywhere(dim, periodic_y):
    """Coarse edge weight = 1/4 of the harmonic mean of the two fine edges that make up the
    coarse edge (in series along it), taken on the fine line through the coarse edge's end
    nodes (injection across: fine row 2J, plane 2K).  Weights drawn independently per edge, so
    an across-edge index that is off (2J+1 for 2J, plane 0 for 2K) or a swapped direction
    changes the result.  Coarse operators on two coarser levels against loops written here."""
    rng = np.random.default_rng(71 + dim + 2 * periodic_y)
    n = (17, 16 if periodic_y else 17, 9 if dim == 3 else 1)
    shape = (n[1], n[0]) if dim == 2 else (n[2], n[1], n[0])
    w = [np.exp(rng.standard_normal(shape)) for _ in range(3)]
    p = orc.Problem(dim=dim, n=n, periodic_y=periodic_y, kind=orc.EDGE, h=(1, 1, 1), ex=w[0], ey=w[1],
                    ez=w[2] if dim == 3 else None)
    o = orc.Oracle(p, levels=3)

    def H(a, b):
        return 2 * a * b / (a + b)

    ex, ey, ez = [a if dim == 3 else a[None] for a in w]
    nl = n
    for l in (3, 2, 1):
        if l < 3:
            nc = ((nl[0] - 1) // 2 + 1, nl[1] // 2 if periodic_y else (nl[1] - 1) // 2 + 1,
                  (nl[2] - 1) // 2 + 1 if dim == 3 else 1)
            cx, cy, cz = (np.zeros((nc[2], nc[1], nc[0])) for _ in range(3))
            for K in range(nc[2]):
                kk = 2 * K if dim == 3 else 0
                for J in range(nc[1]):
                    for I in range(nc[0]):
                        if I + 1 < nc[0]:
                            cx[K, J, I] = 0.25 * H(ex[kk, 2 * J, 2 * I], ex[kk, 2 * J, 2 * I + 1])
                        if J + 1 < nc[1] or periodic_y:
                            cy[K, J, I] = 0.25 * H(ey[kk, 2 * J, 2 * I], ey[kk, 2 * J + 1, 2 * I])
                        if dim == 3 and K + 1 < nc[2]:
                            cz[K, J, I] = 0.25 * H(ez[kk, 2 * J, 2 * I], ez[kk + 1, 2 * J, 2 * I])
            ex, ey, ez, nl = cx, cy, cz, nc
        assert o.dims(l) == nl
        for _ in range(2):
            u = rand_field(o, rng, l)
            if dim == 2:
                want = _hand_apply(u, ex[0], ey[0], None, periodic_y)
            else:
                want = _hand_apply(u, ex, ey, ez, periodic_y)
            assert np.abs(o.apply(u, l) - want).max() <= 1e-13 * np.abs(want).max(), l


# --------------------------------------------------------------------------------------
# the threaded build of the timed CPU baseline
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("smoother,kind,periodic_y,dim", [("rbgs", orc.CONST, False, 2), ("jacobi", orc.SEPARABLE, True, 2),
                                                         ("zebra_y", orc.CELL, False, 2), ("gsadi", orc.SEPARABLE, True, 2),
                                                         ("zebra_x", orc.CONST, False, 3)])
def test_threaded_oracle_is_bit_identical(smoother, kind, periodic_y, dim):
    """The OpenMP build of the oracle (grid rows and lines spread over host cores) computes every
    node exactly as the plain build: two cycles and a defect agree bit for bit."""
    rng = np.random.default_rng(81)
    n = (65, 64 if periodic_y else 65, 17 if dim == 3 else 1)
    if dim == 3:
        n = (33, 33, 17)
    h = (1.0 / (n[0] - 1), 1.0 / n[1] if periodic_y else 1.0 / (n[1] - 1), 1.0 / max(n[2] - 1, 1))
    kw = dict(dim=dim, n=n, periodic_y=periodic_y, kind=kind, h=h)
    if kind == orc.CONST:
        kw["c"] = (0.3 / h[0] ** 2, 1.0 / h[1] ** 2, 1.0 / h[2] ** 2)
    elif kind == orc.SEPARABLE:
        kw.update(sx=rng.uniform(0.5, 2, n[0] - 1), sy=rng.uniform(0.5, 2, n[0]), sz=rng.uniform(0.5, 2, n[0]))
    else:
        cy = n[1] if periodic_y else n[1] - 1
        kw["k"] = np.exp(rng.standard_normal((cy, n[0] - 1) if dim == 2 else (n[2] - 1, cy, n[0] - 1)))
    p = orc.Problem(**kw)
    a = orc.Oracle(p, levels=3, smoother=smoother, omega=0.8 if smoother == "jacobi" else 1.0, dense_max=4096)
    b = orc.Oracle(p, levels=3, smoother=smoother, omega=0.8 if smoother == "jacobi" else 1.0, dense_max=4096,
                   threaded=True)
    f = rng.uniform(-1, 1, a.shape()) * a.unknown_mask()
    x, y = a.zeros(), b.zeros()
    for _ in range(2):
        x, y = a.cycle(x, f), b.cycle(y, f)
    assert np.array_equal(x, y)
    assert np.array_equal(a.defect(x, f), b.defect(y, f))
    assert orc.threads(True) >= 1 and orc.threads(False) == 1


# --------------------------------------------------------------------------------------
# Galerkin coarse operators A_c = R A P (2-D)
# --------------------------------------------------------------------------------------

def _lin_interp_1d(nf):
    """Linear interpolation between the unknowns of a coarse and a fine 1-D Dirichlet grid
    (nf nodes -> (nf - 1) / 2 + 1): fine unknown 2I takes coarse I, 2I +- 1 half of it."""
    nc = (nf - 1) // 2 + 1
    P = np.zeros((nf - 2, nc - 2))
    for I in range(1, nc - 1):
        P[2 * I - 1, I - 1] = 1.0
        P[2 * I - 2, I - 1] = 0.5
        P[2 * I, I - 1] = 0.5
    return P


def _dense_op(o, l):
    """The oracle's operator on level l as a dense matrix over the unknowns (x fastest)."""
    m = o.unknown_mask(l)
    idx = np.flatnonzero(m)
    A = np.zeros((idx.size, idx.size))
    for c, p in enumerate(idx):
        e = np.zeros(m.size)
        e[p] = 1.0
        A[:, c] = o.apply(e.reshape(m.shape), l).ravel()[idx]
    return A


def _cell_problem(n, rng, jump=False):
    h = (1.0 / (n[0] - 1), 1.0 / (n[1] - 1), 1.0)
    k = np.exp(rng.standard_normal((n[1] - 1, n[0] - 1)))
    if jump:
        k[: (n[1] - 1) // 2, : (n[0] - 1) // 2] *= 1e3
    return orc.Problem(dim=2, n=(n[0], n[1], 1), kind=orc.CELL, h=h, k=k)


def test_galerkin_poisson_stencil_closed_form():
    """For the 5-point Laplacian, full weighting and bilinear interpolation, R A P is the 9-point
    stencil (1/H^2) [[-1/4, -1/2, -1/4], [-1/2, 3, -1/2], [-1/4, -1/2, -1/4]], H = 2h (a textbook
    result), at every coarse node whose stencil stays off the boundary."""
    n = 33
    h = 1.0 / (n - 1)
    o = orc.Oracle(orc.Problem(dim=2, n=(n, n, 1), kind=orc.CONST, h=(h, h, 1), c=(1 / h ** 2, 1 / h ** 2, 0)),
                   levels=3, galerkin=True, dense_max=4096)
    st = o.stencil(2)
    want = np.array([[-0.25, -0.5, -0.25], [-0.5, 3.0, -0.5], [-0.25, -0.5, -0.25]]) / (2 * h) ** 2
    nc = o.dims(2)[0]
    for J in range(2, nc - 2):
        for I in range(2, nc - 2):
            assert np.abs(st[J, I] - want).max() <= 1e-13 * np.abs(want).max()


@pytest.mark.parametrize("n", [(17, 9), (17, 17), (33, 17)])
def test_galerkin_equals_dense_rap(n):
    """The oracle's coarse operators on two coarser levels equal R A P built densely here from the
    fine operator, bilinear P (Kronecker product of 1-D linear interpolation) and R = P^T / 4, for
    a cell coefficient that varies from cell to cell."""
    rng = np.random.default_rng(sum(n))
    p = _cell_problem(n, rng)
    o = orc.Oracle(p, levels=3, galerkin=True, dense_max=4096)
    A = _dense_op(o, 3)
    dims = [o.dims(3)]
    for l in (2, 1):
        nf = dims[-1]
        P = np.kron(_lin_interp_1d(nf[1]), _lin_interp_1d(nf[0]))
        A = (P.T / 4.0) @ A @ P
        got = _dense_op(o, l)
        assert np.abs(got - A).max() <= 1e-13 * np.abs(A).max(), l
        assert np.abs(got - got.T).max() <= 1e-13 * np.abs(A).max()
        dims.append(o.dims(l))


def test_galerkin_two_grid_cycle_is_the_textbook_two_grid_method():
    """Two grids, exact coarse solve: one cycle is x <- S^nu2(y + P A_c^-1 R (b - A y)), y = S^nu1(x),
    with A_c = R A P formed densely here."""
    rng = np.random.default_rng(5)
    n = (17, 17)
    p = _cell_problem(n, rng)
    for sm, om in (("jacobi", 0.8), ("rbgs", 1.0)):
        o = orc.Oracle(p, levels=2, smoother=sm, omega=om, nu1=2, nu2=1, galerkin=True, dense_max=4096)
        m = o.unknown_mask()
        idx = np.flatnonzero(m)
        A = _dense_op(o, 2)
        P = np.kron(_lin_interp_1d(n[1]), _lin_interp_1d(n[0]))
        Ac = (P.T / 4.0) @ A @ P
        b = rng.uniform(-1, 1, m.shape) * m
        x = rng.uniform(-1, 1, m.shape) * m
        y = o.smooth(x, b, 2, 0)
        r = (b - o.apply(y)).ravel()[idx]
        e = P @ np.linalg.solve(Ac, (P.T / 4.0) @ r)
        z = y.copy().ravel()
        z[idx] += e
        want = o.smooth(z.reshape(m.shape), b, 1, 0)
        got = o.cycle(x, b)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), sm


def test_galerkin_four_colour_gauss_seidel_invariant():
    """omega = 1: after a Gauss-Seidel sweep on a Galerkin (9-point) level the residual vanishes at
    the colour updated last, (0, 1) in red-first order and (0, 0) in black-first order, and at no
    other colour."""
    rng = np.random.default_rng(6)
    p = _cell_problem((33, 33), rng)
    o = orc.Oracle(p, levels=3, smoother="rbgs", omega=1.0, galerkin=True, dense_max=4096)
    l = 2
    m = o.unknown_mask(l)
    jj, ii = np.indices(m.shape)
    u = rng.standard_normal(m.shape) * m
    g = rng.standard_normal(m.shape) * m
    for order, last in ((0, (0, 1)), (1, (0, 0))):
        r = o.defect(o.smooth(u, g, 1, order, l), g, l)
        sel = m & (ii % 2 == last[0]) & (jj % 2 == last[1])
        assert np.abs(r[sel]).max() <= 1e-12 * np.abs(g).max()
        assert np.abs(r[m & ~sel]).max() > 1e-3 * np.abs(g).max()


def test_galerkin_transposed_cycle_is_the_adjoint():
    """<M b, c> = <b, M^T c> for 1 and 2 cycles from zero: the four-colour order reversed in the
    transposed cycle is the exact transpose of the forward sweeps."""
    rng = np.random.default_rng(7)
    p = _cell_problem((33, 17), rng)
    o = orc.Oracle(p, levels=3, smoother="rbgs", omega=1.0, nu1=2, nu2=1, galerkin=True, dense_max=4096)
    m = o.unknown_mask()
    b = rng.standard_normal(m.shape) * m
    c = rng.standard_normal(m.shape) * m
    for ncyc in (1, 2):
        x, y = o.zeros(), o.zeros()
        for _ in range(ncyc):
            x = o.cycle(x, b)
            y = o.cycle(y, c, transposed=True)
        lhs, rhs = np.vdot(x, c), np.vdot(b, y)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("sm,om", [("jacobi", 0.8), ("rbgs", 1.0)])
def test_galerkin_cycles_converge_to_the_dense_solution(sm, om):
    """F-cycles on four Galerkin levels converge to the dense solution of a problem with a
    coefficient jump of 1e3, where Galerkin coarse operators keep the jump's effect."""
    rng = np.random.default_rng(8)
    p = _cell_problem((33, 33), rng, jump=True)
    o = orc.Oracle(p, levels=4, smoother=sm, omega=om, galerkin=True, dense_max=4096)
    m = o.unknown_mask()
    b = rng.uniform(-1, 1, m.shape) * m
    x, st, cyc, rr, hist = o.solve(b, tol=1e-12, maxit=100)
    assert st == orc.OK
    A = _dense_op(o, 4)
    idx = np.flatnonzero(m)
    xd = np.linalg.solve(A, b.ravel()[idx])
    assert np.abs(x.ravel()[idx] - xd).max() <= 1e-10 * np.abs(xd).max()
    # and faster than rediscretised coarse operators on this jump
    o2 = orc.Oracle(p, levels=4, smoother=sm, omega=om, dense_max=4096)
    cyc2 = o2.solve(b, tol=1e-12, maxit=200)[2]
    print(f"{sm}: Galerkin {cyc} cycles, rediscretised {cyc2}")
    assert cyc < cyc2


def test_galerkin_rejects_what_it_does_not_cover():
    h = 1.0 / 16
    p3 = orc.Problem(dim=3, n=(17, 17, 17), kind=orc.CONST, h=(h, h, h), c=(1, 1, 1))
    with pytest.raises(ValueError):
        orc.Oracle(p3, levels=2, galerkin=True)
    p2 = orc.Problem(dim=2, n=(17, 16, 1), periodic_y=True, kind=orc.CONST, h=(h, h, 1), c=(1, 1, 0))
    with pytest.raises(ValueError):
        orc.Oracle(p2, levels=2, galerkin=True)
    p1 = orc.Problem(dim=2, n=(17, 17, 1), kind=orc.CONST, h=(h, h, 1), c=(1, 1, 0))
    with pytest.raises(ValueError):
        orc.Oracle(p1, levels=2, smoother="zebra_x", galerkin=True)
