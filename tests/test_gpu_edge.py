"""Edge-weight coefficients (MG_COEF_EDGE) on the GPU against the oracle.

Weights varying edge by edge (log-normal, independent), grids refined in two directions and
the spherical shell: the operator and the smoother on every level within 1e-12, one cycle
(plain and transposed) within 1e-11, the oracle's cycle count to 1e-10, and the mixed form
converging.  Cases cover the per-level kernels, the tile sweeps, the y-line kernel, the
single-CTA coarse kernel and the whole cycle inside it.
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
from test_gpu_parity import rel  # noqa: E402


def random_edges(dim, n, periodic_y, seed):
    """A problem with log-normal weights on every edge and a uniform right-hand side."""
    rng = np.random.default_rng(seed)
    n = tuple(n) + (1,) * (3 - len(n))
    shape = (n[1], n[0]) if dim == 2 else (n[2], n[1], n[0])
    w = [np.exp(0.5 * rng.standard_normal(shape)) * 1e3 for _ in range(3)]
    h = (1.0 / (n[0] - 1), 1.0 / n[1] if periodic_y else 1.0 / (n[1] - 1), 1.0 / max(n[2] - 1, 1))
    b = inputs._zero_boundary(rng.uniform(-1, 1, shape), dim, periodic_y)
    return inputs.ProblemSpec(name="edges", dim=dim, n=n if dim == 3 else (n[0], n[1], 1), periodic_y=periodic_y,
                              kind=inputs.EDGE, h=h, ex=w[0], ey=w[1], ez=w[2] if dim == 3 else None, b=b)


CASES = [
    # name, spec factory, levels, smoother, omega
    ("2d-129x65-rbgs", lambda: random_edges(2, (129, 65), False, 1), 5, "rbgs", 1.0),
    ("2d-65x65-zebra_y", lambda: random_edges(2, (65, 65), False, 2), 4, "zebra_y", 1.0),
    ("2d-129x64-per-zebra_x", lambda: random_edges(2, (129, 64), True, 3), 5, "zebra_x", 1.0),
    ("2d-65x65-gsadi", lambda: random_edges(2, (65, 65), False, 4), 4, "gsadi", 1.0),
    ("2d-65x33-jacobi", lambda: random_edges(2, (65, 33), False, 5), 4, "jacobi", 0.8),
    ("2d-129x64-per-gsadi", lambda: random_edges(2, (129, 64), True, 12), 5, "gsadi", 1.0),
    ("3d-33x17x33-rbgs", lambda: random_edges(3, (33, 17, 33), False, 6), 3, "rbgs", 1.0),
    ("3d-17x16x17-per-jacobi", lambda: random_edges(3, (17, 16, 17), True, 7), 3, "jacobi", 0.8),
    ("2d-33x33-rbgs-all-coarse", lambda: random_edges(2, (33, 33), False, 8), 4, "rbgs", 1.0),
    ("stretched-xy-129-gsadi", lambda: inputs.stretched_xy(129, beta_x=4.0, beta_y=-3.0), 7, "gsadi", 1.0),
    ("spherical-129-gsadi", lambda: inputs.spherical_shell(129, 129), 7, "gsadi", 1.0),
    ("spherical-65-rbgs", lambda: inputs.spherical_shell(65, 65), 6, "rbgs", 1.0),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: c[0])
def case(request):
    name, make, L, sm, om = request.param
    sp = make()
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=orc.EDGE, h=sp.h, ex=sp.ex, ey=sp.ey,
                    ez=sp.ez)
    o = orc.Oracle(p, levels=L, smoother=sm, omega=om, dense_max=4096)
    return sp, o, dict(levels=L, smoother=sm, omega=om, max_cycles=100), np.random.default_rng(9)


def test_edge_operator_and_smoother_every_level(case):
    sp, o, kw, rng = case
    s = Solver(sp, **kw)
    for l in range(1, o.levels + 1):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        assert rel(s.apply(u, l), o.apply(u, l)) <= 1e-12
        if l >= 2:
            g = rng.standard_normal(o.shape(l))
            assert rel(s.smooth(u, g, 2, 0, l), o.smooth(u, g, 2, 0, l)) <= 1e-12


def test_edge_cycle_matches_oracle(case):
    sp, o, kw, rng = case
    s = Solver(sp, **kw)
    x = rng.standard_normal(o.shape()) * o.unknown_mask()
    for tr in (False, True):
        assert rel(s.cycle(x, sp.b, tr), o.cycle(x, sp.b, transposed=tr)) <= 1e-11


def test_edge_solve_matches_oracle(case):
    sp, o, kw, rng = case
    x, info = Solver(sp, **kw).solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=kw["max_cycles"])
    assert info["status"] == "MG_OK" and sto == orc.OK
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
    assert rel(x, xo) <= 1e-10


def test_edge_mixed_solve(case):
    sp, o, kw, rng = case
    x, info = Solver(sp, precision="mixed", **kw).solve(sp.b, tol=1e-10)
    assert info["status"] == "MG_OK" and info["relres"] <= 1e-10
