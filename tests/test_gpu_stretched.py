"""Stretched grids (x-refined, separable weights) on the GPU against the oracle.

The strong stretching makes cells thin in x at one end and thin in y at the other, so the
alternating line smoothers carry the solve; one cycle of each smoother matches the oracle
within 1e-11 and the solves take the oracle's cycle counts.
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

CASES = [
    # n, ny, dim, beta, smoother, omega, max cycles
    (129, 65, 2, 6.0, "gsadi", 1.0, 20),
    (129, 65, 2, 6.0, "adi", 0.8, 60),
    (129, 65, 2, 6.0, "zebra_x", 1.0, 200),
    (129, 129, 2, 3.0, "rbgs", 1.0, 200),
    (33, 33, 3, 3.0, "rbgs", 1.0, 200),
    (33, 17, 3, 3.0, "adi", 0.8, 100),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[2]}d-{c[0]}x{c[1]}-b{c[3]}-{c[4]}")
def case(request):
    n, ny, dim, beta, sm, om, mx = request.param
    sp = inputs.stretched_x(n, ny=ny, beta=beta, dim=dim)
    L = inputs.max_levels(sp.n, dim=dim)
    p = orc.Problem(dim=dim, n=sp.n, periodic_y=False, kind=orc.SEPARABLE, h=sp.h, sx=sp.sx, sy=sp.sy, sz=sp.sz)
    o = orc.Oracle(p, levels=L, smoother=sm, omega=om, dense_max=4096)
    return sp, o, dict(levels=L, smoother=sm, omega=om, max_cycles=mx)


def test_stretched_cycle_matches_oracle(case):
    sp, o, kw = case
    s = Solver(sp, **kw)
    x = np.random.default_rng(8).standard_normal(o.shape()) * o.unknown_mask()
    for tr in (False, True):
        assert rel(s.cycle(x, sp.b, tr), o.cycle(x, sp.b, transposed=tr)) <= 1e-11


def test_stretched_solve_matches_oracle(case):
    sp, o, kw = case
    x, info = Solver(sp, **kw).solve(sp.b, tol=1e-10)
    xo, sto, co, rro, ho = o.solve(sp.b, tol=1e-10, maxit=kw["max_cycles"])
    assert info["status"] == "MG_OK" and sto == orc.OK
    if not np.any(np.abs(ho / 1e-10 - 1.0) < 1e-3):
        assert info["cycles"] == co
    assert rel(x, xo) <= 1e-10


def test_stretched_mixed_solve(case):
    sp, o, kw = case
    x, info = Solver(sp, precision="mixed", **kw).solve(sp.b, tol=1e-10)
    assert info["status"] == "MG_OK" and info["relres"] <= 1e-10
