"""The benchmark's own workload at full size.  The problem is the 4097^2 anisotropic Poisson problem
(eps = 1, f ~ U[-1, 1] seed 1) on 12 grids with red-black Gauss-Seidel, nu = 2.  It goes through the
same calls and launch configuration that bench.py times.

The oracle's full F-cycle solve at this size takes most of a minute, so the checks use what the
oracle computes directly:
- the mixed-precision solve meets the 1e-10 relative residual as the oracle's FP64 operator measures
  it, in the benchmark's cycle count (FP32 cycles with the TMA-fed sweeps, one graph launch);
- FP64 single steps on the finest grid match the oracle element by element within 1e-12: the defect,
  and the register-marching red-black sweep that only grids above 513^2 take;
- the TMA sweep and the marching sweep give the same mixed iterates after three refinement steps.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver, FLAG_NO_TMA  # noqa: E402
from test_gpu_parity import rel  # noqa: E402

N = 4097


@pytest.fixture(scope="module")
def problem():
    sp = inputs.anisotropic(n=N, eps=1.0, seed_f=1)
    L = inputs.max_levels(sp.n)
    p = orc.Problem(dim=2, n=sp.n, periodic_y=False, kind=orc.CONST, h=sp.h, c=sp.c)
    o = orc.Oracle(p, levels=L, smoother="rbgs", omega=1.0, nu1=2, nu2=2)
    return sp, L, o


def test_headline_mixed_solve_meets_tolerance_in_the_oracles_residual(problem):
    sp, L, o = problem
    s = Solver(sp, levels=L, smoother="rbgs", omega=1.0, nu1=2, nu2=2, precision="mixed", max_cycles=100)
    b = torch.from_numpy(sp.b).cuda()
    x = torch.zeros_like(b)
    info = s.solve_into(b, x, tol=1e-10)
    xn = x.cpu().numpy()
    rr = o.norm(o.defect(xn, sp.b)) / o.norm(sp.b)
    print(f"4097^2 mixed: {info['cycles']} steps, relres {info['relres']:.3e} (oracle {rr:.3e})")
    assert info["status"] == "MG_OK" and info["cycles"] <= 8
    assert rr <= 1e-10
    # Near 1e-10 each FP64 evaluation of the residual carries about 1e-3 of it in rounding at this
    # size: its 5-point sums hold terms some 1e7 times larger than the result.
    assert abs(rr - info["relres"]) <= 1e-2 * rr


def test_fp64_finest_steps_match_oracle(problem):
    sp, L, o = problem
    s = Solver(sp, levels=L, smoother="rbgs", omega=1.0, nu1=2, nu2=2, precision="fp64", max_cycles=10)
    rng = np.random.default_rng(41)
    u = rng.standard_normal(o.shape()) * o.unknown_mask()
    g = rng.standard_normal(o.shape())
    assert rel(s.defect(u, g), o.defect(u, g)) <= 1e-12
    for sweeps, order in ((1, 0), (2, 1)):
        assert rel(s.smooth(u, g, sweeps, order), o.smooth(u, g, sweeps, order)) <= 1e-12


def test_tma_and_marching_sweeps_agree_at_full_size(problem):
    sp, L, o = problem
    kw = dict(levels=L, smoother="rbgs", omega=1.0, nu1=2, nu2=2, precision="mixed", max_cycles=3)
    xa, ia = Solver(sp, **kw).solve(sp.b, tol=0.0)
    xb, ib = Solver(sp, flags=FLAG_NO_TMA, **kw).solve(sp.b, tol=0.0)
    assert ia["cycles"] == ib["cycles"]
    assert rel(xa, xb.cpu().numpy()) <= 1e-6
