"""Long x-line smoothing (TRIx line Jacobi, GSTRIx zebra, the x half of ADI / GSADI) against the oracle.

Lines of more than 512 unknowns take the one-CTA-per-line kernel (partition of the line over
the CTA's threads, the reduced system by cyclic reduction in shared memory); shorter lines take
the one-warp kernel.  The cases run both at 513, 1023, 2047 and 4095 unknowns per line, with
constant (strong along x), separable, cell and edge coefficients, periodic y, 2-D and 3-D.
y-lines of constant coefficients become x-lines of the axis-swapped problem: the 4097^2
eps = 1e-4 zebra y-line solve of the anisotropy study runs here, both as sweeps and as one
whole FP64 F-cycle against the oracle's.

Bar: the larger of 1e-12 and 4 kappa_G u (u = 2^-53), kappa_G the Gershgorin bound on the
condition number of the line systems.  The oracle's Thomas and the kernel's partitioned solve
are both backward stable on these diagonally dominant lines, each with a forward error of a
few kappa u, so two correct FP64 solves can differ by that much and no less.
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
from test_gpu_parity import spec_of, oracle_of, rel  # noqa: E402
from test_gpu_edge import random_edges  # noqa: E402

EDGE = inputs.EDGE
U64 = 2.0 ** -53


def line_condition_bound(o, axis):
    """Gershgorin bound on the condition number of the line systems C along `axis` (0 = x,
    1 = y) of the oracle's finest level.  C keeps the node's diagonal D and the two in-line
    couplings, so lambda_max <= 2 max D and lambda_min >= min(D - in-line couplings), which is
    (A v)_p for v = 1 on every other line (and every other z-plane in 3-D) at the nodes with
    v = 1: what remains there are the couplings off the line."""
    mask = o.unknown_mask()
    idx = np.indices(o.shape())
    across = idx[-2] if axis == 0 else idx[-1]   # the index that numbers the lines in the plane
    kp = (idx[0] % 2,) if o.prob.dim == 3 else ()
    margin = np.inf
    for p in (0, 1):
        for pk in ((0, 1) if kp else (None,)):
            sel = mask & (across % 2 == p) & ((kp[0] == pk) if kp else True)
            margin = min(margin, o.apply(sel.astype(np.float64))[sel].min())
    return 2.0 * o.diag()[mask].max() / margin


def make(dim, n, per, kind, seed, eps=1.0):
    if kind == EDGE:
        return random_edges(dim, n[:dim], per, seed)
    return spec_of(dim, n, per, kind, np.random.default_rng(seed), eps=eps)


def oracle_for(sp, levels, sm, om):
    if sp.kind == EDGE:
        p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=orc.EDGE, h=sp.h, ex=sp.ex, ey=sp.ey,
                        ez=sp.ez)
        return orc.Oracle(p, levels=levels, smoother=sm, omega=om, dense_max=4096)
    return oracle_of(sp, levels, sm, om)


SWEEP_CASES = [
    # dim, n, periodic, kind, smoother, omega, eps (constant kind: x-weight eps / h^2)
    (2, (515, 9), False, inputs.CONST, "zebra_x", 1.0, 1e3),     # 513 unknowns: the one-CTA kernel
    (2, (515, 10), True, inputs.SEPARABLE, "line_x", 0.7, 1.0),
    (2, (1025, 9), False, inputs.CELL, "zebra_x", 1.0, 1.0),
    (2, (1025, 9), False, EDGE, "line_x", 0.7, 1.0),
    (2, (2049, 9), False, inputs.SEPARABLE, "zebra_x", 1.0, 1.0),
    (2, (2049, 10), True, inputs.CONST, "line_x", 0.7, 1e4),
    (2, (2049, 9), False, EDGE, "gsadi", 1.0, 1.0),
    (2, (4097, 9), False, inputs.CONST, "zebra_x", 1.0, 1e4),
    (2, (4097, 10), True, inputs.CELL, "line_x", 0.7, 1.0),
    (2, (4097, 9), False, inputs.SEPARABLE, "adi", 0.8, 1.0),
    (2, (4097, 9), False, EDGE, "zebra_x", 1.0, 1.0),
    (3, (515, 9, 5), False, inputs.CONST, "line_x", 0.7, 1e3),
    (3, (1025, 8, 5), True, inputs.SEPARABLE, "zebra_x", 1.0, 1.0),
    (3, (2049, 5, 5), False, inputs.CELL, "zebra_x", 1.0, 1.0),
    (3, (4097, 5, 5), False, EDGE, "line_x", 0.7, 1.0),
    # y-lines of the constant kind: x-lines of the axis-swapped problem (4095 unknowns)
    (2, (9, 4097), False, inputs.CONST, "zebra_y", 1.0, 1e-4),
    (2, (9, 2049), False, inputs.CELL, "line_y", 0.7, 1.0),
]


@pytest.mark.parametrize("case", SWEEP_CASES,
                         ids=lambda c: f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'per' if c[2] else 'dir'}-k{c[3]}-{c[4]}")
def test_xline_sweeps_match_oracle(case):
    dim, n, per, kind, sm, om, eps = case
    sp = make(dim, n, per, kind, seed=sum(n) + 7 * kind, eps=eps)
    o = oracle_for(sp, 2, sm, om)
    s = Solver(sp, levels=2, smoother=sm, omega=om, max_cycles=10)
    rng = np.random.default_rng(13)
    u = rng.standard_normal(o.shape()) * o.unknown_mask()
    g = rng.standard_normal(o.shape())
    axes = (0, 1) if sm in ("adi", "gsadi") else ((1,) if sm.endswith("_y") else (0,))
    kappa = max(line_condition_bound(o, a) for a in axes)
    tol = max(1e-12, 4.0 * kappa * U64)
    for sweeps, order in ((1, 0), (2, 1)):
        e = rel(s.smooth(u, g, sweeps, order), o.smooth(u, g, sweeps, order))
        print(f"{case}: kappa_G {kappa:.2e}, error {e:.2e} = {e / (kappa * U64):.3f} kappa_G u")
        assert e <= tol


def test_xline_mixed_sweeps_converge_like_fp64():
    """The FP32 x-line kernels (one CTA a line) in the mixed solve: 1e-10 in the oracle's residual."""
    sp = make(2, (2049, 17), False, inputs.CONST, seed=5, eps=1e3)
    o = oracle_for(sp, 4, "zebra_x", 1.0)
    s = Solver(sp, levels=4, smoother="zebra_x", omega=1.0, precision="mixed", max_cycles=40)
    x, info = s.solve(sp.b, tol=1e-10)
    xn = x.cpu().numpy()
    rr = o.norm(o.defect(xn, sp.b)) / o.norm(sp.b)
    assert info["status"] == "MG_OK" and rr <= 1e-10, (info, rr)


def test_aniso4097_zebra_y_fp64_cycle_matches_oracle():
    """One FP64 F-cycle of the anisotropy study's strongest case (4097^2, eps = 1e-4, zebra y-lines,
    nu = 1, 12 grids) from a random start, against the oracle's cycle.

    What is compared is the correction c = x' - x that the cycle adds (x is the exact input),
    relative to max |c|.  Its rounding has two sources: the line solves (a few kappa_G u,
    kappa_G ~ 2e4 on the finest grid's lines), and the first defect b - A x, whose 5-point sums
    carry terms up to |A||x| ~ 1e4 times the defect.  That rounding, at most u |A||x| per node and
    of random sign, goes through the cycle like a right-hand side; the cycle is close to A^-1, and
    the component that A^-1 amplifies most (by 1 / lambda_min) collects about u |A||x| of it and
    spreads it over N unknowns with amplitude ~ 2 / sqrt(N): about 8 u |A||x| / (lambda_min sqrt(N)),
    1.5e-12 of max |c| here.  The bar is the larger of 1e-11 and 4 kappa_G u.
    """
    sp = inputs.anisotropic(n=4097, eps=1e-4, seed_f=1)
    L = inputs.max_levels(sp.n)
    p = orc.Problem(dim=2, n=sp.n, periodic_y=False, kind=orc.CONST, h=sp.h, c=sp.c)
    o = orc.Oracle(p, levels=L, smoother="zebra_y", omega=1.0, nu1=1, nu2=1, dense_max=4096)
    s = Solver(sp, levels=L, smoother="zebra_y", omega=1.0, nu1=1, nu2=1, precision="fp64", max_cycles=4)
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, o.shape()) * o.unknown_mask()
    kappa = line_condition_bound(o, 1)
    tol = max(1e-11, 4.0 * kappa * U64)
    for tr in (False, True):
        c_or = o.cycle(x, sp.b, transposed=tr) - x
        c_gpu = s.cycle(x, sp.b, transposed=tr).cpu().numpy() - x
        e = rel(c_gpu, c_or)
        print(f"4097^2 eps=1e-4 zebra-y cycle (transposed={tr}): kappa_G {kappa:.2e}, error of the correction "
              f"{e:.2e} (bar {tol:.2e})")
        assert e <= tol
