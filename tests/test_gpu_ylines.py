"""y-line smoothing (TRIy line Jacobi, GSTRIy zebra, the y half of GSADI) over a range of line
lengths, against the oracle.

Narrow grids with long y-lines reach every kernel a y-line can take:
- one thread per line below 4 unknowns;
- the register-resident kernel at each segment count from 1 to 256: Dirichlet and periodic
  lines of 4 to 2048 unknowns, segments of 2 to 8 rows with ragged splits;
- the scratch-array partition kernel above 2048.

Separable, cell and edge coefficients are used, in 2-D and 3-D.  Sweeps on the finest level
match in FP64 within the larger of 1e-12 and 4 kappa u.  Here kappa is the Gershgorin bound on the
line systems' condition number, which reaches 2e6 on the long anisotropic lines.  The
mixed-precision solve (FP32 line kernels) converges.
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

SWEEP_CASES = [
    # dim, n, periodic, kind, smoother, omega
    (2, (9, 5), False, inputs.SEPARABLE, "zebra_y", 1.0),        # 3 unknowns: one thread per line
    (2, (9, 7), False, inputs.SEPARABLE, "zebra_y", 1.0),        # 5: one segment
    (2, (17, 11), False, EDGE, "line_y", 0.7),                   # 9: two segments of 4 and 5
    (2, (9, 4), True, inputs.SEPARABLE, "zebra_y", 1.0),         # 4 periodic: one segment, cyclic
    (2, (9, 6), True, inputs.CELL, "line_y", 0.7),               # 6 periodic
    (2, (17, 18), True, inputs.SEPARABLE, "gsadi", 1.0),         # 18 periodic: 4 segments of 4 and 5
    (2, (33, 35), False, inputs.SEPARABLE, "zebra_y", 1.0),      # 33: 8 segments, ragged
    (2, (17, 66), True, EDGE, "zebra_y", 1.0),                   # 66 periodic: 16 segments
    (2, (9, 259), False, inputs.SEPARABLE, "line_y", 0.7),       # 257: 64 segments
    (2, (9, 1027), False, inputs.SEPARABLE, "zebra_y", 1.0),     # 1025: 256 segments, ragged
    (2, (9, 2048), True, inputs.SEPARABLE, "zebra_y", 1.0),      # 2048 periodic: 256 segments of 8
    (2, (9, 2049), False, EDGE, "gsadi", 1.0),                   # 2047: 256 segments
    (2, (9, 2051), False, inputs.SEPARABLE, "zebra_y", 1.0),     # 2049: the scratch-array kernel
    (2, (9, 2050), True, inputs.CELL, "line_y", 0.7),            # 2050 periodic: scratch-array, cyclic
    (2, (9, 4097), False, EDGE, "zebra_y", 1.0),                 # 4095: scratch-array
    (3, (9, 35, 9), False, inputs.SEPARABLE, "zebra_y", 1.0),    # 3-D, 33 unknowns
    (3, (9, 64, 9), True, EDGE, "gsadi", 1.0),                   # 3-D periodic
    (3, (9, 258, 5), True, inputs.CELL, "line_y", 0.7),          # 3-D, 258 periodic
]


def line_condition_bound(o):
    """Gershgorin bound on the condition number of the y-line systems C of the oracle's finest level.

    C has the node's diagonal D and the two y-couplings w_S, w_N.  Then lambda_max <= max(D + w_S + w_N) <= 2 max D
    and lambda_min >= min(D - w_S - w_N), the couplings off the line.  The margin is read from the
    oracle's operator: A v with v = 1 on every other column (and every other z-plane in 3-D)
    leaves D - w_S - w_N at each node where v = 1.
    """
    mask = o.unknown_mask()
    idx = np.indices(o.shape())
    i = idx[-1]
    kp = (idx[0] % 2,) if o.prob.dim == 3 else ()
    margin = np.inf
    for pi in (0, 1):
        for pk in ((0, 1) if kp else (None,)):
            sel = mask & (i % 2 == pi) & ((kp[0] == pk) if kp else True)
            margin = min(margin, o.apply(sel.astype(np.float64))[sel].min())
    return 2.0 * o.diag()[mask].max() / margin


def make_spec(dim, n, per, kind, seed):
    if kind == EDGE:
        return random_edges(dim, n[:dim], per, seed)
    return spec_of(dim, n, per, kind, np.random.default_rng(seed))


@pytest.mark.parametrize("case", SWEEP_CASES,
                         ids=lambda c: f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'per' if c[2] else 'dir'}-k{c[3]}-{c[4]}")
def test_yline_sweeps_match_oracle(case):
    dim, n, per, kind, sm, om = case
    sp = make_spec(dim, n, per, kind, seed=sum(n) + 7 * kind)
    if kind == EDGE:
        p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=orc.EDGE, h=sp.h, ex=sp.ex, ey=sp.ey,
                        ez=sp.ez)
        o = orc.Oracle(p, levels=2, smoother=sm, omega=om, dense_max=4096)
    else:
        o = oracle_of(sp, 2, sm, om)
    s = Solver(sp, levels=2, smoother=sm, omega=om, max_cycles=10)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(o.shape()) * o.unknown_mask()
    g = rng.standard_normal(o.shape())
    # The oracle's Thomas and the kernels' partitioned solves are both backward stable on these
    # diagonally dominant lines: each one's forward error is a few kappa(C) u (u = 2^-53), so the
    # two differ by up to about 4 kappa_G u.  Observed: 0.6 kappa_G u on the 1025-row line.
    # The bar is the larger of 1e-12 and 4 kappa_G u.
    tol = max(1e-12, 4.0 * line_condition_bound(o) * 2.0 ** -53)
    for sweeps, order in ((1, 0), (2, 1)):
        assert rel(s.smooth(u, g, sweeps, order), o.smooth(u, g, sweeps, order)) <= tol


FP32_CASES = SWEEP_CASES + [
    (2, (129, 1024), True, inputs.SEPARABLE, "zebra_y", 1.0),     # 64 lines of 128 segments
    (2, (257, 513), False, EDGE, "line_y", 0.7),                  # 255 lines of 64 segments, ragged
]


@pytest.mark.parametrize("case", FP32_CASES,
                         ids=lambda c: f"{c[0]}d-{'x'.join(map(str, c[1]))}-{'per' if c[2] else 'dir'}-k{c[3]}-{c[4]}")
def test_yline_fp32_sweeps_match_oracle(case):
    """The single-precision y-line kernels (mixed contexts) against the oracle's FP64 sweep on the
    same FP64 inputs.  Inputs and coefficients are rounded to FP32 and the line
    solves run in FP32, so the bar is the FP64 one with u = 2^-24: max(1e-6, 8 kappa_G u)."""
    dim, n, per, kind, sm, om = case
    sp = make_spec(dim, n, per, kind, seed=sum(n) + 7 * kind)
    if kind == EDGE:
        p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=orc.EDGE, h=sp.h, ex=sp.ex, ey=sp.ey,
                        ez=sp.ez)
        o = orc.Oracle(p, levels=2, smoother=sm, omega=om, dense_max=4096)
    else:
        o = oracle_of(sp, 2, sm, om)
    s = Solver(sp, levels=2, smoother=sm, omega=om, max_cycles=10, precision="mixed")
    rng = np.random.default_rng(12)
    u = rng.standard_normal(o.shape()) * o.unknown_mask()
    g = rng.standard_normal(o.shape())
    kappa = line_condition_bound(o)
    tol = max(1e-6, 8.0 * kappa * 2.0 ** -24)
    for sweeps, order in ((1, 0), (2, 1)):
        e = rel(s.smooth(u, g, sweeps, order), o.smooth(u, g, sweeps, order))
        print(f"{case}: kappa_G {kappa:.2e}, error {e:.2e} = {e / (kappa * 2.0 ** -24):.3f} kappa_G u32")
        assert e <= tol


SOLVE_CASES = [
    # dim, n, periodic, kind, levels, smoother
    (2, (17, 2049), False, inputs.SEPARABLE, 4, "zebra_y"),
    (2, (17, 2048), True, inputs.SEPARABLE, 4, "gsadi"),
    (2, (33, 1024), True, EDGE, 5, "zebra_y"),
    (3, (17, 64, 17), True, inputs.SEPARABLE, 3, "gsadi"),
]


@pytest.mark.parametrize("case", SOLVE_CASES, ids=lambda c: f"{c[0]}d-{'x'.join(map(str, c[1]))}-{c[5]}")
def test_yline_mixed_solve_converges_like_fp64(case):
    dim, n, per, kind, L, sm = case
    sp = make_spec(dim, n, per, kind, seed=3)
    kw = dict(levels=L, smoother=sm, omega=1.0, max_cycles=60)
    _, i64 = Solver(sp, **kw).solve(sp.b, tol=1e-10)
    _, i32 = Solver(sp, precision="mixed", **kw).solve(sp.b, tol=1e-10)
    assert i64["status"] == "MG_OK" and i32["status"] == "MG_OK"
    assert i32["relres"] <= 1e-10
    assert i32["cycles"] <= i64["cycles"] + 2
