"""The TMA-fed FP32 red-black sweep against the register-marching sweep and the oracle.

Both kernels perform the same floating-point operations in the same order, so mixed-
precision solves through either give the same iterates; the bar is 1e-6 relative (a few
FP32 roundings amplified by three cycles) and equality is reported.  Shapes cover a single
128-column strip (n0 = 129), a ragged last strip (n0 = 257: one real column in the third
strip), periodic y with separable coefficients, row counts that leave a ragged last chunk
of rows, several chunk heights, and the sweep that folds in the coarse-grid correction
(every post-smoothing).  The mixed solve through the TMA sweep must meet 1e-10 in the
oracle's FP64 residual.  Solvers here pass tile_nodes=-1 so that even small grids take the
row-streaming kernels; the last test checks the one-pass tile kernel used below the default
threshold against them.
"""
import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver, FLAG_NO_TMA  # noqa: E402
from test_gpu_parity import spec_of, oracle_of, rel  # noqa: E402

CASES = [
    # dim, n, periodic_y, kind, levels, eps
    (2, (129, 129), False, inputs.CONST, 7, 1.0),
    (2, (257, 257), False, inputs.CONST, 8, 1.0),
    (2, (257, 133), False, inputs.CONST, 3, 0.3),
    (2, (513, 200), True, inputs.SEPARABLE, 4, 1.0),
    (2, (129, 128), True, inputs.SEPARABLE, 7, 1.0),
    (2, (1025, 385), False, inputs.SEPARABLE, 8, 1.0),
]


@pytest.mark.parametrize("dim,n,per,kind,L,eps", CASES)
def test_tma_sweep_matches_marching_sweep(dim, n, per, kind, L, eps):
    rng = np.random.default_rng(21)
    sp = spec_of(dim, n, per, kind, rng, eps=eps)
    a = Solver(sp, levels=L, smoother="rbgs", precision="mixed", max_cycles=3, tile_nodes=-1)
    b = Solver(sp, levels=L, smoother="rbgs", precision="mixed", max_cycles=3, flags=FLAG_NO_TMA, tile_nodes=-1)
    xa, ia = a.solve(sp.b, tol=0.0)
    xb, ib = b.solve(sp.b, tol=0.0)
    d = rel(xa, xb.cpu().numpy())
    print(f"TMA vs marching sweep after 3 steps: max rel difference {d:.3e}")
    assert d <= 1e-6
    assert np.allclose(ia["history"], ib["history"], rtol=1e-5, atol=0)


@pytest.mark.parametrize("rows", [1, 2, 3, 7, 64, 500])
def test_tma_sweep_chunk_heights(rows):
    """Rows per warp from 1 (prologue-only chunks) to more than the grid has."""
    rng = np.random.default_rng(22)
    sp = spec_of(2, (257, 97), False, inputs.CONST, rng, eps=0.7)
    a = Solver(sp, levels=6, smoother="rbgs", precision="mixed", max_cycles=3, sweep_rows=rows, tile_nodes=-1)
    b = Solver(sp, levels=6, smoother="rbgs", precision="mixed", max_cycles=3, flags=FLAG_NO_TMA, tile_nodes=-1)
    xa, _ = a.solve(sp.b, tol=0.0)
    xb, _ = b.solve(sp.b, tol=0.0)
    assert rel(xa, xb.cpu().numpy()) <= 1e-6


def test_tma_mixed_solve_meets_tolerance_in_fp64():
    rng = np.random.default_rng(23)
    sp = spec_of(2, (513, 513), False, inputs.CONST, rng, eps=1.0)
    o = oracle_of(sp, 9, "rbgs", 1.0)
    s = Solver(sp, levels=9, smoother="rbgs", precision="mixed", max_cycles=40, tile_nodes=-1)
    x, info = s.solve(sp.b, tol=1e-10)
    xn = x.cpu().numpy()
    rr = o.norm(o.defect(xn, sp.b)) / o.norm(sp.b)
    assert info["status"] == "MG_OK" and rr <= 1e-10, (info, rr)


@pytest.mark.parametrize("kind,per", [(inputs.CONST, False), (inputs.SEPARABLE, True)])
def test_tile_sweep_matches_streaming_sweep(kind, per):
    """Grids at or below the tile threshold smooth with the one-pass tile kernel; it performs
    the same relaxations as the row-streaming sweep (in a different FMA order)."""
    rng = np.random.default_rng(24)
    sp = spec_of(2, (257, 256 if per else 257), per, kind, rng, eps=0.5)
    a = Solver(sp, levels=7, smoother="rbgs", precision="mixed", max_cycles=3, tile_nodes=-1)
    b = Solver(sp, levels=7, smoother="rbgs", precision="mixed", max_cycles=3, tile_nodes=1 << 30)
    xa, _ = a.solve(sp.b, tol=0.0)
    xb, _ = b.solve(sp.b, tol=0.0)
    d = rel(xa, xb.cpu().numpy())
    print(f"tile vs streaming sweep after 3 steps: max rel difference {d:.3e}")
    assert d <= 1e-6
