"""GPU entry points beyond the solve itself: residual norm, host-buffer solve, apply on the
axis-swapped (y-line) layout -- each against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver  # noqa: E402


def _problem(n, kind, rng, periodic=False, eps=1.0):
    n0, n1 = n
    h = (1.0 / (n0 - 1), 1.0 / n1 if periodic else 1.0 / (n1 - 1), 1.0)
    b = rng.uniform(-1, 1, (n1, n0))
    sp = inputs.ProblemSpec(name="t", dim=2, n=(n0, n1, 1), periodic_y=periodic, kind=kind, h=h, b=b)
    if kind == inputs.CONST:
        sp.c = (eps / h[0] ** 2, 1.0 / h[1] ** 2, 0.0)
    elif kind == inputs.SEPARABLE:
        sp.sx, sp.sy, sp.sz = rng.uniform(1, 2, n0 - 1), rng.uniform(1, 2, n0), np.zeros(n0)
    else:
        sp.k = np.exp(rng.standard_normal((n1 if periodic else n1 - 1, n0 - 1)))
    return sp


def _oracle(sp, L, sm):
    return orc.Oracle(orc.Problem(dim=2, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c,
                                  sx=sp.sx, sy=sp.sy, sz=sp.sz, k=sp.k), levels=L, smoother=sm)


@pytest.mark.parametrize("kind,periodic,sm", [(inputs.CONST, False, "rbgs"), (inputs.SEPARABLE, True, "zebra_x"),
                                              (inputs.CELL, False, "zebra_y"), (inputs.CONST, False, "line_y")])
def test_residual_norm_matches_oracle(kind, periodic, sm):
    rng = np.random.default_rng(50)
    sp = _problem((129, 128 if periodic else 65), kind, rng, periodic)
    o = _oracle(sp, 4, sm)
    s = Solver(sp, levels=4, smoother=sm, omega=0.7 if sm.startswith("line") else 1.0)
    for l in (4, 2):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        g = rng.standard_normal(o.shape(l))
        ref = o.norm(o.defect(u, g, l), l)
        got = float(s.residual_norm(u, g, l).item())
        assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sm", ["rbgs", "zebra_y"])
def test_host_buffer_solve_equals_device_solve(precision, sm):
    rng = np.random.default_rng(51)
    sp = _problem((257, 129), inputs.CONST, rng, eps=0.05)
    s = Solver(sp, levels=7, smoother=sm, precision=precision, max_cycles=50)
    xd, info_d = s.solve(sp.b, tol=1e-10)
    xh = np.zeros(sp.shape)
    info_h = s.solve_host(np.ascontiguousarray(sp.b), xh, tol=1e-10)
    assert info_h["cycles"] == info_d["cycles"] and info_h["status"] == "MG_OK"
    assert np.abs(xh - xd.cpu().numpy()).max() <= 1e-13 * np.abs(xh).max()


def test_swapped_axes_operator_and_dims():
    """y-line smoothers run on the axis-swapped problem; the caller-facing layout is unchanged."""
    rng = np.random.default_rng(52)
    sp = _problem((129, 33), inputs.CELL, rng)
    o = _oracle(sp, 3, "zebra_y")
    s = Solver(sp, levels=3, smoother="zebra_y")
    assert s.level_shape(3) == (33, 129) and s.level_shape(1) == (9, 33)
    for l in (1, 2, 3):
        u = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        a = s.apply(u, l).cpu().numpy()
        ref = o.apply(u, l)
        assert np.abs(a - ref).max() <= 1e-12 * np.abs(ref).max()
