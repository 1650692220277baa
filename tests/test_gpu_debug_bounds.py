"""The checking build (-DMG_DEBUG): device-side bounds checks that report MG_EBOUNDS.

Every kernel of the checking build tests the node indices of its global accesses against the
level's arrays; a failed check skips the access, records its site in a device word and makes
the call return MG_EBOUNDS (no trap, no fault).  Here:

- the build identifies itself (mg_debug_build), and the normal build refuses the probe flag;
- solves, adjoint solves, single steps, the gradient and batches over every smoother family,
  coefficient kind, precision and kernel path (TMA, marching and tile sweeps, the single-CTA
  coarse cycle, conjugate gradients, long x-lines, y-lines, Galerkin levels, the float-float
  defect, the persistent batch) run with no check failing, and give the normal build's results;
- the probe (MG_FLAG_TEST_BOUNDS: one check of the index one past the finest grid's last node,
  nothing accessed there) makes a solve return MG_EBOUNDS naming its site, and the context
  still solves afterwards.
"""
import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300 import binding  # noqa: E402
from paper_0805_3041_gb300.binding import (Solver, Batch, MGError, BATCH_PERSISTENT, BATCH_GRAPH,  # noqa: E402
                                           FLAG_NO_GRAPH, FLAG_NO_TMA, FLAG_ADAPTIVE_CORR, FLAG_FMG_START,
                                           FLAG_GALERKIN, FLAG_TEST_BOUNDS)
from test_gpu_parity import spec_of, rel  # noqa: E402
from test_gpu_edge import random_edges  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def checking_build():
    lib = binding.load(debug=True)   # compiled on first use
    assert lib.mg_debug_build() == 1
    assert binding.load().mg_debug_build() == 0


def problem(dim, n, per, kind, seed, eps=1.0):
    if kind == inputs.EDGE:
        return random_edges(dim, n[:dim], per, seed)
    return spec_of(dim, n, per, kind, np.random.default_rng(seed), eps=eps)


CASES = [
    # name, (dim, n, periodic, kind, eps), levels, smoother, precision, flags
    ("tma-sweeps-ff", (2, (2049, 2049), False, inputs.CONST, 1.0), 11, "rbgs", "mixed", 0),
    ("marching", (2, (1025, 1025), False, inputs.SEPARABLE, 1.0), 10, "rbgs", "mixed", FLAG_NO_TMA),
    ("fp64-adaptive", (2, (257, 129), False, inputs.CONST, 1.0), 6, "rbgs", "fp64", FLAG_NO_GRAPH | FLAG_ADAPTIVE_CORR),
    ("periodic-gsadi-fmg", (2, (129, 128), True, inputs.SEPARABLE, 1.0), 5, "gsadi", "mixed", FLAG_FMG_START),
    ("cell-zebra-y", (2, (129, 129), False, inputs.CELL, 1.0), 5, "zebra_y", "fp64", 0),
    ("edge-jacobi", (2, (129, 65), False, inputs.EDGE, 1.0), 4, "jacobi", "fp64", 0),
    ("3d-zebra-x", (3, (33, 33, 33), False, inputs.CONST, 1.0), 3, "zebra_x", "mixed", 0),
    ("3d-cell-rbgs", (3, (33, 33, 33), False, inputs.CELL, 1.0), 4, "rbgs", "fp64", 0),
    ("cg-coarsest", (2, (257, 129), False, inputs.CONST, 1.0), 2, "rbgs", "mixed", 0),
    ("long-x-lines", (2, (2049, 17), False, inputs.CONST, 1e3), 4, "zebra_x", "mixed", 0),
    ("long-y-lines", (2, (65, 1025), False, inputs.SEPARABLE, 1.0), 4, "zebra_y", "fp64", 0),
    ("galerkin", (2, (129, 129), False, inputs.CONST, 1.0), 5, "rbgs", "fp64", FLAG_GALERKIN),
]


def solvers(case, **kw):
    name, (dim, n, per, kind, eps), L, sm, prec, flags = case
    sp = problem(dim, n, per, kind, seed=len(name), eps=eps)
    om = 0.8 if sm == "jacobi" else 1.0
    mk = lambda debug: Solver(sp, levels=L, smoother=sm, omega=om, precision=prec, max_cycles=40, flags=flags,
                              debug=debug, **kw)
    return sp, mk(True), mk(False)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_checked_solves_pass_every_check(case):
    sp, sd, sn = solvers(case)
    xd, infod = sd.solve(sp.b, tol=1e-10)       # MG_EBOUNDS would raise
    xn, infon = sn.solve(sp.b, tol=1e-10)
    e = rel(xd, xn.cpu().numpy())
    print(f"{case[0]}: {infod['cycles']} cycles, relres {infod['relres']:.2e}; against the normal build {e:.1e}")
    assert infod["status"] == infon["status"] == "MG_OK"
    assert infod["cycles"] == infon["cycles"]
    assert e <= (1e-12 if case[4] == "fp64" else 1e-9)
    if case[4] == "fp64" and not (case[5] & FLAG_GALERKIN):
        ld, _ = sd.solve_adjoint(sp.b, tol=1e-10)
        ln, _ = sn.solve_adjoint(sp.b, tol=1e-10)
        assert rel(ld, ln.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4], CASES[7]], ids=lambda c: c[0])
def test_checked_single_steps_pass_every_check(case):
    sp, sd, sn = solvers(case)
    rng = np.random.default_rng(3)
    L = case[2]
    u, g = rng.standard_normal(tuple(sd.shape)), np.asarray(sp.b, dtype=np.float64)
    pairs = [
        (sd.smooth(u, g, 2, 1), sn.smooth(u, g, 2, 1)),
        (sd.defect(u, g), sn.defect(u, g)),
        (sd.restrict(u), sn.restrict(u)),
        (sd.cycle(u, g), sn.cycle(u, g)),
    ]
    if L >= 2:
        uo_d, gc_d = sd.descend(u, g)
        uo_n, gc_n = sn.descend(u, g)
        pairs += [(uo_d, uo_n), (gc_d, gc_n)]
        ec = rng.standard_normal(tuple(sd.level_shape(L - 1)))
        pairs.append((sd.prolong_add(ec, u), sn.prolong_add(ec, u)))
    if case[4] == "mixed":
        pairs.append((sd.outer_defect(u, g)[0], sn.outer_defect(u, g)[0]))
    if case[1][3] == inputs.CELL:
        pairs.append((sd.grad_coeff(u, g), sn.grad_coeff(u, g)))
    for a, b in pairs:
        assert rel(a, b.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("mode", [BATCH_PERSISTENT, BATCH_GRAPH])
def test_checked_batch_passes_every_check(mode):
    specs = [spec_of(2, (n, n), False, inputs.CONST, np.random.default_rng(n)) for n in (65, 129, 257)]
    dev = torch.device("cuda")
    ss = [Solver(sp, levels=5, smoother="rbgs", precision="mixed", max_cycles=40, debug=True) for sp in specs]
    bs = [torch.from_numpy(sp.b).to(dev) for sp in specs]
    xs = [torch.zeros_like(b) for b in bs]
    infos = Batch(ss, bs, xs, mode=mode).solve(tol=1e-10)
    for sp, x, info in zip(specs, xs, infos):
        _, ref = Solver(sp, levels=5, smoother="rbgs", precision="mixed", max_cycles=40).solve(sp.b, tol=1e-10)
        assert info["status"] == "MG_OK" and info["relres"] <= 1e-10 and abs(info["cycles"] - ref["cycles"]) <= 1


def test_probe_returns_ebounds_and_the_context_recovers():
    sp = spec_of(2, (129, 129), False, inputs.CONST, np.random.default_rng(1))
    for extra in (0, FLAG_NO_GRAPH):
        s = Solver(sp, levels=5, smoother="rbgs", flags=FLAG_TEST_BOUNDS | extra, debug=True)
        with pytest.raises(MGError) as ei:
            s.solve(sp.b, tol=1e-10)
        assert ei.value.status == binding.EBOUNDS
        assert "kernels_point.cu" in str(ei.value)
        print(str(ei.value))
        # the word was cleared: a call without the probe on the same context passes
        r = s.defect(np.zeros(s.shape), sp.b)
        want = Solver(sp, levels=5).defect(np.zeros(s.shape), sp.b)
        assert rel(r, want.cpu().numpy()) == 0.0
    # a context without the flag solves as usual
    x, info = Solver(sp, levels=5, smoother="rbgs", debug=True).solve(sp.b, tol=1e-10)
    assert info["status"] == "MG_OK"


def test_normal_build_refuses_the_probe_flag():
    sp = spec_of(2, (65, 65), False, inputs.CONST, np.random.default_rng(2))
    with pytest.raises(MGError) as ei:
        Solver(sp, levels=4, flags=FLAG_TEST_BOUNDS)
    assert ei.value.status == binding.EINVAL
