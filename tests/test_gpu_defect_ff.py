"""The refinement loop's float-float defect against the oracle's FP64 defect.

MG_MIXED contexts (2-D, constant or separable coefficients) evaluate r = b - A x of the FP64
iterate in float-float arithmetic: each FP64 operand split into two floats (47 significant
bits), error-free FP32 sums and products.  Per node the result may differ from the exact
defect by its own FP32 rounding, 2^-24 |r|, plus the pair arithmetic's error, a few 2^-46 of
the largest stencil term, (|b| + |A||x|)_p; the test allows 2^-24 |r| + 16 * 2^-46 (|b| + |A||x|)_p
and prints what it finds.  At an iterate near convergence (relative residual ~2e-11 at 4097^2,
where the 5-point sums cancel terms ~1e7 times the result) the error of the whole defect is
printed relative to ||r|| and bounded relative to ||b||: there the error must stay below the
solver's own estimate, 2^-46 ||(|b| + |A||x|)||, by which the loop stops short of the
tolerance.  MG_FLAG_FP64_DEFECT keeps the FP64 kernel: within its FP32 rounding of the oracle's
defect.  The mixed solve with the float-float loop reports its FP64 residual; on lines so
strongly coupled that the float-float error is near the tolerance (eps = 1e3, error ~7e-11
||b||) the loop moves to FP64 defects and still meets 1e-10 in the oracle's residual.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver, FLAG_FP64_DEFECT  # noqa: E402
from test_gpu_parity import spec_of  # noqa: E402

U32, U46 = 2.0 ** -24, 2.0 ** -46


def oracle_for(sp, levels):
    p = orc.Problem(dim=2, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c, sx=sp.sx, sy=sp.sy)
    return orc.Oracle(p, levels=levels, smoother="rbgs", dense_max=4096)


def abs_terms(o, x, b):
    """(|b| + |A||x|) per node: for positive edge weights |A||x| = 2 D |x| - A |x|."""
    ax = np.abs(x)
    return (np.abs(b) + 2.0 * o.diag() * ax - o.apply(ax)) * o.unknown_mask()


def check(o, s, x, b, label):
    r, sq = s.outer_defect(x, b)
    r = r.cpu().numpy()
    want = o.defect(x, b)
    bound = U32 * np.abs(want) + 16 * U46 * abs_terms(o, x, b)
    err = np.abs(r - want)
    ratio = float((err / np.maximum(bound, 1e-300)).max())
    rel = float(np.linalg.norm(err) / max(np.linalg.norm(want), 1e-300))
    relb = float(np.linalg.norm(err) / np.linalg.norm(b * o.unknown_mask()))
    own = float(np.sum(r ** 2))   # the kernel's sum of its own FP32 values' squares (FP32 partial sums)
    print(f"{label}: max error / bound {ratio:.3f}, ||r - r_exact|| / ||r_exact|| {rel:.2e}, / ||b|| {relb:.2e}, "
          f"sum of squares {sq:.6e} (of its values {own:.6e})")
    assert np.all(err <= bound), label
    assert abs(sq - own) <= 1e-4 * own + 1e-300
    return relb


CASES = [
    ("aniso4097", lambda: inputs.anisotropic(n=4097, eps=1.0, seed_f=1), 12),
    ("ragged-sep-periodic", lambda: spec_of(2, (1543, 1100), True, inputs.SEPARABLE, np.random.default_rng(9)), 2),
    ("const-eps1e-3", lambda: inputs.anisotropic(n=1025, eps=1e-3, seed_f=3), 10),
]


@pytest.mark.parametrize("name,make,L", CASES, ids=[c[0] for c in CASES])
def test_float_float_defect_within_its_bound(name, make, L):
    sp = make()
    o = oracle_for(sp, L)
    s = Solver(sp, levels=L, smoother="rbgs", precision="mixed", max_cycles=40)
    rng = np.random.default_rng(5)
    m = o.unknown_mask()
    # a random iterate (no cancellation), then one near the solution (strong cancellation)
    check(o, s, rng.standard_normal(m.shape) * m, sp.b, f"{name} random x")
    sm = "zebra_y" if name == "const-eps1e-3" else "rbgs"
    s64 = Solver(sp, levels=L, smoother=sm, precision="mixed", max_cycles=40, flags=FLAG_FP64_DEFECT)
    x, info = s64.solve(sp.b, tol=1e-10)
    xn = x.cpu().numpy()
    relb = check(o, s, xn, sp.b, f"{name} converged x (relres {info['relres']:.1e})")
    estimate = U46 * np.linalg.norm(abs_terms(o, xn, sp.b)) / np.linalg.norm(sp.b * m)
    print(f"   error / ||b|| {relb:.2e}, the solver's estimate {estimate:.2e}")
    assert relb <= estimate


def test_fp64_flag_keeps_the_fp64_defect():
    sp = inputs.anisotropic(n=1025, eps=0.5, seed_f=2)
    o = oracle_for(sp, 10)
    s = Solver(sp, levels=10, smoother="rbgs", precision="mixed", flags=FLAG_FP64_DEFECT)
    x, _ = s.solve(sp.b, tol=1e-10)
    xn = x.cpu().numpy()
    r, _ = s.outer_defect(xn, sp.b)
    want = o.defect(xn, sp.b)
    # the FP64 kernel's only difference from the oracle: its rounding to FP32, and FP64 rounding
    # of terms up to |A||x|
    bound = U32 * np.abs(want) + 8 * 2.0 ** -53 * abs_terms(o, xn, sp.b)
    assert np.all(np.abs(r.cpu().numpy() - want) <= bound)


@pytest.mark.parametrize("flags", [0, FLAG_FP64_DEFECT])
def test_mixed_solve_reports_the_fp64_residual(flags):
    """The loop stops on the float-float residual (below the tolerance by its error estimate) and reports the FP64
    one: 1e-10 in the oracle's residual, the same report to 1e-3, graph and kernel by kernel."""
    from paper_0805_3041_gb300.binding import FLAG_NO_GRAPH, FLAG_NO_PDL
    sp = inputs.anisotropic(n=2049, eps=0.3, seed_f=4)
    o = oracle_for(sp, 11)
    xs = []
    for extra in (0, FLAG_NO_GRAPH, FLAG_NO_PDL):
        s = Solver(sp, levels=11, smoother="rbgs", precision="mixed", max_cycles=40, flags=flags | extra)
        x, info = s.solve(sp.b, tol=1e-10)
        xn = x.cpu().numpy()
        xs.append((extra, xn, info["cycles"]))
        rr = o.norm(o.defect(xn, sp.b)) / o.norm(sp.b)
        print(f"flags {flags | extra}: {info['cycles']} steps, report {info['relres']:.4e}, oracle {rr:.4e}")
        assert info["status"] == "MG_OK" and rr <= 1e-10
        assert abs(rr - info["relres"]) <= 1e-3 * rr
    # the device loop, the host loop and ordinary graph edges run the same kernels on the same data,
    # the fused update's buffer swaps included: the same iterate, bit for bit
    for extra, xn, cyc in xs[1:]:
        assert cyc == xs[0][2] and np.array_equal(xn, xs[0][1]), extra


def test_start_vector_meeting_the_tolerance_takes_no_step():
    """The start vector's defect is a float-float one too: a start that already meets the
    tolerance by the defect's error estimate stops the loop before any refinement step, the FP64
    residual after the loop confirms it and is reported, and the iterate comes back unchanged, in
    the device loop and the host loop alike."""
    from paper_0805_3041_gb300.binding import FLAG_NO_GRAPH
    sp = inputs.anisotropic(n=513, eps=1.0, seed_f=6)
    o = oracle_for(sp, 9)
    xs, info0 = Solver(sp, levels=9, smoother="rbgs", precision="mixed", max_cycles=40).solve(sp.b, tol=1e-12)
    assert info0["status"] == "MG_OK" and info0["cycles"] > 0
    b = torch.from_numpy(sp.b).to(xs.device)
    for extra in (0, FLAG_NO_GRAPH):
        s = Solver(sp, levels=9, smoother="rbgs", precision="mixed", max_cycles=40, flags=extra)
        x = xs.clone()
        info = s.solve_into(b, x, tol=1e-10)
        rr = o.norm(o.defect(x.cpu().numpy(), sp.b)) / o.norm(sp.b)
        print(f"flags {extra}: {info['cycles']} steps, report {info['relres']:.4e}, oracle {rr:.4e}")
        assert info["status"] == "MG_OK" and info["cycles"] == 0, (extra, info)
        assert torch.equal(x, xs), extra
        assert rr <= 1e-10 and abs(rr - info["relres"]) <= 1e-2 * rr


def test_strongly_coupled_lines_move_the_loop_to_fp64_defects():
    """x-lines with eps = 1e3 (n = 2049 x 17): the float-float defect's error (~7e-11 ||b|| near
    the solution) is close to the tolerance, so the loop has to finish on FP64 defects; it then
    takes at most one refinement step more than a loop on FP64 defects throughout."""
    from paper_0805_3041_gb300.binding import FLAG_NO_GRAPH
    sp = spec_of(2, (2049, 17), False, inputs.CONST, np.random.default_rng(5), eps=1e3)
    p = orc.Problem(dim=2, n=sp.n, periodic_y=False, kind=sp.kind, h=sp.h, c=sp.c)
    o = orc.Oracle(p, levels=4, smoother="zebra_x", dense_max=4096)
    ref = Solver(sp, levels=4, smoother="zebra_x", precision="mixed", max_cycles=40, flags=FLAG_FP64_DEFECT)
    _, iref = ref.solve(sp.b, tol=1e-10)
    for extra in (0, FLAG_NO_GRAPH):
        s = Solver(sp, levels=4, smoother="zebra_x", precision="mixed", max_cycles=40, flags=extra)
        x, info = s.solve(sp.b, tol=1e-10)
        rr = o.norm(o.defect(x.cpu().numpy(), sp.b)) / o.norm(sp.b)
        print(f"flags {extra}: {info['cycles']} steps (FP64 defects: {iref['cycles']}), report {info['relres']:.3e}, "
              f"oracle {rr:.3e}")
        assert info["status"] == "MG_OK" and rr <= 1e-10
        assert info["cycles"] <= iref["cycles"] + 1
