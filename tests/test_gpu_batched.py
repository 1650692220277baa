"""Batched solves (mg_batch_create / mg_batch_solve / mg_solve_batched) through the C ABI.

In the graph form each instance of a batch runs exactly the kernels its own mg_solve
runs (the same device-side loop, as one branch of one graph), so the batch must
reproduce the individual solves bit for bit, with the same cycle counts; a few instances are also
checked against the oracle's FP64 residual.  Instances: uneven sizes, anisotropies
eps in [1e-3, 1] with the smoother chosen for each, mixed and FP64 precision.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import (Solver, Batch, solve_batched, MGError, FLAG_NO_GRAPH,  # noqa: E402
                                           EINVAL, BATCH_GRAPH)


def instances(count=10, seed=41):
    specs = inputs.batched(count=count, sizes=(65, 129, 257), eps_range=(1e-3, 1.0), seed=seed)
    out = []
    for q, sp in enumerate(specs):
        eps = sp.c[0] * sp.h[0] ** 2
        sm = "rbgs" if eps > 0.2 else "zebra_y"
        prec = "fp64" if q % 4 == 3 else "mixed"
        s = Solver(sp, levels=inputs.max_levels(sp.n), smoother=sm, precision=prec, max_cycles=60)
        out.append((sp, s))
    return out


def tensors(sp, dev="cuda"):
    b = torch.from_numpy(sp.b).to(dev)
    x = torch.zeros_like(b)
    return b, x


def test_batch_matches_individual_solves():
    inst = instances()
    bs, xs = zip(*[tensors(sp) for sp, _ in inst])
    solvers = [s for _, s in inst]
    batch = Batch(solvers, bs, xs, mode=BATCH_GRAPH)
    assert batch.info()[0] == 0
    infos = batch.solve(tol=1e-10)
    for (sp, s), b, x, info in zip(inst, bs, xs, infos):
        xr = torch.zeros_like(b)
        ref = s.solve_into(b, xr, tol=1e-10)
        assert info["status"] == ref["status"] == "MG_OK", (sp.name, info, ref)
        assert info["cycles"] == ref["cycles"], sp.name
        assert torch.equal(x, xr), sp.name
        assert np.array_equal(info["history"], ref["history"]), sp.name
    # the batch can be launched again: same start vectors, same results
    first = [x.clone() for x in xs]
    for x in xs:
        x.zero_()
    again = batch.solve(tol=1e-10)
    for a, b_, x0, x1 in zip(infos, again, first, xs):
        assert a["cycles"] == b_["cycles"] and torch.equal(x0, x1)
    batch.close()


def test_batch_residuals_in_fp64_oracle():
    inst = instances(count=6, seed=42)
    bs, xs = zip(*[tensors(sp) for sp, _ in inst])
    infos = solve_batched([s for _, s in inst], bs, xs, tol=1e-10)
    for (sp, s), x, info in zip(inst, xs, infos):
        o = orc.Oracle(orc.Problem(dim=2, n=sp.n, kind=orc.CONST, h=sp.h, c=sp.c), levels=2,
                       smoother="rbgs", omega=1.0)
        xn = x.cpu().numpy()
        rr = o.norm(o.defect(xn, sp.b)) / o.norm(sp.b)
        assert info["status"] == "MG_OK" and rr <= 1e-10, (sp.name, info, rr)


def test_batch_zero_rhs_and_tolerance_per_call():
    inst = instances(count=3, seed=43)
    bs, xs = zip(*[tensors(sp) for sp, _ in inst])
    bs[1].zero_()
    xs[1].fill_(1.0)
    batch = Batch([s for _, s in inst], bs, xs)
    infos = batch.solve(tol=1e-10)
    assert infos[1]["status"] == "MG_OK" and infos[1]["cycles"] == 0
    assert torch.count_nonzero(xs[1]) == 0
    loose = [x.clone() for x in xs]
    for x in xs:
        x.zero_()
    infos6 = batch.solve(tol=1e-6)
    for a, b_ in zip(infos, infos6):
        assert b_["cycles"] <= a["cycles"]
        assert b_["relres"] <= 1e-6
    del loose
    batch.close()


def test_batch_rejects_bad_sets():
    sp0, sp1 = inputs.anisotropic(n=65, eps=0.5), inputs.anisotropic(n=129, eps=0.5)
    s0 = Solver(sp0, levels=inputs.max_levels(sp0.n), smoother="rbgs", precision="mixed")
    s1 = Solver(sp1, levels=inputs.max_levels(sp1.n), smoother="rbgs", precision="mixed")
    b0, x0 = tensors(sp0)
    b1, x1 = tensors(sp1)
    with pytest.raises(MGError) as e:
        Batch([s0, s0], [b0, b0], [x0, x0])
    assert e.value.status == EINVAL
    s_ng = Solver(sp1, levels=inputs.max_levels(sp1.n), smoother="rbgs", precision="mixed", flags=FLAG_NO_GRAPH)
    with pytest.raises(MGError) as e:
        Batch([s0, s_ng], [b0, b1], [x0, x1])
    assert e.value.status == EINVAL
    with pytest.raises(ValueError):
        Batch([s0, s1], [b0, b0], [x0, x1])   # b1's shape differs from b0's
