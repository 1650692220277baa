"""Per-kernel trace of a solve (MG_FLAG_TRACE, mg_trace_report).

A traced context runs each refinement step (or FP64 cycle) as one graph launch from the host,
with an event after every kernel; the report sums, per kernel launcher and level, the time
between consecutive events.  Checked here: the solve's result is the untraced one's, every
launch of the schedule is accounted for (launches per step times steps), the times are positive
and add up to no more than the solve's wall time, a size query leaves the trace in place, the
report consumes it, and contexts without the flag refuse the call.
"""
import time

import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300 import binding  # noqa: E402
from paper_0805_3041_gb300.binding import Solver, MGError, FLAG_TRACE, FLAG_NO_GRAPH  # noqa: E402
from test_gpu_parity import rel  # noqa: E402


@pytest.mark.parametrize("prec,n", [("mixed", 1025), ("fp64", 257)])
@pytest.mark.parametrize("extra", [0, FLAG_NO_GRAPH])
def test_trace_accounts_for_every_launch(prec, n, extra):
    sp = inputs.anisotropic(n=n, eps=1.0, seed_f=3)
    L = int(np.log2(n - 1))
    s = Solver(sp, levels=L, smoother="rbgs", precision=prec, max_cycles=40, flags=FLAG_TRACE | extra)
    ref = Solver(sp, levels=L, smoother="rbgs", precision=prec, max_cycles=40)
    xr, ir = ref.solve(sp.b, tol=1e-10)
    s.trace_report()                       # start from an empty trace
    k0 = s.launch_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, info = s.solve(sp.b, tol=1e-10)
    wall = (time.perf_counter() - t0) * 1e3
    launches = s.launch_count() - k0
    assert info["cycles"] == ir["cycles"] and rel(x, xr.cpu().numpy()) == 0.0
    # a size query does not consume the trace
    n_bytes = binding.C.c_size_t()
    assert s.lib.mg_trace_report(s.ctx, None, 0, binding.C.byref(n_bytes)) == 0 and n_bytes.value > 64
    rows = s.trace_report()
    traced = sum(r[2] for r in rows)
    total = sum(r[3] for r in rows)
    print(f"{prec} {n}^2 flags {extra}: {info['cycles']} steps, {launches} launches, {traced} traced, "
          f"{total:.3f} of {wall:.3f} ms; top: {rows[:3]}")
    assert rows and all(r[2] > 0 and r[3] > 0 and 1 <= r[1] <= L for r in rows)
    # every kernel of every step is traced (the solve's set-up and final launches are not)
    assert traced % info["cycles"] == 0 and 0 < traced < launches
    assert total <= wall
    assert s.trace_report() == []          # consumed


def test_trace_needs_the_flag():
    sp = inputs.anisotropic(n=65, eps=1.0, seed_f=3)
    s = Solver(sp, levels=5, smoother="rbgs")
    with pytest.raises(MGError) as ei:
        s.trace_report()
    assert ei.value.status == binding.EINVAL
