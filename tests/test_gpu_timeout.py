"""The bounded-wait timeout path of the TMA-fed sweep, made to run out on purpose.

MG_FLAG_TEST_WAIT_TIMEOUT leaves one row copy of the first single-precision TMA sweep of a solve
uncopied: the compute warps' waits on it give up after their cycle budget (about half a
second), they and the producer stop, and the solve reports MG_ETIMEOUT.  No fault, trap or
endless loop is involved.  The context stays usable: a solve without the hook on the same
device gives the right answer afterwards.
"""
import time

import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import (Solver, MGError, FLAG_TEST_WAIT_TIMEOUT,  # noqa: E402
                                           FLAG_NO_GRAPH)

ETIMEOUT = 6


@pytest.mark.parametrize("extra", [0, FLAG_NO_GRAPH], ids=["graph", "host-loop"])
def test_wait_that_runs_out_reports_timeout_and_leaves_the_device_usable(extra):
    sp = inputs.anisotropic(n=257, eps=1.0, seed_f=1)
    kw = dict(levels=inputs.max_levels(sp.n), smoother="rbgs", precision="mixed", max_cycles=20, tile_nodes=-1)
    s = Solver(sp, flags=FLAG_TEST_WAIT_TIMEOUT | extra, **kw)
    t0 = time.perf_counter()
    with pytest.raises(MGError) as e:
        s.solve(sp.b, tol=1e-10)
    elapsed = time.perf_counter() - t0
    assert e.value.status == ETIMEOUT
    assert elapsed < 30.0
    # the device and the library still work: the same problem without the hook
    x2, info2 = Solver(sp, **kw).solve(sp.b, tol=1e-10)
    assert info2["status"] == "MG_OK" and info2["relres"] <= 1e-10
    # and the hooked context, solved again, times out again (the hook re-arms per solve)
    with pytest.raises(MGError) as e:
        s.solve(sp.b, tol=1e-10)
    assert e.value.status == ETIMEOUT
