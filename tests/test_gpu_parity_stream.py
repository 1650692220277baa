"""FP64 parity of the row-streaming red-black sweep (the register-marching kernel that
FP64 grids above the tile threshold use), forced onto small grids with tile_nodes=-1:
sweeps and whole cycles against the oracle at 1e-12, as for the default path."""
import numpy as np
import pytest

from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver  # noqa: E402
from test_gpu_parity import spec_of, oracle_of, rel, TOL64  # noqa: E402

CASES = [
    # dim, n, periodic, kind, levels
    (2, (129, 65), False, inputs.CONST, 5),
    (2, (257, 129), False, inputs.CONST, 6),
    (2, (129, 64), True, inputs.SEPARABLE, 5),
    (2, (385, 97), False, inputs.SEPARABLE, 4),
]


@pytest.mark.parametrize("dim,n,per,kind,L", CASES)
def test_streaming_sweep_and_cycle_match_oracle(dim, n, per, kind, L):
    rng = np.random.default_rng(31)
    sp = spec_of(dim, n, per, kind, rng, eps=0.6)
    o = oracle_of(sp, L, "rbgs", 1.0)
    s = Solver(sp, levels=L, smoother="rbgs", omega=1.0, max_cycles=60, tile_nodes=-1)
    for order in (0, 1):
        u = rng.standard_normal(o.shape()) * o.unknown_mask()
        g = rng.standard_normal(o.shape())
        for sweeps in (1, 3):
            assert rel(s.smooth(u, g, sweeps, order, L), o.smooth(u, g, sweeps, order, L)) <= TOL64
    x = rng.standard_normal(o.shape()) * o.unknown_mask()
    for transposed in (False, True):
        assert rel(s.cycle(x, sp.b, transposed), o.cycle(x, sp.b, transposed=transposed)) <= 1e-11
