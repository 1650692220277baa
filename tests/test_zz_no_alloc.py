"""mg_residual_norm_noalloc: the residual norm for callers that cannot allocate device memory.

The entry point keeps its partial sums in a static device array instead of a caller
workspace.  Through the C ABI it must give the same norm as mg_residual_norm (the
context-based entry point, whose partials live in the workspace) and as the oracle's
norm of its defect, on consecutive calls that reuse the shared array, and reject,
before launching anything, the grids its array cannot serve.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300 import binding  # noqa: E402
from paper_0805_3041_gb300.binding import Solver  # noqa: E402

TOL = 1e-12   # relative, as for the FP64 parity tests


def _abi_args(sp, stream):
    p = binding.Params()
    p.dim = sp.dim
    p.n = (C.c_int * 3)(*[int(v) for v in sp.n])
    p.periodic_y = int(bool(sp.periodic_y))
    p.levels = 1
    p.stream = stream.cuda_stream
    k = binding.Coeffs()
    k.kind = int(sp.kind)
    k.h = (C.c_double * 3)(*[float(v) for v in sp.h])
    k.c = (C.c_double * 3)(*[float(v) for v in (sp.c or (0, 0, 0))])
    keep = []
    for name in ("sx", "sy", "sz", "k"):
        arr = getattr(sp, name)
        if arr is not None:
            t = torch.tensor(np.ascontiguousarray(arr, dtype=np.float64), device="cuda")
            keep.append(t)
            setattr(k, name, t.data_ptr())
    return p, k, keep


def _noalloc(lib, p, k, u, b, out):
    return lib.mg_residual_norm_noalloc(C.byref(p), C.byref(k), C.c_void_p(u.data_ptr()), C.c_void_p(b.data_ptr()),
                                        C.c_void_p(out.data_ptr()))


def _cases():
    rng = np.random.default_rng(60)
    out = []
    sp = inputs.anisotropic(n=1025, eps=0.01, seed_f=61)
    out.append((sp, 10, "rbgs"))
    sp = inputs.annulus_2d(nr=257, nt=256)
    out.append((sp, 7, "zebra_x"))
    sp = inputs.poisson_3d(n=65, seed=62)
    out.append((sp, 6, "rbgs"))
    sp = inputs.stretched_x(n=257, beta=3.0, seed=63)        # separable, 2-D, not periodic
    out.append((sp, 8, "rbgs"))
    return out, rng


def _oracle_norm(sp, u, b):
    """||b - A u||_2 over the unknowns, by the oracle."""
    p = orc.Problem(dim=sp.dim, n=sp.n, periodic_y=sp.periodic_y, kind=sp.kind, h=sp.h, c=sp.c, sx=sp.sx, sy=sp.sy,
                    sz=sp.sz)
    o = orc.Oracle(p, levels=1, smoother="rbgs", dense_max=0)
    return o.norm(o.defect(u, b))


def _zero_boundary(a, sp):
    a = a.copy()
    if sp.dim == 2:
        a[:, 0] = a[:, -1] = 0.0
        if not sp.periodic_y:
            a[0, :] = a[-1, :] = 0.0
    else:
        a[:, :, 0] = a[:, :, -1] = 0.0
        a[0] = a[-1] = 0.0
        if not sp.periodic_y:
            a[:, 0, :] = a[:, -1, :] = 0.0
    return a


def test_noalloc_norm_matches_workspace_norm_on_consecutive_calls():
    lib = binding.load()
    cases, rng = _cases()
    stream = torch.cuda.current_stream()
    for sp, L, sm in cases:
        s = Solver(sp, levels=L, smoother=sm)
        p, k, keep = _abi_args(sp, stream)
        b = torch.tensor(sp.b, device="cuda")
        for call in range(2):   # two calls in a row, the second on a different iterate
            u = torch.tensor(_zero_boundary(rng.standard_normal(sp.shape) * 1e-3, sp), device="cuda")
            ref = float(s.residual_norm(u, b).item())
            want = _oracle_norm(sp, u.cpu().numpy(), sp.b)
            out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            assert _noalloc(lib, p, k, u, b, out) == binding.OK
            stream.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= TOL * ref, (sp.name, call, got, ref)
            assert abs(got - want) <= TOL * want, (sp.name, call, got, want)
        del keep


def test_noalloc_norm_on_a_tall_narrow_grid():
    """2.5 M rows of one unknown: the blocks' row count is raised until gridDim.y stays within
    its limit of 65535 and the partial sums within the array."""
    lib = binding.load()
    n1 = 2_500_002
    rng = np.random.default_rng(64)
    sp = inputs.ProblemSpec(name="tall", dim=2, n=(3, n1, 1), periodic_y=False, kind=inputs.CONST,
                            h=(0.5, 1.0 / (n1 - 1), 1.0), c=(4.0, float(n1 - 1) ** 2, 0.0),
                            b=rng.uniform(-1, 1, (n1, 3)))
    stream = torch.cuda.current_stream()
    p, k, keep = _abi_args(sp, stream)
    b = torch.tensor(sp.b, device="cuda")
    for call in range(2):
        un = _zero_boundary(rng.standard_normal(sp.b.shape) * 1e-6, sp)
        u = torch.tensor(un, device="cuda")
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, p, k, u, b, out) == binding.OK
        stream.synchronize()
        want = _oracle_norm(sp, un, sp.b)
        assert abs(float(out.item()) - want) <= TOL * want, (call, float(out.item()), want)


def test_noalloc_rejects_unsupported_input():
    lib = binding.load()
    sp = inputs.diffusion_cells(n=65)
    stream = torch.cuda.current_stream()
    p, k, keep = _abi_args(sp, stream)
    u = torch.zeros(sp.shape, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, p, k, u, u, out) == binding.EINVAL          # cell coefficients
    sp2 = inputs.anisotropic(n=65, eps=1.0)
    p2, k2, keep2 = _abi_args(sp2, stream)
    p2.n = (C.c_int * 3)(70000, 70000, 1)                              # beyond the node limit
    assert _noalloc(lib, p2, k2, u, u, out) == binding.EINVAL
    assert lib.mg_residual_norm_noalloc(None, C.byref(k2), None, None, None) == binding.EINVAL
    # rows wider than 32 x 65536 unknowns need more partial sums than the array holds: rejected
    # before any launch (the arrays passed are large enough for these grids all the same)
    big = torch.zeros(3_000_000 * 3, dtype=torch.float64, device="cuda")
    p3, k3, keep3 = _abi_args(sp2, stream)
    for n0 in (3_000_000, 32 * 65536 + 3):
        p3.n = (C.c_int * 3)(n0, 3, 1)
        assert _noalloc(lib, p3, k3, big, big, out) == binding.EINVAL
    stream.synchronize()
    assert float(out.item()) == 0.0
