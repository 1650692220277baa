"""Differentiation through the GPU F-cycle: adjoint solve + cell-coefficient gradient.

Checked against torch.autograd.gradcheck (central differences of the whole
solve), against the FP64 oracle's gradient, and against central finite
differences on sampled cells of the 1025^2 log-normal inverse problem.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.autograd import diffusion_solve  # noqa: E402


def _mask(n):
    m = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    m[1:-1, 1:-1] = 1.0
    return m


def test_gradcheck_small_grid():
    n, L = 17, 4
    rng = np.random.default_rng(40)
    k = torch.tensor(np.exp(0.5 * rng.standard_normal((n - 1, n - 1))), device="cuda", requires_grad=True)
    f = torch.tensor(rng.uniform(-1, 1, (n, n)), device="cuda") * _mask(n)
    f.requires_grad_(True)
    uobs = torch.tensor(0.01 * rng.standard_normal((n, n)), device="cuda")

    def loss(k, f):
        u = diffusion_solve(k, f, levels=L, tol=1e-14)
        return ((u - uobs) ** 2).sum()

    assert torch.autograd.gradcheck(loss, (k, f), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_gradient_matches_oracle():
    n, L = 65, 5
    rng = np.random.default_rng(41)
    kk = np.exp(0.7 * rng.standard_normal((n - 1, n - 1)))
    f = rng.uniform(-1, 1, (n, n))
    f[0, :] = f[-1, :] = f[:, 0] = f[:, -1] = 0.0
    uobs = 0.01 * rng.standard_normal((n, n))
    k = torch.tensor(kk, device="cuda", requires_grad=True)
    ft = torch.tensor(f, device="cuda", requires_grad=True)
    u = diffusion_solve(k, ft, levels=L, tol=1e-13)
    m = _mask(n)
    ((u - torch.tensor(uobs, device="cuda")) ** 2 * m).sum().backward()
    h = 1.0 / (n - 1)
    o = orc.Oracle(orc.Problem(dim=2, n=(n, n, 1), kind=orc.CELL, h=(h, h, 1), k=kk), levels=L)
    uo, *_ = o.solve(f, tol=1e-13, maxit=100)
    lam, *_ = o.solve(2 * (uo - uobs) * o.unknown_mask(), tol=1e-13, maxit=100, transposed=True)
    go = o.grad_k(uo, lam)
    gk = k.grad.cpu().numpy()
    assert np.abs(gk - go).max() <= 1e-9 * np.abs(go).max()
    assert np.abs(ft.grad.cpu().numpy() - lam).max() <= 1e-9 * np.abs(lam).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_finite_differences_lognormal_1025(precision):
    """Inverse problem of the differentiation study: 1025^2 nodes, k log-normal (correlation
    16 cells), u_obs = u(k_ref) + 1 % noise, L = ||u - u_obs||^2; dL/dk on 64 random cells
    against central differences with delta = 1e-3 k_c.  The solves stop at 1e-10: this
    smooth-solution problem reaches its FP64 rounding floor of the residual near 2e-11, so
    the step is large enough that the solve error (~1e-10 relative in L) stays far below the
    differenced signal, and small enough that the O(delta^2) truncation is ~1e-6."""
    n, L = 1025, 10
    tol = 1e-10
    sp = inputs.diffusion_cells(n=n, seed_k=5)
    kref = inputs.lognormal_cells(n - 1, corr=16.0, seed=6)
    f = torch.tensor(sp.b, device="cuda")
    with torch.no_grad():
        uref = diffusion_solve(torch.tensor(kref, device="cuda"), f, levels=L, tol=tol)
    noise = torch.tensor(inputs.observation_noise((n, n), seed=7), device="cuda")
    uobs = uref + 0.01 * uref.pow(2).mean().sqrt() * noise
    m = _mask(n)

    def loss(kt):
        u = diffusion_solve(kt, f, levels=L, tol=tol, precision=precision)
        return (((u - uobs) * m) ** 2).sum()

    k = torch.tensor(sp.k, device="cuda", requires_grad=True)
    loss(k).backward()
    g = k.grad.cpu().numpy()
    rng = np.random.default_rng(8)
    cells = [(int(rng.integers(0, n - 1)), int(rng.integers(0, n - 1))) for _ in range(64)]
    errs = []
    with torch.no_grad():
        for c in cells:
            d = 1e-3 * float(sp.k[c])
            kp = torch.tensor(sp.k, device="cuda")
            km = kp.clone()
            kp[c] += d
            km[c] -= d
            fd = (loss(kp).item() - loss(km).item()) / (2 * d)
            errs.append(abs(fd - g[c]))
    scale = np.abs(g).max()
    print(f"{precision}: max |FD - adjoint| / max |grad| over 64 cells = {max(errs) / scale:.2e}")
    assert max(errs) <= 1e-5 * scale


GRAD_CASES = [
    # dim, n, periodic, smoother (zebra_y on a non-periodic cell problem runs axis-swapped)
    (2, (129, 65), False, "rbgs"),
    (2, (129, 64), True, "rbgs"),
    (2, (65, 129), False, "zebra_y"),
    (3, (33, 17, 33), False, "rbgs"),
    (3, (17, 16, 17), True, "jacobi"),
]


@pytest.mark.parametrize("dim,n,per,sm", GRAD_CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_kernel_matches_oracle_on_the_same_fields(dim, n, per, sm, precision):
    """mg_grad_coeff and the oracle's gradient on the same u and lambda (no solve in between):
    dL/dk_c = -sum over the cell's edges of (dw_e/dk_c)(u_p - u_q)(lambda_p - lambda_q), within
    1e-12 of the array max.  The gradient is an FP64 kernel in both precisions."""
    from paper_0805_3041_gb300.binding import Solver
    from test_gpu_parity import spec_of, oracle_of
    rng = np.random.default_rng(sum(n) + 5 * per + dim)
    sp = spec_of(dim, n, per, inputs.CELL, rng)
    o = oracle_of(sp, 2, sm, 1.0)
    s = Solver(sp, levels=2, smoother=sm, omega=1.0, precision=precision, max_cycles=4)
    for trial in range(2):
        u = rng.standard_normal(o.shape()) * o.unknown_mask()
        lam = rng.standard_normal(o.shape()) * o.unknown_mask()
        got = s.grad_coeff(u, lam).cpu().numpy()
        want = o.grad_k(u, lam)
        assert got.shape == want.shape
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
