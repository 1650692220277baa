"""Seeded synthetic problem generators.

These build the inputs of the Poisson-type problems studied in Wallis (2008):
the isotropic and anisotropic operators -eps u_xx - u_yy of section
"Anisotropies", the annulus / cylinder mapped to the unit square of section
"Introduction / Motivation" (gravity potential, Delta Phi = -4 pi G rho, here
with 4 pi G = 1 and a Gaussian density blob), many uneven instances for batched
solves, and log-normal cell coefficient fields for the inverse problem
-div(k grad u) = f.

This module holds problem data only (mesh, right-hand side, edge weights of the
user's discretisation, random fields).  It contains none of the multigrid
method; both the CUDA solver and the CPU oracle take its output unchanged.

Every random draw uses ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

CONST, SEPARABLE, CELL, EDGE = 0, 1, 2, 3


@dataclasses.dataclass
class ProblemSpec:
    """One linear system A u = b on a structured grid.

    Node arrays have numpy shape (n1, n0) in 2D and (n2, n1, n0) in 3D, x fastest.
    ``kind`` selects the coefficient representation:
      CONST:     ``c`` = edge weight per direction (units 1/h^2),
      SEPARABLE: ``sx[i]`` weight of x-edge (i, i+1); ``sy[i]``, ``sz[i]`` weights of
                 the y- and z-edges at x-index i (mapped polar / cylindrical grids),
      CELL:      ``k`` one coefficient per cell, weights k_avg / h^2 formed by the solver,
      EDGE:      ``ex``, ``ey`` (, ``ez``) full node arrays: the weight of the edge from each node
                 to its +x, +y (, +z) neighbour (periodic y: the last row's edge wraps to row 0).
    """
    name: str
    dim: int
    n: tuple
    periodic_y: bool
    kind: int
    h: tuple = (1.0, 1.0, 1.0)
    c: tuple = (1.0, 1.0, 1.0)
    sx: Optional[np.ndarray] = None
    sy: Optional[np.ndarray] = None
    sz: Optional[np.ndarray] = None
    k: Optional[np.ndarray] = None
    ex: Optional[np.ndarray] = None
    ey: Optional[np.ndarray] = None
    ez: Optional[np.ndarray] = None
    b: Optional[np.ndarray] = None
    x0: Optional[np.ndarray] = None

    @property
    def shape(self):
        return (self.n[1], self.n[0]) if self.dim == 2 else (self.n[2], self.n[1], self.n[0])


def max_levels(n, periodic_y=False, dim=2):
    """Largest number of grids for node counts n (Dirichlet: 2^m + 1, periodic y: even)."""
    L = 1
    m = list(n)
    while True:
        ok = (m[0] - 1) % 2 == 0 and m[0] >= 5
        if periodic_y:
            ok = ok and m[1] % 2 == 0 and m[1] >= 4
        else:
            ok = ok and (m[1] - 1) % 2 == 0 and m[1] >= 5
        if dim == 3:
            ok = ok and (m[2] - 1) % 2 == 0 and m[2] >= 5
        if not ok:
            return L
        m[0] = (m[0] - 1) // 2 + 1
        m[1] = m[1] // 2 if periodic_y else (m[1] - 1) // 2 + 1
        if dim == 3:
            m[2] = (m[2] - 1) // 2 + 1
        L += 1


def _zero_boundary(a, dim, periodic_y):
    a = a.copy()
    if dim == 2:
        a[:, 0] = 0.0
        a[:, -1] = 0.0
        if not periodic_y:
            a[0, :] = 0.0
            a[-1, :] = 0.0
    else:
        a[:, :, 0] = 0.0
        a[:, :, -1] = 0.0
        a[0] = 0.0
        a[-1] = 0.0
        if not periodic_y:
            a[:, 0, :] = 0.0
            a[:, -1, :] = 0.0
    return a


def poisson_sin(n=129):
    """-Laplace u = 2 pi^2 sin(pi x) sin(pi y) on the unit square, zero Dirichlet data.

    Its discrete solution is a multiple of the right-hand side (an eigenvector of
    the 5-point operator)."""
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    f = 2.0 * math.pi ** 2 * np.outer(np.sin(math.pi * x), np.sin(math.pi * x))
    b = _zero_boundary(f, 2, False)
    return ProblemSpec(name=f"poisson_sin_{n}", dim=2, n=(n, n, 1), periodic_y=False, kind=CONST,
                       h=(h, h, 1.0), c=(1.0 / h ** 2, 1.0 / h ** 2, 0.0), b=b, x0=np.zeros_like(b))


def anisotropic(n=4097, eps=1.0, seed_f=1, seed_x=2, random_start=False, dtype=np.float64):
    """-eps u_xx - u_yy = f, f i.i.d. uniform[-1, 1]; start vector zero or uniform[-1, 1]."""
    h = 1.0 / (n - 1)
    rng = np.random.default_rng(seed_f)
    b = _zero_boundary(rng.uniform(-1.0, 1.0, size=(n, n)), 2, False).astype(dtype)
    if random_start:
        x0 = _zero_boundary(np.random.default_rng(seed_x).uniform(-1.0, 1.0, size=(n, n)), 2, False).astype(dtype)
    else:
        x0 = np.zeros((n, n), dtype=dtype)
    return ProblemSpec(name=f"aniso_{n}_eps{eps:g}", dim=2, n=(n, n, 1), periodic_y=False, kind=CONST,
                       h=(h, h, 1.0), c=(eps / h ** 2, 1.0 / h ** 2, 0.0), b=b, x0=x0)


def _blob(X, Y, Z=None, centre=(-0.55, 0.0, 0.5), width=0.1):
    d2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2
    if Z is not None:
        d2 = d2 + (Z - centre[2]) ** 2
    return np.exp(-d2 / (2.0 * width ** 2))


def annulus_2d(nr=2049, nt=2048, r0=0.1, r1=1.0, seed=3, noise=0.1):
    """Annulus r in [r0, r1], theta periodic, mapped to the unit square (x = radius, y = angle).

    The polar Poisson equation multiplied by r gives the symmetric form
    -d/dr(r du/dr) - (1/r) d^2u/dtheta^2 = r f, whose 5-point discretisation has
    edge weights r_{i+1/2}/h_r^2 (x-edges) and 1/(r_i h_t^2) (y-edges).
    f = Gaussian density blob centred at (r, theta) = (0.55, pi) plus uniform noise.
    """
    hr = (r1 - r0) / (nr - 1)
    ht = 2.0 * math.pi / nt
    r = r0 + hr * np.arange(nr)
    rh = r0 + hr * (np.arange(nr - 1) + 0.5)
    t = ht * np.arange(nt)
    R, T = np.meshgrid(r, t)                   # (nt, nr)
    f = _blob(R * np.cos(T), R * np.sin(T))
    f = f + noise * np.random.default_rng(seed).uniform(-1.0, 1.0, size=f.shape)
    b = _zero_boundary(R * f, 2, True)
    sx = rh / hr ** 2
    sy = 1.0 / (r * ht ** 2)
    return ProblemSpec(name=f"annulus_{nr}x{nt}", dim=2, n=(nr, nt, 1), periodic_y=True, kind=SEPARABLE,
                       h=(hr, ht, 1.0), sx=sx, sy=sy, sz=np.zeros(nr), b=b, x0=np.zeros_like(b))


def cylinder_3d(nr=257, nt=256, nz=257, r0=0.1, r1=1.0, seed=3, noise=0.1):
    """Cylinder shell (r, theta, z) in [r0, r1] x [0, 2 pi) x [0, 1], theta periodic.

    r-weighted form -d/dr(r du/dr) - (1/r) u_tt - r u_zz = r f; edge weights
    r_{i+1/2}/h_r^2, 1/(r_i h_t^2), r_i/h_z^2; blob centred at (r, theta, z) = (0.55, pi, 0.5)."""
    hr = (r1 - r0) / (nr - 1)
    ht = 2.0 * math.pi / nt
    hz = 1.0 / (nz - 1)
    r = r0 + hr * np.arange(nr)
    rh = r0 + hr * (np.arange(nr - 1) + 0.5)
    t = ht * np.arange(nt)
    z = hz * np.arange(nz)
    Z, T, R = np.meshgrid(z, t, r, indexing="ij")   # (nz, nt, nr)
    f = _blob(R * np.cos(T), R * np.sin(T), Z)
    f = f + noise * np.random.default_rng(seed).uniform(-1.0, 1.0, size=f.shape)
    b = _zero_boundary(R * f, 3, True)
    return ProblemSpec(name=f"cylinder_{nr}x{nt}x{nz}", dim=3, n=(nr, nt, nz), periodic_y=True,
                       kind=SEPARABLE, h=(hr, ht, hz), sx=rh / hr ** 2, sy=1.0 / (r * ht ** 2),
                       sz=r / hz ** 2, b=b, x0=np.zeros_like(b))


def stretched_x(n=129, ny=None, beta=3.0, dim=2, manufactured=False, seed=12):
    """-Laplace u = f on the unit square (cube) on a grid stretched in x (section "Anisotropies":
    refinement in one direction), y (and z) uniform.

    Nodes x_i = (exp(beta s_i) - 1) / (exp(beta) - 1), s_i = i / (n - 1): spacings grow
    geometrically away from x = 0 (ratio exp(beta h0) between neighbours, exp(beta) end to end);
    the even nodes form the same family on the coarser grid.  Finite-volume form on the dual
    cells, divided by the nominal h0 = 1 / (n - 1) times hy (hy hz in 3-D) so that a uniform grid
    gives the usual 1/h^2 weights:

        x-edge (i, i+1): 1 / (hx_{i+1/2} h0),  y-edge at x_i: hbar_i / (h0 hy^2),
        z-edge at x_i: hbar_i / (h0 hz^2),     right-hand side: f_i hbar_i / h0,

    hbar_i = (hx_{i-1/2} + hx_{i+1/2}) / 2 the dual-cell width.  The weights depend on x only:
    a separable-coefficient problem.  manufactured=True takes f = d pi^2 prod sin(pi x_d) (exact
    solution prod sin(pi x_d)); otherwise f is uniform in [-1, 1].
    """
    ny = n if ny is None else ny
    nz = n if dim == 3 else 1
    s = np.arange(n) / (n - 1)
    x = np.expm1(beta * s) / np.expm1(beta) if beta != 0 else s
    hx = np.diff(x)
    hbar = np.empty(n)
    hbar[1:-1] = 0.5 * (hx[:-1] + hx[1:])
    hbar[0], hbar[-1] = 0.5 * hx[0], 0.5 * hx[-1]
    h0 = 1.0 / (n - 1)
    hy = 1.0 / (ny - 1)
    hz = 1.0 / (nz - 1) if dim == 3 else 1.0
    y = hy * np.arange(ny)
    if dim == 2:
        shape = (ny, n)
        if manufactured:
            f = 2 * math.pi ** 2 * np.outer(np.sin(math.pi * y), np.sin(math.pi * x))
        else:
            f = np.random.default_rng(seed).uniform(-1.0, 1.0, shape)
        scale = hbar[None, :] / h0
    else:
        z = hz * np.arange(nz)
        shape = (nz, ny, n)
        if manufactured:
            f = 3 * math.pi ** 2 * np.einsum("k,j,i->kji", np.sin(math.pi * z), np.sin(math.pi * y),
                                             np.sin(math.pi * x))
        else:
            f = np.random.default_rng(seed).uniform(-1.0, 1.0, shape)
        scale = hbar[None, None, :] / h0
    b = _zero_boundary(f * scale, dim, False)
    sp = ProblemSpec(name=f"stretched_x{n}_b{beta:g}", dim=dim, n=(n, ny, nz), periodic_y=False, kind=SEPARABLE,
                     h=(h0, hy, hz), sx=1.0 / (hx * h0), sy=hbar / (h0 * hy ** 2),
                     sz=(hbar / (h0 * hz ** 2)) if dim == 3 else np.zeros(n), b=b, x0=np.zeros_like(b))
    sp.x_nodes = x
    return sp


def _stretched_nodes(n, beta):
    """Nodes (e^{beta s} - 1) / (e^beta - 1), s = i / (n - 1), their spacings, and the dual-cell
    widths (half a spacing at the two ends)."""
    s = np.arange(n) / (n - 1)
    x = np.expm1(beta * s) / np.expm1(beta) if beta != 0 else s
    hx = np.diff(x)
    hbar = np.empty(n)
    hbar[1:-1] = 0.5 * (hx[:-1] + hx[1:])
    hbar[0], hbar[-1] = 0.5 * hx[0], 0.5 * hx[-1]
    return x, hx, hbar


def stretched_xy(n=129, ny=None, beta_x=3.0, beta_y=-3.0, manufactured=False, seed=13):
    """-Laplace u = f on the unit square on a grid refined in both directions (section
    "Anisotropies": combinations of one-direction refinements), nodes as in stretched_x per axis
    (beta < 0 clusters at the far end).  Finite-volume weights divided by the nominal cell area
    h0x h0y: x-edge (i, i+1) at row j: hbar_y(j) / (hx_{i+1/2} h0x h0y), y-edge (j, j+1) at
    column i: hbar_x(i) / (hy_{j+1/2} h0x h0y), right-hand side f hbar_x hbar_y / (h0x h0y).  The
    weights vary in both directions: an edge-weight (EDGE) problem."""
    ny = n if ny is None else ny
    x, hx, hbx = _stretched_nodes(n, beta_x)
    y, hy, hby = _stretched_nodes(ny, beta_y)
    h0x, h0y = 1.0 / (n - 1), 1.0 / (ny - 1)
    area = h0x * h0y
    ex = np.zeros((ny, n))
    ey = np.zeros((ny, n))
    ex[:, :-1] = hby[:, None] / (hx[None, :] * area)
    ey[:-1, :] = hbx[None, :] / (hy[:, None] * area)
    if manufactured:
        f = 2 * math.pi ** 2 * np.outer(np.sin(math.pi * y), np.sin(math.pi * x))
    else:
        f = np.random.default_rng(seed).uniform(-1.0, 1.0, (ny, n))
    b = _zero_boundary(f * np.outer(hby, hbx) / area, 2, False)
    sp = ProblemSpec(name=f"stretched_xy{n}x{ny}", dim=2, n=(n, ny, 1), periodic_y=False, kind=EDGE,
                     h=(h0x, h0y, 1.0), ex=ex, ey=ey, b=b, x0=np.zeros_like(b))
    sp.x_nodes, sp.y_nodes = x, y
    return sp


def spherical_shell(nr=129, nt=129, r0=0.5, r1=1.0, t0=math.pi / 8, t1=7 * math.pi / 8, manufactured=False,
                    seed=14):
    """Axisymmetric Poisson problem in spherical coordinates (r, theta) on the shell
    r0 <= r <= r1 between the cones theta = t0 and t1, mapped to the unit square (x = r,
    y = theta), zero Dirichlet data.  Multiplied by the volume factor r^2 sin(theta), the
    operator is -d/dr(r^2 sin(theta) du/dr) - d/dtheta(sin(theta) du/dtheta) = r^2 sin(theta) f,
    whose 5-point form has edge weights r_{i+1/2}^2 sin(theta_j) / h_r^2 (x-edges) and
    sin(theta_{j+1/2}) / h_t^2 (y-edges): they vary in both directions (EDGE).
    manufactured=True takes u = sin(pi (r - r0) / (r1 - r0)) sin(pi (theta - t0) / (t1 - t0))
    and f = -Laplace u in spherical coordinates; otherwise f is uniform in [-1, 1]."""
    hr, ht = (r1 - r0) / (nr - 1), (t1 - t0) / (nt - 1)
    r = r0 + hr * np.arange(nr)
    t = t0 + ht * np.arange(nt)
    rh = r0 + hr * (np.arange(nr - 1) + 0.5)
    th = t0 + ht * (np.arange(nt - 1) + 0.5)
    ex = np.zeros((nt, nr))
    ey = np.zeros((nt, nr))
    ex[:, :-1] = np.outer(np.sin(t), rh ** 2) / hr ** 2
    ey[:-1, :] = np.outer(np.sin(th), np.ones(nr)) / ht ** 2
    T, R = np.meshgrid(t, r, indexing="ij")
    if manufactured:
        a, c = math.pi / (r1 - r0), math.pi / (t1 - t0)
        Rf, Rd, Rdd = np.sin(a * (R - r0)), a * np.cos(a * (R - r0)), -a * a * np.sin(a * (R - r0))
        Tf, Td, Tdd = np.sin(c * (T - t0)), c * np.cos(c * (T - t0)), -c * c * np.sin(c * (T - t0))
        f = -(Tf * (Rdd + 2.0 * Rd / R) + Rf / R ** 2 * (Tdd + Td * np.cos(T) / np.sin(T)))
    else:
        f = np.random.default_rng(seed).uniform(-1.0, 1.0, (nt, nr))
    b = _zero_boundary(R ** 2 * np.sin(T) * f, 2, False)
    sp = ProblemSpec(name=f"spherical_{nr}x{nt}", dim=2, n=(nr, nt, 1), periodic_y=False, kind=EDGE,
                     h=(hr, ht, 1.0), ex=ex, ey=ey, b=b, x0=np.zeros_like(b))
    sp.r_nodes, sp.t_nodes = r, t
    return sp


def poisson_3d(n=33, seed=11):
    """-Laplace u = f on the unit cube, f uniform[-1, 1]."""
    h = 1.0 / (n - 1)
    b = _zero_boundary(np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, n, n)), 3, False)
    return ProblemSpec(name=f"poisson3d_{n}", dim=3, n=(n, n, n), periodic_y=False, kind=CONST,
                       h=(h, h, h), c=(1.0 / h ** 2,) * 3, b=b, x0=np.zeros_like(b))


def batched(count=256, sizes=(65, 129, 257, 513, 1025), eps_range=(1e-3, 1.0), seed=4):
    """Independent anisotropic instances of uneven size: N uniform over ``sizes``,
    eps log-uniform in ``eps_range``, f uniform[-1, 1]."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        n = int(rng.choice(sizes))
        eps = float(math.exp(rng.uniform(math.log(eps_range[0]), math.log(eps_range[1]))))
        h = 1.0 / (n - 1)
        b = _zero_boundary(rng.uniform(-1.0, 1.0, size=(n, n)), 2, False)
        out.append(ProblemSpec(name=f"batch{q}_{n}_eps{eps:.3g}", dim=2, n=(n, n, 1), periodic_y=False,
                               kind=CONST, h=(h, h, 1.0), c=(eps / h ** 2, 1.0 / h ** 2, 0.0), b=b,
                               x0=np.zeros_like(b)))
    return out


def lognormal_cells(ncells=1024, corr=16.0, seed=5):
    """k = exp(g) per cell, g = N(0,1) noise smoothed by a periodic Gaussian filter of
    standard deviation ``corr`` cells and renormalised to zero mean, unit variance."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((ncells, ncells))
    fy = np.fft.fftfreq(ncells)[:, None]
    fx = np.fft.fftfreq(ncells)[None, :]
    filt = np.exp(-2.0 * math.pi ** 2 * corr ** 2 * (fx ** 2 + fy ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(g) * filt))
    g = (g - g.mean()) / g.std()
    return np.exp(g)


def diffusion_cells(n=1025, seed_k=5, corr=16.0):
    """-div(k grad u) = f on the unit square with a log-normal cell field k and a
    Gaussian blob source centred at (0.55, 0.5)."""
    h = 1.0 / (n - 1)
    k = lognormal_cells(n - 1, corr=corr, seed=seed_k)
    x = np.arange(n) * h
    X, Y = np.meshgrid(x, x)
    f = _blob(X, Y, centre=(0.55, 0.5, 0.0))
    b = _zero_boundary(f, 2, False)
    return ProblemSpec(name=f"diffusion_{n}", dim=2, n=(n, n, 1), periodic_y=False, kind=CELL,
                       h=(h, h, 1.0), k=k, b=b, x0=np.zeros_like(b))


def observation_noise(shape, seed=7):
    """Standard normal noise used to perturb the synthetic observation u_obs."""
    return np.random.default_rng(seed).standard_normal(shape)
