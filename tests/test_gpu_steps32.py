"""Single-precision kernels against the FP64 oracle, element by element.

The mixed form runs its F-cycles in FP32: the TMA-fed red-black sweep in its three
modes (plain; iterate starting at zero; coarse correction folded in), the streamed
defect + full weighting, and on grids up to 1025^2 the tile kernels that run two
sweeps, or two sweeps with the defect and restriction, in one pass.  Here each runs
as one step of an MG_MIXED context (inputs rounded to FP32, outputs widened) and is
compared with the oracle's FP64 step on the same inputs:

- mg_step_smooth: S^s(u, g) against the oracle's sweeps;
- mg_step_descend: the pre-smoothing sweeps from u (mode 0) or from zero (mode 1),
  then R(g - A u): against the oracle's sweeps, defect and restriction;
- mg_step_ascend: u + P ec then the post-smoothing sweeps (mode 2 folds the
  correction into the first): against the oracle's prolongation and sweeps;
- mg_step_defect / restrict / prolong: the plain FP32 kernels.

The bar.  A step rounds its FP64 inputs to FP32 (relative 2^-24 each) and runs a
few FP32 operations per node: a sweep sums 5 products and 4 terms, whose rounding
errors are each at most 2^-24 of the running magnitude, which the inputs bound.
Two sweeps, then a defect and a 9-point restriction, chain under 40 such roundings,
so the error is below 40 * 2^-24 = 2.4e-6 of the output's scale.  The inputs are
random and independent (u ~ N(0,1), g = A v with v ~ N(0,1)), so no output is a
small difference of large terms and the array max is that scale: FP32_BAR = 2.4e-6
of the array max.  The measured errors are printed.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_0805_3041_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0805_3041_gb300.binding import Solver  # noqa: E402
from test_gpu_parity import rel, spec_of, oracle_of  # noqa: E402

FP32_BAR = 40 * 2.0 ** -24


def _aniso4097():
    return inputs.anisotropic(n=4097, eps=1.0, seed_f=1)


def _ragged(kind, periodic):
    rng = np.random.default_rng(71 + kind + 2 * periodic)
    return spec_of(2, (1543, 1100 if periodic else 1101), periodic, kind, rng, eps=0.3)


# name, spec builder, levels, levels whose steps are checked
CASES = [
    # the benchmark's workload: TMA sweeps on 4097^2 and 2049^2, tile kernels on 1025^2
    ("aniso4097", _aniso4097, 12, (12, 11, 10)),
    # ragged rows (1541 unknowns, 13 strips of 128 columns) and ragged bands
    ("ragged-const", lambda: _ragged(inputs.CONST, False), 2, (2,)),
    ("ragged-sep", lambda: _ragged(inputs.SEPARABLE, False), 2, (2,)),
    ("ragged-sep-periodic", lambda: _ragged(inputs.SEPARABLE, True), 2, (2,)),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: c[0])
def pair(request):
    name, make, L, check = request.param
    sp = make()
    o = oracle_of(sp, L, "rbgs", 1.0)
    s = Solver(sp, levels=L, smoother="rbgs", omega=1.0, nu1=2, nu2=2, precision="mixed", max_cycles=4)
    return name, sp, o, s, check, np.random.default_rng(hash(name) % 2 ** 32)


def _inputs(o, l, rng):
    m = o.unknown_mask(l)
    u = rng.standard_normal(o.shape(l)) * m
    g = o.apply(rng.standard_normal(o.shape(l)) * m, l)
    return u, g


def _check(what, got, want):
    e = rel(got, want)
    print(f"  {what}: {e:.2e} ({e / 2.0 ** -24:.1f} u32)")
    assert e <= FP32_BAR, (what, e)


def test_fp32_sweeps(pair):
    name, sp, o, s, check, rng = pair
    for l in check:
        u, g = _inputs(o, l, rng)
        for sweeps, order in ((1, 0), (2, 1)):
            _check(f"{name} l={l} smooth s={sweeps} o={order}", s.smooth(u, g, sweeps, order, l),
                   o.smooth(u, g, sweeps, order, l))


def test_fp32_descend(pair):
    name, sp, o, s, check, rng = pair
    for l in check:
        u, g = _inputs(o, l, rng)
        for start, tr in (("u", False), ("zero", False), ("u", True)):
            u0 = u if start == "u" else None
            uo, gc = s.descend(u0, g, l, transposed=tr)
            ref = o.smooth(u if start == "u" else o.zeros(l), g, 2, 1 if tr else 0, l)
            _check(f"{name} l={l} descend from {start} tr={tr}: sweeps", uo, ref)
            _check(f"{name} l={l} descend from {start} tr={tr}: R(g - Au)", gc, o.restrict(o.defect(ref, g, l), l))


def test_fp32_ascend(pair):
    name, sp, o, s, check, rng = pair
    for l in check:
        u, g = _inputs(o, l, rng)
        ec = rng.standard_normal(o.shape(l - 1)) * o.unknown_mask(l - 1)
        for tr in (False, True):
            got = s.ascend(ec, u, g, l, transposed=tr)
            ref = o.smooth(o.prolong_add(ec, u, 1.0, l), g, 2, 1 if tr else 0, l)
            _check(f"{name} l={l} ascend tr={tr}", got, ref)


def test_fp32_defect_and_transfers(pair):
    name, sp, o, s, check, rng = pair
    for l in check:
        u, g = _inputs(o, l, rng)
        _check(f"{name} l={l} defect", s.defect(u, g, l), o.defect(u, g, l))
        r = rng.standard_normal(o.shape(l)) * o.unknown_mask(l)
        _check(f"{name} l={l} restrict", s.restrict(r, l), o.restrict(r, l))
        ec = rng.standard_normal(o.shape(l - 1)) * o.unknown_mask(l - 1)
        _check(f"{name} l={l} prolong", s.prolong_add(ec, u, 1.0, l), o.prolong_add(ec, u, 1.0, l))
