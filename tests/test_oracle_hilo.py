"""Oracle pins of hi + lo coarse storage (Sec. 2.1.2, eq. conservation).

The coarse block of a BL5/3 patch carries the patch's trapezoid-weighted
mass; in FP32 the lifting rounds, so the FP32 samples (hi) keep it only to
about 1e-7 per patch.  With hi + lo the coarse block is also formed in FP64
from the same nodes and lo = fl32(c64 - hi) is kept beside hi.  Check A: the
FP64 coarse-domain mass after an encode (2^(2L) times the trapezoid sum of
hi + lo) equals the FP64 mass of the nodes before it to 1e-12 relative.

The pins below fix the oracle to what the mathematics says, not to itself:
the node sums before an encode are compared with an exactly rounded sum of
the imported values (math.fsum), the conservation identity is what the
transform must satisfy whatever its rounding, a field on which the FP32
lifting is exact must give lo = 0, and lo must be a rounding-sized
correction (a transposed or misplaced sample is not).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import inputs

N, P, L = 128, 32, 3


def check_a(s):
    """Per field: |hi + lo - pre| and the scale it is measured against."""
    st, h = s.stats(), s.hilo_sums()
    err = np.abs(st["coef_sums"] + h["lo_sums"] - h["pre_sums"])
    err_hi = np.abs(st["coef_sums"] - h["pre_sums"])
    scale = st["coef_abs_sums"] + h["lo_abs_sums"]
    return err, err_hi, scale


CASES = [
    ("d2q9", dict(store="bf16", tau=0.6), lambda: inputs.shear_wave(N, seed=0)),
    ("euler2d", dict(store="i8", periodic=(False, False), cfl=0.4), lambda: inputs.four_quadrant(N)),
    ("transport", dict(store="f32", periodic=(False, False), velocity=(0.9, 0.9), cfl=0.45, length=2.0),
     lambda: inputs.transport_gaussian(N)),
    ("swe", dict(store="f32", periodic=(False, False), cfl=0.4), lambda: inputs.swe_square(N)),
]


@pytest.mark.parametrize("scheme,kw,init", CASES, ids=[c[0] for c in CASES])
def test_check_a_every_encode(scheme, kw, init):
    """Check A after the initial encode and after each of three steps."""
    s = O.OracleSim(scheme, "bl53", N, N, P, L, 1e-4, prec="f32", hilo=True, **kw)
    s.init_macro(init())
    worst_hi = 0.0
    for k in range(4):
        err, err_hi, scale = check_a(s)
        assert np.all(err <= 1e-12 * scale), (k, err / scale)
        worst_hi = max(worst_hi, float(np.max(err_hi / np.where(scale > 0, scale, 1.0))))
        s.step(1)
    # the FP32 samples alone miss it by FP32 rounding: the check can fail
    assert worst_hi > 1e-12


def test_pre_sums_are_the_imported_mass():
    """The node sums before an encode, against an exactly rounded sum of the
    imported values (periodic grid: every unique node once)."""
    rng = np.random.default_rng(7)
    s = O.OracleSim("d2q9", "bl53", N, N, P, L, 1e-3, prec="f32", store="bf16", tau=0.6, hilo=True)
    v = (1.0 / 9.0 + 0.01 * rng.standard_normal((9, N, N))).astype(np.float32).astype(np.float64)
    s.import_field(-1, v)
    pre = s.hilo_sums()["pre_sums"]
    for f in range(9):
        want = math.fsum(v[f].ravel())
        assert abs(pre[f] - want) <= 1e-15 * math.fsum(np.abs(v[f]).ravel())
    err, _, scale = check_a(s)
    assert np.all(err <= 1e-12 * scale)


def test_lo_is_zero_where_fp32_lifting_is_exact():
    """Small integers: every FP32 lifting operation of three levels is exact
    (sums of a few integers, halved and quartered, fit in 24 bits), so
    hi = c64 and lo = 0 at every sample, in every patch; a lo taken at a
    misplaced sample would not vanish on these unsymmetric values."""
    rng = np.random.default_rng(11)
    s = O.OracleSim("transport", "bl53", N, N, P, L, 0.0, prec="f32", store="f32", velocity=(0.9, 0.9), hilo=True)
    s.import_field(-1, rng.integers(0, 16, size=(1, N, N)).astype(np.float64))
    assert np.all(s.coarse_lo() == 0.0)
    err, _, scale = check_a(s)
    assert np.all(err <= 1e-12 * scale)
    # a smooth non-polynomial field rounds, and lo takes the difference up
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    s.import_field(-1, (1.0 + 1e-3 * np.sin(0.37 * x) * np.cos(0.21 * y))[None])
    assert np.any(s.coarse_lo() != 0.0)


def test_lo_is_a_rounding_correction():
    """|lo| stays within a few FP32 roundings of the coarse samples' size, so
    a misplaced FP64 sample (a transposed block, a wrong level) shows; the
    trapezoid weights are symmetric in x and y, so Check A alone would not
    see a transposition."""
    s = O.OracleSim("d2q9", "bl53", N, N, P, L, 1e-4, prec="f32", store="bf16", tau=0.6, hilo=True)
    s.init_macro(inputs.shear_wave(N, seed=3))
    s.step(2)
    lo = s.coarse_lo()
    assert np.max(np.abs(lo)) <= 2.0 ** -19 * (4.0 / 9.0) * 1.2
    assert np.max(np.abs(lo)) > 0.0


def test_hilo_needs_fp32_bl53():
    with pytest.raises(RuntimeError):
        O.OracleSim("d2q9", "bl53", N, N, P, L, 1e-4, prec="f64", store="f64", hilo=True)
    with pytest.raises(RuntimeError):
        O.OracleSim("d2q9", "haar", N, N, P, L, 1e-4, prec="f32", store="f32", hilo=True)


def test_check_a_d3q19():
    """The same in three dimensions (2^(3L) times the trapezoid sum over the
    three axes): D3Q19, 64^3, P 32, L 3, BF16 details, the initial encode
    and two steps."""
    n = 64
    s = O.OracleSim3("bl53", n, n, n, 32, 3, 1e-6, prec="f32", store="bf16", tau=0.55, hilo=True)
    s.init_macro(inputs.taylor_green_3d(n))
    worst_hi = 0.0
    for k in range(3):
        st, h = s.stats(), s.hilo_sums()
        scale = st["coef_abs_sums"] + h["lo_abs_sums"]
        assert np.all(np.abs(st["coef_sums"] + h["lo_sums"] - h["pre_sums"]) <= 1e-12 * scale), k
        worst_hi = max(worst_hi, float(np.max(np.abs(st["coef_sums"] - h["pre_sums"]) / scale)))
        lo = s.coarse_lo()
        assert 0.0 < np.max(np.abs(lo)) <= 2.0 ** -19 * (1.0 / 3.0) * 1.2
        if k < 2:
            s.step(1)
    assert worst_hi > 1e-12
