"""GPU parity of hi + lo coarse storage (Sec. 2.1.2, eq. conservation).

With the option on, every encode of an FP32 BL5/3 patch also forms its
coarse block in FP64 from the same FP32 nodes and keeps lo = fl32(c64 - hi)
beside each FP32 coarse sample hi of the record.  Checked here through the
C-ABI against the oracle (whose FP64 coarse path is pinned by Check A and by
exact cases in test_oracle_hilo.py):

- the records are byte-identical with and without the option (the FP32
  path is untouched) and byte-identical to the oracle's;
- the lo parts equal the oracle's bit for bit;
- Check A: the FP64 coarse-domain mass after each encode (field_sum +
  field_sum_lo) equals the FP64 mass of the nodes before it (the oracle's
  node sums, or an exactly rounded sum of imported values) to 1e-12
  relative, where the FP32 samples alone miss it by FP32 rounding.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Sim, inputs

pytestmark = pytest.mark.gpu

N = 256
CASES = [
    ("d2q9_bf16_p64", "d2q9", 64, 4, dict(store="bf16", tau=0.6), lambda: inputs.shear_wave(N, seed=1)),
    ("d2q9_bf16_p32", "d2q9", 32, 3, dict(store="bf16", tau=0.6), lambda: inputs.shear_wave(N, seed=2)),
    ("euler_i8", "euler2d", 64, 4, dict(store="i8", periodic=(False, False), cfl=0.4),
     lambda: inputs.four_quadrant(N)),
    ("transport_l3", "transport", 64, 3,
     dict(store="f32", periodic=(False, False), cfl=0.45, velocity=(0.9, 0.9), length=2.0),
     lambda: inputs.transport_gaussian(N)),
    ("swe_p64", "swe", 64, 4, dict(store="f32", periodic=(False, False), cfl=0.4), lambda: inputs.swe_square(N)),
]


def check_a_rel(g_stats, pre, scale):
    return np.abs(g_stats["field_sum"] + g_stats["field_sum_lo"] - pre) / scale


@pytest.mark.parametrize("name,scheme,P,L,kw,init", CASES, ids=[c[0] for c in CASES])
def test_hilo_bitwise_and_check_a(name, scheme, P, L, kw, init):
    eps = 1e-4
    g = Sim(scheme, "bl53", N, N, P, L, eps, prec="f32", coarse_hilo=True, **kw)
    o = O.OracleSim(scheme, "bl53", N, N, P, L, eps, prec="f32", hilo=True, **kw)
    ref = Sim(scheme, "bl53", N, N, P, L, eps, prec="f32", **kw)  # the option off
    f = init()
    for s in (g, o, ref):
        s.init_macro(f)
    worst_hi = 0.0
    for k in range(4):
        if k:
            for s in (g, o, ref):
                s.step(1)
        g.sync()
        ref.sync()
        for p in range(g.npatch):
            rg = g.record(p)
            assert rg == o.record(p), "patch %d record differs from the oracle after %d steps" % (p, k)
            assert rg == ref.record(p), "patch %d record changed by the option after %d steps" % (p, k)
        lo_g, lo_o = g.coarse_lo(), o.coarse_lo()
        assert np.array_equal(lo_g.view(np.uint32), lo_o.view(np.uint32)), "lo parts differ after %d steps" % k
        st, ost, h = g.stats(), o.stats(), o.hilo_sums()
        scale = ost["coef_abs_sums"] + h["lo_abs_sums"]
        scale = np.where(scale > 0, scale, 1.0)
        # the lo sums: the same terms in another order
        assert np.all(np.abs(st["field_sum_lo"] - h["lo_sums"]) <= 1e-15 * scale)
        rel = check_a_rel(st, h["pre_sums"], scale)
        assert np.all(rel <= 1e-12), (k, rel)
        worst_hi = max(worst_hi, float(np.max(np.abs(st["field_sum"] - h["pre_sums"]) / scale)))
    assert worst_hi > 1e-12  # the FP32 samples alone do not conserve to 1e-12
    # the lo parts are compressed bytes; the option costs F x NC floats a patch
    nc = ((P >> L) + 1) ** 2
    assert g.compressed_bytes() - ref.compressed_bytes() == g.npatch * g.F * nc * 4


def test_hilo_check_a_full_size_import():
    """2048^2 D2Q9, P 64, L 4, BF16 details (the headline workload's
    configuration): one encode of imported FP32 populations; Check A
    against an exactly rounded sum of the imported values, no oracle."""
    n = 2048
    rng = np.random.default_rng(3)
    g = Sim("d2q9", "bl53", n, n, 64, 4, 1e-3, prec="f32", store="bf16", tau=0.6, coarse_hilo=True)
    v = (1.0 / 9.0 + 1e-3 * rng.standard_normal((9, n, n))).astype(np.float32)
    g.import_field(-1, v)
    st = g.stats()
    for f in range(9):
        want = math.fsum(v[f].astype(np.float64).ravel())
        scale = math.fsum(np.abs(v[f].astype(np.float64)).ravel())
        assert abs(st["field_sum"][f] + st["field_sum_lo"][f] - want) <= 1e-12 * scale
        assert abs(st["field_sum"][f] - want) > 1e-12 * scale  # hi alone misses it
    lo = g.coarse_lo()
    assert np.isfinite(lo).all() and np.max(np.abs(lo)) < 2.0 ** -18


def test_hilo_needs_a_kernel_that_keeps_it():
    with pytest.raises(RuntimeError):  # FP64 compute keeps its coarse samples in FP64 already
        Sim("d2q9", "bl53", 128, 128, 32, 3, 1e-4, prec="f64", store="f64", coarse_hilo=True)
    with pytest.raises(RuntimeError):  # L = 1: 33 x 33 coarse samples do not fit the staging area
        Sim("transport", "bl53", 128, 128, 64, 1, 0.01, prec="f32", store="f32", velocity=(0.9, 0.9),
            coarse_hilo=True)
    g = Sim("d2q9", "bl53", 128, 128, 32, 3, 1e-4, prec="f32", store="bf16")
    g.init_macro(inputs.shear_wave(128))
    with pytest.raises(RuntimeError):  # the option is off
        g.coarse_lo()


def test_hilo_d3q19_bitwise_and_check_a():
    """D3Q19, 64^3, P 32, L 3, BF16 details: records unchanged by the option
    and equal to the oracle's, lo parts bit for bit, Check A at the initial
    encode and after each of two steps."""
    from paper_2302_09883_gb300 import Sim3
    n = 64
    g = Sim3(n, n, n, 32, 3, 1e-6, store="bf16", tau=0.55, coarse_hilo=True)
    ref = Sim3(n, n, n, 32, 3, 1e-6, store="bf16", tau=0.55)
    o = O.OracleSim3("bl53", n, n, n, 32, 3, 1e-6, prec="f32", store="bf16", tau=0.55, hilo=True)
    f = inputs.taylor_green_3d(n)
    for s in (g, ref, o):
        s.init_macro(f)
    worst_hi = 0.0
    for k in range(3):
        if k:
            for s in (g, ref, o):
                s.step(1)
        g.sync()
        ref.sync()
        for p in range(g.npatch):
            rg = g.record(p)
            assert rg == o.record(p) and rg == ref.record(p), (p, k)
        assert np.array_equal(g.coarse_lo().view(np.uint32), o.coarse_lo().view(np.uint32)), k
        st, ost, h = g.stats(), o.stats(), o.hilo_sums()
        scale = ost["coef_abs_sums"] + h["lo_abs_sums"]
        assert np.all(np.abs(st["field_sum_lo"] - h["lo_sums"]) <= 1e-15 * scale)
        assert np.all(np.abs(st["field_sum"] + st["field_sum_lo"] - h["pre_sums"]) <= 1e-12 * scale), k
        worst_hi = max(worst_hi, float(np.max(np.abs(st["field_sum"] - h["pre_sums"]) / scale)))
    assert worst_hi > 1e-12


def test_hilo_stats_paths_and_what_does_not_take_it():
    """The queued statistics carry the lo sums like wcs_stats; batches and the
    learned threshold have no hi + lo kernel and say so."""
    from paper_2302_09883_gb300 import Batch, learned
    n = 128
    g = Sim("d2q9", "bl53", n, n, 32, 3, 1e-4, prec="f32", store="bf16", tau=0.6, coarse_hilo=True)
    g.init_macro(inputs.shear_wave(n, seed=5))
    g.step(2)
    g.stats_enqueue(1)
    q = g.stats_collect(1)
    st = g.stats()
    assert np.array_equal(q["field_sum_lo"], st["field_sum_lo"]) and np.any(st["field_sum_lo"] != 0.0)
    assert np.array_equal(q["field_sum"], st["field_sum"])
    with pytest.raises(RuntimeError):
        Batch([g])
    with pytest.raises(RuntimeError):
        learned.use_mlp(g, learned.Mlp(18, seed=0))
