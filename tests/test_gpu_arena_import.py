"""GPU: state import (wcs_import_field), arenas sized from the measured live
bytes (arena_factor 0) with a step that overflowed re-run transparently, and
the resident-bytes account.  Every state is compared byte for byte with the
oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Sim, Sim3, inputs

pytestmark = pytest.mark.gpu


def same_records(g, o, what=""):
    g.sync()
    for p in range(g.npatch):
        assert g.record(p) == o.record(p), "patch %d record differs %s" % (p, what)


def test_import_all_fields_matches_oracle_then_steps():
    # A state produced by another run (5 steps from a shear wave), handed
    # over as FP32 planes: the import re-encodes it exactly as the oracle does.
    n, P, L, eps = 256, 64, 4, 1e-4
    src = Sim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)
    src.init_macro(inputs.shear_wave(n, seed=21))
    src.step(5)
    state = src.export_field(-1, dtype=np.float32)
    src.close()
    rng = np.random.default_rng(3)
    state = (state + rng.normal(scale=1e-4, size=state.shape)).astype(np.float32)
    g = Sim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)
    o = O.OracleSim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)
    g.import_field(-1, state)  # initialises a fresh simulation
    o.import_field(-1, state.astype(np.float64))
    same_records(g, o, "after the import")
    assert g.stats()["step"] == 0
    g.step(6)
    o.step(6)
    same_records(g, o, "6 steps after the import")
    assert np.array_equal(g.export_field(-1), o.export_all())


@pytest.mark.parametrize("scheme,store,periodic", [("d2q9", "bf16", (True, True)), ("euler2d", "i8", (False, False))])
def test_import_one_field_keeps_step_and_matches_oracle(scheme, store, periodic):
    n, P, L, eps = 256, 64, 4, 1e-4
    f = inputs.shear_wave(n, seed=22) if scheme == "d2q9" else inputs.four_quadrant(n)
    kw = dict(tau=0.6) if scheme == "d2q9" else dict(cfl=-0.15)
    g = Sim(scheme, "bl53", n, n, P, L, eps, prec="f32", store=store, periodic=periodic, **kw)
    o = O.OracleSim(scheme, "bl53", n, n, P, L, eps, prec="f32", store=store, periodic=periodic, **kw)
    g.init_macro(f)
    o.init_macro(f)
    g.step(4)
    o.step(4)
    q = 2
    v = g.export_field(q)
    v = v * (1.0 + 0.01 * np.sin(np.arange(v.size).reshape(v.shape) * 0.37))
    g.import_field(q, v)
    o.import_field(q, v)
    same_records(g, o, "after importing field %d" % q)
    st = g.stats()
    assert st["step"] == 4 and st["time"] == o.stats()["time"]
    g.step(5)
    o.step(5)
    same_records(g, o, "5 steps after the import")


def test_import_3d_roundtrip():
    # 3-D: importing the decoded state gives it back to within the FP32
    # transform round trip (eps 0 keeps every coefficient), mass included.
    n = 32
    g = np.arange(n) * (2 * np.pi / n)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    ux = 0.04 * np.sin(x) * np.cos(y) * np.cos(z)
    uy = -0.04 * np.cos(x) * np.sin(y) * np.cos(z)
    s = Sim3(n, n, n, 16, 3, 0.0, store="f32", tau=0.55)
    s.init_macro([np.ones_like(ux), ux, uy, np.zeros_like(ux)])
    s.step(3)
    a = s.export_field(-1, dtype=np.float32)
    m0 = s.stats()["mass"]
    s.import_field(-1, a)
    b = s.export_field(-1, dtype=np.float32)
    assert np.max(np.abs(b - a)) <= 1e-6 * np.max(np.abs(a))
    assert abs(s.stats()["mass"] - m0) <= 1e-6 * m0
    s.close()


def test_auto_arena_reruns_overflowed_steps_exactly():
    # A sharp bump at a small eps: the acoustic front carries details into
    # patches that had none, so the live bytes grow about fivefold in 300
    # steps, past the capacity fitted after the first encode.  The steps
    # that overflowed are re-run with larger arenas; the result is the
    # oracle's, byte for byte.
    n, P, L, eps = 512, 64, 4, 1e-7
    f = inputs.gaussian_bump(n, amp=0.1, sigma=2.0)
    g = Sim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)  # arena_factor 0: automatic
    o = O.OracleSim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)
    g.init_macro(f)
    o.init_macro(f)
    cap0 = g.stats()["arena_capacity"]
    live0 = g.stats()["live_bytes"]
    assert cap0 < 2 * live0 + 64 * 1024
    g.step(300)
    o.step(300)
    same_records(g, o, "after 300 steps")
    st = g.stats()
    assert st["step"] == 300
    assert st["arena_reruns"] > 0
    assert st["arena_capacity"] > cap0
    assert st["live_bytes"] <= st["arena_capacity"]
    assert np.array_equal(g.export_field(-1), o.export_all())


def test_auto_arena_resident_bytes_on_the_2048_workload():
    # 2048^2 shear wave, P 64, L 4, BF16, eps 1e-3: every byte the simulation
    # holds, not only its records, stays under a tenth of one uncompressed
    # FP32 state.
    n = 2048
    g = Sim("d2q9", "bl53", n, n, 64, 4, 1e-3, prec="f32", store="bf16", tau=0.6)
    g.init_macro(inputs.shear_wave(n, seed=0))
    g.step(20)
    st = g.stats()
    assert st["resident_bytes"] == g.resident_bytes()
    assert st["resident_bytes"] >= 2 * st["arena_capacity"]
    assert st["live_bytes"] <= st["arena_capacity"]
    assert 10 * st["resident_bytes"] <= st["uncompressed_bytes"]
    g.close()


def test_fixed_arena_overflow_still_reported():
    from paper_2302_09883_gb300._lib import WcsError
    n = 512
    f = inputs.gaussian_bump(n, amp=0.1, sigma=2.0)
    g = Sim("d2q9", "bl53", n, n, 64, 4, 1e-8, prec="f32", store="bf16", tau=0.6, arena_factor=0.02)
    g.init_macro(f)
    g.step(60)
    with pytest.raises(WcsError) as ei:
        g.sync()
    assert ei.value.status == 3
    assert g.stats()["arena_reruns"] == 0


def test_survivor_count_matches_oracle_records():
    n, P, L = 256, 64, 4
    f = inputs.shear_wave(n, seed=23)
    for eps in (1e-6, 1e-4):
        g = Sim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)
        o = O.OracleSim("d2q9", "bl53", n, n, P, L, eps, prec="f32", store="bf16", tau=0.6)
        g.init_macro(f)
        o.init_macro(f)
        g.step(3)
        o.step(3)
        want = 0
        for p in range(o.npatch):
            r = o.record(p)
            rows = np.frombuffer(r, np.uint32, 4 * 9, 16).reshape(9, 4)
            want += int(rows[:, 2].sum() + rows[:, 3].sum())
        assert g.survivors() == want
        g.close()


def test_async_stats_equal_the_synchronous_ones():
    # wcs_stats_enqueue / wcs_stats_collect give, for each step, exactly what
    # wcs_stats gives after that step (same sums in the same order)
    n = 256
    a = Sim("d2q9", "bl53", n, n, 64, 4, 1e-5, prec="f32", store="bf16", tau=0.6)
    b = Sim("d2q9", "bl53", n, n, 64, 4, 1e-5, prec="f32", store="bf16", tau=0.6)
    f = inputs.shear_wave(n, seed=3)
    a.init_macro(f)
    b.init_macro(f)
    got = []
    for k in range(6):
        a.step(1)
        a.stats_enqueue(k % 4)
        if k >= 3:
            got.append(a.stats_collect((k - 3) % 4))
    for k in range(3, 6):
        got.append(a.stats_collect(k % 4))
    for k in range(6):
        b.step(1)
        want = b.stats()
        g = got[k]
        assert g["step"] == want["step"] == k + 1
        assert np.array_equal(g["field_sum"], want["field_sum"]) and g["mass"] == want["mass"]
        assert g["live_bytes"] == want["live_bytes"] and g["status"] == 0
    from paper_2302_09883_gb300._lib import WcsError
    with pytest.raises(WcsError):
        a.stats_collect(0)  # nothing queued in that slot any more
