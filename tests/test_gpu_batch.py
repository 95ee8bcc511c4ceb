"""Batched stepping (many independent simulations per launch, CUDA graph of
six steps) and the patch-size autotuner, against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Batch, Sim, autotune, inputs

pytestmark = pytest.mark.gpu


def _pair(n, P, L, prec, store, wavelet, fields, tau):
    g = Sim("d2q9", wavelet, n, n, P, L, 1e-4, prec=prec, store=store, tau=tau, arena_factor=0.5)
    o = O.OracleSim("d2q9", wavelet, n, n, P, L, 1e-4, prec=prec, store=store, tau=tau)
    g.init_macro(fields)
    o.init_macro(fields)
    return g, o


def test_batch_of_mixed_grids_matches_the_oracle():
    # three kernel kinds (BF16 P=64, BF16 P=32, FP64 Haar) and four grid sizes
    specs = [(128, 64, 4, "f32", "bf16", "bl53"), (256, 32, 3, "f32", "bf16", "bl53"),
             (64, 64, 4, "f32", "bf16", "bl53"), (128, 32, 3, "f64", "f64", "haar")]
    pairs = []
    for k, (n, P, L, prec, store, wv) in enumerate(specs):
        f = inputs.gaussian_bump(n, amp=0.05 + 0.01 * k, sigma=4.0 + 3 * k, center=(0.3 * n, 0.6 * n))
        pairs.append(_pair(n, P, L, prec, store, wv, f, tau=0.7))
    b = Batch([g for g, _ in pairs])
    for chunk in (3, 14):  # single launches to the 6-step boundary, graph replays, remainder
        b.step(chunk)
        for g, o in pairs:
            o.step(chunk)
        b.sync()
        for g, o in pairs:
            for p in range(g.npatch):
                assert g.record(p) == o.record(p)
    for g, o in pairs:
        assert np.array_equal(g.export_field(-1), o.export_all())
    b.close()


def test_batch_rejects_out_of_band_steps():
    from paper_2302_09883_gb300._lib import WcsError
    f = inputs.gaussian_bump(128)
    a = Sim("d2q9", "bl53", 128, 128, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.7)
    c = Sim("d2q9", "bl53", 128, 128, 32, 3, 1e-4, prec="f32", store="bf16", tau=0.7)
    a.init_macro(f)
    c.init_macro(f)
    b = Batch([a, c])
    a.step(1)
    with pytest.raises(WcsError):
        b.step(1)
    b.close()


def test_autotune_picks_a_runnable_candidate_and_caches_it():
    f = inputs.shear_wave(512, seed=7)
    best, ms = autotune("d2q9", "bl53", 512, 512, 1e-4, f, candidates=((64, 4), (32, 3), (16, 2)), tau=0.6)
    assert best in (0, 1)
    assert ms[0] > 0 and ms[1] > 0 and ms[2] < 0  # P=16 has no compiled kernel
    assert ms[best] == min(m for m in ms if m > 0)
    best2, ms2 = autotune("d2q9", "bl53", 512, 512, 1e-4, f, candidates=((64, 4), (32, 3), (16, 2)), tau=0.6)
    assert best2 == best and ms2 == ms


def test_merged_batch_is_one_launch_per_step_and_matches_the_oracle():
    # the two patch sizes of the autotuner (64/4 and 32/3, BF16) in one
    # persistent launch per step, larger patches first
    specs = [(256, 64, 4), (128, 32, 3), (192, 64, 4), (96, 32, 3), (64, 32, 3)]
    pairs = []
    for k, (n, P, L) in enumerate(specs):
        f = inputs.gaussian_bump(n, amp=0.03 + 0.02 * k, sigma=3.0 + 2 * k, center=(0.4 * n, 0.55 * n))
        pairs.append(_pair(n, P, L, "f32", "bf16", "bl53", f, tau=0.65))
    b = Batch([g for g, _ in pairs])
    launches, grid = b.launches_per_step()
    assert launches == 1 and grid > 0
    for chunk in (2, 13):
        b.step(chunk)
        for g, o in pairs:
            o.step(chunk)
        b.sync()
        for g, o in pairs:
            for p in range(g.npatch):
                assert g.record(p) == o.record(p)
    # the launch-shape tuner (persistent grid against one block per item)
    # keeps the records exact
    nitems = sum(g.npatch for g, _ in pairs)
    ms = b.tune_launch([grid, nitems], steps=6)
    assert len(ms) == 2 and min(ms) > 0
    for g, o in pairs:
        o.step(12)
    b.sync()
    for g, o in pairs:
        assert np.array_equal(g.export_field(-1), o.export_all())
    b.close()


def test_batch_catches_up_after_an_arena_overflow():
    # automatic arenas, a narrow bump and a tiny eps: the records grow many
    # times over as the acoustic waves spread, so a simulation outgrows the
    # room the batch gave it, freezes, and wcs_batch_sync re-runs its lost
    # steps alone; the records stay those of the oracle, and the batch keeps
    # stepping with the new arenas
    specs = [(256, 64, 4), (128, 32, 3)]
    pairs = []
    for n, P, L in specs:
        f = inputs.gaussian_bump(n, amp=0.05, sigma=2.0, center=(0.5 * n, 0.5 * n))
        g = Sim("d2q9", "bl53", n, n, P, L, 1e-9, prec="f32", store="bf16", tau=0.6)
        o = O.OracleSim("d2q9", "bl53", n, n, P, L, 1e-9, prec="f32", store="bf16", tau=0.6)
        g.init_macro(f)
        o.init_macro(f)
        pairs.append((g, o))
    b = Batch([g for g, _ in pairs])
    for chunk in (60, 12):
        b.step(chunk)
        b.sync()
        for g, o in pairs:
            o.step(chunk)
            for p in range(g.npatch):
                assert g.record(p) == o.record(p)
    assert sum(g.stats()["arena_reruns"] for g, _ in pairs) > 0
    b.close()
