"""GPU parity of the paper's two FV workloads against the oracle: linear
transport with the upwind flux (Sec. 3.1.2) over the level sweep and the
three threshold rules, and shallow water with the Godunov flux (Sec. 3.2.4).
Records byte for byte, decoded fields and times bit for bit, at every level
and rule; the uncompressed baselines bit for bit against the oracle's
reference runs."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Dense, Sim, inputs

pytestmark = pytest.mark.gpu

TR = dict(periodic=(False, False), cfl=0.45, velocity=(0.9, 0.9), length=2.0)


def pair(scheme, n, P, L, eps, prec, store, rule, fields, steps_at, **kw):
    g = Sim(scheme, "bl53", n, n, P, L, eps, prec=prec, store=store, rule=rule, **kw)
    o = O.OracleSim(scheme, "bl53", n, n, P, L, eps, prec=prec, store=store, rule=rule, **kw)
    g.init_macro(fields)
    o.init_macro(fields)
    done = 0
    for s in [0] + list(steps_at):
        g.step(s - done)
        o.step(s - done)
        done = s
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p), "patch %d record differs after %d steps" % (p, s)
    return g, o


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("rule", ["const", "accum", "capped"])
def test_transport_levels_and_rules_bitwise(L, rule):
    # the paper's setup: 128^2 on [-1, 1]^2, 2 x 2 patches of 65 nodes,
    # velocity (0.9, 0.9), CFL 0.45, to t = 0.5 (64 steps)
    f = inputs.transport_gaussian(128)
    g, o = pair("transport", 128, 64, L, 0.01, "f32", "f32", rule, f, (1, 17, 64), **TR)
    assert np.array_equal(g.export_field(-1), o.export_all())
    st = g.stats()
    assert st["time"] == o.stats()["time"] and abs(st["time"] - 0.5) < 1e-6


def test_transport_fp64_periodic_conserves_mass():
    rng = np.random.default_rng(4)
    f = [1.0 + 0.2 * rng.random((128, 128))]
    kw = dict(periodic=(True, True), cfl=0.45, velocity=(0.9, -0.5), length=2.0)
    g, o = pair("transport", 128, 32, 3, 1e-3, "f64", "f64", "capped", f, (1, 40), **kw)
    assert np.array_equal(g.export_field(-1), o.export_all())
    assert abs(g.stats()["mass"] - f[0].sum()) <= 1e-12 * f[0].sum()


def test_swe_fp32_fixed_step_bitwise():
    # the cost-study geometry: 129^2 nodes on [0, 1]^2, outflow, the raised
    # square, dt = 10 s / 38245, 4 levels, c = 5e-4
    n = 128
    dth = (10.0 / 38245) * n
    kw = dict(periodic=(False, False), cfl=-dth, gravity=9.81, length=1.0)
    g, o = pair("swe", n, 64, 4, 5e-4, "f32", "f32", "capped", inputs.swe_square(n), (1, 30, 120), **kw)
    assert np.array_equal(g.export_field(-1), o.export_all())
    assert g.stats()["time"] == o.stats()["time"]


def test_swe_fp32_cfl_step_bitwise():
    n = 128
    kw = dict(periodic=(False, False), cfl=0.4, gravity=9.81, length=1.0)
    g, o = pair("swe", n, 64, 4, 1e-3, "f32", "f32", "const", inputs.swe_square(n), (1, 25), **kw)
    assert np.array_equal(g.export_field(-1), o.export_all())
    assert g.stats()["time"] == o.stats()["time"]


def test_swe_fp64_periodic_bitwise_and_conservative():
    n = 128
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    h = 1.0 + 0.4 * np.exp(-50 * ((X - 0.4) ** 2 + (Y - 0.6) ** 2))
    f = [h, 0.1 * np.sin(2 * np.pi * Y), np.zeros_like(h)]
    kw = dict(periodic=(True, True), cfl=0.4, gravity=9.81, length=1.0)
    g, o = pair("swe", n, 32, 3, 1e-4, "f64", "f64", "capped", f, (1, 20), **kw)
    assert np.array_equal(g.export_field(-1), o.export_all())
    assert abs(g.stats()["mass"] - h.sum()) <= 1e-12 * h.sum()


@pytest.mark.parametrize("scheme", ["transport", "swe"])
def test_dense_fv_baselines_match_oracle_reference(scheme):
    n = 128
    if scheme == "transport":
        f, kw, steps = inputs.transport_gaussian(n), TR, 64
    else:
        f, kw, steps = inputs.swe_square(n), dict(periodic=(False, False), cfl=0.4, gravity=9.81, length=1.0), 60
    d = Dense(scheme, n, n, **kw)
    r = O.OracleRef(scheme, "bl53", n, n, prec="f32", **kw)
    d.init_macro(f)
    r.init_macro(f)
    d.step(steps)
    r.step(steps)
    for q in range(d.F):
        assert np.array_equal(d.export_field(q), r.export_field(q))


@pytest.mark.parametrize("rule", ["const", "capped"])
def test_transport_cdf97_bitwise(rule):
    # the CDF 9/7 wavelet (Sec. 2.1.2's second-order alternative) in the
    # same fused step: records and fields bit for bit against the oracle
    f = inputs.transport_gaussian(128)
    g, o = pair_wv("transport", "cdf97", 128, 64, 4, 0.01, rule, f, (1, 20, 64), **TR)
    assert np.array_equal(g.export_field(-1), o.export_all())


def pair_wv(scheme, wv, n, P, L, eps, rule, fields, steps_at, **kw):
    g = Sim(scheme, wv, n, n, P, L, eps, prec="f32", store="f32", rule=rule, **kw)
    o = O.OracleSim(scheme, wv, n, n, P, L, eps, prec="f32", store="f32", rule=rule, **kw)
    g.init_macro(fields)
    o.init_macro(fields)
    done = 0
    for s in [0] + list(steps_at):
        g.step(s - done)
        o.step(s - done)
        done = s
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p), "patch %d record differs after %d steps" % (p, s)
    return g, o


@pytest.mark.parametrize("scheme", ["euler2d", "transport"])
def test_ring_free_ghosts_one_patch_along_an_axis(scheme):
    # ring-free FV ghosts when the neighbour across a periodic border is the
    # patch itself (one patch along x) and the other axis has outflow
    # borders: records byte for byte and fields bit for bit (FP64)
    nx, ny, P = 32, 96, 32
    x = np.arange(nx + 0) / nx
    y = np.arange(ny + 1) / ny
    X, Y = np.meshgrid(x, y)
    if scheme == "euler2d":
        f = [1.0 + 0.3 * np.exp(-40 * ((X - 0.5) ** 2 + (Y - 0.3) ** 2)), 0.2 * np.sin(2 * np.pi * X),
             0.1 * np.cos(2 * np.pi * X) * Y, 1.0 + 0.2 * np.exp(-30 * ((X - 0.4) ** 2 + (Y - 0.6) ** 2))]
        kw = dict(periodic=(True, False), cfl=0.4, gamma=1.4)
    else:
        f = [1.0 + np.exp(-30 * ((X - 0.5) ** 2 + (Y - 0.4) ** 2))]
        kw = dict(periodic=(True, False), cfl=0.45, velocity=(0.7, -0.4), length=1.0)
    g = Sim(scheme, "bl53", nx, ny, P, 3, 1e-4, prec="f64", store="f64", rule="capped", **kw)
    o = O.OracleSim(scheme, "bl53", nx, ny, P, 3, 1e-4, prec="f64", store="f64", rule="capped", **kw)
    g.init_macro(f)
    o.init_macro(f)
    for chunk in (1, 15):
        g.step(chunk)
        o.step(chunk)
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p)
    assert np.array_equal(g.export_field(-1), o.export_all())
