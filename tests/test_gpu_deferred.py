"""Patch size and levels left to the autotuner (patch = 0 and/or levels = 0
at creation): the choice is made in wcs_init_macro on the caller's fields,
among the compiled kernels of the configuration, and the simulation is then
the same as one created with that (P, L) directly: records byte for byte."""
import numpy as np
import pytest

from paper_2302_09883_gb300 import Sim, Sim3, inputs

pytestmark = pytest.mark.gpu


def test_d2q9_both_left_to_the_autotuner():
    n = 512
    f = inputs.shear_wave(n, seed=4)
    g = Sim("d2q9", "bl53", n, n, 0, 0, 1e-4, prec="f32", store="bf16", tau=0.6)
    assert g.patch_config() == (0, 0) and g.npatch == 0
    g.init_macro(f)
    P, L = g.patch_config()
    assert (P, L) in ((64, 4), (32, 3)) and g.npatch == (n // P) ** 2
    d = Sim("d2q9", "bl53", n, n, P, L, 1e-4, prec="f32", store="bf16", tau=0.6)
    d.init_macro(f)
    g.step(3)
    d.step(3)
    g.sync()
    d.sync()
    for p in range(g.npatch):
        assert g.record(p) == d.record(p), p
    assert np.array_equal(g.export_field(-1), d.export_field(-1))
    assert g.stats()["step"] == 3


def test_transport_levels_left_to_the_autotuner():
    n = 128
    kw = dict(periodic=(False, False), cfl=0.45, velocity=(0.9, 0.9), length=2.0)
    g = Sim("transport", "bl53", n, n, 64, 0, 0.01, prec="f32", store="f32", **kw)
    g.init_macro(inputs.transport_gaussian(n))
    P, L = g.patch_config()
    assert P == 64 and 1 <= L <= 5
    d = Sim("transport", "bl53", n, n, 64, L, 0.01, prec="f32", store="f32", **kw)
    d.init_macro(inputs.transport_gaussian(n))
    g.step(4)
    d.step(4)
    assert np.array_equal(g.export_field(-1), d.export_field(-1))


def test_d3q19_left_to_the_autotuner():
    n = 64
    g = Sim3(n, n, n, 0, 0, 1e-6, store="bf16", tau=0.55)
    g.init_macro(inputs.taylor_green_3d(n))
    P, L = g.patch_config()
    assert (P, L) in ((32, 3), (16, 3)) and g.npatch == (n // P) ** 3
    g.step(2)
    g.sync()
    assert g.stats()["step"] == 2


def test_deferred_simulation_starts_from_the_init():
    g = Sim("d2q9", "bl53", 256, 256, 0, 0, 1e-3, prec="f32", store="bf16", tau=0.6)
    with pytest.raises(RuntimeError):
        g.import_field(-1, np.full((9, 256, 256), 1.0 / 9.0))
    with pytest.raises(RuntimeError):
        g.step(1)
    g.init_macro(inputs.shear_wave(256))
    g.step(1)
    g.sync()
