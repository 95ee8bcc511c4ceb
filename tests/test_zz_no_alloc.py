"""The export entry point that allocates no device memory.

wcs_export_field_noalloc serves callers that cannot call cudaMalloc when
they read a field back (device memory already taken by their simulations, or
a loop that must not pay for an allocation and its implicit device-wide
synchronisation).  It stages the decoded field in one fixed library-wide
device array instead of a temporary buffer.  These checks call it through
the C-ABI and compare it with wcs_export_field, which allocates its own
temporary buffer, on two calls in a row.  The file sorts last so that a run
stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2302_09883_gb300 import Sim, inputs
from paper_2302_09883_gb300 import _lib as B

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 << 20


def _noalloc(sim, field, dtype):
    shape = ((sim.F,) if field < 0 else ()) + (sim.G[1], sim.G[0])
    out = np.empty(shape, dtype=np.float64 if dtype == 0 else np.float32)
    st = B.lib().wcs_export_field_noalloc(sim.h, field, out.ctypes.data, dtype)
    return st, out


def test_noalloc_export_matches_export_field_on_two_calls():
    f = inputs.shear_wave(256, seed=5)
    sim = Sim("d2q9", "bl53", 256, 256, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    sim.init_macro(f)
    sim.step(4)
    for call in range(2):
        for field, dtype in [(3, 0), (-1, 1)]:
            want = sim.export_field(field, dtype=np.float64 if dtype == 0 else np.float32)
            st, got = _noalloc(sim, field, dtype)
            assert st == 0, B.lib().wcs_last_error(sim.h)
            # both paths run the same decode kernel: bit-identical output
            assert np.array_equal(got, want), "call %d field %d dtype %d" % (call, field, dtype)
        sim.step(3)
    sim.close()


def test_noalloc_export_rejects_requests_above_the_staging_size():
    n = 1024  # 9 fields x 1024^2 doubles = 72 MiB > 16 MiB
    sim = Sim("d2q9", "bl53", n, n, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    sim.init_macro(inputs.shear_wave(n, seed=6))
    out = np.empty((9, n, n), np.float64)
    st = B.lib().wcs_export_field_noalloc(sim.h, -1, out.ctypes.data, 0)
    assert st == 1
    assert b"staging array" in B.lib().wcs_last_error(sim.h)
    # one field of 1024^2 doubles (8 MiB) fits and matches the allocating path
    st, got = _noalloc(sim, 0, 0)
    assert st == 0
    assert np.array_equal(got, sim.export_field(0))
    sim.close()


def test_noalloc_export_3d_and_alternating_sizes():
    # The 3-D decode goes through its own kernel; and the shared array keeps
    # the previous call's bytes, so a smaller export right after a larger one
    # (from another simulation) must still return exactly its own field.
    from paper_2302_09883_gb300 import Sim3
    n3 = 64
    g = np.arange(n3, dtype=np.float64) * (2.0 * np.pi / n3)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    u0 = 0.04
    ux = u0 * np.sin(x) * np.cos(y) * np.cos(z)
    uy = -u0 * np.cos(x) * np.sin(y) * np.cos(z)
    s3 = Sim3(n3, n3, n3, 32, 3, 1e-6, store="bf16", tau=0.55)
    s3.init_macro([np.ones_like(ux), ux, uy, np.zeros_like(ux)])
    s3.step(2)
    big = Sim("d2q9", "bl53", 512, 512, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    big.init_macro(inputs.shear_wave(512, seed=7))
    small = Sim("d2q9", "bl53", 128, 128, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    small.init_macro(inputs.shear_wave(128, seed=8))
    small.step(2)
    for call in range(2):
        out3 = np.empty((n3, n3, n3), np.float32)
        st = B.lib().wcs_export_field_noalloc(s3.h, 5, out3.ctypes.data, 1)
        assert st == 0, B.lib().wcs_last_error(s3.h)
        assert np.array_equal(out3, s3.export_field(5, dtype=np.float32))
        st, got = _noalloc(big, -1, 1)  # 9 x 512^2 floats = 9 MiB
        assert st == 0
        assert np.array_equal(got, big.export_field(-1, dtype=np.float32))
        st, got = _noalloc(small, 4, 0)
        assert st == 0
        assert np.array_equal(got, small.export_field(4))
        s3.step(1)
        big.step(1)
        small.step(1)
    for s in (s3, big, small):
        s.close()
