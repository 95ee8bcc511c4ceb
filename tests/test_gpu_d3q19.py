"""GPU parity of the 3-D path (D3Q19, folded BL5/3, FP32 compute) against
the FP32 instantiation of the oracle: records byte-identical, decoded fields
bit-identical, FP64 coarse sums bit-identical."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Sim3, inputs

pytestmark = pytest.mark.gpu


def run_pair3(dims, P, L, eps, store, fields, steps, check_at=(), tau=0.55, arena=0.5):
    nx, ny, nz = dims
    g = Sim3(nx, ny, nz, P, L, eps, store=store, tau=tau, arena_factor=arena)
    o = O.OracleSim3("bl53", nx, ny, nz, P, L, eps, prec="f32", store=store, tau=tau)
    g.init_macro(fields)
    o.init_macro(fields)
    done = 0
    for s in sorted(set([0] + list(check_at) + [steps])):
        g.step(s - done)
        o.step(s - done)
        done = s
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p), "patch %d record differs after %d steps" % (p, s)
    return g, o


@pytest.mark.parametrize("store", ["bf16", "f32"])
def test_d3q19_p16_matches_fp32_oracle_bitwise(store):
    # 32^3 Taylor-Green vortex, 8 patches of 16^3 (17^3 nodes), 3 levels
    f = inputs.taylor_green_3d(32, u0=0.04)
    g, o = run_pair3((32, 32, 32), 16, 3, 1e-4, store, f, 4, check_at=(1,))
    a, b = g.export_field(-1), o.export_all()
    assert np.array_equal(a, b)
    sg, so = g.stats(), o.stats()
    assert O.sums_agree(sg["field_sum"], so)


def test_d3q19_p32_matches_fp32_oracle_bitwise():
    # 64^3, 8 patches of 32^3 (33^3 nodes), BF16 details
    f = inputs.taylor_green_3d(64, u0=0.04)
    g, o = run_pair3((64, 64, 64), 32, 3, 1e-4, "bf16", f, 2, check_at=(1,))
    assert np.array_equal(g.export_field(-1), o.export_all())


def test_d3q19_non_cubic_grid_with_a_single_patch_along_z():
    # 2 x 3 x 1 patches: along z a patch is its own neighbour; shear wave along y + noise
    f = inputs.shear_wave_3d(32, 48, 16, u0=0.02, axis=1, noise=1e-4, seed=3)
    g, o = run_pair3((32, 48, 16), 16, 3, 1e-4, "bf16", f, 3, check_at=(1,))
    assert np.array_equal(g.export_field(-1), o.export_all())
    assert o.stats()["shared_mismatch"] == 0


def test_d3q19_eps_zero_tracks_the_uncompressed_run():
    f = inputs.taylor_green_3d(32, u0=0.04)
    g = Sim3(32, 32, 32, 16, 3, 0.0, store="f32", tau=0.55, arena_factor=2.0)
    r = O.OracleRef3(32, 32, 32, prec="f64", tau=0.55)
    g.init_macro(f)
    r.init_macro(f)
    g.step(5)
    r.step(5)
    a, b = g.export_field(-1), r.export_all()
    # FP32 arithmetic against the FP64 reference: the 2-D paths' bar
    for i in range(19):
        assert np.linalg.norm(a[i] - b[i]) <= 1e-5 * np.linalg.norm(b[i])
    st = g.stats()
    m0 = float(np.sum(f[0]))
    assert abs(st["mass"] - m0) <= 1e-5 * m0
    assert np.all(np.abs(st["momentum"]) <= 1e-5 * m0)


def test_d3q19_arena_overflow_is_reported():
    from paper_2302_09883_gb300._lib import WcsError
    f = inputs.taylor_green_3d(32, u0=0.04)
    g = Sim3(32, 32, 32, 16, 3, 0.0, store="f32", tau=0.55, arena_factor=0.01)
    with pytest.raises(WcsError) as ei:
        g.init_macro(f)
    assert ei.value.status == 3


def test_d3q19_dense_baseline_matches_oracle_reference():
    from paper_2302_09883_gb300 import Dense3
    d = Dense3(32, 32, 16, tau=0.55)
    r = O.OracleRef3(32, 32, 16, prec="f32", tau=0.55)
    f16 = [a[:16] for a in inputs.taylor_green_3d(32, u0=0.04)]
    d.init_macro(f16)
    r.init_macro(f16)
    d.step(7)
    r.step(7)
    b = r.export_all()
    for i in range(19):
        assert np.array_equal(d.export_field(i), b[i])


def test_d3q19_only_coarse_blocks_survive_at_huge_eps():
    f = inputs.taylor_green_3d(32, u0=0.04)
    g, o = run_pair3((32, 32, 32), 16, 3, 1e30, "bf16", f, 3, check_at=(1,))
    assert np.array_equal(g.export_field(-1), o.export_all())
    assert O.sums_agree(g.stats()["field_sum"], o.stats())
