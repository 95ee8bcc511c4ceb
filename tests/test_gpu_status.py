"""Failure reporting without a GPU fault: a non-finite macroscopic value at
one node makes the encode of the state report E_NAN.  The node is away from
every coarse sample, so the report relies on the lifting carrying the NaN
or infinity into the coarse block, which is the only place the 2-D kernels
check."""
import numpy as np
import pytest

from paper_2302_09883_gb300 import Sim, Sim3, inputs
from paper_2302_09883_gb300._lib import WcsError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("case", ["d2q9_bl53_bf16", "d2q9_haar_f64", "euler_bl53_i8"])
def test_non_finite_node_is_reported(bad, case):
    if case == "d2q9_bl53_bf16":
        sc, wv, n, P, L, prec, store, kw = "d2q9", "bl53", 256, 64, 4, "f32", "bf16", dict(tau=0.6)
        f = inputs.shear_wave(n, seed=3)
        per = (True, True)
    elif case == "d2q9_haar_f64":
        sc, wv, n, P, L, prec, store, kw = "d2q9", "haar", 128, 32, 3, "f64", "f64", dict(tau=0.8)
        f = inputs.shear_wave(n, seed=4)
        per = (True, True)
    else:
        sc, wv, n, P, L, prec, store, kw = "euler2d", "bl53", 256, 64, 4, "f32", "i8", dict(cfl=0.4)
        f = inputs.four_quadrant(n)
        per = (False, False)
    f = [np.array(x, dtype=np.float64, copy=True) for x in f]
    f[1][37, 101] = bad  # node (x 101, y 37): no axis is a multiple of 2^L
    g = Sim(sc, wv, n, n, P, L, 1e-4, prec=prec, store=store, periodic=per, **kw)
    with pytest.raises(WcsError) as ei:
        g.init_macro(f)
        g.step(1)
        g.sync()
    assert "E_NAN" in str(ei.value)


def test_non_finite_node_is_reported_d3q19():
    rho, ux, uy, uz = [np.array(x, dtype=np.float64, copy=True) for x in inputs.shear_wave_3d(64, 64, 64, seed=5)]
    ux[21, 37, 13] = np.nan
    g = Sim3(64, 64, 64, 32, 3, 1e-6, store="bf16", tau=0.8)
    with pytest.raises(WcsError) as ei:
        g.init_macro([rho, ux, uy, uz])
        g.step(1)
        g.sync()
    assert "E_NAN" in str(ei.value)


def test_finite_state_steps_cleanly():
    n = 256
    g = Sim("d2q9", "bl53", n, n, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    g.init_macro(inputs.shear_wave(n, seed=3))
    g.step(3)
    g.sync()
    assert g.stats()["status"] == 0


def test_zero_steps_change_nothing():
    # the degenerate calls: zero steps (alone and in a batch) and repeated
    # syncs leave records, step count and FP64 sums as they were
    from paper_2302_09883_gb300 import Batch
    n = 128
    a = Sim("d2q9", "bl53", n, n, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    a.init_macro(inputs.shear_wave(n, seed=5))
    a.step(3)
    a.sync()
    recs = [a.record(p) for p in range(a.npatch)]
    st = a.stats()
    a.step(0)
    a.sync()
    a.sync()
    b = Batch([a])
    b.step(0)
    b.sync()
    b.close()
    st2 = a.stats()
    assert [a.record(p) for p in range(a.npatch)] == recs
    assert st2["step"] == st["step"] == 3 and np.array_equal(st2["field_sum"], st["field_sum"])
