"""The C-ABI library on the CPU (no GPU needed): it loads, exports every
function include/wcsim.h declares, and rejects bad arguments before any CUDA
call with the documented status and a message."""
import ctypes as C
import os
import re

import pytest

from paper_2302_09883_gb300 import _lib as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_2302_09883_gb300 import build
        build.build()
    L = B.lib()
    L.wcs_last_error.restype = C.c_char_p
    return L


def declared():
    hdr = open(os.path.join(ROOT, "include", "wcsim.h")).read()
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(wcs_\w+)\s*\(", hdr, re.M)))


def test_library_exports_every_declared_function(L):
    names = declared()
    assert len(names) >= 39
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


def _grid(dims, n, mask):
    g = B.Grid()
    g.dims = dims
    for a in range(3):
        g.n[a] = n[a]
    g.periodic_mask = mask
    return g


def _opts(store="bf16", prec="f32", wavelet="bl53", rule="const"):
    o = B.Opts()
    o.wavelet, o.rule, o.detail_store, o.compute = B.WAVELET[wavelet], B.RULE[rule], B.STORE[store], B.PREC[prec]
    o.tau = 0.6
    return o


def _create(L, g, scheme, P, Lv, eps, o):
    h = C.c_void_p()
    st = L.wcs_create_sim(C.byref(g), B.SCHEME[scheme], P, Lv, eps, C.byref(o), C.byref(h))
    return st, h, L.wcs_last_error(None).decode()


@pytest.mark.parametrize("case,want,msg", [
    ("ragged_2d", 1, "multiple of the patch"),
    ("empty_grid", 1, "multiple of the patch"),
    ("negative_eps", 1, "eps"),
    ("no_kernel", 7, "no compiled kernel"),
    ("d2q9_outflow", 1, "periodic"),
    ("bad_rule", 1, "rule"),
    ("ragged_3d", 1, "multiple of the patch"),
    ("d3q19_outflow", 1, "periodic"),
    ("d3q19_fp64", 7, "FP32"),
    ("d3q19_no_kernel", 7, "no compiled 3-D kernel"),
    ("d3q19_on_2d_grid", 1, "D3Q19"),
    ("deferred_no_fit", 7, "fits the grid"),
    ("deferred_negative", 1, ">= 0"),
    ("hilo_fp64", 7, "hi + lo"),
    ("deferred_outflow_d2q9", 1, "periodic"),
    ("deferred_bad_rule", 1, "rule"),
])
def test_create_rejects_bad_arguments_without_a_gpu(L, case, want, msg):
    g2 = _grid(2, (256, 256, 1), 3)
    g3 = _grid(3, (64, 64, 64), 7)
    if case == "ragged_2d":
        r = _create(L, _grid(2, (250, 256, 1), 3), "d2q9", 64, 4, 1e-3, _opts())
    elif case == "empty_grid":
        r = _create(L, _grid(2, (0, 256, 1), 3), "d2q9", 64, 4, 1e-3, _opts())
    elif case == "negative_eps":
        r = _create(L, g2, "d2q9", 64, 4, -1.0, _opts())
    elif case == "no_kernel":
        r = _create(L, g2, "d2q9", 128, 5, 1e-3, _opts())
    elif case == "d2q9_outflow":
        r = _create(L, _grid(2, (256, 256, 1), 1), "d2q9", 64, 4, 1e-3, _opts())
    elif case == "bad_rule":
        o = _opts()
        o.rule = 9
        r = _create(L, g2, "d2q9", 64, 4, 1e-3, o)
    elif case == "ragged_3d":
        r = _create(L, _grid(3, (64, 60, 64), 7), "d3q19", 32, 3, 1e-3, _opts())
    elif case == "d3q19_outflow":
        r = _create(L, _grid(3, (64, 64, 64), 3), "d3q19", 32, 3, 1e-3, _opts())
    elif case == "d3q19_fp64":
        r = _create(L, g3, "d3q19", 32, 3, 1e-3, _opts(store="f64", prec="f64"))
    elif case == "d3q19_no_kernel":
        r = _create(L, g3, "d3q19", 32, 2, 1e-3, _opts())
    elif case == "deferred_no_fit":  # 80 cells: no compiled P (32, 64) divides them
        r = _create(L, _grid(2, (80, 80, 1), 3), "d2q9", 0, 0, 1e-3, _opts())
    elif case == "deferred_negative":
        r = _create(L, g2, "d2q9", 0, -1, 1e-3, _opts())
    elif case == "deferred_outflow_d2q9":
        r = _create(L, _grid(2, (256, 256, 1), 1), "d2q9", 0, 0, 1e-3, _opts())
    elif case == "deferred_bad_rule":
        o = _opts()
        o.rule = 7
        r = _create(L, g2, "d2q9", 0, 4, 1e-3, o)
    elif case == "hilo_fp64":
        o = _opts(store="f64", prec="f64")
        o.coarse_hilo = 1
        r = _create(L, _grid(2, (128, 128, 1), 3), "d2q9", 32, 3, 1e-3, o)
    else:
        r = _create(L, g2, "d3q19", 32, 3, 1e-3, _opts())
    st, h, text = r
    assert st == want and not h.value
    assert msg in text


def test_deferred_patch_choice_waits_for_the_init(L):
    """patch = levels = 0: the handle exists, nothing is chosen or allocated
    before wcs_init_macro, and calls that need a state are refused."""
    st, h, _ = _create(L, _grid(2, (256, 256, 1), 3), "d2q9", 0, 0, 1e-3, _opts())
    assert st == 0 and h.value
    P, Lv = C.c_int(-1), C.c_int(-1)
    assert L.wcs_patch_config(h, C.byref(P), C.byref(Lv)) == 0 and (P.value, Lv.value) == (0, 0)
    npatch, nf, gx, gy = C.c_int64(-1), C.c_int(), C.c_int64(), C.c_int64()
    assert L.wcs_shape(h, C.byref(npatch), C.byref(nf), C.byref(gx), C.byref(gy)) == 0
    assert (npatch.value, nf.value, gx.value, gy.value) == (0, 9, 256, 256)
    assert L.wcs_step(h, 1) == 1 and "init" in L.wcs_last_error(h).decode()
    stats = B.StepStats()
    assert L.wcs_stats(h, C.byref(stats)) == 1
    assert L.wcs_compressed_bytes(h) == -1
    L.wcs_destroy(h)


def test_null_arguments_are_rejected(L):
    o, g = _opts(), _grid(2, (256, 256, 1), 3)
    h = C.c_void_p()
    assert L.wcs_create_sim(None, 0, 64, 4, 1e-3, C.byref(o), C.byref(h)) == 1
    assert L.wcs_create_sim(C.byref(g), 0, 64, 4, 1e-3, None, C.byref(h)) == 1
    assert L.wcs_step(None, 1) == 1
    assert L.wcs_sync(None) == 1
    assert L.wcs_export_field(None, 0, None, 0, 0) == 1
    assert L.wcs_compressed_bytes(None) == -1
    assert L.wcs_shape3(None, None, None, None) == 1
    L.wcs_destroy(None)  # accepted


def test_learned_part_rejects_bad_sizes(L):
    m = C.c_void_p()
    assert L.wcs_mlp_create(0, C.byref(m)) == 1
    assert L.wcs_mlp_create(65, C.byref(m)) == 1
    assert L.wcs_mlp_nparam(None) == -1
    # features/labels: null device pointers, a grid that is not a multiple of the patch
    assert L.wcs_features_labels(None, 9, 256, 256, 0, 64, 4, 1e-4, None, None, None) == 1
    assert L.wcs_features_labels(C.c_void_p(16), 9, 250, 256, 0, 64, 4, 1e-4, C.c_void_p(16), C.c_void_p(16),
                                 None) == 1


def test_batch_and_autotune_reject_bad_arguments(L):
    b = C.c_void_p()
    assert L.wcs_batch_create(None, 0, C.byref(b)) == 1
    g3 = _grid(3, (64, 64, 64), 7)
    o = _opts()
    P = (C.c_int * 1)(32)
    Lv = (C.c_int * 1)(3)
    best = C.c_int()
    assert L.wcs_autotune(C.byref(g3), B.SCHEME["d3q19"], C.byref(o), 1e-3, P, Lv, 1, None, 0, 0, 2, C.byref(best),
                          None) == 7
