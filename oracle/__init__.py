"""CPU oracle of the compressed-patch time step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import
this package.  The library under paper_2302_09883_gb300/ never does.

The arithmetic lives in plain C++ (oracle/*.hpp), FP64, with an FP32
instantiation of the same source for decisions the GPU takes in FP32.
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

SCHEME = {"d2q9": 0, "d3q19": 1, "euler2d": 2, "transport": 3, "swe": 4}
WAVELET = {"bl53": 0, "haar": 1, "cdf97": 2}
STORE = {"f64": 0, "f32": 1, "bf16": 2, "i8": 3}
RULE = {"const": 0, "accum": 1, "capped": 2}
PREC = {"f64": 0, "f32": 1}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
        dp = C.POINTER(C.c_double)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [i32, i32, i32, i32, i32, i64, i64, i32, i32, i32, dbl, dbl, dbl, dbl]
        L.orc_destroy.argtypes = [vp]
        L.orc_init_macro.argtypes = [vp, dp, dp, dp, dp]
        L.orc_step.argtypes = [vp, i64]
        L.orc_import.argtypes = [vp, i32, dp]
        L.orc_set_fv.argtypes = [vp, dbl, dbl, dbl, dbl]
        L.orc_entropy_code.restype = i64
        L.orc_entropy_code.argtypes = [vp, C.c_char_p, i64]
        L.orc_rans.restype = i64
        L.orc_rans.argtypes = [C.c_char_p, i64, C.c_char_p, i64, C.c_char_p]
        L.orc_rans_freqs.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
        L.orc_set_threads.restype = i32
        L.orc_set_threads.argtypes = [i32]
        L.orc_export_field.argtypes = [vp, i32, dp]
        L.orc_export_all.argtypes = [vp, dp]
        L.orc_set_patch_eps.argtypes = [vp, C.POINTER(C.c_double)]
        L.orc_track_features.argtypes = [vp, i32]
        L.orc_features.argtypes = [vp, dp]
        L.orc_npatch.restype = i64
        L.orc_npatch.argtypes = [vp]
        L.orc_record_bytes.restype = i64
        L.orc_record_bytes.argtypes = [vp, i64]
        L.orc_record.argtypes = [vp, i64, C.c_char_p, i64]
        L.orc_stats.argtypes = [vp, dp]
        L.orc_set_hilo.argtypes = [vp, i32]
        L.orc_count_ops.argtypes = [i32, i32, C.POINTER(i64)]
        L.orc_coarse_lo.argtypes = [vp, C.POINTER(C.c_float)]
        L.orc_hilo_sums.argtypes = [vp, dp]
        L.orc_ref_create.restype = vp
        L.orc_ref_create.argtypes = [i32, i32, i32, i64, i64, i32, dbl, dbl, dbl]
        L.orc_ref_init_macro.argtypes = [vp, dp, dp, dp, dp]
        L.orc_ref_step.argtypes = [vp, i64]
        L.orc_ref_export_field.argtypes = [vp, i32, dp]
        L.orc_ref_time.restype = dbl
        L.orc_ref_time.argtypes = [vp]
        L.orc_dwt.argtypes = [i32, i32, i64, i32, i32, i32, dp]
        L.orc_dwt_pyramid.argtypes = [i32, i64, i32, i32, dp]
        L.orc_layout.argtypes = [i32, i32, i64, i32, C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                                 C.POINTER(C.c_uint8), C.POINTER(C.c_int64)]
        L.orc_band_factor.restype = dbl
        L.orc_band_factor.argtypes = [i32, i32, i64, i32, i32, i32]
        L.orc_encode.restype = i64
        L.orc_encode.argtypes = [i32, i32, i64, i32, i32, i32, i32, dbl, i32, dp, C.c_char_p, i64]
        L.orc_decode.argtypes = [i32, i32, i64, i32, i32, i32, C.c_char_p, i64, dp]
        L.orc_bf16.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_uint16), i64]
        L.orc_d2q9_equilibrium.argtypes = [i32, dbl, dbl, dbl, dp]
        L.orc_d2q9_collide.argtypes = [i32, dp, dbl]
        L.orc_rusanov.argtypes = [dp, dp, i32, i32, dbl, dp]
        L.orc_sw_riemann.argtypes = [dbl, dbl, dbl, dbl, dbl, dbl, dbl, dp]
        L.orc_sw_flux.argtypes = [dp, dp, i32, i32, dbl, dp]
        L.orc_patch_features.argtypes = [i32, i32, i64, i32, i32, dp, dp]
        L.orc_patch_label.argtypes = [i32, i32, i64, i32, i32, dp, dbl, dp, i32]
        L.orc_patch_features_f32.argtypes = [i32, i32, i64, i32, i32, dp, dp]
        L.orc_eps_grid.restype = dbl
        L.orc_eps_grid.argtypes = [i32]
        L.orc_mlp_forward.argtypes = [i32, i32, dp, dp, i32, dp]
        L.orc_mlp_loss_grad.restype = dbl
        L.orc_mlp_loss_grad.argtypes = [i32, i32, dp, dp, dp, i32, dp]
        L.orc_d3q19_equilibrium.argtypes = [i32, dbl, dbl, dbl, dbl, dp]
        L.orc_d3q19_collide.argtypes = [i32, dp, dbl]
        L.orc3_create.restype = vp
        L.orc3_create.argtypes = [i32, i32, i32, i32, i64, i64, i64, i32, i32, dbl, dbl]
        L.orc3_ref_create.restype = vp
        L.orc3_ref_create.argtypes = [i32, i64, i64, i64, dbl]
        L.orc3_destroy.argtypes = [vp]
        L.orc3_init_macro.argtypes = [vp, dp, dp, dp, dp]
        L.orc3_step.argtypes = [vp, i64]
        L.orc3_export_all.argtypes = [vp, dp]
        L.orc3_npatch.restype = i64
        L.orc3_npatch.argtypes = [vp]
        L.orc3_record_bytes.restype = i64
        L.orc3_record_bytes.argtypes = [vp, i64]
        L.orc3_record.argtypes = [vp, i64, C.c_char_p, i64]
        L.orc3_stats.argtypes = [vp, dp]
        L.orc3_set_patch_eps.argtypes = [vp, dp]
        L.orc3_track_features.argtypes = [vp, i32]
        L.orc3_set_hilo.argtypes = [vp, i32]
        L.orc3_step_patch.argtypes = [i32, i32, i32, i32, dbl, dbl, i64, dp, C.c_char_p, i64, C.POINTER(i64)]
        L.orc3_coarse_lo.argtypes = [vp, C.POINTER(C.c_float)]
        L.orc3_hilo_sums.argtypes = [vp, dp]
        L.orc3_features.argtypes = [vp, dp]
        L.orc_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle: " + lib().orc_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _macro_ptrs(fields):
    arrs = [np.ascontiguousarray(f, dtype=np.float64) for f in fields]
    while len(arrs) < 4:
        arrs.append(arrs[0])
    return arrs, [_dp(a) for a in arrs[:4]]


def nfields(scheme):
    return {"d2q9": 9, "d3q19": 19, "euler2d": 4, "transport": 1, "swe": 3}[scheme]


class OracleSim:
    """Compressed-patch run (2-D).  Global arrays are (ny_nodes, nx_nodes)."""

    def __init__(self, scheme, wavelet, nx, ny, P, L, eps, prec="f64", store="f64", rule="const",
                 periodic=(True, True), tau=0.8, cfl=0.4, gamma=1.4, velocity=(0.0, 0.0), gravity=9.81, length=1.0,
                 hilo=False):
        self.scheme, self.wavelet, self.prec = scheme, wavelet, prec
        self.P, self.L = P, L
        pmask = int(periodic[0]) | (int(periodic[1]) << 1)
        self.G = [n + 1 if (wavelet != "haar" and not per) else n for n, per in zip((nx, ny), periodic)]
        self.F = nfields(scheme)
        self.h = lib().orc_create(SCHEME[scheme], WAVELET[wavelet], PREC[prec], STORE[store], RULE[rule],
                                  nx, ny, pmask, P, L, eps, tau, cfl, gamma)
        if not self.h:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        _check(lib().orc_set_fv(self.h, velocity[0], velocity[1], gravity, length))
        self.hilo = bool(hilo)
        if hilo:
            _check(lib().orc_set_hilo(self.h, 1))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def init_macro(self, fields):
        arrs, ptrs = _macro_ptrs(fields)
        _check(lib().orc_init_macro(self.h, *ptrs))

    def step(self, n=1):
        _check(lib().orc_step(self.h, n))

    def import_field(self, f, values):
        """Replace field f (-1: all, shape (F, ny, nx)) and re-encode."""
        a = np.ascontiguousarray(values, np.float64)
        _check(lib().orc_import(self.h, f, _dp(a)))

    def export_field(self, f):
        out = np.empty((self.G[1], self.G[0]), np.float64)
        _check(lib().orc_export_field(self.h, f, _dp(out)))
        return out

    def export_all(self):
        out = np.empty((self.F, self.G[1], self.G[0]), np.float64)
        _check(lib().orc_export_all(self.h, _dp(out)))
        return out

    def set_patch_eps(self, eps):
        e = np.ascontiguousarray(eps, np.float64)
        assert e.shape == (self.npatch,)
        _check(lib().orc_set_patch_eps(self.h, _dp(e)))

    def track_features(self, on=True):
        lib().orc_track_features(self.h, int(on))

    def features(self):
        """Features (npatch, 6L) of every patch at its last encode."""
        out = np.zeros((self.npatch, n_features(2, self.L)), np.float64)
        _check(lib().orc_features(self.h, _dp(out)))
        return out

    @property
    def npatch(self):
        return lib().orc_npatch(self.h)

    def record(self, p):
        n = lib().orc_record_bytes(self.h, p)
        buf = C.create_string_buffer(n)
        _check(lib().orc_record(self.h, p, buf, n))
        return buf.raw[:n]

    def entropy_code(self):
        """The rANS-coded state of the current records (bytes)."""
        n = lib().orc_entropy_code(self.h, None, 0)
        if n < 0:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        buf = C.create_string_buffer(n)
        lib().orc_entropy_code(self.h, buf, n)
        return buf.raw[:n]

    def stats(self):
        out = np.zeros(48, np.float64)
        _check(lib().orc_stats(self.h, _dp(out)))
        return {"coef_sums": out[:self.F].copy(), "nstep": int(out[20]), "time": out[21],
                "shared_mismatch": int(out[22]), "compressed_bytes": int(out[23]),
                "coef_abs_sums": out[24:24 + self.F].copy(), "n_terms": self.npatch * self.n_coarse}

    @property
    def n_coarse(self):
        return ((self.P >> self.L) + (1 if self.wavelet != "haar" else 0)) ** 2

    def coarse_lo(self):
        """hi + lo coarse storage: the lo parts of the current state,
        (npatch, F, NC1^2) float32, sample iy NC1 + ix."""
        out = np.zeros((self.npatch, self.F, self.n_coarse), np.float32)
        _check(lib().orc_coarse_lo(self.h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def hilo_sums(self):
        """hi + lo: per field the lo parts' share of the coarse-domain mass,
        the sums of its absolute terms, and the FP64 trapezoid node sums of
        the state just before its encode."""
        out = np.zeros(72, np.float64)
        _check(lib().orc_hilo_sums(self.h, _dp(out)))
        return {"lo_sums": out[:self.F].copy(), "lo_abs_sums": out[24:24 + self.F].copy(),
                "pre_sums": out[48:48 + self.F].copy()}


class OracleRef:
    """Uncompressed run of the same scheme on the global arrays."""

    def __init__(self, scheme, wavelet, nx, ny, prec="f64", periodic=(True, True), tau=0.8, cfl=0.4, gamma=1.4,
                 velocity=(0.0, 0.0), gravity=9.81, length=1.0):
        pmask = int(periodic[0]) | (int(periodic[1]) << 1)
        self.G = [n + 1 if (wavelet != "haar" and not per) else n for n, per in zip((nx, ny), periodic)]
        self.F = nfields(scheme)
        self.h = lib().orc_ref_create(SCHEME[scheme], WAVELET[wavelet], PREC[prec], nx, ny, pmask, tau, cfl, gamma)
        if not self.h:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        _check(lib().orc_set_fv(self.h, velocity[0], velocity[1], gravity, length))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def init_macro(self, fields):
        arrs, ptrs = _macro_ptrs(fields)
        _check(lib().orc_ref_init_macro(self.h, *ptrs))

    def step(self, n=1):
        _check(lib().orc_ref_step(self.h, n))

    def export_field(self, f):
        out = np.empty((self.G[1], self.G[0]), np.float64)
        _check(lib().orc_ref_export_field(self.h, f, _dp(out)))
        return out

    @property
    def time(self):
        return lib().orc_ref_time(self.h)


def dwt(u, wavelet, P, L, inverse=False, prec="f64"):
    """Tensor lifting transform of a d-D block (returns a new array)."""
    a = np.ascontiguousarray(u, dtype=np.float64).copy()
    _check(lib().orc_dwt(WAVELET[wavelet], a.ndim, P, L, int(inverse), PREC[prec], _dp(a)))
    return a


def dwt_pyramid(u, wavelet, P, L, inverse=False):
    """Mallat-pyramid transform of a 2-D block (FP64; returns a new array)."""
    a = np.ascontiguousarray(u, dtype=np.float64).copy()
    _check(lib().orc_dwt_pyramid(WAVELET[wavelet], P, L, int(inverse), _dp(a)))
    return a


def layout(wavelet, dims, P, L):
    """Per node position (row-major, x fastest): band id, edge-line and
    coarse flags."""
    sizes = np.zeros(4, np.int64)
    _check(lib().orc_layout(WAVELET[wavelet], dims, P, L, None, None, None,
                            sizes.ctypes.data_as(C.POINTER(C.c_int64))))
    n = int(sizes[0])
    band = np.zeros(n, np.int32)
    edge = np.zeros(n, np.uint8)
    coarse = np.zeros(n, np.uint8)
    _check(lib().orc_layout(WAVELET[wavelet], dims, P, L, band.ctypes.data_as(C.POINTER(C.c_int32)),
                            edge.ctypes.data_as(C.POINTER(C.c_uint8)), coarse.ctypes.data_as(C.POINTER(C.c_uint8)),
                            sizes.ctypes.data_as(C.POINTER(C.c_int64))))
    return {"band": band, "edge": edge.astype(bool), "coarse": coarse.astype(bool), "n_all": n,
            "n_c": int(sizes[1]), "n_w": int(sizes[2]), "nb": int(sizes[3])}


def band_factor(wavelet, dims, P, L, band, rule):
    return lib().orc_band_factor(WAVELET[wavelet], dims, P, L, band, RULE[rule])


def encode(coef, wavelet, P, L, eps, prec="f64", store="f64", rule="const"):
    """coef: (F, E, E[, E]) transformed coefficients in place.  Returns bytes."""
    c = np.ascontiguousarray(coef, dtype=np.float64)
    dims = c.ndim - 1
    cap = c.size * 8 + 4096 + 64 * c.shape[0]
    buf = C.create_string_buffer(cap)
    n = lib().orc_encode(WAVELET[wavelet], dims, P, L, PREC[prec], STORE[store], RULE[rule], eps, c.shape[0],
                         _dp(c), buf, cap)
    if n < 0:
        raise RuntimeError("oracle: " + lib().orc_last_error().decode())
    return buf.raw[:n]


def decode(rec, nfields_, shape, wavelet, P, L, prec="f64", store="f64"):
    out = np.zeros((nfields_,) + tuple(shape), np.float64)
    _check(lib().orc_decode(WAVELET[wavelet], len(shape), P, L, PREC[prec], STORE[store], rec, len(rec), _dp(out)))
    return out


def bf16_bits(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(x.shape, np.uint16)
    lib().orc_bf16(x.ctypes.data_as(C.POINTER(C.c_float)), out.ctypes.data_as(C.POINTER(C.c_uint16)), x.size)
    return out


def d2q9_equilibrium(rho, ux, uy, prec="f64"):
    out = np.zeros(9, np.float64)
    lib().orc_d2q9_equilibrium(PREC[prec], rho, ux, uy, _dp(out))
    return out


def d2q9_collide(f, tau, prec="f64"):
    g = np.ascontiguousarray(f, dtype=np.float64).copy()
    lib().orc_d2q9_collide(PREC[prec], _dp(g), tau)
    return g


def rusanov(WL, WR, nx, ny, gamma=1.4):
    a = np.ascontiguousarray(WL, np.float64)
    b = np.ascontiguousarray(WR, np.float64)
    out = np.zeros(4, np.float64)
    lib().orc_rusanov(_dp(a), _dp(b), nx, ny, gamma, _dp(out))
    return out


# ----------------------------------------------------------- learned part
def n_features(dims, L):
    return 2 * ((1 << dims) - 1) * L


def patch_features(u, wavelet, P, L, prec="f64"):
    """u: (F, E, E) or (F, E, E, E) node values of one patch -> features
    (groups (l, S) in order, energy then max); prec: precision of the
    transforms."""
    a = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(n_features(a.ndim - 1, L), np.float64)
    fn = lib().orc_patch_features if prec == "f64" else lib().orc_patch_features_f32
    _check(fn(WAVELET[wavelet], a.ndim - 1, P, L, a.shape[0], _dp(a), _dp(out)))
    return out


def patch_label(u, wavelet, P, L, delta, prec="f64"):
    """log10 of the largest admissible eps of a patch (grid + bisection);
    prec: precision of the transforms (tests and sums are FP64)."""
    a = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(1, np.float64)
    _check(lib().orc_patch_label(WAVELET[wavelet], a.ndim - 1, P, L, a.shape[0], _dp(a), delta, _dp(out), PREC[prec]))
    return float(out[0])


def eps_grid(k):
    return lib().orc_eps_grid(k)


def mlp_nparam(nin, nh):
    return nh * nin + nh + nh * nh + nh + nh + 1


def mlp_forward(w, X, nin, nh):
    w = np.ascontiguousarray(w, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    y = np.zeros(X.shape[0], np.float64)
    lib().orc_mlp_forward(nin, nh, _dp(w), _dp(X), X.shape[0], _dp(y))
    return y


def mlp_loss_grad(w, X, t, nin, nh):
    w = np.ascontiguousarray(w, np.float64)
    X = np.ascontiguousarray(X, np.float64)
    t = np.ascontiguousarray(t, np.float64)
    g = np.zeros(mlp_nparam(nin, nh), np.float64)
    loss = lib().orc_mlp_loss_grad(nin, nh, _dp(w), _dp(X), _dp(t), X.shape[0], _dp(g))
    return loss, g


# ------------------------------------------------------------------ D3Q19
def d3q19_equilibrium(rho, ux, uy, uz, prec="f64"):
    out = np.zeros(19, np.float64)
    lib().orc_d3q19_equilibrium(PREC[prec], rho, ux, uy, uz, _dp(out))
    return out


def d3q19_collide(f, tau, prec="f64"):
    a = np.array(f, np.float64)
    lib().orc_d3q19_collide(PREC[prec], _dp(a), tau)
    return a


def _macro3(fields):
    arrs = [np.ascontiguousarray(a, np.float64) for a in fields]
    assert len(arrs) == 4 and all(a.ndim == 3 for a in arrs)
    return arrs, [_dp(a) for a in arrs]


class _Run3:
    def __del__(self):
        if getattr(self, "h", None):
            lib().orc3_destroy(self.h)
            self.h = None

    def init_macro(self, fields):
        """fields: rho, ux, uy, uz as (nz, ny, nx) arrays."""
        arrs, ptrs = _macro3(fields)
        _check(lib().orc3_init_macro(self.h, *ptrs))

    def step(self, n=1):
        _check(lib().orc3_step(self.h, n))

    def export_all(self):
        out = np.empty((19,) + self.shape, np.float64)
        _check(lib().orc3_export_all(self.h, _dp(out)))
        return out


class OracleSim3(_Run3):
    """Compressed-patch D3Q19 run on a periodic (nz, ny, nx) grid."""

    def __init__(self, wavelet, nx, ny, nz, P, L, eps, prec="f64", store="f64", rule="const", tau=0.8, hilo=False):
        self.P, self.L, self.shape = P, L, (nz, ny, nx)
        self.h = lib().orc3_create(WAVELET[wavelet], PREC[prec], STORE[store], RULE[rule], nx, ny, nz, P, L, eps,
                                   tau)
        if not self.h:
            raise RuntimeError("oracle: " + lib().orc_last_error().decode())
        self.hilo = bool(hilo)
        if hilo:
            _check(lib().orc3_set_hilo(self.h, 1))

    def coarse_lo(self):
        """hi + lo: the lo parts, (npatch, 19, NC1^3) float32."""
        out = np.zeros((self.npatch, 19, ((self.P >> self.L) + 1) ** 3), np.float32)
        _check(lib().orc3_coarse_lo(self.h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def hilo_sums(self):
        """hi + lo: lo sums, their absolute terms, node sums before the last
        encode (per field)."""
        out = np.zeros(72, np.float64)
        _check(lib().orc3_hilo_sums(self.h, _dp(out)))
        return {"lo_sums": out[:19].copy(), "lo_abs_sums": out[24:43].copy(), "pre_sums": out[48:67].copy()}

    @property
    def npatch(self):
        return lib().orc3_npatch(self.h)

    def record(self, p):
        n = lib().orc3_record_bytes(self.h, p)
        buf = C.create_string_buffer(n)
        _check(lib().orc3_record(self.h, p, buf, n))
        return buf.raw[:n]

    def set_patch_eps(self, eps):
        e = np.ascontiguousarray(eps, np.float64)
        assert e.shape == (self.npatch,)
        _check(lib().orc3_set_patch_eps(self.h, _dp(e)))

    def track_features(self, on=True):
        lib().orc3_track_features(self.h, int(on))

    def features(self):
        """Features (npatch, 42 for L = 3) of every patch at its last encode."""
        out = np.zeros((self.npatch, n_features(3, self.L)), np.float64)
        _check(lib().orc3_features(self.h, _dp(out)))
        return out

    def stats(self):
        out = np.zeros(48, np.float64)
        _check(lib().orc3_stats(self.h, _dp(out)))
        return {"coef_sums": out[:19].copy(), "nstep": int(out[20]), "shared_mismatch": int(out[22]),
                "compressed_bytes": int(out[23]), "coef_abs_sums": out[24:43].copy(),
                "n_terms": self.npatch * ((self.P >> self.L) + 1) ** 3}


def count_ops(P, L):
    """Operations (+, -, *, / each one) the oracle executes for one 2-D BL5/3
    patch of P+1 nodes per axis: (forward transform of one field, its inverse,
    one D2Q9 collision of a node)."""
    out = (C.c_int64 * 3)()
    _check(lib().orc_count_ops(P, L, out))
    return int(out[0]), int(out[1]), int(out[2])


def d3q19_patch_step(block, P, L, eps, tau, store="bf16", rule="const", pid=0):
    """One FP32 D3Q19 step of a single patch: block (19, P+3, P+3, P+3) is
    the decoded state on the patch's nodes and the layer around them
    ([f][z][y][x], index 0 = node -1); returns the record (bytes) that
    OracleSim3 would write for patch pid."""
    b = np.ascontiguousarray(block, np.float64)
    assert b.shape == (19, P + 3, P + 3, P + 3)
    cap = 64 * 19 * (P + 1) ** 3 + 4096
    buf = C.create_string_buffer(cap)
    nb = C.c_int64()
    _check(lib().orc3_step_patch(STORE[store], RULE[rule], P, L, eps, tau, pid, _dp(b), buf, cap, C.byref(nb)))
    return buf.raw[:nb.value]


class OracleRef3(_Run3):
    """Uncompressed D3Q19 run on a periodic (nz, ny, nx) grid."""

    def __init__(self, nx, ny, nz, prec="f64", tau=0.8):
        self.shape = (nz, ny, nx)
        self.h = lib().orc3_ref_create(PREC[prec], nx, ny, nz, tau)


def sums_agree(got, stats):
    """True if GPU coarse-block sums equal the oracle's plain FP64 sums up to
    the rounding of two summation orders: each order errs by at most
    gamma_(n-1) * sum|terms| (n terms, gamma_k = k u / (1 - k u),
    u = 2^-53), so two orders differ by at most twice that."""
    u = 2.0 ** -53
    k = stats["n_terms"] - 1
    gamma = k * u / (1.0 - k * u)
    want, ab = stats["coef_sums"], stats["coef_abs_sums"]
    return bool(np.all(np.abs(np.asarray(got) - want) <= 2.0 * gamma * ab))


def set_threads(n):
    """Threads of the oracle's parallel loops (0: default); returns the count."""
    return lib().orc_set_threads(int(n))


def sw_riemann(hL, uL, tL, hR, uR, tR, g=9.81):
    """Shallow-water Riemann solution along a normal: (h, un, ut) at x/t = 0
    and the star state (h*, u*)."""
    out = np.zeros(5, np.float64)
    _check(lib().orc_sw_riemann(hL, uL, tL, hR, uR, tR, g, _dp(out)))
    return out[:3], out[3], out[4]


def sw_flux(WL, WR, nx, ny, g=9.81):
    a = np.ascontiguousarray(WL, np.float64)
    b = np.ascontiguousarray(WR, np.float64)
    out = np.zeros(3, np.float64)
    _check(lib().orc_sw_flux(_dp(a), _dp(b), nx, ny, g, _dp(out)))
    return out


def rans_roundtrip(data):
    """(coded bytes, decoded bytes) of an order-0 rANS round trip of data with
    the table of its own byte counts."""
    n = len(data)
    cap = 2 * n + 64
    coded = C.create_string_buffer(cap)
    dec = C.create_string_buffer(max(n, 1))
    m = lib().orc_rans(bytes(data), n, coded, cap, dec)
    if m < 0:
        raise RuntimeError("oracle: " + lib().orc_last_error().decode())
    return coded.raw[:m], dec.raw[:n]


def rans_freqs(counts):
    c = np.ascontiguousarray(counts, np.uint64)
    f = np.zeros(256, np.uint32)
    _check(lib().orc_rans_freqs(c.ctypes.data_as(C.POINTER(C.c_uint64)), f.ctypes.data_as(C.POINTER(C.c_uint32))))
    return f
