"""Python front end of the C-ABI: a compressed-patch simulation and the
uncompressed baseline.  PyTorch supplies the CUDA stream and, when the caller
passes device tensors, the device memory of inputs and outputs."""
import ctypes as C

import numpy as np

from . import _lib as B


def _grid(nx, ny, periodic):
    g = B.Grid()
    g.dims = 2
    g.n[0], g.n[1], g.n[2] = nx, ny, 1
    g.periodic_mask = int(periodic[0]) | (int(periodic[1]) << 1)
    return g


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _field_ptrs(fields):
    """Host numpy arrays or CUDA tensors -> (keepalive, pointer array, is_device)."""
    keep, ptrs, dev = [], [], None
    for f in fields:
        if hasattr(f, "data_ptr"):
            import torch
            t = f.to(torch.float64).contiguous()
            keep.append(t)
            ptrs.append(t.data_ptr())
            d = 1 if t.is_cuda else 0
        else:
            a = np.ascontiguousarray(f, dtype=np.float64)
            keep.append(a)
            ptrs.append(a.ctypes.data)
            d = 0
        if dev is None:
            dev = d
        elif dev != d:
            raise ValueError("mixed host/device inputs")
    if dev:
        # the tensors were produced on torch's stream; the library reads them
        # on its own stream, so the producer must have finished
        import torch
        torch.cuda.synchronize()
    arr = (C.c_void_p * len(ptrs))(*ptrs)
    return keep, arr, dev or 0


class Sim:
    """One compressed-patch simulation on the current CUDA device."""

    def __init__(self, scheme, wavelet, nx, ny, P, L, eps, prec="f32", store="bf16", rule="const",
                 periodic=(True, True), tau=0.8, cfl=0.4, gamma=1.4, arena_factor=0.0, stream=None,
                 velocity=(0.0, 0.0), gravity=9.81, length=1.0, coarse_hilo=False):
        self.scheme, self.P, self.L = scheme, P, L
        o = B.Opts()
        o.wavelet, o.rule, o.detail_store, o.compute = B.WAVELET[wavelet], B.RULE[rule], B.STORE[store], B.PREC[prec]
        o.tau, o.cfl, o.gamma, o.arena_factor = tau, cfl, gamma, arena_factor
        o.velocity[0], o.velocity[1], o.gravity, o.length = velocity[0], velocity[1], gravity, length
        o.coarse_hilo = int(bool(coarse_hilo))
        o.cuda_stream = _stream_ptr(stream)
        h = C.c_void_p()
        g = _grid(nx, ny, periodic)
        B.check(B.lib().wcs_create_sim(C.byref(g), B.SCHEME[scheme], P, L, eps, C.byref(o), C.byref(h)), None)
        self.h = h
        npatch, nf, gx, gy = C.c_int64(), C.c_int(), C.c_int64(), C.c_int64()
        B.lib().wcs_shape(h, C.byref(npatch), C.byref(nf), C.byref(gx), C.byref(gy))
        self.npatch, self.F, self.G = npatch.value, nf.value, (gx.value, gy.value)

    def close(self):
        if getattr(self, "h", None):
            B.lib().wcs_destroy(self.h)
            self.h = None

    __del__ = close

    def init_macro(self, fields):
        keep, arr, dev = _field_ptrs(fields)
        B.check(B.lib().wcs_init_macro(self.h, arr, len(fields), dev), self.h)
        if not (self.P and self.L):  # P or L 0: the autotuner chose them in the init
            self._refresh_shape()

    def _refresh_shape(self):
        P, L = C.c_int(), C.c_int()
        B.check(B.lib().wcs_patch_config(self.h, C.byref(P), C.byref(L)), self.h)
        self.P, self.L = P.value, L.value
        npatch, nf = C.c_int64(), C.c_int()
        B.lib().wcs_shape(self.h, C.byref(npatch), C.byref(nf), None, None)
        self.npatch = npatch.value

    def patch_config(self):
        """(P, L) of the simulation (0 before the init when left to the
        autotuner)."""
        return self.P, self.L

    def step(self, n=1):
        B.check(B.lib().wcs_step(self.h, n), self.h)

    def sync(self):
        B.check(B.lib().wcs_sync(self.h), self.h)

    def export_field(self, f, out=None, dtype=np.float64):
        """Decoded field f ([ny][nx]); f = -1 gives all fields.  `out` may be a
        CUDA tensor (device export) or a host numpy array."""
        shape = ((self.F,) if f < 0 else ()) + (self.G[1], self.G[0])
        dt = 0 if np.dtype(dtype) == np.float64 else 1
        if out is None:
            out = np.empty(shape, dtype=dtype)
        if hasattr(out, "data_ptr"):
            B.check(B.lib().wcs_export_field(self.h, f, out.data_ptr(), 1 if out.is_cuda else 0, dt), self.h)
            if out.is_cuda:
                self.sync()  # a device export is enqueued on the simulation's stream
        else:
            B.check(B.lib().wcs_export_field(self.h, f, out.ctypes.data, 0, dt), self.h)
        return out

    def compressed_bytes(self):
        return B.lib().wcs_compressed_bytes(self.h)

    def resident_bytes(self):
        return B.lib().wcs_resident_bytes(self.h)

    def entropy_code(self):
        """The current records entropy-coded by the library (rANS; bytes)."""
        n = C.c_int64()
        B.check(B.lib().wcs_entropy_code(self.h, None, 0, C.byref(n)), self.h)
        buf = C.create_string_buffer(max(n.value, 1))
        B.check(B.lib().wcs_entropy_code(self.h, buf, n.value, C.byref(n)), self.h)
        return buf.raw[:n.value]

    def survivors(self):
        """Detail coefficients kept in the current state (all patches, fields)."""
        k = B.lib().wcs_survivors(self.h)
        if k < 0:
            B.check(6, self.h)
        return k

    def import_field(self, f, values):
        """Replace field f (-1: all fields, shape (F, ...)) of the current
        state by dense values (numpy float64/float32, or a CUDA tensor) and
        re-encode."""
        if hasattr(values, "data_ptr"):
            import torch
            t = values.contiguous()
            dt = 0 if t.dtype == torch.float64 else 1
            if dt == 1 and t.dtype != torch.float32:
                t = t.to(torch.float32)
            if t.is_cuda:
                torch.cuda.synchronize()
            B.check(B.lib().wcs_import_field(self.h, f, t.data_ptr(), 1 if t.is_cuda else 0, dt), self.h)
            return
        a = np.ascontiguousarray(values)
        if a.dtype != np.float32:
            a = a.astype(np.float64)
        dt = 0 if a.dtype == np.float64 else 1
        B.check(B.lib().wcs_import_field(self.h, f, a.ctypes.data, 0, dt), self.h)

    def _stats_dict(self, s):
        return {"step": s.step, "time": s.time, "field_sum": np.array(s.field_sum[:self.F]), "mass": s.mass,
                "momentum": np.array(s.momentum[:3 if len(self.G) == 3 else 2]), "energy": s.energy, "smax": s.smax,
                "live_bytes": s.live_bytes, "resident_bytes": s.resident_bytes,
                "uncompressed_bytes": s.uncompressed_bytes, "status": s.status,
                "arena_capacity": s.arena_capacity, "arena_reruns": s.arena_reruns,
                "field_sum_lo": np.array(s.field_sum_lo[:self.F])}

    def stats(self):
        s = B.StepStats()
        B.check(B.lib().wcs_stats(self.h, C.byref(s)), self.h)
        return self._stats_dict(s)

    def stats_enqueue(self, slot=0):
        """Queues the statistics of the state the enqueued steps lead to into
        pinned slot `slot` (0..3) without synchronising."""
        B.check(B.lib().wcs_stats_enqueue(self.h, slot), self.h)

    def stats_collect(self, slot=0):
        """Waits for slot `slot` and returns what stats() gave for that step."""
        s = B.StepStats()
        B.check(B.lib().wcs_stats_collect(self.h, slot, C.byref(s)), self.h)
        return self._stats_dict(s)

    def coarse_lo(self):
        """hi + lo coarse storage: the lo parts of the current state,
        (npatch, F, NC1^dims) float32, coarse sample iy NC1 + ix (3-D:
        (iz NC1 + iy) NC1 + ix)."""
        nc = ((self.P >> self.L) + 1) ** len(self.G)
        out = np.zeros((self.npatch, self.F, nc), np.float32)
        B.check(B.lib().wcs_coarse_lo(self.h, out.ctypes.data_as(C.POINTER(C.c_float)), out.size), self.h)
        return out

    def record(self, p):
        n = C.c_int64()
        B.lib().wcs_export_record(self.h, p, None, 0, C.byref(n))
        buf = C.create_string_buffer(max(n.value, 1))
        B.check(B.lib().wcs_export_record(self.h, p, buf, n.value, C.byref(n)), self.h)
        return buf.raw[:n.value]

    @property
    def stream(self):
        return B.lib().wcs_stream(self.h)


class Sim3(Sim):
    """One compressed-patch D3Q19 simulation on a periodic (nz, ny, nx) grid
    (folded BL5/3, FP32 compute)."""

    def __init__(self, nx, ny, nz, P, L, eps, store="bf16", rule="const", tau=0.8, arena_factor=0.0, stream=None,
                 coarse_hilo=False):
        self.scheme, self.P, self.L = "d3q19", P, L
        o = B.Opts()
        o.wavelet, o.rule, o.detail_store, o.compute = B.WAVELET["bl53"], B.RULE[rule], B.STORE[store], B.PREC["f32"]
        o.tau, o.arena_factor = tau, arena_factor
        o.coarse_hilo = int(bool(coarse_hilo))
        o.cuda_stream = _stream_ptr(stream)
        g = B.Grid()
        g.dims = 3
        g.n[0], g.n[1], g.n[2] = nx, ny, nz
        g.periodic_mask = 7
        h = C.c_void_p()
        B.check(B.lib().wcs_create_sim(C.byref(g), B.SCHEME["d3q19"], P, L, eps, C.byref(o), C.byref(h)), None)
        self.h = h
        npatch, nf = C.c_int64(), C.c_int()
        nodes = (C.c_int64 * 3)()
        B.check(B.lib().wcs_shape3(h, C.byref(npatch), C.byref(nf), nodes), h)
        self.npatch, self.F, self.G = npatch.value, nf.value, (nodes[0], nodes[1], nodes[2])

    def export_field(self, f, out=None, dtype=np.float64):
        """Decoded field f ([nz][ny][nx]); f = -1 gives all fields."""
        shape = ((self.F,) if f < 0 else ()) + (self.G[2], self.G[1], self.G[0])
        dt = 0 if np.dtype(dtype) == np.float64 else 1
        if out is None:
            out = np.empty(shape, dtype=dtype)
        if hasattr(out, "data_ptr"):
            B.check(B.lib().wcs_export_field(self.h, f, out.data_ptr(), 1 if out.is_cuda else 0, dt), self.h)
            if out.is_cuda:
                self.sync()  # a device export is enqueued on the simulation's stream
        else:
            B.check(B.lib().wcs_export_field(self.h, f, out.ctypes.data, 0, dt), self.h)
        return out


class Dense:
    """Uncompressed FP32 baseline of the same scheme."""

    def __init__(self, scheme, nx, ny, periodic=(True, True), tau=0.8, cfl=0.4, gamma=1.4, stream=None,
                 velocity=(0.0, 0.0), gravity=9.81, length=1.0):
        o = B.Opts()
        o.tau, o.cfl, o.gamma = tau, cfl, gamma
        o.velocity[0], o.velocity[1], o.gravity, o.length = velocity[0], velocity[1], gravity, length
        o.cuda_stream = _stream_ptr(stream)
        g = _grid(nx, ny, periodic)
        h = C.c_void_p()
        st = B.lib().wcs_dense_create(C.byref(g), B.SCHEME[scheme], C.byref(o), C.byref(h))
        if st != 0:
            raise B.WcsError(st, "dense baseline create failed")
        self.h = h
        self.F = {"d2q9": 9, "euler2d": 4, "transport": 1, "swe": 3}[scheme]
        self.G = tuple(n if per else n + 1 for n, per in zip((nx, ny), periodic))

    def close(self):
        if getattr(self, "h", None):
            B.lib().wcs_dense_destroy(self.h)
            self.h = None

    __del__ = close

    def init_macro(self, fields):
        keep, arr, dev = _field_ptrs(fields)
        st = B.lib().wcs_dense_init_macro(self.h, arr, len(fields), dev)
        if st != 0:
            raise B.WcsError(st, "dense init failed")

    def step(self, n=1):
        st = B.lib().wcs_dense_step(self.h, n)
        if st != 0:
            raise B.WcsError(st, "dense step failed")

    def export_field(self, f, dtype=np.float64):
        out = np.empty((self.G[1], self.G[0]), dtype=dtype)
        st = B.lib().wcs_dense_export_field(self.h, f, out.ctypes.data, 0, 0 if np.dtype(dtype) == np.float64 else 1)
        if st != 0:
            raise B.WcsError(st, "dense export failed")
        return out

    def nbytes(self):
        return B.lib().wcs_dense_bytes(self.h)


class Dense3(Dense):
    """Uncompressed FP32 D3Q19 baseline on a periodic (nz, ny, nx) grid."""

    def __init__(self, nx, ny, nz, tau=0.8, stream=None):
        o = B.Opts()
        o.tau = tau
        o.cuda_stream = _stream_ptr(stream)
        g = B.Grid()
        g.dims = 3
        g.n[0], g.n[1], g.n[2] = nx, ny, nz
        g.periodic_mask = 7
        h = C.c_void_p()
        st = B.lib().wcs_dense_create(C.byref(g), B.SCHEME["d3q19"], C.byref(o), C.byref(h))
        if st != 0:
            raise B.WcsError(st, "dense baseline create failed")
        self.h = h
        self.F = 19
        self.G = (nx, ny, nz)

    def export_field(self, f, out=None, dtype=np.float64):
        """Field f ([nz][ny][nx]); `out` may be a CUDA tensor (device copy)."""
        dt = 0 if np.dtype(dtype) == np.float64 else 1
        if out is None:
            out = np.empty((self.G[2], self.G[1], self.G[0]), dtype=dtype)
        if hasattr(out, "data_ptr"):
            st = B.lib().wcs_dense_export_field(self.h, f, out.data_ptr(), 1 if out.is_cuda else 0, dt)
        else:
            st = B.lib().wcs_dense_export_field(self.h, f, out.ctypes.data, 0, dt)
        if st != 0:
            raise B.WcsError(st, "dense export failed")
        return out
