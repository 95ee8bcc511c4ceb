"""Batches of independent simulations and the patch-size autotuner (C-ABI
wrappers: the batching, graph capture and timing run in the library)."""
import ctypes as C

import numpy as np

from . import _lib as B
from .sim import Sim, _field_ptrs, _grid, _stream_ptr


class Batch:
    """Advances many initialised simulations (same stream, same step) with one
    graph launch per six steps."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        st = B.lib().wcs_batch_create(arr, len(self.sims), C.byref(h))
        if st != 0:
            raise B.WcsError(st, B.lib().wcs_batch_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            B.lib().wcs_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def step(self, n=1):
        st = B.lib().wcs_batch_step(self.h, n)
        if st != 0:
            raise B.WcsError(st, B.lib().wcs_batch_last_error(self.h).decode())

    def sync(self):
        st = B.lib().wcs_batch_sync(self.h)
        if st != 0:
            raise B.WcsError(st, B.lib().wcs_batch_last_error(self.h).decode())

    def launches_per_step(self):
        """(kernel launches per step, grid of the merged launch or 0)."""
        n, g = C.c_int(), C.c_int()
        B.check(B.lib().wcs_batch_launches_per_step(self.h, C.byref(n), C.byref(g)), None)
        return n.value, g.value

    def tune_launch(self, grids, steps=6):
        """Times each candidate grid of the merged launch and keeps the
        fastest; returns the ms per step of each (advances the batch)."""
        n = len(grids)
        ms = (C.c_double * n)()
        st = B.lib().wcs_batch_tune_launch(self.h, (C.c_int * n)(*grids), n, steps, ms)
        if st != 0:
            raise B.WcsError(st, B.lib().wcs_batch_last_error(self.h).decode())
        return list(ms)


def autotune(scheme, wavelet, nx, ny, eps, fields, candidates=((64, 4), (32, 3)), prec="f32", store="bf16",
             rule="const", periodic=(True, True), tau=0.8, cfl=0.4, gamma=1.4, steps=20, stream=None):
    """Index of the fastest (P, L) candidate on these initial fields, and the
    measured ms per step of each (negative: not runnable)."""
    o = B.Opts()
    o.wavelet, o.rule, o.detail_store, o.compute = B.WAVELET[wavelet], B.RULE[rule], B.STORE[store], B.PREC[prec]
    o.tau, o.cfl, o.gamma, o.arena_factor = tau, cfl, gamma, 0.0
    o.cuda_stream = _stream_ptr(stream)
    g = _grid(nx, ny, periodic)
    n = len(candidates)
    P = (C.c_int * n)(*[c[0] for c in candidates])
    L = (C.c_int * n)(*[c[1] for c in candidates])
    keep, arr, dev = _field_ptrs(fields)
    best = C.c_int(-1)
    ms = (C.c_double * n)()
    B.check(B.lib().wcs_autotune(C.byref(g), B.SCHEME[scheme], C.byref(o), eps, P, L, n, arr, len(fields), dev, steps,
                                 C.byref(best), ms), None)
    return best.value, list(ms)
