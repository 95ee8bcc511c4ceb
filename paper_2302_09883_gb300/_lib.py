"""ctypes binding of libwcsim.so (include/wcsim.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels.  There is no
fallback: if the shared library is missing the import of a simulation fails.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwcsim.so")

SCHEME = {"d2q9": 0, "d3q19": 1, "euler2d": 2, "transport": 3, "swe": 4}
WAVELET = {"bl53": 0, "haar": 1, "cdf97": 2}
RULE = {"const": 0, "accum": 1, "capped": 2}
STORE = {"f64": 0, "f32": 1, "bf16": 2, "i8": 3}
PREC = {"f64": 0, "f32": 1}
STATUS = {0: "OK", 1: "E_ARG", 2: "E_OOM", 3: "E_ARENA_FULL", 4: "E_NAN", 5: "E_TIMEOUT", 6: "E_CUDA",
          7: "E_UNSUPPORTED"}


class WcsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Grid(C.Structure):
    _fields_ = [("dims", C.c_int), ("n", C.c_int64 * 3), ("periodic_mask", C.c_uint32)]


class Opts(C.Structure):
    _fields_ = [("wavelet", C.c_int), ("rule", C.c_int), ("detail_store", C.c_int), ("compute", C.c_int),
                ("tau", C.c_double), ("cfl", C.c_double), ("gamma", C.c_double), ("arena_factor", C.c_double),
                ("cuda_stream", C.c_void_p), ("velocity", C.c_double * 2), ("gravity", C.c_double),
                ("length", C.c_double), ("coarse_hilo", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("time", C.c_double), ("field_sum", C.c_double * 19), ("mass", C.c_double),
                ("momentum", C.c_double * 3), ("energy", C.c_double), ("smax", C.c_double),
                ("live_bytes", C.c_int64), ("resident_bytes", C.c_int64), ("uncompressed_bytes", C.c_int64),
                ("status", C.c_uint32), ("arena_capacity", C.c_int64), ("arena_reruns", C.c_int64),
                ("field_sum_lo", C.c_double * 19)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libwcsim.so is not built (run __graft_entry__.build() or "
                               "python paper_2302_09883_gb300/build.py); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        L.wcs_create_sim.argtypes = [C.POINTER(Grid), i32, i32, i32, C.c_double, C.POINTER(Opts), C.POINTER(vp)]
        L.wcs_destroy.argtypes = [vp]
        L.wcs_init_macro.argtypes = [vp, C.POINTER(vp), i32, i32]
        L.wcs_step.argtypes = [vp, i64]
        L.wcs_sync.argtypes = [vp]
        L.wcs_export_field.argtypes = [vp, i32, vp, i32, i32]
        L.wcs_export_field_noalloc.argtypes = [vp, i32, vp, i32]
        L.wcs_compressed_bytes.restype = i64
        L.wcs_compressed_bytes.argtypes = [vp]
        L.wcs_resident_bytes.restype = i64
        L.wcs_resident_bytes.argtypes = [vp]
        L.wcs_import_field.argtypes = [vp, i32, vp, i32, i32]
        L.wcs_entropy_code.argtypes = [vp, vp, i64, C.POINTER(i64)]
        L.wcs_survivors.restype = i64
        L.wcs_survivors.argtypes = [vp]
        L.wcs_stats.argtypes = [vp, C.POINTER(StepStats)]
        L.wcs_stats_enqueue.argtypes = [vp, i32]
        L.wcs_stats_collect.argtypes = [vp, i32, C.POINTER(StepStats)]
        L.wcs_export_record.argtypes = [vp, i64, vp, i64, C.POINTER(i64)]
        L.wcs_coarse_lo.argtypes = [vp, C.POINTER(C.c_float), i64]
        L.wcs_patch_config.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.wcs_shape.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]
        L.wcs_shape3.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i64)]
        L.wcs_stream.restype = vp
        L.wcs_stream.argtypes = [vp]
        L.wcs_last_error.restype = C.c_char_p
        L.wcs_last_error.argtypes = [vp]
        L.wcs_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp)]
        L.wcs_batch_destroy.argtypes = [vp]
        L.wcs_batch_step.argtypes = [vp, i64]
        L.wcs_batch_sync.argtypes = [vp]
        L.wcs_batch_launches_per_step.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.wcs_batch_tune_launch.argtypes = [vp, C.POINTER(i32), i32, i32, C.POINTER(C.c_double)]
        L.wcs_batch_last_error.restype = C.c_char_p
        L.wcs_batch_last_error.argtypes = [vp]
        L.wcs_autotune.argtypes = [C.POINTER(Grid), i32, C.POINTER(Opts), C.c_double, C.POINTER(i32), C.POINTER(i32),
                                   i32, C.POINTER(vp), i32, i32, i32, C.POINTER(i32), C.POINTER(C.c_double)]
        fp = C.POINTER(C.c_float)
        L.wcs_features_labels.argtypes = [vp, i32, i64, i64, i32, i32, i32, C.c_double, vp, vp, vp]
        L.wcs_features_labels3.argtypes = [vp, i32, i64, i64, i64, i32, i32, C.c_double, vp, vp, vp]
        L.wcs_mlp_create.argtypes = [i32, C.POINTER(vp)]
        L.wcs_mlp_destroy.argtypes = [vp]
        L.wcs_mlp_nparam.argtypes = [vp]
        L.wcs_mlp_set_weights.argtypes = [vp, fp]
        L.wcs_mlp_get_weights.argtypes = [vp, fp]
        L.wcs_mlp_grad.argtypes = [vp, vp, vp, i32, fp, fp]
        L.wcs_mlp_train.argtypes = [vp, vp, vp, i32, C.POINTER(i32), i32, i32, C.c_float, fp]
        L.wcs_mlp_fit.argtypes = [vp, vp, vp, i32, C.POINTER(i32), i32, i32, C.c_float, C.c_double, fp,
                                  C.POINTER(C.c_double)]
        L.wcs_mlp_forward.argtypes = [vp, vp, i32, vp]
        L.wcs_sim_use_mlp.argtypes = [vp, vp, C.c_double, C.c_double]
        L.wcs_sim_set_patch_eps.argtypes = [vp, C.POINTER(C.c_double)]
        L.wcs_sim_patch_data.argtypes = [vp, fp, C.POINTER(C.c_double)]
        L.wcs_dense_create.argtypes = [C.POINTER(Grid), i32, C.POINTER(Opts), C.POINTER(vp)]
        L.wcs_dense_destroy.argtypes = [vp]
        L.wcs_dense_init_macro.argtypes = [vp, C.POINTER(vp), i32, i32]
        L.wcs_dense_step.argtypes = [vp, i64]
        L.wcs_dense_export_field.argtypes = [vp, i32, vp, i32, i32]
        L.wcs_dense_bytes.restype = i64
        L.wcs_dense_bytes.argtypes = [vp]
        _lib = L
    return _lib


def check(status, handle=None):
    if status != 0:
        msg = lib().wcs_last_error(handle)
        raise WcsError(status, msg.decode() if msg else "")
