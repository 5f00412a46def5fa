"""ctypes declarations of libflashmap.so (include/flashmap.h).

The library is built in-tree by paper_2609_19190_gb300/build.py.  Loading
fails loudly when it is missing: there is no CPU or Python fallback.
"""
import ctypes as C
import os

from . import build as _build

FR_OK = 0
STATUS_NAMES = {
    0: "FR_OK", 1: "FR_ERR_INVALID_ARG", 2: "FR_ERR_EMPTY_MASK",
    3: "FR_ERR_TOO_MANY_LEVELS", 4: "FR_ERR_OOM", 5: "FR_ERR_CUDA",
    6: "FR_ERR_TIMEOUT", 7: "FR_ERR_UNSUPPORTED", 8: "FR_ERR_MISMATCH", 9: "FR_ERR_IO",
}

FR_FBN, FR_FBW = 0, 1
FR_ANCHOR_VOI_MIN, FR_ANCHOR_ZERO_FLOOR = 0, 1
FR_NUM_FEATURES = 101
FR_NUM_BENCH_FEATURES = 93  # ids 0..92: the benchmark maps (the default selection)
FR_SCALAR_STDDEV = 101  # scalar extraction only: the standard deviation (no map)
FR_NUM_SCALAR_FEATURES = 102
FR_NUM_DIRECTIONS = 13
FR_H5_NONE, FR_H5_GZIP, FR_H5_LZF = 0, 1, 2


class MapParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("spacing", C.c_double * 3),
        ("disc_mode", C.c_int32), ("bin_count", C.c_int32),
        ("bin_width", C.c_double), ("fbw_anchor", C.c_int32),
        ("kernel_radius", C.c_int32), ("glcm_distance", C.c_int32),
        ("feature_mask", C.c_uint64 * 2),
        ("kurtosis_excess", C.c_int32), ("device", C.c_int32),
        ("mask_on_device", C.c_int32), ("aggregation", C.c_int32),
        ("range_given", C.c_int32), ("range_min", C.c_int32), ("range_max", C.c_int32),
    ]


class Tune(C.Structure):
    _fields_ = [
        ("brick_x", C.c_int32), ("brick_y", C.c_int32), ("brick_z", C.c_int32),
        ("voxels_per_item", C.c_int32), ("consumer_warps", C.c_int32),
        ("stages", C.c_int32), ("ctas_per_sm", C.c_int32),
    ]


class H5Options(C.Structure):
    _fields_ = [
        ("codec", C.c_int32), ("level", C.c_int32), ("shuffle", C.c_int32),
        ("threads", C.c_int32), ("chunk", C.c_int32 * 3),
    ]


class H5Source(C.Structure):
    _fields_ = [
        ("image", C.c_void_p), ("mask", C.c_void_p), ("origin", C.c_double * 3),
        ("source_id", C.c_char_p),
    ]


# Every symbol include/flashmap.h declares, with (restype, argtypes).
_P = C.c_void_p
SIGNATURES = {
    "fr_map_params_init": (None, [C.POINTER(MapParams), C.c_int32, C.c_int32, C.c_int32]),
    "fr_map_plan": (C.c_int, [C.POINTER(MapParams), _P, C.POINTER(Tune), C.POINTER(_P)]),
    "fr_map_run": (C.c_int, [_P, _P, _P, _P]),
    "fr_map_run_host": (C.c_int, [_P, _P, _P, _P]),
    "fr_map_sync_status": (C.c_int, [_P]),
    "fr_plan_query": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                C.POINTER(C.c_size_t)]),
    "fr_plan_voxel_index": (C.c_int, [_P, _P, _P]),
    "fr_plan_levels": (C.c_int, [_P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int32)]),
    "fr_scatter_dense": (C.c_int, [_P, _P, _P, _P]),
    "fr_debug_record_ints": (C.c_int64, [_P, C.c_int32]),
    "fr_debug_matrices": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, _P, _P]),
    "fr_plan_last_kernel_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "fr_batch_last_kernel_ms": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "fr_map_destroy": (None, [_P]),
    "fr_batch_plan": (C.c_int, [C.POINTER(MapParams), C.POINTER(_P), C.c_int32,
                                C.POINTER(Tune), C.POINTER(_P)]),
    "fr_batch_query": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "fr_batch_run": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), _P]),
    "fr_batch_sync_status": (C.c_int, [_P]),
    "fr_batch_destroy": (None, [_P]),
    "fr_scalar_plan": (C.c_int, [C.POINTER(MapParams), _P, C.POINTER(_P)]),
    "fr_scalar_run": (C.c_int, [_P, _P, _P, _P]),
    "fr_scalar_sync_status": (C.c_int, [_P]),
    "fr_scalar_query": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_size_t)]),
    "fr_scalar_destroy": (None, [_P]),
    "fr_voxel_list_noalloc": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int64,
                                        C.POINTER(C.c_int64), C.c_int32, _P]),
    "fr_server_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(Tune),
                                   C.POINTER(_P)]),
    "fr_server_add": (C.c_int, [_P, C.POINTER(MapParams), _P, _P, _P, C.POINTER(C.c_int64)]),
    "fr_server_step": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_int32)]),
    "fr_server_poll": (C.c_int, [_P, C.c_int32, _P, _P, C.c_int32, C.POINTER(C.c_int32)]),
    "fr_server_release": (C.c_int, [_P, C.c_int64]),
    "fr_server_query": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_size_t)]),
    "fr_server_destroy": (None, [_P]),
    "fr_h5_options_init": (C.c_int, [C.POINTER(H5Options)]),
    "fr_h5_write_maps": (C.c_int, [C.c_char_p, C.POINTER(MapParams), C.POINTER(H5Source), _P,
                                   C.c_int32, C.c_int64, _P, C.POINTER(H5Options)]),
    "fr_h5_write_scalar": (C.c_int, [C.c_char_p, C.POINTER(MapParams), C.POINTER(H5Source), _P,
                                     C.c_int32, C.POINTER(H5Options)]),
    "fr_feature_count": (C.c_int32, []),
    "fr_measure_alu_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]),
    "fr_debug_wait_fault": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "fr_scalar_feature_count": (C.c_int32, []),
    "fr_feature_name": (C.c_char_p, [C.c_int32]),
    "fr_status_string": (C.c_char_p, [C.c_int]),
    "fr_direction": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32)]),
}

_lib = None


def library_path():
    return _build.LIB_PATH


def load(build_if_missing=True):
    """Load libflashmap.so (building it first if allowed and missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libflashmap.so is not built (%s); run __graft_entry__.build()" % path)
        _build.build()
    L = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class FlashmapError(RuntimeError):
    def __init__(self, where, status):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, STATUS_NAMES.get(status, "?"), status))


def check(where, status):
    if status != FR_OK:
        raise FlashmapError(where, status)
