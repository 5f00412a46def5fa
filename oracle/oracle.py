"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this
module.  It loads oracle/lib/liboracle.so (building it with g++ when it is
missing) and wraps each C entry point with numpy arrays.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

NUM_FEATURES = 101
NUM_SCALAR_FEATURES = 102
NUM_BENCH = 93  # ids 0..92: the spatial benchmark set
NUM_DIRS = 13
FBN, FBW = 0, 1
ANCHOR_VOI_MIN, ANCHOR_ZERO_FLOOR = 0, 1
AGG_AVERAGE, AGG_MERGED = 0, 1


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("spacing", C.c_double * 3),
        ("disc_mode", C.c_int32), ("bin_count", C.c_int32),
        ("bin_width", C.c_double), ("fbw_anchor", C.c_int32),
        ("radius", C.c_int32), ("distance", C.c_int32),
        ("kurtosis_excess", C.c_int32), ("aggregation", C.c_int32),
        ("range_given", C.c_int32), ("range_min", C.c_int32), ("range_max", C.c_int32),
    ]


def make_params(shape, *, disc_mode=FBN, bin_count=16, bin_width=25.0,
                fbw_anchor=ANCHOR_VOI_MIN, radius=1, distance=1,
                spacing=(1.0, 1.0, 1.0), kurtosis_excess=1, aggregation=0, value_range=None):
    nz, ny, nx = shape
    p = Params()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.spacing[:] = list(spacing)
    p.disc_mode, p.bin_count, p.bin_width = disc_mode, bin_count, bin_width
    p.fbw_anchor, p.radius, p.distance = fbw_anchor, radius, distance
    p.kurtosis_excess = kurtosis_excess
    p.aggregation = aggregation
    if value_range is not None:
        p.range_given, p.range_min, p.range_max = 1, int(value_range[0]), int(value_range[1])
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.fro_feature_name.restype = C.c_char_p
        L.fro_feature_name.argtypes = [C.c_int32]
        L.fro_discretise.argtypes = [P(Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                     P(C.c_int32), P(C.c_int32), P(C.c_int32)]
        L.fro_map_voxels.argtypes = [P(Params), C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_void_p, C.c_int64, C.c_void_p, C.c_int32]
        L.fro_matrices.argtypes = [P(Params), C.c_void_p, C.c_int32, C.c_int64] + [C.c_void_p] * 7
        L.fro_scalar.argtypes = [P(Params), C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.fro_glcm_features.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.fro_glrlm_features.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p]
        L.fro_glszm_features.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p]
        L.fro_gldm_features.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
        L.fro_ngtdm_features.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.fro_firstorder_features.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                              C.c_double, C.c_int32, C.c_void_p]
        L.fro_glcm_mcc.restype = C.c_double
        L.fro_glcm_mcc.argtypes = [C.c_void_p, C.c_int32]
        L.fro_direction.argtypes = [C.c_int32] + [P(C.c_int32)] * 3
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def feature_names():
    L = lib()
    return [L.fro_feature_name(i).decode() for i in range(NUM_FEATURES)]


def scalar_feature_names():
    L = lib()
    return [L.fro_feature_name(i).decode() for i in range(NUM_SCALAR_FEATURES)]


def directions():
    L = lib()
    out = []
    for i in range(NUM_DIRS):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        L.fro_direction(i, C.byref(a), C.byref(b), C.byref(c))
        out.append((a.value, b.value, c.value))
    return out


class OracleError(RuntimeError):
    pass


def discretise(params, image, mask):
    """Returns (levels uint8 [Z,Y,X], Ng, xmin, xmax)."""
    image = np.ascontiguousarray(image, dtype=np.int16)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    levels = np.zeros(image.shape, dtype=np.uint8)
    ng, xmin, xmax = C.c_int32(), C.c_int32(), C.c_int32()
    rc = lib().fro_discretise(C.byref(params), _ptr(image), _ptr(mask), _ptr(levels),
                              C.byref(ng), C.byref(xmin), C.byref(xmax))
    if rc != 0:
        raise OracleError("fro_discretise failed with code %d" % rc)
    return levels, ng.value, xmin.value, xmax.value


def map_voxels(params, image, levels, ng, voxels, nthreads=0):
    """Feature maps [101, n] (float64) at the listed linear voxel indices."""
    image = np.ascontiguousarray(image, dtype=np.int16)
    levels = np.ascontiguousarray(levels, dtype=np.uint8)
    vox = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty((NUM_FEATURES, vox.size), dtype=np.float64)
    rc = lib().fro_map_voxels(C.byref(params), _ptr(image), _ptr(levels), ng, _ptr(vox),
                              vox.size, _ptr(out), int(nthreads))
    if rc != 0:
        raise OracleError("fro_map_voxels failed with code %d" % rc)
    return out


def map_volume(params, image, mask, nthreads=0):
    """Discretise and map every VOI voxel (z-major order).

    Returns (maps [101, n_voi], voxel linear indices, levels, Ng)."""
    levels, ng, _, _ = discretise(params, image, mask)
    vox = np.flatnonzero(np.asarray(mask).reshape(-1)).astype(np.int64)
    return map_voxels(params, image, levels, ng, vox, nthreads), vox, levels, ng


def scalar(params, image, levels, ng):
    """The 102 features of the whole VOI (scalar extraction): the 101 map
    features and the scalar-only standard deviation (id 101)."""
    image = np.ascontiguousarray(image, dtype=np.int16)
    levels = np.ascontiguousarray(levels, dtype=np.uint8)
    out = np.empty(NUM_SCALAR_FEATURES)
    rc = lib().fro_scalar(C.byref(params), _ptr(image), _ptr(levels), ng, _ptr(out))
    if rc != 0:
        raise OracleError("fro_scalar failed with code %d" % rc)
    return out


def matrices(params, levels, ng, voxel):
    """Dense integer matrices of one voxel's sub-VOI, as a dict."""
    s = 2 * params.radius + 1
    w = s ** 3
    levels = np.ascontiguousarray(levels, dtype=np.uint8)
    out = {
        "glcm": np.zeros((NUM_DIRS, ng, ng), np.int32),
        "glrlm": np.zeros((NUM_DIRS, ng, s), np.int32),
        "glszm": np.zeros((ng, w), np.int32),
        "gldm": np.zeros((ng, 27), np.int32),
        "ngtdm_n": np.zeros(ng, np.int32),
        "ngtdm_sl": np.zeros(ng, np.int64),
        "hist": np.zeros(ng, np.int32),
    }
    rc = lib().fro_matrices(C.byref(params), _ptr(levels), ng, int(voxel),
                            *[_ptr(out[k]) for k in ("glcm", "glrlm", "glszm", "gldm",
                                                     "ngtdm_n", "ngtdm_sl", "hist")])
    if rc != 0:
        raise OracleError("fro_matrices failed with code %d" % rc)
    return out


def glcm_features(counts):
    counts = np.ascontiguousarray(counts, dtype=np.float64)
    out = np.empty(24)
    lib().fro_glcm_features(_ptr(counts), counts.shape[0], _ptr(out))
    return out


def glrlm_features(counts, n_vox):
    counts = np.ascontiguousarray(counts, dtype=np.float64)
    out = np.empty(16)
    lib().fro_glrlm_features(_ptr(counts), counts.shape[0], counts.shape[1], float(n_vox), _ptr(out))
    return out


def glszm_features(counts, n_vox):
    counts = np.ascontiguousarray(counts, dtype=np.float64)
    out = np.empty(16)
    lib().fro_glszm_features(_ptr(counts), counts.shape[0], counts.shape[1], float(n_vox), _ptr(out))
    return out


def gldm_features(counts):
    counts = np.ascontiguousarray(counts, dtype=np.float64)
    out = np.empty(14)
    lib().fro_gldm_features(_ptr(counts), counts.shape[0], counts.shape[1], _ptr(out))
    return out


def ngtdm_features(n, s):
    n = np.ascontiguousarray(n, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty(5)
    lib().fro_ngtdm_features(_ptr(n), _ptr(s), n.size, _ptr(out))
    return out


def firstorder_features(x, g, ng, voxel_volume=1.0, kurtosis_excess=1):
    x = np.ascontiguousarray(x, dtype=np.int32)
    g = np.ascontiguousarray(g, dtype=np.int32)
    out = np.empty(18)
    lib().fro_firstorder_features(_ptr(x), _ptr(g), x.size, ng, float(voxel_volume),
                                  int(kurtosis_excess), _ptr(out))
    return out


def glcm_mcc(counts):
    counts = np.ascontiguousarray(counts, dtype=np.float64)
    return lib().fro_glcm_mcc(_ptr(counts), counts.shape[0])
