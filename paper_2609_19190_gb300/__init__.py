"""GB300-native radiomic spatial mapping.

Thin Python binding of libflashmap.so (include/flashmap.h): argument
marshalling only.  Every step of the mapping (discretisation, VOI list,
window gather, texture matrices, features) runs in the library's sm_103a
kernels; PyTorch supplies device memory and streams.  There is no CPU
fallback: without the built library and a GB300 device the calls raise.

The functions keep the C names:

    p = fr_map_params_init(nx, ny, nz, disc_mode=FR_FBW, bin_width=25.0, ...)
    plan = fr_map_plan(p, mask)                 # mask: torch uint8 (cpu or cuda)
    out = fr_map_run(plan, image)               # image: torch int16 cuda
    fr_map_sync_status(plan)
    fr_map_destroy(plan)
"""
import ctypes as C

from . import _lib
from ._lib import (FR_ANCHOR_VOI_MIN, FR_ANCHOR_ZERO_FLOOR, FR_FBN, FR_FBW,  # noqa: F401
                   FR_H5_GZIP, FR_H5_LZF, FR_H5_NONE, FR_NUM_DIRECTIONS, FR_NUM_FEATURES,
                   FR_NUM_SCALAR_FEATURES, FR_SCALAR_STDDEV,
                   FlashmapError, MapParams, Tune, check)

__all__ = [
    "fr_map_params_init", "fr_map_plan", "fr_map_run", "fr_map_run_host",
    "fr_map_sync_status", "fr_plan_query", "fr_plan_voxel_index", "fr_plan_levels",
    "fr_scatter_dense", "fr_debug_matrices", "fr_map_destroy", "fr_batch_plan",
    "fr_plan_last_kernel_ms", "fr_batch_last_kernel_ms",
    "fr_batch_run", "fr_batch_sync_status", "fr_batch_query", "fr_batch_destroy",
    "fr_feature_names", "fr_direction", "FR_FBN", "FR_FBW", "MapParams", "Tune",
    "FlashmapError", "fr_h5_write_maps", "fr_h5_write_scalar", "fr_debug_wait_fault",
]

FAMILIES = {
    "firstorder": range(0, 18), "glcm": range(18, 42), "glrlm": range(42, 58),
    "glszm": range(58, 74), "gldm": range(74, 88), "ngtdm": range(88, 93),
    # IBSI extras completing Table 2's 101-map default set
    "extras": range(93, 101),
}


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def feature_mask(ids):
    words = [0, 0]
    for f in ids:
        words[f >> 6] |= 1 << (f & 63)
    return words


def fr_map_params_init(nx, ny, nz, **fields):
    """fr_map_params_init plus keyword overrides; `features` (iterable of ids)
    sets the feature mask, `spacing` a 3-tuple."""
    L = _lib.load()
    p = MapParams()
    L.fr_map_params_init(C.byref(p), nx, ny, nz)
    feats = fields.pop("features", None)
    if feats is not None:
        w = feature_mask(feats)
        p.feature_mask[0], p.feature_mask[1] = w[0], w[1]
    sp = fields.pop("spacing", None)
    if sp is not None:
        p.spacing[:] = list(sp)
    vr = fields.pop("value_range", None)  # (min, max) of the discretisation
    if vr is not None:
        p.range_given, p.range_min, p.range_max = 1, int(vr[0]), int(vr[1])
    for k, v in fields.items():
        if not hasattr(p, k):
            raise AttributeError("fr_map_params has no field %r" % k)
        setattr(p, k, v)
    return p


def selected_features(params, n=FR_NUM_FEATURES):
    return [f for f in range(n)
            if (params.feature_mask[f >> 6] >> (f & 63)) & 1]


def _tune(tune):
    if tune is None:
        return None
    if isinstance(tune, Tune):
        return C.byref(tune)
    t = Tune()
    for k, v in dict(tune).items():
        setattr(t, k, int(v))
    return C.byref(t)


class Plan:
    """Handle of an fr_plan (C pointer) plus the parameters it was made with."""

    def __init__(self, handle, params, device):
        self.handle = handle
        self.params = params
        self.device = device
        n_voi, n_rows, nbytes = C.c_int64(), C.c_int32(), C.c_size_t()
        check("fr_plan_query", _lib.load().fr_plan_query(handle, C.byref(n_voi), C.byref(n_rows),
                                                          C.byref(nbytes)))
        self.n_voi, self.n_rows, self.device_bytes = n_voi.value, n_rows.value, nbytes.value
        self.features = selected_features(params)

    def __del__(self):
        try:
            fr_map_destroy(self)
        except Exception:
            pass


def fr_map_plan(params, mask, tune=None):
    """Plan a mapping.  mask: torch uint8 tensor [nz, ny, nx] on the CPU or on
    the plan's CUDA device (or a numpy array, treated as host memory)."""
    torch = _torch()
    L = _lib.load()
    if not isinstance(mask, torch.Tensor):
        mask = torch.from_numpy(mask)
    mask = mask.to(torch.uint8).contiguous()
    params.mask_on_device = 1 if mask.is_cuda else 0
    if mask.is_cuda:
        params.device = mask.device.index or 0
    h = C.c_void_p()
    check("fr_map_plan", L.fr_map_plan(C.byref(params), C.c_void_p(mask.data_ptr()),
                                       _tune(tune), C.byref(h)))
    return Plan(h, params, params.device)


def fr_map_run(plan, image, out=None, stream=None):
    """Map an int16 CUDA image [nz, ny, nx]; returns out [n_rows, n_voi] float32."""
    torch = _torch()
    assert image.is_cuda and image.dtype == torch.int16 and image.is_contiguous()
    if out is None:
        out = torch.empty((plan.n_rows, plan.n_voi), dtype=torch.float32, device=image.device)
    check("fr_map_run", _lib.load().fr_map_run(plan.handle, C.c_void_p(image.data_ptr()),
                                               C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def fr_map_run_host(plan, image, out=None, stream=None):
    """Map a host int16 image (torch CPU tensor, pinned for DMA) into a host
    float32 output; synchronous.  Returns out."""
    torch = _torch()
    assert not image.is_cuda and image.dtype == torch.int16 and image.is_contiguous()
    if out is None:
        out = torch.empty((plan.n_rows, plan.n_voi), dtype=torch.float32).pin_memory()
    check("fr_map_run_host", _lib.load().fr_map_run_host(
        plan.handle, C.c_void_p(image.data_ptr()), C.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


class ScalarPlan:
    """Handle of an fr_scalar (whole-VOI scalar extraction)."""

    def __init__(self, handle, params):
        self.handle = handle
        self.params = params
        n_voi, nf, nbytes = C.c_int64(), C.c_int32(), C.c_size_t()
        check("fr_scalar_query", _lib.load().fr_scalar_query(handle, C.byref(n_voi), C.byref(nf),
                                                              C.byref(nbytes)))
        self.n_voi, self.n_features, self.device_bytes = n_voi.value, nf.value, nbytes.value
        self.features = selected_features(params, FR_NUM_SCALAR_FEATURES)

    def __del__(self):
        try:
            fr_scalar_destroy(self)
        except Exception:
            pass


def fr_scalar_plan(params, mask):
    """Plan a scalar extraction (mask as for fr_map_plan)."""
    torch = _torch()
    L = _lib.load()
    if not isinstance(mask, torch.Tensor):
        mask = torch.from_numpy(mask)
    mask = mask.to(torch.uint8).contiguous()
    params.mask_on_device = 1 if mask.is_cuda else 0
    if mask.is_cuda:
        params.device = mask.device.index or 0
    h = C.c_void_p()
    check("fr_scalar_plan", L.fr_scalar_plan(C.byref(params), C.c_void_p(mask.data_ptr()),
                                             C.byref(h)))
    return ScalarPlan(h, params)


def fr_scalar_run(sp, image, out=None, stream=None):
    """Features of the whole VOI of an int16 CUDA image [nz, ny, nx]; returns
    out [n_features] float64 on the device."""
    torch = _torch()
    assert image.is_cuda and image.dtype == torch.int16 and image.is_contiguous()
    if out is None:
        out = torch.empty((sp.n_features,), dtype=torch.float64, device=image.device)
    check("fr_scalar_run", _lib.load().fr_scalar_run(sp.handle, C.c_void_p(image.data_ptr()),
                                                     C.c_void_p(out.data_ptr()),
                                                     _stream_ptr(stream)))
    return out


def fr_scalar_sync_status(sp):
    check("fr_scalar_sync_status", _lib.load().fr_scalar_sync_status(sp.handle))


def fr_scalar_destroy(sp):
    if getattr(sp, "handle", None):
        _lib.load().fr_scalar_destroy(sp.handle)
        sp.handle = None


def fr_map_sync_status(plan):
    check("fr_map_sync_status", _lib.load().fr_map_sync_status(plan.handle))


def fr_plan_query(plan):
    return plan.n_voi, plan.n_rows, plan.device_bytes


def fr_plan_voxel_index(plan, stream=None):
    torch = _torch()
    idx = torch.empty(plan.n_voi, dtype=torch.int32, device="cuda:%d" % plan.device)
    check("fr_plan_voxel_index", _lib.load().fr_plan_voxel_index(
        plan.handle, C.c_void_p(idx.data_ptr()), _stream_ptr(stream)))
    return idx


def fr_plan_levels(plan):
    """(levels uint8 cuda [nz,ny,nx], Ng, xmin, xmax) of the last run."""
    torch = _torch()
    p = plan.params
    lev = torch.empty((p.nz, p.ny, p.nx), dtype=torch.uint8, device="cuda:%d" % plan.device)
    ng, lo, hi = C.c_int32(), C.c_int32(), C.c_int32()
    torch.cuda.synchronize()
    check("fr_plan_levels", _lib.load().fr_plan_levels(
        plan.handle, C.c_void_p(lev.data_ptr()), C.byref(ng), C.byref(lo), C.byref(hi)))
    return lev, ng.value, lo.value, hi.value


def fr_scatter_dense(plan, out, stream=None):
    torch = _torch()
    p = plan.params
    dense = torch.empty((plan.n_rows, p.nz, p.ny, p.nx), dtype=torch.float32, device=out.device)
    check("fr_scatter_dense", _lib.load().fr_scatter_dense(
        plan.handle, C.c_void_p(out.data_ptr()), C.c_void_p(dense.data_ptr()), _stream_ptr(stream)))
    return dense


def fr_measure_alu_peak(device=0):
    """(int32 add, int32 multiply-add, fp32 FMA) lane operations per second
    measured on the device."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    check("fr_measure_alu_peak", _lib.load().fr_measure_alu_peak(int(device), C.byref(a),
                                                                  C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def fr_debug_wait_fault(plan, item, wait_limit_ns=0):
    """Testing hook of the bounded device waits: later runs of the plan
    leave work item `item`'s halo buffer unfilled (-1: none) and bound every
    wait by wait_limit_ns (0: the default)."""
    check("fr_debug_wait_fault", _lib.load().fr_debug_wait_fault(plan.handle, int(item),
                                                                 int(wait_limit_ns)))


def fr_debug_matrices(plan, image, cols, ng, stream=None):
    """Integer matrices of the listed output columns, as numpy arrays:
    dict of hist [n,ng], glcm [n,13,ng,ng], glrlm [n,13,ng,s], glszm [n,ng,w],
    gldm [n,ng,27], ngtdm_n [n,ng], ngtdm_sl [n,ng] (int64), nv [n]."""
    import numpy as np
    torch = _torch()
    L = _lib.load()
    stride = L.fr_debug_record_ints(plan.handle, ng)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    n = cols.size
    rec = torch.zeros((n, stride), dtype=torch.int32, device=image.device)
    check("fr_debug_matrices", L.fr_debug_matrices(
        plan.handle, C.c_void_p(image.data_ptr()), cols.ctypes.data_as(C.c_void_p), n, ng,
        C.c_void_p(rec.data_ptr()), _stream_ptr(stream)))
    torch.cuda.synchronize()
    r = rec.cpu().numpy()
    s = int(r[0, 1])
    w = int(r[0, 2])
    out = {"nv": r[:, 3].copy()}
    o = 4
    def take(shape):
        nonlocal o
        size = int(np.prod(shape))
        a = r[:, o:o + size].reshape((n,) + tuple(shape))
        o += size
        return a
    out["hist"] = take((ng,))
    out["glcm"] = take((13, ng, ng))
    out["glrlm"] = take((13, ng, s))
    out["glszm"] = take((ng, w))
    out["gldm"] = take((ng, 27))
    out["ngtdm_n"] = take((ng,))
    o = (o + 1) & ~1
    out["ngtdm_sl"] = np.ascontiguousarray(r[:, o:o + 2 * ng]).view(np.int64).reshape(n, ng)
    return out


def fr_plan_last_kernel_ms(plan):
    ms = C.c_float()
    check("fr_plan_last_kernel_ms", _lib.load().fr_plan_last_kernel_ms(plan.handle, C.byref(ms)))
    return ms.value


def fr_batch_last_kernel_ms(batch):
    ms = C.c_float()
    check("fr_batch_last_kernel_ms", _lib.load().fr_batch_last_kernel_ms(batch.handle, C.byref(ms)))
    return ms.value


def fr_map_destroy(plan):
    if getattr(plan, "handle", None):
        _lib.load().fr_map_destroy(plan.handle)
        plan.handle = None


class Batch:
    def __init__(self, handle, params_list):
        self.handle = handle
        self.params = params_list
        L = _lib.load()
        self.n_voi, self.n_rows = [], []
        for i in range(len(params_list)):
            n, r = C.c_int64(), C.c_int32()
            check("fr_batch_query", L.fr_batch_query(handle, i, C.byref(n), C.byref(r)))
            self.n_voi.append(n.value)
            self.n_rows.append(r.value)

    def __del__(self):
        try:
            fr_batch_destroy(self)
        except Exception:
            pass


def fr_batch_plan(params_list, masks, tune=None):
    torch = _torch()
    L = _lib.load()
    n = len(params_list)
    arr = (MapParams * n)()
    keep = []
    ptrs = (C.c_void_p * n)()
    for i, (p, m) in enumerate(zip(params_list, masks)):
        if not isinstance(m, torch.Tensor):
            m = torch.from_numpy(m)
        m = m.to(torch.uint8).contiguous()
        keep.append(m)
        p.mask_on_device = 1 if m.is_cuda else 0
        arr[i] = p
        ptrs[i] = m.data_ptr()
    h = C.c_void_p()
    check("fr_batch_plan", L.fr_batch_plan(arr, ptrs, n, _tune(tune), C.byref(h)))
    return Batch(h, list(params_list))


def fr_batch_run(batch, images, outs=None, stream=None):
    torch = _torch()
    n = len(batch.params)
    if outs is None:
        outs = [torch.empty((batch.n_rows[i], batch.n_voi[i]), dtype=torch.float32,
                            device=images[i].device) for i in range(n)]
    ip = (C.c_void_p * n)(*[im.data_ptr() for im in images])
    op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    check("fr_batch_run", _lib.load().fr_batch_run(batch.handle, ip, op, _stream_ptr(stream)))
    return outs


def fr_batch_sync_status(batch):
    check("fr_batch_sync_status", _lib.load().fr_batch_sync_status(batch.handle))


def fr_batch_query(batch, i):
    return batch.n_voi[i], batch.n_rows[i]


def fr_batch_destroy(batch):
    if getattr(batch, "handle", None):
        _lib.load().fr_batch_destroy(batch.handle)
        batch.handle = None


def fr_voxel_list_noalloc(mask, stream=None):
    """Linear indices of the nonzero voxels of a uint8 CUDA mask [nz, ny, nx]
    (z-major), computed without any device allocation by the library; the
    output tensor is the caller's (allocated here by torch)."""
    torch = _torch()
    assert mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous()
    nz, ny, nx = mask.shape
    with torch.cuda.device(mask.device):
        if stream is None:
            stream = torch.cuda.current_stream(mask.device)
        voi = torch.empty(mask.numel(), dtype=torch.int32, device=mask.device)
        n = C.c_int64()
        check("fr_voxel_list_noalloc", _lib.load().fr_voxel_list_noalloc(
            C.c_void_p(mask.data_ptr()), nx, ny, nz, C.c_void_p(voi.data_ptr()), voi.numel(),
            C.byref(n), mask.device.index or 0, C.c_void_p(stream.cuda_stream)))
    return voi[:n.value]


def fr_feature_names():
    L = _lib.load()
    return [L.fr_feature_name(i).decode() for i in range(L.fr_feature_count())]


def fr_direction(i):
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    check("fr_direction", _lib.load().fr_direction(i, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


_CODECS = {"none": FR_H5_NONE, "gzip": FR_H5_GZIP, "lzf": FR_H5_LZF}


def _h5_args(image, mask, origin, source_id, codec, level, shuffle, threads, chunk):
    import numpy as np
    img = np.ascontiguousarray(_host(image), dtype=np.int16)
    msk = np.ascontiguousarray(_host(mask), dtype=np.uint8)
    src = _lib.H5Source()
    src.image = img.ctypes.data
    src.mask = msk.ctypes.data
    src.origin[:] = [float(v) for v in origin]
    src.source_id = None if source_id is None else str(source_id).encode()
    opt = _lib.H5Options()
    check("fr_h5_options_init", _lib.load().fr_h5_options_init(C.byref(opt)))
    opt.codec = _CODECS[codec]
    opt.level = int(level)
    opt.shuffle = 1 if shuffle else 0
    opt.threads = int(threads)
    opt.chunk[:] = list(chunk) if chunk is not None else [0, 0, 0]
    return img, msk, src, opt


def _host(x):
    import numpy as np
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def fr_h5_write_maps(path, params, image, mask, maps, voxel_index, origin=(0.0, 0.0, 0.0),
                     source_id=None, codec="gzip", level=4, shuffle=True, threads=0,
                     chunk=None):
    """Write one spatial extraction to an HDF5 file (host side).  image / mask:
    [nz][ny][nx] int16 / uint8; maps: float32 [rows][n_voi] (fr_map_run's
    output, cpu or cuda); voxel_index: int32 [n_voi] (fr_plan_voxel_index)."""
    import numpy as np
    img, msk, src, opt = _h5_args(image, mask, origin, source_id, codec, level, shuffle, threads,
                                  chunk)
    m = np.ascontiguousarray(_host(maps), dtype=np.float32)
    vi = np.ascontiguousarray(_host(voxel_index), dtype=np.int32)
    check("fr_h5_write_maps", _lib.load().fr_h5_write_maps(
        str(path).encode(), C.byref(params), C.byref(src), C.c_void_p(m.ctypes.data),
        m.shape[0], m.shape[1], C.c_void_p(vi.ctypes.data), C.byref(opt)))


def fr_h5_write_scalar(path, params, image, mask, values, origin=(0.0, 0.0, 0.0),
                       source_id=None, codec="gzip", level=4, shuffle=True, threads=0,
                       chunk=None):
    """Write one scalar extraction (float64 values in feature-id order, as
    fr_scalar_run gives) to an HDF5 file (host side)."""
    import numpy as np
    img, msk, src, opt = _h5_args(image, mask, origin, source_id, codec, level, shuffle, threads,
                                  chunk)
    v = np.ascontiguousarray(_host(values), dtype=np.float64)
    check("fr_h5_write_scalar", _lib.load().fr_h5_write_scalar(
        str(path).encode(), C.byref(params), C.byref(src), C.c_void_p(v.ctypes.data), v.size,
        C.byref(opt)))
