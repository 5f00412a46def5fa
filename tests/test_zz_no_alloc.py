"""The allocation-free entry point fr_voxel_list_noalloc, called through the C
ABI and checked against the planned entry point's voxel list
(fr_plan_voxel_index) on two calls in a row.

The entry point serves callers that cannot allocate device memory (their
memory belongs to another allocator's pool, or they must not allocate while
running): it uses only the library's fixed static scratch.  The output is
integer, so the check is exact.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu


def _call(L, mask_dev, nx, ny, nz, voi, capacity, device=0):
    import torch
    n = C.c_int64(-1)
    stream = torch.cuda.current_stream()
    rc = L.fr_voxel_list_noalloc(C.c_void_p(mask_dev.data_ptr()), nx, ny, nz,
                                 C.c_void_p(voi.data_ptr()), capacity, C.byref(n), device,
                                 C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, n.value


def test_noalloc_voxel_list_matches_planned_list_on_two_calls():
    import torch

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import _lib
    L = _lib.load()
    _, tiny_mask = synth.tiny(seed=1)
    shape = (23, 31, 29)  # odd extents, not a multiple of the warp width
    ell = synth.ellipsoid(shape, (14.0, 15.0, 11.0), (13.0, 11.0, 9.5))
    for mask in (tiny_mask, ell):  # two calls in a row, different sizes
        nz, ny, nx = mask.shape
        plan = fm.fr_map_plan(fm.fr_map_params_init(nx, ny, nz), torch.from_numpy(mask))
        ref = fm.fr_plan_voxel_index(plan)
        mdev = torch.from_numpy(mask).cuda()
        voi = torch.full((mask.size,), -1, dtype=torch.int32, device="cuda")
        rc, n = _call(L, mdev, nx, ny, nz, voi, voi.numel())
        assert rc == 0
        assert n == plan.n_voi == int(mask.sum())
        assert torch.equal(voi[:n], ref)
        assert bool((voi[n:] == -1).all())
        assert np.array_equal(voi[:n].cpu().numpy(), np.flatnonzero(mask.reshape(-1)))


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch

    from paper_2609_19190_gb300 import _lib
    L = _lib.load()
    # more rows (ny * nz) than the static scratch holds: refused before any work
    mask = torch.ones((500, 600, 1), dtype=torch.uint8, device="cuda")
    voi = torch.full((16,), -1, dtype=torch.int32, device="cuda")
    rc, _ = _call(L, mask, 1, 600, 500, voi, voi.numel())
    assert rc == 7
    assert bool((voi == -1).all())
    # an output too small: the count is reported, the output left untouched
    mask = torch.ones((4, 4, 4), dtype=torch.uint8, device="cuda")
    rc, n = _call(L, mask, 4, 4, 4, voi, 10)
    assert rc == 1 and n == 64
    assert bool((voi == -1).all())


def test_noalloc_allocates_nothing_and_handles_edges():
    # after a first call (which looks up the static scratch once), further
    # calls leave the device's free memory unchanged: the output is the
    # caller's and the scratch is the static array
    import torch

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import _lib
    L = _lib.load()
    mask = torch.from_numpy(synth.tiny(seed=1)[1]).cuda()
    nz, ny, nx = mask.shape
    voi = torch.full((mask.numel(),), -1, dtype=torch.int32, device="cuda")
    rc, n = _call(L, mask, nx, ny, nz, voi, voi.numel())
    assert rc == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rc, n2 = _call(L, mask, nx, ny, nz, voi, voi.numel())
        assert rc == 0 and n2 == n
    assert torch.cuda.mem_get_info()[0] == free0
    # a capacity of exactly n is enough
    exact = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rc, n3 = _call(L, mask, nx, ny, nz, exact, n)
    assert rc == 0 and n3 == n and torch.equal(exact, voi[:n])
    # an empty mask: zero voxels, the output untouched
    empty = torch.zeros((5, 6, 7), dtype=torch.uint8, device="cuda")
    out = torch.full((8,), -1, dtype=torch.int32, device="cuda")
    rc, n0 = _call(L, empty, 7, 6, 5, out, out.numel())
    assert rc == 0 and n0 == 0 and bool((out == -1).all())
    # the Python wrapper gives the same list
    assert torch.equal(fm.fr_voxel_list_noalloc(mask), voi[:n])
