"""GPU tests of the C-ABI entry points beyond plain parity: determinism,
host-buffer runs, dense scatter, batching (bit-identical to the plain path),
launch-shape independence, feature subsets, error statuses and edge cases."""
import numpy as np
import pytest

import gpu_helpers as H
import parity
from oracle import oracle as O
from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu

ALL = list(range(101))  # the 93 benchmark maps and the 8 IBSI extras (Table 2)


def _fm():
    import paper_2609_19190_gb300 as fm
    return fm


def _torch():
    import torch
    return torch


def _ct(seed=2, shape=(20, 30, 33), semi=(14.0, 12.0, 8.0)):
    img = synth.ct_like(shape, seed)
    mask = synth.ellipsoid(shape, ((shape[2] - 1) / 2, (shape[1] - 1) / 2, (shape[0] - 1) / 2), semi)
    return img, mask


def _plan_run(img, mask, tune=None, **kw):
    fm, torch = _fm(), _torch()
    nz, ny, nx = img.shape
    p = fm.fr_map_params_init(nx, ny, nz, **kw)
    plan = fm.fr_map_plan(p, torch.from_numpy(mask), tune=tune)
    out = fm.fr_map_run(plan, torch.from_numpy(img).cuda())
    fm.fr_map_sync_status(plan)
    return plan, out


def test_two_runs_are_bit_identical():
    img, mask = _ct()
    plan, a = _plan_run(img, mask, disc_mode=1, bin_width=25.0, kernel_radius=2)
    b = _fm().fr_map_run(plan, _torch().from_numpy(img).cuda())
    assert _torch().equal(a.view(_torch().int32), b.view(_torch().int32))


def test_host_buffer_run_matches_device_run():
    torch, fm = _torch(), _fm()
    img, mask = _ct(seed=3)
    plan, dev_out = _plan_run(img, mask, disc_mode=0, bin_count=32, kernel_radius=1)
    host_img = torch.from_numpy(img).pin_memory()
    host_out = fm.fr_map_run_host(plan, host_img)
    assert torch.equal(host_out.view(torch.int32), dev_out.cpu().view(torch.int32))


def test_scatter_dense_places_columns_and_nan():
    torch, fm = _torch(), _fm()
    img, mask = _ct(seed=4)
    plan, out = _plan_run(img, mask, disc_mode=1, bin_width=25.0, kernel_radius=1,
                          features=[0, 18, 92])
    dense = fm.fr_scatter_dense(plan, out).cpu().numpy()
    vox = np.flatnonzero(mask.reshape(-1))
    flat = dense.reshape(3, -1)
    np.testing.assert_array_equal(flat[:, vox], out.cpu().numpy())
    outside = np.ones(flat.shape[1], bool)
    outside[vox] = False
    assert np.all(np.isnan(flat[:, outside]))


def test_feature_subset_rows_equal_full_rows():
    torch = _torch()
    img, mask = _ct(seed=5)
    feats = [0, 41, 50, 63, 80, 92]
    _, full = _plan_run(img, mask, disc_mode=1, bin_width=25.0, kernel_radius=2)
    _, sub = _plan_run(img, mask, disc_mode=1, bin_width=25.0, kernel_radius=2, features=feats)
    assert torch.equal(sub.view(torch.int32), full[feats].view(torch.int32))


@pytest.mark.parametrize("tune", [
    dict(brick_x=16, brick_y=8, brick_z=8, voxels_per_item=64, consumer_warps=8, stages=2),
    dict(brick_x=4, brick_y=2, brick_z=2, voxels_per_item=5, consumer_warps=3, stages=3),
    dict(brick_x=32, brick_y=16, brick_z=4, voxels_per_item=1024, consumer_warps=16, stages=1),
])
def test_launch_shape_does_not_change_results(tune):
    torch = _torch()
    img, mask = _ct(seed=6)
    kw = dict(disc_mode=1, bin_width=25.0, kernel_radius=2)
    _, ref = _plan_run(img, mask, **kw)
    _, got = _plan_run(img, mask, tune=tune, **kw)
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))


def test_batch_is_bit_identical_to_plain_and_replays():
    torch, fm = _torch(), _fm()
    cases = [
        (*_ct(seed=7), dict(disc_mode=0, bin_count=16, kernel_radius=1)),
        (*_ct(seed=8, shape=(16, 25, 21), semi=(9.0, 11.0, 7.0)),
         dict(disc_mode=1, bin_width=25.0, kernel_radius=3)),
        (*_ct(seed=9), dict(disc_mode=0, bin_count=64, kernel_radius=2, features=list(range(18, 42)))),
    ]
    params, masks, imgs, refs = [], [], [], []
    for img, mask, kw in cases:
        nz, ny, nx = img.shape
        params.append(fm.fr_map_params_init(nx, ny, nz, **kw))
        masks.append(torch.from_numpy(mask))
        imgs.append(torch.from_numpy(img).cuda())
        _, ref = _plan_run(img, mask, **kw)
        refs.append(ref)
    b = fm.fr_batch_plan(params, masks)
    for rep in range(2):
        outs = fm.fr_batch_run(b, imgs)
        fm.fr_batch_sync_status(b)
        for o, r in zip(outs, refs):
            assert torch.equal(o.view(torch.int32), r.view(torch.int32))
    fm.fr_batch_destroy(b)


def test_single_voxel_voi_and_isolated_voxels():
    img, mask = _ct(seed=10)
    m1 = np.zeros_like(mask)
    m1[10, 15, 16] = 1
    m1[2, 2, 2] = 1
    m1[2, 2, 4] = 1  # two voxels two apart: each window holds one or two
    got, plan, feats = H.gpu_map(img, m1, features=ALL, disc_mode=0, bin_count=8,
                                 kernel_radius=1)
    ref, _, _, _ = H.oracle_map(img, m1, disc_mode=0, bin_count=8, kernel_radius=1)
    parity.assert_close(got, ref[feats], [O.feature_names()[f] for f in feats])


def test_voi_on_the_borders_odd_extent_radius3():
    rng = np.random.default_rng(11)
    img = rng.integers(-200, 200, size=(9, 11, 13)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.8).astype(np.uint8)
    kw = dict(disc_mode=0, bin_count=12, kernel_radius=3)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    ref, _, _, _ = H.oracle_map(img, mask, **kw)
    parity.assert_close(got, ref[feats], [O.feature_names()[f] for f in feats])


def test_max_radius_seven():
    rng = np.random.default_rng(12)
    img = rng.integers(0, 40, size=(15, 16, 17)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.6).astype(np.uint8)
    kw = dict(disc_mode=0, bin_count=6, kernel_radius=7)
    vox = synth.sample_voxels(mask, 150, seed=1)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    cols = np.searchsorted(np.flatnonzero(mask.reshape(-1)), vox)
    ref, _, _, _ = H.oracle_map(img, mask, voxels=vox, **kw)
    parity.assert_close(got[:, cols], ref[feats], [O.feature_names()[f] for f in feats])


def test_glcm_distance_two_and_zero_floor_anchor():
    img, mask = _ct(seed=13)
    kw = dict(disc_mode=1, bin_width=20.0, fbw_anchor=1, kernel_radius=2, glcm_distance=2)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    ref, _, _, _ = H.oracle_map(img, mask, **kw)
    parity.assert_close(got, ref[feats], [O.feature_names()[f] for f in feats])


def test_constant_and_two_level_images():
    img = np.full((10, 10, 10), 37, np.int16)
    mask = np.zeros_like(img, dtype=np.uint8)
    mask[1:9, 1:9, 1:9] = 1
    for im in (img, np.where((np.indices(img.shape).sum(0) % 2) == 0, 10, 90).astype(np.int16)):
        got, plan, feats = H.gpu_map(im, mask, features=ALL, disc_mode=0, bin_count=4,
                                     kernel_radius=2)
        ref, _, _, _ = H.oracle_map(im, mask, disc_mode=0, bin_count=4, kernel_radius=2)
        parity.assert_close(got, ref[feats], [O.feature_names()[f] for f in feats])


def test_many_levels_use_the_slab_and_match():
    # FBN 255 on uniform noise: windows with far more than 24 levels
    rng = np.random.default_rng(14)
    img = rng.integers(0, 5000, size=(10, 12, 12)).astype(np.int16)
    mask = np.ones(img.shape, np.uint8)
    kw = dict(disc_mode=0, bin_count=255, kernel_radius=2)
    vox = synth.sample_voxels(mask, 200, seed=2)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    ref, _, _, _ = H.oracle_map(img, mask, voxels=vox, **kw)
    cols = np.searchsorted(np.flatnonzero(mask.reshape(-1)), vox)
    parity.assert_close(got[:, cols], ref[feats], [O.feature_names()[f] for f in feats])


def test_too_many_levels_is_reported():
    fm, torch = _fm(), _torch()
    img = np.zeros((4, 4, 4), np.int16)
    img[0, 0, 0] = 3000
    mask = np.ones(img.shape, np.uint8)
    p = fm.fr_map_params_init(4, 4, 4, disc_mode=fm.FR_FBW, bin_width=1.0)
    plan = fm.fr_map_plan(p, torch.from_numpy(mask))
    fm.fr_map_run(plan, torch.from_numpy(img).cuda())
    with pytest.raises(fm.FlashmapError) as e:
        fm.fr_map_sync_status(plan)
    assert e.value.status == 3


def test_empty_mask_is_reported():
    fm, torch = _fm(), _torch()
    p = fm.fr_map_params_init(4, 4, 4)
    with pytest.raises(fm.FlashmapError) as e:
        fm.fr_map_plan(p, torch.zeros((4, 4, 4), dtype=torch.uint8))
    assert e.value.status == 2
