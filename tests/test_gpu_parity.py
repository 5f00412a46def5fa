"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Integer outputs (gray levels, VOI list, every texture-matrix count) must be
bit-exact; float maps within max(1e-6, 1e-4 |oracle|) with identical
finite / non-finite patterns.  Inputs are the seeded synthetic workloads.
"""
import numpy as np
import pytest

import gpu_helpers as H
import parity
from oracle import oracle as O
from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu

NAMES = None
ALL = list(range(101))  # the 93 benchmark maps and the 8 IBSI extras (Table 2)


def names():
    global NAMES
    if NAMES is None:
        NAMES = O.feature_names()
    return NAMES


def _check(img, mask, features=None, tune=None, voxels=None, **kw):
    got, plan, feats = H.gpu_map(img, mask, features=features, tune=tune, **kw)
    if voxels is None:
        ref, vox, _, _ = H.oracle_map(img, mask, **kw)
        cols = np.arange(got.shape[1])
    else:
        allvox = np.flatnonzero(mask.reshape(-1))
        cols = np.searchsorted(allvox, voxels)
        ref, vox, _, _ = H.oracle_map(img, mask, voxels=voxels, **kw)
    ref = ref[feats]
    parity.assert_close(got[:, cols], ref, [names()[f] for f in feats])
    return plan


def _crop_ct(seed=2, shape=(24, 40, 44), semi=(19.0, 16.0, 10.0)):
    img = synth.ct_like(shape, seed)
    mask = synth.ellipsoid(shape, ((shape[2] - 1) / 2, (shape[1] - 1) / 2, (shape[0] - 1) / 2),
                           semi)
    return img, mask


def test_tiny_glcm_and_first_order_full():
    # 32^3 uniform 0..255, ball r=10, FBN 16, r=1: GLCM 24 + first order 18
    img, mask = synth.tiny(seed=1)
    _check(img, mask, features=list(range(42)), disc_mode=0, bin_count=16, kernel_radius=1)


def test_tiny_fbn24_r2_many_levels_per_window():
    # uniform noise with 24 bins: most 5^3 windows hold 22-24 levels, the top
    # of what the shared-memory arena takes (every family's matrices over
    # high compact levels; MCC on more than 12 levels)
    img, mask = synth.tiny(seed=1)
    _check(img, mask, features=ALL, disc_mode=0, bin_count=24, kernel_radius=2)


def test_tiny_all_101_full():
    img, mask = synth.tiny(seed=1)
    _check(img, mask, features=ALL, disc_mode=0, bin_count=16, kernel_radius=1)


def test_tiny_default_is_the_93_benchmark_maps():
    img, mask = synth.tiny(seed=1)
    plan = _check(img, mask, disc_mode=0, bin_count=16, kernel_radius=1)
    assert plan.features == list(range(93))


@pytest.mark.parametrize("r", [1, 2, 3])
def test_ct_crop_all_101_fbw(r):
    img, mask = _crop_ct()
    _check(img, mask, features=ALL, disc_mode=1, bin_width=25.0, kernel_radius=r)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_ct_crop_all_101_merged_aggregation(r):
    # GLCM and GLRLM over the sum of the 13 directional matrices
    img, mask = _crop_ct(seed=6, shape=(16, 28, 32), semi=(14.0, 12.0, 7.0))
    _check(img, mask, features=ALL, disc_mode=1, bin_width=25.0, kernel_radius=r, aggregation=1)


def test_tiny_merged_aggregation_fbn16():
    img, mask = synth.tiny(seed=1)
    _check(img, mask, disc_mode=0, bin_count=16, kernel_radius=1, aggregation=1)


def test_ct_crop_fbn64_r3_slab_path():
    # FBN 64 makes windows with more than 32 levels or a level range >= 64
    # possible; the kernel then uses its global slab.
    img, mask = _crop_ct(seed=5)
    _check(img, mask, features=ALL, disc_mode=0, bin_count=64, kernel_radius=3)


@pytest.mark.parametrize("r", [1, 2])
def test_ct_crop_glcm_only_fbn64(r):
    # GLCM alone (no later family clears the big region between voxels):
    # windows of up to 9 levels take the one-lane-per-direction path, larger
    # ones the count-matrix path, interleaved in every warp; both must leave
    # the shared region as they found it
    img, mask = _crop_ct(seed=9)
    _check(img, mask, features=list(range(18, 42)) + [96, 97], disc_mode=0, bin_count=64,
           kernel_radius=r)


def test_levels_and_voxel_list_bit_exact():
    import paper_2609_19190_gb300 as fm
    for img, mask, kw in [
        (*synth.tiny(seed=1), dict(disc_mode=0, bin_count=16)),
        (*_crop_ct(), dict(disc_mode=1, bin_width=25.0)),
        (*_crop_ct(), dict(disc_mode=1, bin_width=7.3, fbw_anchor=1)),
        (*_crop_ct(), dict(disc_mode=0, bin_count=255)),
    ]:
        got, plan, _ = H.gpu_map(img, mask, features=[0], **kw)
        lev, ng, xmin, xmax = fm.fr_plan_levels(plan)
        op = H.oracle_params(img.shape, **kw)
        rlev, rng_, rmin, rmax = O.discretise(op, img, mask)
        assert (ng, xmin, xmax) == (rng_, rmin, rmax)
        assert np.array_equal(lev.cpu().numpy(), rlev)
        idx = fm.fr_plan_voxel_index(plan).cpu().numpy()
        assert np.array_equal(idx, np.flatnonzero(mask.reshape(-1)))


@pytest.mark.parametrize("r", [1, 2, 3])
def test_texture_matrices_bit_exact(r):
    import torch

    import paper_2609_19190_gb300 as fm
    img, mask = _crop_ct(seed=7)
    kw = dict(disc_mode=1, bin_width=25.0, kernel_radius=r)
    _, plan, _ = H.gpu_map(img, mask, **kw)
    op = H.oracle_params(img.shape, **kw)
    levels, ng, _, _ = O.discretise(op, img, mask)
    allvox = np.flatnonzero(mask.reshape(-1))
    cols = synth.sample_voxels(mask, 40, seed=r)
    cols = np.searchsorted(allvox, cols).astype(np.int32)
    m = fm.fr_debug_matrices(plan, torch.from_numpy(img).cuda(), cols, ng)
    for t, c in enumerate(cols):
        ref = O.matrices(op, levels, ng, int(allvox[c]))
        for key in ("hist", "glcm", "glrlm", "glszm", "gldm", "ngtdm_n", "ngtdm_sl"):
            assert np.array_equal(m[key][t], ref[key]), (key, t, c)
        assert m["nv"][t] == ref["hist"].sum()
