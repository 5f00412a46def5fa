"""Parity at the full workload sizes, in the launch configuration bench.py
times (default tune), on seeded samples of output columns that the oracle
computes one by one; matrices bit-exact on a smaller sample."""
import numpy as np
import pytest

import gpu_helpers as H
import parity
from oracle import oracle as O
from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu


def _sampled(img, mask, n, seed, **kw):
    vox = synth.sample_voxels(mask, n, seed)
    got, plan, feats = H.gpu_map(img, mask, **kw)
    cols = np.searchsorted(np.flatnonzero(mask.reshape(-1)), vox)
    ref, _, _, _ = H.oracle_map(img, mask, voxels=vox, **kw)
    fails, summary = parity.compare(got[:, cols], ref[feats], [O.feature_names()[f] for f in feats])
    assert not fails, "\n".join(fails[:20])
    return plan, vox, cols


def test_ct_plain_full_size_sampled():
    # 128x128x64 CT-like, ellipsoidal VOI (200,336 voxels), FBW 25, r = 2
    img, mask = synth.ct_plain(seed=2)
    _sampled(img, mask, 3000, 21, disc_mode=1, bin_width=25.0, kernel_radius=2)


def test_ct_large_full_size_sampled_with_matrices():
    import torch

    import paper_2609_19190_gb300 as fm
    # 256x256x128 CT-like, union of three ellipsoids (~2.0M voxels), FBN 64, r = 3
    img, mask = synth.ct_large(seed=3)
    kw = dict(disc_mode=0, bin_count=64, kernel_radius=3)
    plan, vox, cols = _sampled(img, mask, 1500, 22, **kw)
    op = H.oracle_params(img.shape, **kw)
    levels, ng, _, _ = O.discretise(op, img, mask)
    sub = cols[:60].astype(np.int32)
    m = fm.fr_debug_matrices(plan, torch.from_numpy(img).cuda(), sub, ng)
    for t, c in enumerate(sub):
        ref = O.matrices(op, levels, ng, int(vox[t]))
        for key in ("hist", "glcm", "glrlm", "glszm", "gldm", "ngtdm_n", "ngtdm_sl"):
            assert np.array_equal(m[key][t], ref[key]), (key, t)


def test_tiny_full_size_all_columns():
    # 32^3 uniform, ball VOI r=10, FBN 16, r = 1 -- every column
    img, mask = synth.tiny(seed=1)
    got, plan, feats = H.gpu_map(img, mask, disc_mode=0, bin_count=16, kernel_radius=1)
    ref, _, _, _ = H.oracle_map(img, mask, disc_mode=0, bin_count=16, kernel_radius=1)
    parity.assert_close(got, ref[feats], [O.feature_names()[f] for f in feats])


def test_batched_workload_items_against_oracle_sampled():
    # the first 6 requests of the batched workload (128x128x64 CT-like volumes,
    # log-uniform VOI sizes, r in {1,2,3}, FBN 16/32/64), one batched launch,
    # each VOI checked on 200 seeded voxels against the oracle
    import torch

    import paper_2609_19190_gb300 as fm
    params, masks, imgs, host, kws = [], [], [], [], []
    for i in range(6):
        img, mask, r, bins = synth.batch_item(i)
        kw = dict(disc_mode=0, bin_count=bins, kernel_radius=r)
        nz, ny, nx = img.shape
        params.append(fm.fr_map_params_init(nx, ny, nz, features=list(range(101)), **kw))
        masks.append(torch.from_numpy(mask))
        imgs.append(torch.from_numpy(img).cuda())
        host.append((img, mask))
        kws.append(kw)
    b = fm.fr_batch_plan(params, masks)
    outs = fm.fr_batch_run(b, imgs)
    fm.fr_batch_sync_status(b)
    names = O.feature_names()
    for (img, mask), kw, out in zip(host, kws, outs):
        allvox = np.flatnonzero(mask.reshape(-1))
        vox = synth.sample_voxels(mask, 200, 31)
        ref, _, _, _ = H.oracle_map(img, mask, voxels=vox, **kw)
        cols = np.searchsorted(allvox, vox)
        got = out.cpu().numpy().astype(np.float64)[:, cols]
        parity.assert_close(got, ref, names)
    fm.fr_batch_destroy(b)
