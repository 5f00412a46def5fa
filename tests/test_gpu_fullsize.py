"""Parity at the full workload sizes, in the launch configuration bench.py
times (default tune), against the FP64 oracle (all host cores).

* the 128x128x64 CT-like volume (200,336 VOI voxels): every column;
* the 256x256x128 CT-like volume (2.0M VOI voxels, r = 3): every column,
  compared chunk by chunk, and the integer matrices of seeded voxels;
* the 64 VOIs of the batched workload in one batched launch: every voxel of
  the r = 1 VOIs and a seeded 5 % of the r = 2, 3 VOIs;
* served requests (continuous batching): every voxel of the r = 1 requests
  and a seeded 5 % of the others;
* map-path cases with non-unit spacing (TotalEnergy) and raw kurtosis.
"""
import numpy as np
import pytest

import gpu_helpers as H
import parity
from oracle import oracle as O
from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu

ALL = list(range(101))  # the 93 benchmark maps and the 8 IBSI extras
NAMES = None


def _names(feats):
    global NAMES
    if NAMES is None:
        NAMES = O.feature_names()
    return [NAMES[f] for f in feats]


def _check_columns(got, img, mask, vox, cols, feats, chunk=200000, **kw):
    """Oracle at the voxels vox (columns cols of got), chunk by chunk."""
    fails = []
    for a in range(0, len(vox), chunk):
        ref, _, _, _ = H.oracle_map(img, mask, voxels=vox[a:a + chunk], **kw)
        f, _ = parity.compare(got[:, cols[a:a + chunk]], ref[feats], _names(feats))
        fails += ["cols %d..: %s" % (a, s) for s in f]
    assert not fails, "\n".join(fails[:20])


def _sample_fraction(mask, frac, seed):
    n = max(1, int(round(frac * int(mask.sum()))))
    return synth.sample_voxels(mask, n, seed)


def test_ct_plain_every_column():
    # 128x128x64 CT-like, ellipsoidal VOI (200,336 voxels), FBW 25, r = 2
    img, mask = synth.ct_plain(seed=2)
    kw = dict(disc_mode=1, bin_width=25.0, kernel_radius=2)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int64)
    assert got.shape[1] == vox.size == 200336
    _check_columns(got, img, mask, vox, np.arange(vox.size), feats, **kw)


@pytest.mark.parametrize("kw", [
    dict(spacing=(0.7, 0.8, 2.0)),
    dict(kurtosis_excess=0),
    dict(spacing=(1.5, 0.5, 3.0), kurtosis_excess=0),
])
def test_ct_plain_spacing_and_raw_kurtosis_sampled(kw):
    # TotalEnergy scales with the voxel volume; kurtosis without the -3
    img, mask = synth.ct_plain(seed=2)
    kw = dict(disc_mode=1, bin_width=25.0, kernel_radius=2, **kw)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    vox = synth.sample_voxels(mask, 4000, 23)
    cols = np.searchsorted(np.flatnonzero(mask.reshape(-1)), vox)
    _check_columns(got, img, mask, vox, cols, feats, **kw)
    if "spacing" in kw:
        vv = float(np.prod(kw["spacing"]))
        np.testing.assert_allclose(got[1], vv * got[0], rtol=1e-6)


def test_ct_large_every_column_with_matrices():
    import torch

    import paper_2609_19190_gb300 as fm
    # 256x256x128 CT-like, union of three ellipsoids (~2.0M voxels), FBN 64, r = 3
    img, mask = synth.ct_large(seed=3)
    kw = dict(disc_mode=0, bin_count=64, kernel_radius=3)
    got, plan, feats = H.gpu_map(img, mask, features=ALL, **kw)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int64)
    assert got.shape[1] == vox.size > 1900000
    _check_columns(got, img, mask, vox, np.arange(vox.size), feats, chunk=250000, **kw)
    # integer matrices, bit-exact, at seeded voxels
    op = H.oracle_params(img.shape, **kw)
    levels, ng, _, _ = O.discretise(op, img, mask)
    svox = synth.sample_voxels(mask, 60, 22)
    sub = np.searchsorted(vox, svox).astype(np.int32)
    m = fm.fr_debug_matrices(plan, torch.from_numpy(img).cuda(), sub, ng)
    for t in range(sub.size):
        ref = O.matrices(op, levels, ng, int(svox[t]))
        for key in ("hist", "glcm", "glrlm", "glszm", "gldm", "ngtdm_n", "ngtdm_sl"):
            assert np.array_equal(m[key][t], ref[key]), (key, t)


def test_tiny_full_size_all_columns():
    # 32^3 uniform, ball VOI r=10, FBN 16, r = 1 -- every column
    img, mask = synth.tiny(seed=1)
    got, plan, feats = H.gpu_map(img, mask, disc_mode=0, bin_count=16, kernel_radius=1)
    ref, _, _, _ = H.oracle_map(img, mask, disc_mode=0, bin_count=16, kernel_radius=1)
    parity.assert_close(got, ref[feats], _names(feats))


def test_batched_workload_every_voi():
    # the 64 VOIs of the batched workload (128x128x64 CT-like volumes,
    # log-uniform VOI sizes, r in {1,2,3}, FBN 16/32/64) in one batched
    # launch: every voxel at r = 1, a seeded 5 % at r = 2, 3
    import torch

    import paper_2609_19190_gb300 as fm
    params, masks, imgs, host, kws = [], [], [], [], []
    for i in range(64):
        img, mask, r, bins = synth.batch_item(i)
        kw = dict(disc_mode=0, bin_count=bins, kernel_radius=r)
        nz, ny, nx = img.shape
        params.append(fm.fr_map_params_init(nx, ny, nz, features=ALL, **kw))
        masks.append(torch.from_numpy(mask))
        imgs.append(torch.from_numpy(img).cuda())
        host.append((img, mask))
        kws.append(kw)
    b = fm.fr_batch_plan(params, masks)
    outs = fm.fr_batch_run(b, imgs)
    fm.fr_batch_sync_status(b)
    radii = set()
    for i, ((img, mask), kw, out) in enumerate(zip(host, kws, outs)):
        allvox = np.flatnonzero(mask.reshape(-1))
        r = kw["kernel_radius"]
        radii.add(r)
        vox = allvox.astype(np.int64) if r == 1 else _sample_fraction(mask, 0.05, 31 + i)
        cols = np.searchsorted(allvox, vox)
        _check_columns(out.cpu().numpy().astype(np.float64), img, mask, vox, cols, ALL, **kw)
    assert radii == {1, 2, 3}
    fm.fr_batch_destroy(b)


def test_served_requests_every_r1_request_and_a_sample_of_the_rest():
    # requests of the served workload (log-normal sizes, median 50k voxels),
    # continuous batching at 100 req/s: every voxel of the r = 1 requests, a
    # seeded 5 % of the r = 2, 3 requests
    import torch

    from paper_2609_19190_gb300 import serve
    reqs = synth.served_requests(16, seed=200, max_voxels=400000)
    imgs = {}
    for k, rq in enumerate(reqs):
        if rq["shape"] not in imgs:
            imgs[rq["shape"]] = torch.from_numpy(synth.ct_like(rq["shape"], 500 + k)).cuda()
    stats = serve.serve(reqs, imgs, rate=100.0, seed=3, voxel_budget=131072, keep_outputs=True)
    assert stats["requests"] == len(reqs)
    assert {rq["radius"] for rq in reqs} == {1, 2, 3}
    for i, rq in enumerate(reqs):
        img = imgs[rq["shape"]].cpu().numpy()
        mask = rq["mask"]
        allvox = np.flatnonzero(mask.reshape(-1))
        vox = allvox.astype(np.int64) if rq["radius"] == 1 else \
            _sample_fraction(mask, 0.05, 41 + i)
        cols = np.searchsorted(allvox, vox)
        got = stats["outputs"][i].cpu().numpy().astype(np.float64)
        _check_columns(got, img, mask, vox, cols, list(range(93)),
                       kernel_radius=rq["radius"], **rq["disc"])
