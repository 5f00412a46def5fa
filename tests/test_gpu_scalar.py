"""Scalar extraction (fr_scalar_*): the features of the whole VOI, through
the C ABI, against the FP64 oracle's whole-VOI evaluation.

The GPU takes these features in FP64 from exact integer counts, so the bar is
tighter than for the FP32 maps: |gpu - oracle| <= 1e-8 max(1, |oracle|),
identical NaN pattern; MCC comes from the FP32 eigen-solver and keeps the
maps' bar max(1e-6, 1e-4 |oracle|).
"""
import numpy as np
import pytest

import gpu_helpers as H
from oracle import oracle as O
from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu

MCC = 41
MAPS = list(range(101))  # the 93 benchmark features and the 8 IBSI extras (Table 2)
ALL = list(range(102))  # and the scalar-only standard deviation (id 101)


def _gpu_scalar(img, mask, **kw):
    import torch

    import paper_2609_19190_gb300 as fm
    nz, ny, nx = img.shape
    feats = kw.pop("features", None)
    if feats is not None:
        kw["features"] = feats
    p = fm.fr_map_params_init(nx, ny, nz, **kw)
    sp = fm.fr_scalar_plan(p, torch.from_numpy(np.ascontiguousarray(mask)))
    out = fm.fr_scalar_run(sp, torch.from_numpy(np.ascontiguousarray(img)).cuda())
    fm.fr_scalar_sync_status(sp)
    return out.cpu().numpy(), sp


def _oracle_scalar(img, mask, **kw):
    kw = {k: v for k, v in kw.items() if k != "features"}
    p = H.oracle_params(img.shape, **kw)
    levels, ng, _, _ = O.discretise(p, img, mask)
    return O.scalar(p, img, levels, ng)


def _assert_scalar_close(got, ref, feats):
    names = O.scalar_feature_names()
    bad = []
    for k, f in enumerate(feats):
        g, r = got[k], ref[f]
        if np.isnan(r) or np.isnan(g):
            if np.isnan(r) != np.isnan(g):
                bad.append("%s: gpu %r oracle %r" % (names[f], g, r))
            continue
        tol = max(1e-6, 1e-4 * abs(r)) if f == MCC else 1e-8 * max(1.0, abs(r))
        if abs(g - r) > tol:
            bad.append("%s: gpu %.12g oracle %.12g" % (names[f], g, r))
    assert not bad, "\n".join(bad)


def _check(img, mask, **kw):
    got, sp = _gpu_scalar(img, mask, **dict(kw))
    ref = _oracle_scalar(img, mask, **kw)
    _assert_scalar_close(got, ref, sp.features)
    return got, sp


def _crop_ct(seed, shape, semi):
    img = synth.ct_like(shape, seed)
    mask = synth.ellipsoid(shape, ((shape[2] - 1) / 2, (shape[1] - 1) / 2, (shape[0] - 1) / 2),
                           semi)
    return img, mask


def test_scalar_tiny_fbn16():
    img, mask = synth.tiny(seed=1)
    _check(img, mask, disc_mode=0, bin_count=16, features=ALL)


@pytest.mark.parametrize("agg", [0, 1])
def test_scalar_ct_crop_fbw(agg):
    img, mask = _crop_ct(3, (24, 40, 44), (19.0, 16.0, 10.0))
    _check(img, mask, disc_mode=1, bin_width=25.0, aggregation=agg, spacing=(0.8, 0.8, 2.0),
           features=ALL)


def test_scalar_ct_plain_full_size_fbw25():
    # the 128 x 128 x 64 CT-like volume, VOI of 200,336 voxels, all 101 features
    img, mask = synth.ct_plain(seed=2)
    _check(img, mask, disc_mode=1, bin_width=25.0, features=ALL)


def test_scalar_fbn64_delta2_subset():
    img, mask = _crop_ct(4, (20, 36, 30), (14.0, 16.0, 9.0))
    feats = [0, 4, 8, 18, 24, 30, 31, 41, 42, 48, 58, 64, 74, 88, 90, 93, 95, 96, 97, 99]
    _check(img, mask, disc_mode=0, bin_count=64, glcm_distance=2, features=feats)


def test_scalar_equals_map_where_windows_cover_the_voi():
    # VOI inside a 7^3 box, r = 7: every map value is the scalar value
    rng = np.random.default_rng(60)
    img = rng.integers(-300, 300, size=(16, 16, 16)).astype(np.int16)
    mask = np.zeros(img.shape, np.uint8)
    mask[5:12, 4:11, 6:13] = rng.random((7, 7, 7)) < 0.75
    kw = dict(disc_mode=0, bin_count=12)
    sc, _ = _gpu_scalar(img, mask, features=ALL, **dict(kw))
    maps, plan, feats = H.gpu_map(img, mask, features=MAPS, kernel_radius=7, **kw)
    for f in feats:
        if f == MCC:
            continue
        col = maps[f]
        tol = np.maximum(1e-6, 1e-4 * np.abs(sc[f]))
        assert np.all(np.abs(col - sc[f]) <= tol) or (np.isnan(sc[f]) and np.all(np.isnan(col))), f


def test_scalar_runs_are_bit_identical():
    img, mask = _crop_ct(5, (20, 30, 30), (12.0, 13.0, 8.0))
    import torch

    import paper_2609_19190_gb300 as fm
    nz, ny, nx = img.shape
    p = fm.fr_map_params_init(nx, ny, nz, disc_mode=1, bin_width=25.0, features=ALL)
    sp = fm.fr_scalar_plan(p, torch.from_numpy(mask))
    dimg = torch.from_numpy(img).cuda()
    a = fm.fr_scalar_run(sp, dimg).cpu().numpy()
    b = fm.fr_scalar_run(sp, dimg).cpu().numpy()
    fm.fr_scalar_sync_status(sp)
    # every feature, GLSZM included: its cell sums are exact fixed-point
    # integer sums, independent of the zone table's slot order
    for _ in range(3):
        c = fm.fr_scalar_run(sp, dimg).cpu().numpy()
        assert np.array_equal(a.view(np.int64), c.view(np.int64))
    assert np.array_equal(a.view(np.int64), b.view(np.int64))
    fm.fr_scalar_sync_status(sp)


def test_scalar_too_many_levels_reports_and_writes_nan():
    import torch

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import _lib
    rng = np.random.default_rng(61)
    img = rng.integers(-20000, 20000, size=(8, 8, 8)).astype(np.int16)
    mask = np.ones(img.shape, np.uint8)
    p = fm.fr_map_params_init(8, 8, 8, disc_mode=1, bin_width=10.0)
    sp = fm.fr_scalar_plan(p, torch.from_numpy(mask))
    out = fm.fr_scalar_run(sp, torch.from_numpy(img).cuda())
    with pytest.raises(_lib.FlashmapError) as e:
        fm.fr_scalar_sync_status(sp)
    assert e.value.status == 3
    assert bool(torch.isnan(out).all())
