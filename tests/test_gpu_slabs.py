"""z-slab sharding through the library on one GPU: each slab of one volume,
with its r-slice halo, is planned on its own with the whole VOI's intensity
range (fr_map_params.range_given), and the slabs' owned columns reassemble
the whole-volume maps bit for bit (every map value of a voxel depends only
on its window, and every slab discretises as the whole volume does)."""
import numpy as np
import pytest

from paper_2609_19190_gb300 import dist as D
from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world,kw", [
    (2, dict(disc_mode=1, bin_width=25.0, kernel_radius=2)),
    (3, dict(disc_mode=0, bin_count=64, kernel_radius=3)),
    (5, dict(disc_mode=1, bin_width=25.0, fbw_anchor=1, kernel_radius=1)),
])
def test_slabs_reassemble_the_whole_volume_bit_for_bit(world, kw):
    import torch

    import paper_2609_19190_gb300 as fm
    img = synth.ct_like((40, 48, 44), 17)
    mask = synth.ellipsoid(img.shape, (21.5, 23.5, 19.5), (19.0, 21.0, 18.0))
    nz, ny, nx = img.shape
    feats = list(range(fm.FR_NUM_FEATURES))
    p = fm.fr_map_params_init(nx, ny, nz, features=feats, **kw)
    plan = fm.fr_map_plan(p, torch.from_numpy(mask))
    whole = fm.fr_map_run(plan, torch.from_numpy(img).cuda()).cpu().numpy()
    fm.fr_map_sync_status(plan)
    vals = img[mask > 0]
    rng = (int(vals.min()), int(vals.max()))
    parts = [D.map_slab(img, mask, world, k, rng, features=feats, **kw).cpu().numpy()
             for k in range(world)]
    assert sum(p.shape[1] for p in parts) == whole.shape[1]
    got = np.concatenate(parts, axis=1)
    assert np.array_equal(got.view(np.int32), whole.view(np.int32))


def test_a_slab_without_the_global_range_discretises_differently():
    # the reason for the field: a slab's own range differs from the VOI's
    import torch

    import paper_2609_19190_gb300 as fm
    img = synth.ct_like((24, 32, 32), 18)
    # a ramp along z puts the VOI's largest values in the upper slab
    img = (img.astype(np.int32) + 40 * np.arange(24)[:, None, None]).astype(np.int16)
    mask = synth.ellipsoid(img.shape, (15.5, 15.5, 11.5), (14.0, 14.0, 11.0))
    kw = dict(disc_mode=0, bin_count=32, kernel_radius=1, features=[0, 2, 17, 18])
    z0, z1, h0, h1 = D.slab_plan(24, 1, 2, 0)
    sub = np.ascontiguousarray(mask[h0:h1])
    vals = img[mask > 0]
    own = img[h0:h1][sub > 0]
    assert (own.min(), own.max()) != (vals.min(), vals.max())
    p_own = fm.fr_map_params_init(32, 32, h1 - h0, **kw)
    p_glob = fm.fr_map_params_init(32, 32, h1 - h0, value_range=(vals.min(), vals.max()), **kw)
    a_plan = fm.fr_map_plan(p_own, torch.from_numpy(sub))
    b_plan = fm.fr_map_plan(p_glob, torch.from_numpy(sub))
    dimg = torch.from_numpy(np.ascontiguousarray(img[h0:h1])).cuda()
    fm.fr_map_run(a_plan, dimg)
    fm.fr_map_run(b_plan, dimg)
    la, nga, lo_a, hi_a = fm.fr_plan_levels(a_plan)
    lb, ngb, lo_b, hi_b = fm.fr_plan_levels(b_plan)
    assert (lo_b, hi_b) == (int(vals.min()), int(vals.max()))
    assert (lo_a, hi_a) != (lo_b, hi_b)
