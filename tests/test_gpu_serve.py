"""Continuous batching (fr_server_*): results are the same alone and in the
mix, a request that arrives while a large one is being mapped finishes first,
and admission waits for memory."""
import numpy as np
import pytest

from paper_2609_19190_gb300 import synth

pytestmark = pytest.mark.gpu


def _images(requests):
    import torch
    imgs = {}
    for k, rq in enumerate(requests):
        if rq["shape"] not in imgs:
            imgs[rq["shape"]] = torch.from_numpy(synth.ct_like(rq["shape"], 400 + k)).cuda()
    return imgs


def _alone(rq, img):
    import torch

    import paper_2609_19190_gb300 as fm
    nz, ny, nx = rq["shape"]
    p = fm.fr_map_params_init(nx, ny, nz, kernel_radius=rq["radius"], **rq["disc"])
    plan = fm.fr_map_plan(p, torch.from_numpy(rq["mask"]))
    out = fm.fr_map_run(plan, img)
    fm.fr_map_sync_status(plan)
    return out


def test_served_results_equal_alone_and_in_the_mix():
    import torch

    from paper_2609_19190_gb300 import serve
    reqs = synth.served_requests(10, seed=5, median=6000.0, max_voxels=60000)
    imgs = _images(reqs)
    stats = serve.serve(reqs, imgs, rate=300.0, seed=1, voxel_budget=3000, keep_outputs=True)
    assert stats["requests"] == len(reqs)
    assert stats["steps"] > len(reqs)  # requests shared steps, more than one each
    for i, rq in enumerate(reqs):
        ref = _alone(rq, imgs[rq["shape"]])
        got = stats["outputs"][i]
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32)), i
    assert stats["p50_s"] <= stats["p99_s"]
    # and against the oracle on seeded voxels of two requests
    import gpu_helpers as H
    import parity
    from oracle import oracle as O
    for i in (0, len(reqs) - 1):
        rq = reqs[i]
        img = imgs[rq["shape"]].cpu().numpy()
        mask = rq["mask"]
        vox = synth.sample_voxels(mask, 100, 17)
        cols = np.searchsorted(np.flatnonzero(mask.reshape(-1)), vox)
        ref, _, _, _ = H.oracle_map(img, mask, voxels=vox, kernel_radius=rq["radius"], **rq["disc"])
        got = stats["outputs"][i].cpu().numpy().astype(np.float64)[:, cols]
        parity.assert_close(got, ref[:93], O.feature_names()[:93])  # the 93 benchmark maps


def test_late_small_request_overtakes_a_large_one():
    import torch

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import serve
    big = synth.served_requests(1, seed=11, median=150000.0, sigma=0.01)[0]
    small = synth.served_requests(1, seed=12, median=3000.0, sigma=0.01)[0]
    imgs = _images([big, small])
    srv = serve.Server()
    outs = []
    ids = []
    for rq in (big, small):
        nz, ny, nx = rq["shape"]
        p = fm.fr_map_params_init(nx, ny, nz, kernel_radius=rq["radius"], **rq["disc"])
        out = torch.empty((93, rq["n_voi"]), dtype=torch.float32, device="cuda")
        outs.append(out)
        ids.append(srv.add(p, rq["mask"], imgs[rq["shape"]], out))
        if rq is big:
            srv.step(4096)  # the big request is on the GPU when the small one arrives
    order = []
    while len(order) < 2:
        srv.step(4096)
        order += [rid for rid, st in srv.poll(wait=True)]
    assert order[0] == ids[1] and order[1] == ids[0]
    for rid in ids:
        srv.release(rid)
    srv.close()
    for rq, out in zip((big, small), outs):
        ref = _alone(rq, imgs[rq["shape"]])
        assert torch.equal(out.view(torch.int32), ref.view(torch.int32))


def test_admission_waits_for_memory():
    from paper_2609_19190_gb300 import serve
    reqs = synth.served_requests(6, seed=7, median=8000.0, max_voxels=40000)
    imgs = _images(reqs)
    est = [serve.request_bytes(r["shape"], r["n_voi"], 93) for r in reqs]
    budget = int(max(est) * 1.5)
    stats = serve.serve(reqs, imgs, rate=0.0, seed=2, voxel_budget=20000, hbm_budget=budget)
    assert stats["requests"] == len(reqs)
    assert stats["peak_admitted_bytes"] <= budget


def test_served_requests_drain_to_hdf5(tmp_path):
    # each finished request is written to its own HDF5 file on host threads;
    # the file's dense maps hold exactly the served values at the VOI voxels
    import h5read

    import paper_2609_19190_gb300 as fm
    from paper_2609_19190_gb300 import serve
    reqs = synth.served_requests(4, seed=9, median=5000.0, max_voxels=30000)
    imgs = _images(reqs)
    stats = serve.serve(reqs, imgs, rate=200.0, seed=3, voxel_budget=4000, keep_outputs=True,
                        drain_dir=str(tmp_path), drain_codec="lzf")
    assert len(stats["drained"]) == len(reqs)
    names = fm.fr_feature_names()
    for i in (0, len(reqs) - 1):
        rq = reqs[i]
        f = h5read.File(tmp_path / ("request_%d.h5" % i))
        vox = np.flatnonzero(rq["mask"].reshape(-1))
        got = stats["outputs"][i].cpu().numpy()
        np.testing.assert_array_equal(f.root.members["mask"].data, rq["mask"])
        np.testing.assert_array_equal(f.root.members["image"].data,
                                      imgs[rq["shape"]].cpu().numpy())
        for r in (0, 18, 41, 58, 92):
            dense = f.root.members["maps"].members[names[r]].data.reshape(-1)
            np.testing.assert_array_equal(dense[vox].view(np.uint32), got[r].view(np.uint32))
            outside = np.ones(dense.size, bool)
            outside[vox] = False
            assert np.isnan(dense[outside]).all()
