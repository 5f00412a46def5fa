"""The multi-rank host logic on CPU with two gloo ranks (no GPU): sharded
independent VOIs and z-slab sharding with halos and a global intensity range
reassemble exactly the single-process result (mapping done by the FP64
oracle standing in for each rank's device work, with the same given
discretisation range the library takes); slowest-rank timing."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_19190_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _volumes():
    rng = np.random.default_rng(40)
    out = []
    for k in range(5):
        shape = (6 + k, 7, 8)
        img = rng.integers(-300, 300, size=shape).astype(np.int16)
        mask = (rng.random(shape) < 0.3 + 0.1 * k).astype(np.uint8)
        out.append((img, mask))
    return out


def _map(img, mask, vox=None, rng_override=None):
    from oracle import oracle as O
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=8, radius=1,
                      value_range=rng_override)
    levels, ng, lo, hi = O.discretise(p, img, mask)
    if vox is None:
        vox = np.flatnonzero(mask.reshape(-1))
    return O.map_voxels(p, img, levels, ng, vox, nthreads=1)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = D.rank_world()
        assert (r, w) == (rank, world)
        # 1) independent VOIs dealt by size
        vols = _volumes()
        mine = D.shard_units([int(m.sum()) for _, m in vols], world, rank)
        res = {i: _map(*vols[i]) for i in mine}
        # 2) one volume in z-slabs with halos and the global range
        rng = np.random.default_rng(41)
        img = rng.integers(-500, 500, size=(11, 6, 7)).astype(np.int16)
        mask = (rng.random(img.shape) < 0.6).astype(np.uint8)
        z0, z1, h0, h1 = D.slab_plan(img.shape[0], 1, world, rank)
        sub_img, sub_mask = img[h0:h1], mask[h0:h1]
        own = np.zeros_like(sub_mask)
        own[z0 - h0:z1 - h0] = sub_mask[z0 - h0:z1 - h0]
        vals = img[z0:z1][mask[z0:z1] > 0]
        lo, hi = D.global_range(vals.min(), vals.max())
        vox = np.flatnonzero(own.reshape(-1))
        slab = _map(sub_img, sub_mask, vox, rng_override=(lo, hi))
        # 3) slowest-rank timing
        t = D.max_over_ranks(1.0 + rank)
        q.put((rank, mine, res, (z0, z1), slab, t, (lo, hi)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reassemble_the_single_process_result():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    vols = _volumes()
    owned = sorted(i for g in got for i in g[1])
    assert owned == list(range(len(vols)))  # every VOI exactly once
    loads = [sum(int(vols[i][1].sum()) for i in g[1]) for g in got]
    assert max(loads) - min(loads) <= max(int(m.sum()) for _, m in vols)
    for g in got:
        for i, maps in g[2].items():
            np.testing.assert_array_equal(maps, _map(*vols[i]))
    # slabs cover z exactly once and reassemble the whole-volume maps
    rng = np.random.default_rng(41)
    img = rng.integers(-500, 500, size=(11, 6, 7)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.6).astype(np.uint8)
    full = _map(img, mask)
    got.sort(key=lambda g: g[0])
    zs = [g[3] for g in got]
    assert zs[0][0] == 0 and zs[-1][1] == img.shape[0] and zs[0][1] == zs[1][0]
    assembled = np.concatenate([g[4] for g in got], axis=1)
    np.testing.assert_array_equal(assembled, full)
    assert all(g[6] == (int(img[mask > 0].min()), int(img[mask > 0].max())) for g in got)
    assert all(g[5] == 2.0 for g in got)


def test_slab_plan_and_sharding_properties():
    for nz in (1, 5, 64, 127):
        for world in (1, 2, 3, 8):
            for r in (1, 3):
                spans = [D.slab_plan(nz, r, world, k) for k in range(world)]
                assert spans[0][0] == 0 and spans[-1][1] == nz
                for (a0, a1, h0, h1), (b0, _, _, _) in zip(spans, spans[1:]):
                    assert a1 == b0
                for a0, a1, h0, h1 in spans:
                    assert h0 == max(0, a0 - r) and h1 == min(nz, a1 + r)
    sizes = [5, 9, 1, 7, 7, 3]
    parts = [D.shard_units(sizes, 3, k) for k in range(3)]
    assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
