"""Multi-rank host logic (one process per GPU, torch.distributed).

Every map voxel is independent, so the work shards with no exchange on the
data path: independent VOIs (or requests) are dealt to ranks by size, and a
single large volume splits into z-slabs whose windows need an r-slice halo
copied to each rank; the only exchange is the VOI's global intensity range
(min / max), so every rank discretises identically.  Timing takes the
slowest rank.
"""
import os


def rank_world():
    """(rank, world, local_rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def _reduce(value, op, device=None):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value, device=None):
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX, device)


def global_range(vmin, vmax, device=None):
    """Global (min, max) of per-rank intensity ranges."""
    import torch.distributed as dist
    lo = _reduce(float(vmin), dist.ReduceOp.MIN, device)
    hi = _reduce(float(vmax), dist.ReduceOp.MAX, device)
    return int(lo), int(hi)


def shard_units(sizes, world, rank):
    """Indices of the units (VOIs, requests) this rank maps: longest first to
    the least-loaded rank, so the ranks' voxel totals stay balanced."""
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        w = min(range(world), key=lambda k: (load[k], k))
        owner[i] = w
        load[w] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def slab_plan(nz, radius, world, rank):
    """z-slab of a volume for this rank: (own_z0, own_z1, halo_z0, halo_z1).
    Output columns are the VOI voxels with own_z0 <= z < own_z1; the rank
    needs the image and mask of halo_z0 <= z < halo_z1 (radius more on each
    side, clipped), so every window it evaluates is complete."""
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    z1 = z0 + base + (1 if rank < extra else 0)
    return z0, z1, max(0, z0 - radius), min(nz, z1 + radius)


def map_slab(image, mask, world, rank, value_range, device=0, stream=None, **params):
    """Map this rank's z-slab of one volume through the library.

    The slab and its halo (slab_plan) are planned on their own with the whole
    VOI's intensity range `value_range` = (min, max) (global_range gives it
    across ranks), so the slab discretises exactly as the whole volume does.
    Returns float32 [rows, n_own] on the device: the columns of the VOI
    voxels with own_z0 <= z < own_z1, in the whole volume's column order
    (z-major), so the ranks' results concatenate to the whole volume's maps.
    image: int16 numpy [nz, ny, nx]; mask: uint8 numpy; params: keyword
    fields of fr_map_params (kernel_radius required)."""
    import numpy as np
    import torch

    import paper_2609_19190_gb300 as fm
    nz, ny, nx = image.shape
    z0, z1, h0, h1 = slab_plan(nz, params["kernel_radius"], world, rank)
    sub_mask = np.ascontiguousarray(mask[h0:h1])
    before = int(np.count_nonzero(sub_mask[:z0 - h0]))
    own = int(np.count_nonzero(sub_mask[z0 - h0:z1 - h0]))
    p = fm.fr_map_params_init(nx, ny, h1 - h0, value_range=value_range, device=device, **params)
    if own == 0:
        rows = len(fm.selected_features(p))
        return torch.empty((rows, 0), dtype=torch.float32, device="cuda:%d" % device)
    plan = fm.fr_map_plan(p, torch.from_numpy(sub_mask))
    img = torch.from_numpy(np.ascontiguousarray(image[h0:h1])).to("cuda:%d" % device)
    out = fm.fr_map_run(plan, img, stream=stream)
    fm.fr_map_sync_status(plan)
    fm.fr_map_destroy(plan)
    # columns are z-major, so the owned slices are one contiguous block
    return out[:, before:before + own]
