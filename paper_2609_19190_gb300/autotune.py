"""Launch-shape autotuner for the mapping kernel.

Times a small set of candidate shapes (brick, voxels per work item, consumer
warps per CTA, halo stages) on the caller's own workload and keeps the
fastest, cached in a JSON file (FLASHMAP_TUNE_CACHE, else
~/.cache/flashmap_tune.json) under a key of the batch's composition: the set
of kernel radii, the level-count bucket, the feature families and the
bucket of VOI sizes (a batch of many small VOIs wants finer work items than
one of a few large ones).  Every candidate gives bit-identical maps (the
per-voxel computation does not depend on the launch shape), so only time
decides.
"""
import json
import os

CANDIDATES = (
    dict(brick_x=8, brick_y=4, brick_z=4, voxels_per_item=16, consumer_warps=16, stages=1),
    dict(brick_x=8, brick_y=4, brick_z=4, voxels_per_item=16, consumer_warps=16, stages=3),
    dict(brick_x=8, brick_y=4, brick_z=4, voxels_per_item=16, consumer_warps=16, stages=2),
    dict(brick_x=16, brick_y=8, brick_z=8, voxels_per_item=16, consumer_warps=16, stages=1),
    dict(brick_x=16, brick_y=8, brick_z=8, voxels_per_item=32, consumer_warps=16, stages=1),
    dict(brick_x=16, brick_y=4, brick_z=4, voxels_per_item=16, consumer_warps=16, stages=1),
    dict(brick_x=8, brick_y=8, brick_z=4, voxels_per_item=16, consumer_warps=16, stages=1),
    dict(brick_x=8, brick_y=4, brick_z=4, voxels_per_item=16, consumer_warps=8, stages=1),
)


def cache_path():
    return os.environ.get("FLASHMAP_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "flashmap_tune.json"))


def _families(features):
    fam = 0
    for f in features:
        fam |= 1 << (0 if f < 18 else 1 if f < 42 else 2 if f < 58 else 3 if f < 74 else
                     4 if f < 88 else 5 if f < 93 else 0 if f < 96 else 1 if f < 98 else 4)
    return fam


def key_of(params_list, sizes):
    """Cache key of a batch: radii present, largest level-count bucket, the
    union of feature families, and the power-of-two bucket of the median VOI
    size."""
    import paper_2609_19190_gb300 as fm
    radii = sorted({p.kernel_radius for p in params_list})
    ng = max(p.bin_count if p.disc_mode == fm.FR_FBN else 255 for p in params_list)
    bucket = 16 if ng <= 16 else 32 if ng <= 32 else 64 if ng <= 64 else 255
    fam = 0
    for p in params_list:
        fam |= _families(fm.selected_features(p))
    med = sorted(sizes)[len(sizes) // 2]
    return "r%s_ng%d_f%d_v%d" % ("".join(map(str, radii)), bucket, fam,
                                 max(0, int(med).bit_length() - 1))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _time_batch(params_list, masks, images, tune, reps=2):
    import paper_2609_19190_gb300 as fm
    b = fm.fr_batch_plan(params_list, masks, tune=tune)
    fm.fr_batch_run(b, images)
    best = None
    for _ in range(reps):
        fm.fr_batch_run(b, images)
        ms = fm.fr_batch_last_kernel_ms(b)
        best = ms if best is None else min(best, ms)
    fm.fr_batch_sync_status(b)
    fm.fr_batch_destroy(b)
    return best


def pick(params_list, masks, images, candidates=CANDIDATES, use_cache=True):
    """Best launch shape for a batch.  Returns (tune dict, {candidate index:
    kernel ms})."""
    sizes = [int(m.sum()) for m in masks]
    key = key_of(params_list, sizes)
    cache = _load() if use_cache else {}
    if key in cache:
        return dict(cache[key]["tune"]), cache[key].get("timings", {})
    timings = {}
    for k, cand in enumerate(candidates):
        timings[k] = _time_batch(params_list, masks, images, cand)
    best = min(timings, key=timings.get)
    cache[key] = {"tune": dict(candidates[best]), "timings": timings}
    if use_cache:
        _store(cache)
    return dict(candidates[best]), timings
