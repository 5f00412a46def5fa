"""Launch-shape autotuner for the mapping kernel.

Times a small set of candidate shapes (brick, voxels per work item, consumer
warps per CTA, halo stages) on the caller's own workload and keeps the
fastest, cached by a key of (kernel radius, level-count bucket, feature
families) in a JSON file (FLASHMAP_TUNE_CACHE, else
~/.cache/flashmap_tune.json).  Every candidate gives bit-identical maps (the
per-voxel computation does not depend on the launch shape), so only time
decides.
"""
import json
import os

CANDIDATES = (
    dict(brick_x=8, brick_y=4, brick_z=4, voxels_per_item=16, consumer_warps=16, stages=1),
    dict(brick_x=8, brick_y=4, brick_z=4, voxels_per_item=32, consumer_warps=16, stages=1),
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


def key_of(params):
    import paper_2609_19190_gb300 as fm
    ng = params.bin_count if params.disc_mode == fm.FR_FBN else 255
    bucket = 16 if ng <= 16 else 32 if ng <= 32 else 64 if ng <= 64 else 255
    return "r%d_ng%d_f%d" % (params.kernel_radius, bucket,
                             _families(fm.selected_features(params)))


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
    """Best launch shape for a batch (the key of its largest VOI).  Returns
    (tune dict, {candidate index: kernel ms})."""
    sizes = [int(m.sum()) for m in masks]
    key = key_of(params_list[sizes.index(max(sizes))])
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
