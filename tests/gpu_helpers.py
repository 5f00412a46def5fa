"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np

from oracle import oracle as O


def oracle_params(shape, disc_mode=0, bin_count=16, bin_width=25.0, fbw_anchor=0,
                  kernel_radius=1, glcm_distance=1, spacing=(1.0, 1.0, 1.0), kurtosis_excess=1,
                  aggregation=0):
    return O.make_params(shape, disc_mode=disc_mode, bin_count=bin_count, bin_width=bin_width,
                         fbw_anchor=fbw_anchor, radius=kernel_radius, distance=glcm_distance,
                         spacing=spacing, kurtosis_excess=kurtosis_excess,
                         aggregation=aggregation)


def gpu_map(img, mask, features=None, tune=None, **kw):
    """(out float64 [rows, n_voi], plan, feature ids) through fr_map_plan/run."""
    import torch

    import paper_2609_19190_gb300 as fm
    nz, ny, nx = img.shape
    if features is not None:
        kw["features"] = features
    p = fm.fr_map_params_init(nx, ny, nz, **kw)
    plan = fm.fr_map_plan(p, torch.from_numpy(np.ascontiguousarray(mask)), tune=tune)
    out = fm.fr_map_run(plan, torch.from_numpy(np.ascontiguousarray(img)).cuda())
    fm.fr_map_sync_status(plan)
    return out.cpu().numpy().astype(np.float64), plan, plan.features


def oracle_map(img, mask, voxels=None, nthreads=0, **kw):
    """(maps [93, n], voxels, levels, ng) from the oracle for all VOI voxels
    (z-major) or the listed ones."""
    kw = {k: v for k, v in kw.items() if k != "features"}
    p = oracle_params(img.shape, **kw)
    levels, ng, _, _ = O.discretise(p, img, mask)
    if voxels is None:
        voxels = np.flatnonzero(mask.reshape(-1)).astype(np.int64)
    return O.map_voxels(p, img, levels, ng, voxels, nthreads), voxels, levels, ng
