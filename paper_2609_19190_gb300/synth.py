"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws volumes and masks; it holds none of the method's
arithmetic, and both the CUDA path and the CPU oracle consume its arrays.
Arrays are C-contiguous [Z, Y, X]: int16 images, uint8 masks (1 = VOI).

The paper's own data (a 61 x 55 x 39 breast-MRI crop holding a 50,613-voxel
lesion VOI, tiled to larger sizes; "Spatial concordance" and "End-to-end
processing-time evaluation") is not available; these generators stand in
for it:

* ``tiny``      32^3 i.i.d. uniform 0..255, ball mask of radius 10.
* ``ct_like``   smooth Gaussian-mixture tissue classes (means -900, -50, 40,
                300 HU; smooth per-class deviation fields of sd 60, 30, 20, 40)
                plus i.i.d. Gaussian noise of sd 15, rounded to int16.
* ``ct_plain``  128 x 128 x 64 CT-like volume, ellipsoidal VOI (~200k voxels).
* ``ct_large``  256 x 256 x 128 CT-like volume, union of three ellipsoids
                (~2.0M voxels).
* ``batch``     64 CT-like 128 x 128 x 64 volumes with ellipsoidal VOIs of
                log-uniform size in [4k, 400k] voxels.
* ``paper_tiled`` a 61 x 55 x 39 MR-like volume with a blob VOI of ~38.7 % of
                the box, repeated along the axes without interpolation.
"""
import numpy as np

CT_CLASS_MEANS = (-900.0, -50.0, 40.0, 300.0)
CT_CLASS_SDS = (60.0, 30.0, 20.0, 40.0)
CT_NOISE_SD = 15.0
CT_SMOOTH_SIGMA = 6.0


def _smooth_noise(rng, shape, sigma):
    """Unit-variance white noise low-passed by a Gaussian of width sigma
    (voxels), periodic boundary, computed with real FFTs in float32."""
    noise = rng.standard_normal(shape, dtype=np.float32)
    spec = np.fft.rfftn(noise)
    freqs = [np.fft.fftfreq(n) for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    gain = np.ones(spec.shape, dtype=np.float32)
    for axis, f in enumerate(freqs):
        g = np.exp(-2.0 * (np.pi * sigma * f) ** 2).astype(np.float32)
        sh = [1] * len(shape)
        sh[axis] = f.size
        gain = gain * g.reshape(sh)
    field = np.fft.irfftn(spec * gain, s=shape, axes=tuple(range(len(shape)))).astype(np.float32)
    field -= field.mean()
    sd = field.std()
    return field / (sd if sd > 0 else 1.0)


def ct_like(shape, seed):
    """CT-like int16 volume [Z, Y, X]: argmax of four smooth fields picks the
    tissue class; each class adds its own smooth deviation field; i.i.d.
    Gaussian noise (sd 15) on top; rounded and clipped to int16."""
    rng = np.random.default_rng(seed)
    best = None
    label = np.zeros(shape, dtype=np.int8)
    for c in range(len(CT_CLASS_MEANS)):
        f = _smooth_noise(rng, shape, CT_SMOOTH_SIGMA)
        if best is None:
            best = f
        else:
            take = f > best
            label[take] = c
            best = np.where(take, f, best)
    img = np.zeros(shape, dtype=np.float32)
    for c, (mu, sd) in enumerate(zip(CT_CLASS_MEANS, CT_CLASS_SDS)):
        dev = _smooth_noise(rng, shape, CT_SMOOTH_SIGMA)
        sel = label == c
        img[sel] = mu + sd * dev[sel]
    img += rng.normal(0.0, CT_NOISE_SD, size=shape).astype(np.float32)
    return np.clip(np.rint(img), -32768, 32767).astype(np.int16)


def ellipsoid(shape, centre_xyz, semi_xyz):
    """uint8 mask of the voxels whose centres lie in the ellipsoid."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = centre_xyz
    ax, ay, az = semi_xyz
    q = ((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 + ((z - cz) / az) ** 2
    return (q <= 1.0).astype(np.uint8)


def tiny(seed=1):
    """32^3 int16 i.i.d. uniform 0..255 and a ball mask of radius 10 centred at
    (15.5, 15.5, 15.5)."""
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=(32, 32, 32)).astype(np.int16)
    mask = ellipsoid((32, 32, 32), (15.5, 15.5, 15.5), (10.0, 10.0, 10.0))
    return img, mask


def ct_plain(seed=2):
    """128 x 128 x 64 (X x Y x Z) CT-like volume; ellipsoidal VOI with
    semi-axes (52, 40, 23) voxels about the centre (~200k voxels)."""
    shape = (64, 128, 128)
    img = ct_like(shape, seed)
    mask = ellipsoid(shape, (63.5, 63.5, 31.5), (52.0, 40.0, 23.0))
    return img, mask


LARGE_ELLIPSOIDS = (
    ((100.0, 120.0, 60.0), (85.0, 72.0, 48.0)),
    ((165.0, 140.0, 66.0), (76.3, 78.5, 43.6)),
    ((128.0, 180.0, 64.0), (65.4, 50.1, 39.2)),
)


def ct_large(seed=3):
    """256 x 256 x 128 CT-like volume; VOI = union of three ellipsoids
    (~2.0M voxels)."""
    shape = (128, 256, 256)
    img = ct_like(shape, seed)
    mask = np.zeros(shape, dtype=np.uint8)
    for c, s in LARGE_ELLIPSOIDS:
        mask |= ellipsoid(shape, c, s)
    return img, mask


def batch_item(index, base_seed=100):
    """One request of the batched workload: a CT-like 128 x 128 x 64 volume
    with an ellipsoidal VOI of log-uniform size in [4k, 400k] voxels and a
    random aspect ratio; radius in {1, 2, 3}; bin count in {16, 32, 64}.
    Returns (image, mask, radius, bin_count)."""
    seed = base_seed + index
    rng = np.random.default_rng(seed)
    target = float(np.exp(rng.uniform(np.log(4000.0), np.log(400000.0))))
    aspect = rng.uniform(0.7, 1.3, size=3)
    # volume of an ellipsoid = 4/3 pi a b c; pick a scale that meets target
    scale = (target / (4.0 / 3.0 * np.pi * np.prod(aspect))) ** (1.0 / 3.0)
    semi = np.minimum(aspect * scale, np.array([62.0, 62.0, 30.5]))
    radius = int(rng.integers(1, 4))
    bins = int(rng.choice([16, 32, 64]))
    shape = (64, 128, 128)
    img = ct_like(shape, seed)
    mask = ellipsoid(shape, (63.5, 63.5, 31.5), tuple(semi))
    return img, mask, radius, bins


def batch_small_item(index, base_seed=1000):
    """One VOI of the many-small-VOIs batch: an ellipsoidal VOI of
    log-uniform size in [4k, 20k] voxels, random aspect ratio and centre, in
    one of 16 CT-like 64 x 64 x 64 volumes (index mod 16); radius in {1, 2,
    3}; bin count in {16, 32, 64}.  One such VOI leaves most of the chip idle
    in a launch of its own.  Returns (image, mask, radius, bin_count)."""
    seed = base_seed + index
    rng = np.random.default_rng(seed)
    target = float(np.exp(rng.uniform(np.log(4000.0), np.log(20000.0))))
    aspect = rng.uniform(0.7, 1.3, size=3)
    scale = (target / (4.0 / 3.0 * np.pi * np.prod(aspect))) ** (1.0 / 3.0)
    semi = np.minimum(aspect * scale, np.array([24.0, 24.0, 24.0]))
    radius = int(rng.integers(1, 4))
    bins = int(rng.choice([16, 32, 64]))
    centre = tuple(31.5 + rng.uniform(-6.0, 6.0, size=3))
    shape = (64, 64, 64)
    img = _ct_shared(shape, base_seed + index % 16)
    mask = ellipsoid(shape, centre, tuple(semi))
    return img, mask, radius, bins


_CT_SHARED = {}


def _ct_shared(shape, seed):
    """ct_like(shape, seed), computed once per process (callers must not
    modify it)."""
    key = (tuple(shape), seed)
    if key not in _CT_SHARED:
        _CT_SHARED[key] = ct_like(shape, seed)
    return _CT_SHARED[key]


def paper_tiled(reps=(1, 1, 1), seed=300):
    """A 61 x 55 x 39 (X x Y x Z) MR-like volume (positive smooth intensities)
    with a blob VOI of ~50.6k voxels (38.7 % of the box), repeated reps =
    (rx, ry, rz) times along the axes without interpolation."""
    shape = (39, 55, 61)
    rng = np.random.default_rng(seed)
    base = 400.0 + 120.0 * _smooth_noise(rng, shape, 3.0)
    base += rng.normal(0.0, 20.0, size=shape)
    img = np.clip(np.rint(base), 0, 4095).astype(np.int16)
    blob = _smooth_noise(rng, shape, 5.0)
    # keep the 50,613 voxels (38.7 % of the box) with the largest blob field
    keep = np.argsort(blob.reshape(-1), kind="stable")[-50613:]
    mask = np.zeros(blob.size, dtype=np.uint8)
    mask[keep] = 1
    mask = mask.reshape(shape)
    rx, ry, rz = reps
    return np.tile(img, (rz, ry, rx)), np.tile(mask, (rz, ry, rx))


def sample_voxels(mask, n, seed):
    """A seeded uniform sample (without replacement, sorted) of n VOI voxel
    linear indices."""
    vox = np.flatnonzero(mask.reshape(-1))
    if n >= vox.size:
        return vox.astype(np.int64)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(vox, size=n, replace=False)).astype(np.int64)


SERVED_SHAPES = ((32, 64, 64), (64, 64, 64), (64, 128, 128), (128, 128, 128), (128, 256, 256))


def served_requests(n, seed=200, median=50000.0, sigma=1.0, max_voxels=2000000,
                    min_voxels=1000, templates=None):
    """Requests of the served workload: ellipsoidal VOIs of log-normal size
    (median 50k voxels, sigma_ln 1.0, truncated to [1k, 2M]) with a random
    aspect ratio, each in the smallest standard CT-like volume shape that holds
    it; kernel radius uniform in {1, 2, 3}; FBN 64 or FBW 25 HU; all 93 maps.
    Returns a list of dicts with keys shape, mask, radius, disc (parameter
    overrides) and n_voi."""
    if templates is not None and templates < n:
        # n arrivals drawn from `templates` distinct requests, in turn (keeps
        # the host memory of long request streams bounded)
        base = served_requests(templates, seed, median, sigma, max_voxels, min_voxels)
        return [base[k % templates] for k in range(n)]
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        target = float(np.clip(np.exp(rng.normal(np.log(median), sigma)), min_voxels, max_voxels))
        aspect = rng.uniform(0.75, 1.25, size=3)
        scale = (target / (4.0 / 3.0 * np.pi * np.prod(aspect))) ** (1.0 / 3.0)
        semi = aspect * scale  # x, y, z
        shape = SERVED_SHAPES[-1]
        for sh in SERVED_SHAPES:
            if semi[0] <= sh[2] / 2 - 1 and semi[1] <= sh[1] / 2 - 1 and semi[2] <= sh[0] / 2 - 1:
                shape = sh
                break
        semi = np.minimum(semi, [shape[2] / 2 - 1, shape[1] / 2 - 1, shape[0] / 2 - 1])
        centre = ((shape[2] - 1) / 2, (shape[1] - 1) / 2, (shape[0] - 1) / 2)
        mask = ellipsoid(shape, centre, tuple(semi))
        radius = int(rng.integers(1, 4))
        disc = dict(disc_mode=0, bin_count=64) if rng.random() < 0.5 else \
            dict(disc_mode=1, bin_width=25.0)
        out.append(dict(shape=shape, mask=mask, radius=radius, disc=disc,
                        n_voi=int(mask.sum())))
    return out
