"""HDF5 drain (fr_h5_write_maps / fr_h5_write_scalar): the files read back,
value by value, through an independent reader of the HDF5 format
(tests/h5read.py), which is itself checked first on a file written by the
HDF5 library.  Host only: no GPU."""
import os

import numpy as np
import pytest

import h5read
import paper_2609_19190_gb300 as fm
from paper_2609_19190_gb300 import _lib

LIBHDF5_FILE = None
try:
    import scipy
    LIBHDF5_FILE = os.path.join(os.path.dirname(scipy.__file__), "io", "matlab", "tests", "data",
                                "testhdf5_7.4_GLNX86.mat")
except ImportError:  # pragma: no cover
    pass


def test_reader_reads_a_file_written_by_the_hdf5_library():
    # SciPy's MATLAB 7.3 test file (HDF5 library output, 512-byte user block):
    # one double column testdouble = 0 : pi/4 : 2 pi with MATLAB_class "double"
    if LIBHDF5_FILE is None or not os.path.exists(LIBHDF5_FILE):
        pytest.skip("SciPy's HDF5 test file is not installed")
    f = h5read.File(LIBHDF5_FILE)
    assert f.base == 512
    items = dict(h5read.walk(f.root))
    assert list(items) == ["/testdouble"]
    ds = items["/testdouble"]
    assert ds.shape == (9, 1) and ds.dtype == np.float64
    np.testing.assert_allclose(ds.data[:, 0], np.arange(9) * np.pi / 4, rtol=0, atol=1e-15)
    assert ds.attrs["MATLAB_class"].tobytes() == b"double"


def _volume(seed, shape, frac=0.5, hole=True):
    rng = np.random.default_rng(seed)
    img = rng.integers(-1000, 1000, size=shape).astype(np.int16)
    mask = (rng.random(shape) < frac).astype(np.uint8)
    if hole:  # a slab of the volume outside the VOI: whole chunks without a voxel
        mask[:, :, : shape[2] // 2] = 0
    return img, mask


def _maps(seed, rows, n):
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((rows, n)).astype(np.float32)
    m[rng.random((rows, n)) < 0.05] = np.nan
    return m


def _expected_dense(maps, vox, shape):
    out = np.full((maps.shape[0],) + shape, np.nan, np.float32).reshape(maps.shape[0], -1)
    out[:, vox] = maps
    return out.reshape((maps.shape[0],) + shape)


@pytest.mark.parametrize("codec,shuffle", [("none", False), ("gzip", True), ("gzip", False),
                                           ("lzf", True)])
def test_spatial_file_round_trip(tmp_path, codec, shuffle):
    shape = (13, 17, 19)
    img, mask = _volume(1, shape)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int32)
    feats = list(range(101))  # 101 maps: several symbol-table nodes in /maps
    p = fm.fr_map_params_init(shape[2], shape[1], shape[0], features=feats, disc_mode=fm.FR_FBW,
                              bin_width=25.0, kernel_radius=2, spacing=(0.7, 0.8, 2.5))
    maps = _maps(2, len(feats), vox.size)
    path = tmp_path / ("maps_%s.h5" % codec)
    fm.fr_h5_write_maps(path, p, img, mask, maps, vox, origin=(1.5, -2.0, 30.0),
                        source_id="synthetic seed 1", codec=codec, shuffle=shuffle, threads=3,
                        chunk=(5, 8, 7))
    f = h5read.File(path)
    root = f.root
    assert set(root.members) == {"image", "mask", "maps"}
    np.testing.assert_array_equal(root.members["image"].data, img)
    np.testing.assert_array_equal(root.members["mask"].data, mask)
    a = root.attrs
    assert a["mode"].tobytes().rstrip(b"\0") == b"spatial"
    assert list(a["shape_zyx"]) == list(shape)
    np.testing.assert_array_equal(a["spacing_xyz_mm"], [0.7, 0.8, 2.5])
    np.testing.assert_array_equal(a["origin_xyz_mm"], [1.5, -2.0, 30.0])
    assert a["discretisation"].tobytes().rstrip(b"\0") == b"FBW"
    assert float(a["bin_width"][0]) == 25.0 and int(a["kernel_radius"][0]) == 2
    assert list(a["feature_ids"]) == feats
    assert a["source"].tobytes().rstrip(b"\0") == b"synthetic seed 1"
    names = fm.fr_feature_names()
    dense = _expected_dense(maps, vox, shape)
    got = root.members["maps"].members
    assert set(got) == {names[k] for k in feats}
    for r, k in enumerate(feats):
        ds = got[names[k]]
        assert int(ds.attrs["feature_id"][0]) == k and ds.chunks == (5, 8, 7)
        # bit-exact, NaN outside the VOI and where the map is NaN
        np.testing.assert_array_equal(ds.data.view(np.uint32), dense[r].view(np.uint32))
        ids = {fl[0] for fl in ds.filters}
        assert ids == {"none": set(), "gzip": {1} | ({2} if shuffle else set()),
                       "lzf": {2, 32000}}[codec]


def test_map_chunks_without_voi_voxels_are_not_stored(tmp_path):
    shape = (8, 8, 16)
    img, mask = _volume(3, shape, frac=1.0)  # x < 8 empty, x >= 8 full
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int32)
    p = fm.fr_map_params_init(16, 8, 8, features=[0, 18])
    maps = _maps(4, 2, vox.size)
    path = tmp_path / "holes.h5"
    fm.fr_h5_write_maps(path, p, img, mask, maps, vox, chunk=(8, 8, 8))
    f = h5read.File(path)
    ds = f.root.members["maps"].members[fm.fr_feature_names()[18]]
    # the dataset's B-tree lists only the chunk at x = 8; the other reads as NaN
    assert ds.stored == [(0, 0, 8)]
    assert f.root.members["image"].stored == [(0, 0, 0), (0, 0, 8)]
    assert np.isnan(ds.data[:, :, :8]).all()
    np.testing.assert_array_equal(ds.data.reshape(-1)[vox], maps[1])


def test_chunk_grid_is_bounded_to_one_btree_node(tmp_path):
    shape = (20, 24, 28)
    img, mask = _volume(5, shape, hole=False)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int32)
    p = fm.fr_map_params_init(28, 24, 20, features=[7])
    maps = _maps(6, 1, vox.size)
    path = tmp_path / "grid.h5"
    fm.fr_h5_write_maps(path, p, img, mask, maps, vox, chunk=(2, 2, 2))
    ds = h5read.File(path).root.members["maps"].members[fm.fr_feature_names()[7]]
    n = np.prod([-(-s // c) for s, c in zip(shape, ds.chunks)])
    assert n <= 64
    np.testing.assert_array_equal(ds.data.reshape(-1)[vox], maps[0])


def test_scalar_file_round_trip(tmp_path):
    shape = (6, 7, 8)
    img, mask = _volume(7, shape, hole=False)
    feats = [0, 5, 18, 41, 42, 58, 74, 88, 93, 100]
    p = fm.fr_map_params_init(8, 7, 6, features=feats)
    vals = np.random.default_rng(8).standard_normal(len(feats))
    vals[3] = np.nan
    path = tmp_path / "scalar.h5"
    fm.fr_h5_write_scalar(path, p, img, mask, vals, codec="lzf")
    f = h5read.File(path)
    g = f.root.members["features"].members
    names = [n.rstrip(b"\0").decode() for n in g["names"].data]
    assert names == [fm.fr_feature_names()[k] for k in feats]
    np.testing.assert_array_equal(g["values"].data.view(np.uint64), vals.view(np.uint64))
    assert f.root.attrs["mode"].tobytes().rstrip(b"\0") == b"scalar"
    np.testing.assert_array_equal(f.root.members["image"].data, img)


def test_drain_errors():
    shape = (4, 4, 4)
    img, mask = _volume(9, shape, hole=False)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int32)
    p = fm.fr_map_params_init(4, 4, 4, features=[0, 1])
    with pytest.raises(_lib.FlashmapError) as e:  # one row for two selected maps
        fm.fr_h5_write_maps("/nonexistent-dir/x.h5", p, img, mask, _maps(1, 1, vox.size), vox)
    assert e.value.status == 1
    with pytest.raises(_lib.FlashmapError) as e:  # the file cannot be created
        fm.fr_h5_write_maps("/nonexistent-dir/x.h5", p, img, mask, _maps(1, 2, vox.size), vox)
    assert e.value.status == 9
    bad = vox.copy()
    bad[0] = 64  # outside the 4^3 volume
    with pytest.raises(_lib.FlashmapError) as e:
        fm.fr_h5_write_maps("/nonexistent-dir/x.h5", p, img, mask, _maps(1, 2, vox.size), bad)
    assert e.value.status == 1


@pytest.mark.parametrize("shape,chunk", [((1, 1, 1), None), ((3, 2, 5), (8, 8, 8)),
                                         ((2, 9, 4), (1, 1, 1)), ((40, 3, 3), None)])
def test_spatial_edge_shapes(tmp_path, shape, chunk):
    # a single voxel, chunks larger than the volume (clamped), tiny chunks
    # (grown to at most 64), a long thin volume
    img, mask = _volume(11, shape, frac=1.0, hole=False)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int32)
    p = fm.fr_map_params_init(shape[2], shape[1], shape[0], features=[0, 92, 100])
    maps = _maps(12, 3, vox.size)
    path = tmp_path / "edge.h5"
    fm.fr_h5_write_maps(path, p, img, mask, maps, vox, codec="gzip", chunk=chunk)
    f = h5read.File(path)
    names = fm.fr_feature_names()
    dense = _expected_dense(maps, vox, shape)
    for r, k in enumerate([0, 92, 100]):
        ds = f.root.members["maps"].members[names[k]]
        assert all(c <= s for c, s in zip(ds.chunks, shape))
        assert np.prod([-(-s // c) for s, c in zip(shape, ds.chunks)]) <= 64
        np.testing.assert_array_equal(ds.data.view(np.uint32), dense[r].view(np.uint32))
    np.testing.assert_array_equal(f.root.members["image"].data, img)


def test_options_defaults_and_bad_options():
    opt = _lib.H5Options()
    assert _lib.load().fr_h5_options_init(opt) == 0
    assert (opt.codec, opt.level, opt.shuffle, opt.threads) == (fm.FR_H5_GZIP, 4, 1, 0)
    assert list(opt.chunk) == [0, 0, 0]
    shape = (4, 4, 4)
    img, mask = _volume(13, shape, hole=False)
    vox = np.flatnonzero(mask.reshape(-1)).astype(np.int32)
    p = fm.fr_map_params_init(4, 4, 4, features=[0])
    for kw in (dict(codec="gzip", level=10), dict(codec="gzip", level=-1)):
        with pytest.raises(_lib.FlashmapError) as e:
            fm.fr_h5_write_maps("/nonexistent-dir/x.h5", p, img, mask, _maps(1, 1, vox.size), vox,
                                **kw)
        assert e.value.status == 1
