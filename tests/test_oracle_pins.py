"""Pins of the FP64 CPU oracle against facts fixed by the mathematics:
closed forms on phantoms, invariants, special cases that reduce to library
routines, and brute force by a second independent enumerator (naive_py).

None of these values comes from the CUDA path.  Feature definitions: IBSI,
which the paper's backends follow (Introduction; "IBSI compliance tests");
feature families and counts: Table 2.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import naive_py as NP
from oracle import oracle as O

FO, GLCM, GLRLM, GLSZM, GLDM, NGTDM = (slice(0, 18), slice(18, 42), slice(42, 58),
                                        slice(58, 74), slice(74, 88), slice(88, 93))


def names():
    return O.feature_names()


def _levels_params(levels, radius, ng, distance=1):
    p = O.make_params(levels.shape, disc_mode=O.FBN, bin_count=ng, radius=radius,
                      distance=distance)
    return p


def _lin(shape, z, y, x):
    return (z * shape[1] + y) * shape[2] + x


# --------------------------------------------------------------- discretisation

def test_fbn_ramp_closed_form():
    # x = 0..N-1 with FBN n: level = floor(n x / (N-1)) + 1, top value -> n.
    N, n = 1000, 16
    img = np.arange(N, dtype=np.int16).reshape(1, 1, N)
    mask = np.ones_like(img, dtype=np.uint8)
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=n)
    lev, ng, xmin, xmax = O.discretise(p, img, mask)
    x = np.arange(N)
    expect = np.minimum(n * x // (N - 1) + 1, n)
    assert ng == n and xmin == 0 and xmax == N - 1
    assert np.array_equal(lev.reshape(-1), expect)


def test_fbn_interval_membership_all_int16():
    # every int16 value: level g iff xmin + (g-1) D <= x < xmin + g D,
    # D = (xmax - xmin) / Ng, with x = xmax in the top bin (exact rationals).
    vals = np.arange(-32768, 32768, dtype=np.int32)
    img = vals.astype(np.int16).reshape(1, 256, 256)
    mask = np.ones(img.shape, np.uint8)
    for n in (1, 7, 64, 255):
        p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=n)
        lev, ng, xmin, xmax = O.discretise(p, img, mask)
        lev = lev.reshape(-1).astype(np.int64)
        assert lev.min() == 1 and lev.max() == n
        assert np.all(np.diff(lev) >= 0)
        # bin edges: first x of each level
        D = Fraction(xmax - xmin, n)
        for g in range(1, n + 1):
            first = xmin + (g - 1) * D
            first_int = math.ceil(first)
            idx = np.searchsorted(vals, first_int)
            assert lev[idx] == g
            if idx > 0:
                assert lev[idx - 1] == g - 1


@pytest.mark.parametrize("w", [25.0, 7.5, 0.3])
def test_fbw_interval_membership(w):
    rng = np.random.default_rng(4)
    img = rng.integers(-1200, 600, size=(6, 7, 8)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.7).astype(np.uint8)
    if w < 1:
        img = (img // 100).astype(np.int16)  # keep Ng <= 255
    p = O.make_params(img.shape, disc_mode=O.FBW, bin_width=w)
    lev, ng, xmin, xmax = O.discretise(p, img, mask)
    wf = Fraction(w)
    for x, g in zip(img[mask > 0].tolist(), lev[mask > 0].tolist()):
        # (x - xmin) / w in [g - 1, g)
        q = Fraction(int(x) - xmin) / wf
        assert g - 1 <= q < g
    assert ng == math.floor(Fraction(xmax - xmin) / wf) + 1
    assert np.all(lev[mask == 0] == 0)


def test_fbw_zero_floor_anchor():
    img = np.array([[[-37, -12, 0, 24, 25, 49, 51]]], np.int16)
    mask = np.ones_like(img, dtype=np.uint8)
    p = O.make_params(img.shape, disc_mode=O.FBW, bin_width=25.0,
                      fbw_anchor=O.ANCHOR_ZERO_FLOOR)
    lev, ng, _, _ = O.discretise(p, img, mask)
    # anchor floor(-37/25)*25 = -50: bins [-50,-25) [-25,0) [0,25) [25,50) [50,75)
    assert lev.reshape(-1).tolist() == [1, 2, 3, 3, 4, 4, 5]
    assert ng == 5


def test_discretise_errors():
    img = np.zeros((2, 2, 2), np.int16)
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=8)
    with pytest.raises(O.OracleError):
        O.discretise(p, img, np.zeros(img.shape, np.uint8))
    img2 = np.array([[[0, 3000]]], np.int16)
    p2 = O.make_params(img2.shape, disc_mode=O.FBW, bin_width=10.0)
    with pytest.raises(O.OracleError):
        O.discretise(p2, img2, np.ones(img2.shape, np.uint8))
    # constant VOI with FBN: all level 1
    lev, ng, _, _ = O.discretise(p, img + 5, np.ones(img.shape, np.uint8))
    assert np.all(lev == 1) and ng == 8


# --------------------------------------------------------------- phantoms

def _phantom(kind, r=2, size=7, ng=None):
    z, y, x = np.meshgrid(*[np.arange(size)] * 3, indexing="ij")
    if kind == "constant":
        lev = np.full((size,) * 3, 3, np.uint8)
        ng = ng or 4
    else:
        lev = (1 + (x + y + z) % 2).astype(np.uint8)
        ng = ng or 2
    c = size // 2
    return lev, ng, _lin(lev.shape, c, c, c)


def _pairs_full(s, d, delta=1):
    return int(np.prod([s - delta * abs(k) for k in d]))


def test_glcm_constant_closed_form():
    lev, ng, v = _phantom("constant")
    p = _levels_params(lev, 2, ng)
    m = O.matrices(p, lev, ng, v)["glcm"]
    for k, d in enumerate(O.directions()):
        expect = np.zeros((ng, ng), np.int64)
        expect[2, 2] = 2 * _pairs_full(5, d)
        assert np.array_equal(m[k], expect), d


def test_glcm_checkerboard_closed_form():
    lev, ng, v = _phantom("checker")
    p = _levels_params(lev, 2, ng)
    m = O.matrices(p, lev, ng, v)["glcm"]
    for k, d in enumerate(O.directions()):
        l1 = sum(abs(t) for t in d)
        T = m[k].sum()
        assert T == 2 * _pairs_full(5, d)
        if l1 % 2 == 1:  # axis and body diagonals: level always changes
            assert m[k][0, 0] == 0 and m[k][1, 1] == 0 and m[k][0, 1] == m[k][1, 0] == T // 2
        else:  # face diagonals: level never changes
            assert m[k][0, 1] == 0 and m[k][1, 0] == 0


def test_glcm_symmetry_and_totals_random():
    rng = np.random.default_rng(5)
    for trial in range(6):
        shape = (5, 6, 7)
        ng = int(rng.integers(2, 9))
        lev = rng.integers(1, ng + 1, size=shape).astype(np.uint8)
        lev[rng.random(shape) < 0.3] = 0
        r = int(rng.integers(1, 3))
        delta = int(rng.integers(1, 3))
        p = _levels_params(lev, r, ng, delta)
        for v in np.flatnonzero(lev.reshape(-1))[:5]:
            m = O.matrices(p, lev, ng, int(v))["glcm"]
            z, y, x = np.unravel_index(v, shape)
            cube, _ = NP.sub_voi(lev, None, (z, y, x), r)
            ref = NP.glcm(cube, ng, delta)
            assert np.array_equal(m, ref)
            for k, d in enumerate(O.directions()):
                assert np.array_equal(m[k], m[k].T)
                a, b = NP._shift_pairs(cube, d, delta)
                assert m[k].sum() == 2 * a.size


def test_glcm_features_checkerboard_axis():
    P = np.array([[0.0, 1.0], [1.0, 0.0]])
    f = dict(zip(names()[GLCM], O.glcm_features(P)))
    expect = {
        "glcm_Autocorrelation": 2.0, "glcm_JointAverage": 1.5,
        "glcm_ClusterProminence": 0.0, "glcm_ClusterShade": 0.0,
        "glcm_ClusterTendency": 0.0, "glcm_Contrast": 1.0, "glcm_Correlation": -1.0,
        "glcm_DifferenceAverage": 1.0, "glcm_DifferenceEntropy": 0.0,
        "glcm_DifferenceVariance": 0.0, "glcm_JointEnergy": 0.5,
        "glcm_JointEntropy": 1.0, "glcm_Imc1": -1.0,
        "glcm_Imc2": math.sqrt(1 - math.exp(-2.0)), "glcm_Idm": 0.5,
        "glcm_Idmn": 0.8, "glcm_Id": 0.5, "glcm_Idn": 2.0 / 3.0,
        "glcm_InverseVariance": 1.0, "glcm_MaximumProbability": 0.5,
        "glcm_SumAverage": 3.0, "glcm_SumEntropy": 0.0, "glcm_SumSquares": 0.25,
        "glcm_MCC": 1.0,
    }
    for k, v in expect.items():
        assert f[k] == pytest.approx(v, abs=1e-12), k


def test_glcm_features_constant():
    P = np.zeros((4, 4))
    P[2, 2] = 200
    f = dict(zip(names()[GLCM], O.glcm_features(P)))
    assert f["glcm_Idm"] == 1 and f["glcm_Id"] == 1 and f["glcm_Contrast"] == 0
    assert f["glcm_JointEnergy"] == 1 and f["glcm_JointEntropy"] == 0
    assert f["glcm_MaximumProbability"] == 1 and f["glcm_Imc2"] == 0
    assert f["glcm_Autocorrelation"] == 9 and f["glcm_SumAverage"] == 6
    for k in ("glcm_Correlation", "glcm_Imc1", "glcm_MCC"):
        assert math.isnan(f[k]), k
    assert np.all(np.isnan(O.glcm_features(np.zeros((3, 3)))))


def test_glcm_two_level_closed_forms():
    # counts [[a, b], [b, c]]: Correlation = phi = (ac - b^2)/((a+b)(b+c)),
    # MCC = |phi|, Contrast = 2b / T, JointAverage = 1 + (b + c)/T.
    rng = np.random.default_rng(6)
    for _ in range(50):
        a, b, c = (int(t) for t in rng.integers(1, 40, size=3))
        T = a + 2 * b + c
        f = dict(zip(names()[GLCM], O.glcm_features(np.array([[a, b], [b, c]]))))
        phi = (a * c - b * b) / ((a + b) * (b + c))
        assert f["glcm_Correlation"] == pytest.approx(phi, rel=1e-12, abs=1e-14)
        assert f["glcm_MCC"] == pytest.approx(abs(phi), rel=1e-10, abs=1e-12)
        assert f["glcm_Contrast"] == pytest.approx(2 * b / T, rel=1e-12)
        assert f["glcm_JointAverage"] == pytest.approx(1 + (b + c) / T, rel=1e-12)
        assert f["glcm_MaximumProbability"] == pytest.approx(max(a, b, c) / T)


def test_mcc_against_literal_q_eigenvalues():
    rng = np.random.default_rng(7)
    for _ in range(40):
        ng = int(rng.integers(2, 12))
        A = rng.integers(0, 6, size=(ng, ng)).astype(float)
        A[rng.random((ng, ng)) < 0.4] = 0
        C = A + A.T
        if C.sum() == 0:
            continue
        got = O.glcm_mcc(C)
        ref = NP.mcc_literal(C)
        if math.isnan(ref):
            assert math.isnan(got)
        else:
            assert got == pytest.approx(ref, abs=1e-7)


def test_glcm_features_against_naive_random():
    rng = np.random.default_rng(8)
    for _ in range(40):
        ng = int(rng.integers(2, 10))
        A = rng.integers(0, 5, size=(ng, ng)).astype(float)
        A[rng.random((ng, ng)) < 0.5] = 0
        C = A + A.T
        got = O.glcm_features(C)
        ref = NP.glcm_features(C, ng)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-7, equal_nan=True)


def test_glrlm_constant_and_checkerboard():
    s = 5
    lev, ng, v = _phantom("constant")
    p = _levels_params(lev, 2, ng)
    m = O.matrices(p, lev, ng, v)["glrlm"]
    for k, d in enumerate(O.directions()):
        # one run per line of the cube; sum_j j r = N_v
        assert m[k].sum() == s ** 3 - _pairs_full(s, d)
        assert (m[k][2] * np.arange(1, s + 1)).sum() == s ** 3
        if sum(abs(t) for t in d) == 1:
            assert m[k][2, s - 1] == s * s
    lev, ng, v = _phantom("checker")
    p = _levels_params(lev, 2, ng)
    m = O.matrices(p, lev, ng, v)["glrlm"]
    for k, d in enumerate(O.directions()):
        if sum(abs(t) for t in d) % 2 == 1:
            assert m[k][:, 1:].sum() == 0 and m[k][:, 0].sum() == s ** 3


def test_glrlm_run_starts_invariant_random():
    rng = np.random.default_rng(9)
    for _ in range(6):
        shape = (6, 6, 6)
        ng = int(rng.integers(2, 5))
        lev = rng.integers(1, ng + 1, size=shape).astype(np.uint8)
        lev[rng.random(shape) < 0.25] = 0
        r = int(rng.integers(1, 3))
        p = _levels_params(lev, r, ng)
        for v in np.flatnonzero(lev.reshape(-1))[:4]:
            z, y, x = np.unravel_index(v, shape)
            cube, _ = NP.sub_voi(lev, None, (z, y, x), r)
            m = O.matrices(p, lev, ng, int(v))["glrlm"]
            assert np.array_equal(m, NP.glrlm(cube, ng))
            nv = int((cube > 0).sum())
            for k in range(13):
                assert (m[k] * np.arange(1, 2 * r + 2)).sum() == nv


def test_glszm_phantoms_and_scipy_label():
    lev, ng, v = _phantom("constant")
    p = _levels_params(lev, 2, ng)
    z = O.matrices(p, lev, ng, v)["glszm"]
    assert z[2, 124] == 1 and z.sum() == 1
    lev, ng, v = _phantom("checker")
    p = _levels_params(lev, 2, ng)
    z = O.matrices(p, lev, ng, v)["glszm"]
    # 26-connectivity joins same-parity voxels (edge neighbours): one zone per level
    assert z.sum() == 2
    assert z[0].sum() == 1 and z[1].sum() == 1
    assert (z * np.arange(1, 126)).sum() == 125
    # isolated voxels: a sparse mask where no two VOI voxels touch
    iso = np.zeros((7, 7, 7), np.uint8)
    iso[1::2, 1::2, 1::2] = 2
    p = _levels_params(iso, 3, 2)
    z = O.matrices(p, iso, 2, _lin(iso.shape, 3, 3, 3))["glszm"]
    assert z[1, 0] == 27 and z.sum() == 27
    rng = np.random.default_rng(10)
    for _ in range(6):
        shape = (6, 6, 6)
        ng = int(rng.integers(2, 4))
        lev = rng.integers(1, ng + 1, size=shape).astype(np.uint8)
        lev[rng.random(shape) < 0.3] = 0
        p = _levels_params(lev, 2, ng)
        for v in np.flatnonzero(lev.reshape(-1))[:4]:
            zz, yy, xx = np.unravel_index(v, shape)
            cube, _ = NP.sub_voi(lev, None, (zz, yy, xx), 2)
            m = O.matrices(p, lev, ng, int(v))["glszm"]
            assert np.array_equal(m, NP.glszm(cube, ng))


def test_gldm_closed_forms():
    lev, ng, v = _phantom("constant")
    p = _levels_params(lev, 2, ng)
    m = O.matrices(p, lev, ng, v)["gldm"]
    # full 5^3 cube: a voxel with b coordinates on the cube boundary has
    # 3^(3-b) 2^b - 1 neighbours; there are C(3,b) 2^b 3^(3-b) such voxels.
    for b in range(4):
        k = 3 ** (3 - b) * 2 ** b - 1
        count = math.comb(3, b) * 2 ** b * 3 ** (3 - b)
        assert m[2, k] == count
    assert m.sum() == 125
    lev, ng, v = _phantom("checker")
    p = _levels_params(lev, 2, ng)
    m = O.matrices(p, lev, ng, v)["gldm"]
    assert m.sum() == 125
    # interior voxels of the cube (3^3 = 27) have the 12 edge neighbours equal
    assert m[:, 12].sum() >= 27


def test_gldm_ngtdm_against_naive_random():
    L = math.lcm(*range(1, 27))
    rng = np.random.default_rng(11)
    for _ in range(6):
        shape = (6, 6, 6)
        ng = int(rng.integers(2, 6))
        lev = rng.integers(1, ng + 1, size=shape).astype(np.uint8)
        lev[rng.random(shape) < 0.35] = 0
        r = int(rng.integers(1, 3))
        p = _levels_params(lev, r, ng)
        for v in np.flatnonzero(lev.reshape(-1))[:4]:
            zz, yy, xx = np.unravel_index(v, shape)
            cube, _ = NP.sub_voi(lev, None, (zz, yy, xx), r)
            m = O.matrices(p, lev, ng, int(v))
            assert np.array_equal(m["gldm"], NP.gldm(cube, ng))
            assert m["gldm"].sum() == (cube > 0).sum()
            n, s = NP.ngtdm_exact(cube, ng)
            assert m["ngtdm_n"].tolist() == n
            for i in range(ng):
                exact = s[i] * L
                assert exact.denominator == 1
                assert int(m["ngtdm_sl"][i]) == exact.numerator


def test_ngtdm_constant_and_two_level():
    f = O.ngtdm_features(np.array([0, 0, 125.0]), np.zeros(3))
    assert math.isnan(f[0]) and f[1] == 0.0 and math.isnan(f[2]) and f[3] == 0
    assert math.isnan(f[4])
    # two levels i=1, 2 with n = (n1, n2), s = (s1, s2):
    n1, n2, s1, s2 = 30.0, 10.0, 4.5, 7.25
    N = n1 + n2
    p1, p2 = n1 / N, n2 / N
    f = O.ngtdm_features(np.array([n1, n2]), np.array([s1, s2]))
    sps = p1 * s1 + p2 * s2
    assert f[0] == pytest.approx(1 / sps)
    assert f[1] == pytest.approx((2 * p1 * p2) / 2 * (s1 + s2) / N)
    assert f[2] == pytest.approx(sps / (2 * abs(p1 - 2 * p2)))
    assert f[3] == pytest.approx(2 * (p1 * s1 + p2 * s2) / (p1 + p2) / N)
    assert f[4] == pytest.approx(2 * (p1 + p2) / (s1 + s2))
    # levels 2 and 3 with n = (3, 2): 2 p_2 = 3 p_3 exactly, so busyness has a
    # zero denominator and is undefined, although 2 (0.6) - 3 (0.4) is not 0
    # in binary floating point
    f = O.ngtdm_features(np.array([0.0, 3.0, 2.0]), np.array([0.0, 1.5, 2.5]))
    assert 2 * 0.6 - 3 * 0.4 != 0.0
    assert math.isnan(f[2]) and math.isfinite(f[0]) and math.isfinite(f[4])


def test_ibsi_extras_closed_forms_and_identities():
    # ramp 0..10: median 5, median absolute deviation 30/11, CoV sqrt(10)/5,
    # P25 = 2.5, P75 = 7.5, QCoD = 0.5
    img = np.arange(11, dtype=np.int16).reshape(1, 1, 11)
    mask = np.ones_like(img, dtype=np.uint8)
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=4)
    lev, ng, _, _ = O.discretise(p, img, mask)
    f = O.scalar(p, img, lev, ng)
    assert f[93] == pytest.approx(30 / 11, rel=1e-14)
    assert f[94] == pytest.approx(math.sqrt(10) / 5, rel=1e-14)
    assert f[95] == pytest.approx(0.5, rel=1e-14)
    # the scalar-only standard deviation: the population variance of 0..10 is
    # (11^2 - 1) / 12 = 10
    assert f[101] == pytest.approx(math.sqrt(10), rel=1e-14)
    assert f[101] == pytest.approx(math.sqrt(f[16]), rel=1e-14)
    # on random windows: sum variance = cluster tendency and dissimilarity =
    # difference average (identities of a symmetric GLCM), dependence count
    # percentage = 1 (every voxel has a dependence count), GLNUN = GLNU / N_v
    rng = np.random.default_rng(52)
    img = rng.integers(0, 70, size=(7, 7, 7)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.7).astype(np.uint8)
    maps, vox, levels, ng = _oracle_maps(img, mask, disc_mode=O.FBN, bin_count=6, radius=2)
    nv = np.array([O.matrices(O.make_params(img.shape, disc_mode=O.FBN, bin_count=6, radius=2),
                              levels, ng, v)["hist"].sum() for v in vox])
    np.testing.assert_allclose(maps[96], maps[22], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(maps[97], maps[25], rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(maps[99], np.ones(len(vox)))
    np.testing.assert_allclose(maps[98], maps[76] / nv, rtol=1e-12)


def test_firstorder_closed_form_ramp():
    n = 11
    x = np.arange(n)
    f = dict(zip(names()[FO], O.firstorder_features(x, np.ones(n), 1)))
    assert f["firstorder_Mean"] == 5 and f["firstorder_Median"] == 5
    assert f["firstorder_Variance"] == pytest.approx((n * n - 1) / 12)
    assert f["firstorder_Skewness"] == pytest.approx(0, abs=1e-15)
    assert f["firstorder_Kurtosis"] == pytest.approx(-6 * (n * n + 1) / (5 * (n * n - 1)))
    assert f["firstorder_Energy"] == (n - 1) * n * (2 * n - 1) / 6
    assert f["firstorder_10Percentile"] == 1 and f["firstorder_90Percentile"] == 9
    assert f["firstorder_InterquartileRange"] == 5 and f["firstorder_Range"] == 10
    assert f["firstorder_MeanAbsoluteDeviation"] == pytest.approx(30 / 11)
    assert f["firstorder_RobustMeanAbsoluteDeviation"] == pytest.approx(20 / 9)
    assert f["firstorder_Entropy"] == 0 and f["firstorder_Uniformity"] == 1
    g = O.firstorder_features(x, np.ones(n), 1, kurtosis_excess=0)
    assert g[15] == pytest.approx(f["firstorder_Kurtosis"] + 3)
    one = O.firstorder_features(np.array([7]), np.array([1]), 1)
    assert math.isnan(one[14]) and math.isnan(one[15]) and one[16] == 0


def test_firstorder_against_numpy_scipy():
    rng = np.random.default_rng(12)
    for _ in range(30):
        n = int(rng.integers(2, 400))
        x = rng.integers(-1000, 1000, size=n)
        g = rng.integers(1, 9, size=n)
        got = O.firstorder_features(x, g, 8, voxel_volume=0.5)
        ref = NP.firstorder_features(x, g, 8, vvox=0.5)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-9)


# --------------------------------------------------------------- whole maps

def _oracle_maps(img, mask, **kw):
    p = O.make_params(img.shape, **kw)
    maps, vox, levels, ng = O.map_volume(p, img, mask, nthreads=2)
    return maps, vox, levels, ng


@pytest.mark.parametrize("r", [1, 2])
def test_maps_against_naive_enumerator(r):
    rng = np.random.default_rng(20 + r)
    img = rng.integers(0, 60, size=(6, 6, 6)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.75).astype(np.uint8)
    maps, vox, levels, ng = _oracle_maps(img, mask, disc_mode=O.FBN, bin_count=5,
                                         radius=r, spacing=(0.5, 0.8, 2.0))
    ref = NP.map_voxels(levels, img, ng, vox, r, vvox=0.8)
    np.testing.assert_allclose(maps, ref, rtol=1e-9, atol=1e-8, equal_nan=True)


def test_map_equals_scalar_when_window_covers_voi():
    # VOI inside a 3x3x3 box, r = 2: every window holds the whole VOI.
    rng = np.random.default_rng(30)
    img = rng.integers(-50, 50, size=(7, 7, 7)).astype(np.int16)
    mask = np.zeros(img.shape, np.uint8)
    mask[2:5, 2:5, 2:5] = (rng.random((3, 3, 3)) < 0.8)
    maps, vox, levels, ng = _oracle_maps(img, mask, disc_mode=O.FBN, bin_count=6, radius=2)
    whole = levels.copy()
    cube = np.zeros((5, 5, 5), np.int64)
    raw = np.zeros((5, 5, 5), np.int64)
    cube[1:4, 1:4, 1:4] = whole[2:5, 2:5, 2:5]
    raw[1:4, 1:4, 1:4] = img[2:5, 2:5, 2:5]
    scalar = NP.features_of_cube(cube, raw, ng)
    for k in range(maps.shape[1]):
        np.testing.assert_allclose(maps[:, k], scalar, rtol=1e-9, atol=1e-9, equal_nan=True)


@pytest.mark.parametrize("r", [1, 2])
def test_merged_maps_against_naive_enumerator(r):
    rng = np.random.default_rng(40 + r)
    img = rng.integers(0, 60, size=(6, 7, 6)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.75).astype(np.uint8)
    maps, vox, levels, ng = _oracle_maps(img, mask, disc_mode=O.FBN, bin_count=5,
                                         radius=r, aggregation=O.AGG_MERGED)
    ref = NP.map_voxels(levels, img, ng, vox, r, merged=True)
    np.testing.assert_allclose(maps, ref, rtol=1e-9, atol=1e-8, equal_nan=True)


def test_merged_linear_features_are_weighted_direction_means():
    # A feature linear in p = M / sum(M) over the merged matrix sum_d M_d is
    # the mean of the per-direction values weighted by each direction's total
    # (pairs for GLCM, runs for GLRLM); RunPercentage sum_d N_d / (13 N_v)
    # is exactly the plain direction mean.
    rng = np.random.default_rng(44)
    img = rng.integers(0, 90, size=(7, 7, 7)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.7).astype(np.uint8)
    kw = dict(disc_mode=O.FBN, bin_count=7, radius=2)
    mrg, vox, levels, ng = _oracle_maps(img, mask, aggregation=O.AGG_MERGED, **kw)
    avg, _, _, _ = _oracle_maps(img, mask, **kw)
    p = O.make_params(img.shape, **kw)
    lin_glcm = [18, 19, 23, 25, 32, 33, 34, 35, 36, 38]
    lin_glrlm = [42, 43, 52, 53, 54, 55, 56, 57]
    for k in range(0, len(vox), 7):
        mats = O.matrices(p, levels, ng, vox[k])
        nv = int(mats["hist"].sum())
        T = mats["glcm"].reshape(13, -1).sum(1).astype(np.float64)
        fg = np.array([O.glcm_features(mats["glcm"][d]) for d in range(13)])
        ok = T > 0
        want = (T[ok, None] * fg[ok][:, [f - 18 for f in lin_glcm]]).sum(0) / T[ok].sum()
        np.testing.assert_allclose(mrg[lin_glcm, k], want, rtol=1e-10, atol=1e-12)
        N = mats["glrlm"].reshape(13, -1).sum(1).astype(np.float64)
        fr = np.array([O.glrlm_features(mats["glrlm"][d], nv) for d in range(13)])
        want = (N[:, None] * fr[:, [f - 42 for f in lin_glrlm]]).sum(0) / N.sum()
        np.testing.assert_allclose(mrg[lin_glrlm, k], want, rtol=1e-10, atol=1e-12)
        assert mrg[48, k] == pytest.approx(avg[48, k], rel=1e-12)
    # families without a direction are the same in both modes
    np.testing.assert_array_equal(mrg[:18], avg[:18])
    np.testing.assert_array_equal(mrg[58:96], avg[58:96])
    np.testing.assert_array_equal(mrg[98:], avg[98:])


@pytest.mark.parametrize("kw", [dict(disc_mode=O.FBN, bin_count=6),
                                dict(disc_mode=O.FBW, bin_width=30.0),
                                dict(disc_mode=O.FBN, bin_count=5, aggregation=O.AGG_MERGED)])
def test_scalar_against_naive_whole_cube(kw):
    # scalar extraction = the features of the whole VOI, by brute force
    rng = np.random.default_rng(50)
    img = rng.integers(-100, 100, size=(9, 11, 10)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.6).astype(np.uint8)
    p = O.make_params(img.shape, spacing=(0.7, 1.0, 1.5), **kw)
    lev, ng, _, _ = O.discretise(p, img, mask)
    got = O.scalar(p, img, lev, ng)
    S = max(img.shape)
    cube = np.zeros((S, S, S), np.int64)
    raw = np.zeros((S, S, S), np.int64)
    cube[:9, :11, :10] = lev
    raw[:9, :11, :10] = img
    ref = NP.features_of_cube(cube, raw, ng, vvox=0.7 * 1.0 * 1.5,
                              merged=kw.get("aggregation", 0) == O.AGG_MERGED)
    np.testing.assert_allclose(got[:101], ref, rtol=1e-9, atol=1e-9, equal_nan=True)
    # the scalar-only statistic: numpy's population standard deviation
    assert got[101] == pytest.approx(float(np.std(img[mask > 0].astype(np.float64))), rel=1e-12)


def test_scalar_equals_every_map_value_when_windows_cover_the_voi():
    rng = np.random.default_rng(51)
    img = rng.integers(0, 500, size=(12, 12, 12)).astype(np.int16)
    mask = np.zeros(img.shape, np.uint8)
    mask[4:9, 3:8, 5:10] = rng.random((5, 5, 5)) < 0.7
    kw = dict(disc_mode=O.FBN, bin_count=8, radius=5)
    maps, vox, levels, ng = _oracle_maps(img, mask, **kw)
    sc = O.scalar(O.make_params(img.shape, **kw), img, levels, ng)
    for k in range(maps.shape[1]):
        np.testing.assert_allclose(maps[:, k], sc[:101], rtol=1e-12, atol=1e-12, equal_nan=True)


def test_map_flip_permutation_translation_equivariance():
    rng = np.random.default_rng(31)
    img = rng.integers(0, 40, size=(7, 6, 5)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.7).astype(np.uint8)
    kw = dict(disc_mode=O.FBN, bin_count=6, radius=1)
    base, vox, _, _ = _oracle_maps(img, mask, **kw)
    base_vol = np.full((O.NUM_FEATURES,) + img.shape, np.nan)
    base_vol.reshape(O.NUM_FEATURES, -1)[:, vox] = base
    for transform in (lambda a: a[::-1], lambda a: a[:, ::-1], lambda a: a[:, :, ::-1],
                      lambda a: np.transpose(a, (2, 0, 1)), lambda a: np.transpose(a, (1, 2, 0))):
        t_img = np.ascontiguousarray(transform(img))
        t_mask = np.ascontiguousarray(transform(mask))
        got, t_vox, _, _ = _oracle_maps(t_img, t_mask, **kw)
        vol = np.full((O.NUM_FEATURES,) + t_img.shape, np.nan)
        vol.reshape(O.NUM_FEATURES, -1)[:, t_vox] = got
        expect = np.stack([np.ascontiguousarray(transform(base_vol[f])) for f in range(O.NUM_FEATURES)])
        np.testing.assert_allclose(vol, expect, rtol=1e-9, atol=1e-9, equal_nan=True)
    # translation: zero padding outside the mask changes nothing
    pad_img = np.pad(img, 3, constant_values=0)
    pad_mask = np.pad(mask, 3, constant_values=0)
    got, _, _, _ = _oracle_maps(pad_img, pad_mask, **kw)
    np.testing.assert_allclose(got, base, rtol=0, atol=0, equal_nan=True)


def test_feature_names_are_the_101_default_maps():
    # Table 2: the 93-map benchmark column first, then the 8 maps that complete
    # the 101-map default column (+3 statistics, +2 GLCM, +3 NGLDM)
    n = names()
    assert len(n) == 101 and len(set(n)) == 101
    fam = [k.split("_")[0] for k in n]
    assert [fam[:93].count(f) for f in ("firstorder", "glcm", "glrlm", "glszm", "gldm", "ngtdm")] == \
        [18, 24, 16, 16, 14, 5]
    assert [fam.count(f) for f in ("firstorder", "glcm", "glrlm", "glszm", "gldm", "ngtdm")] == \
        [21, 26, 16, 16, 17, 5]
    assert sorted(O.directions()) == sorted(
        d for d in itertools.product((-1, 0, 1), repeat=3) if d > (0, 0, 0))


def test_given_discretisation_range():
    # the VOI's own range given explicitly changes nothing; a z-slab given the
    # whole VOI's range gets the whole volume's levels on its voxels; a
    # narrower range clamps (FBN 4 over [10, 30]: x <= 10 -> 1, x >= 30 -> 4)
    rng = np.random.default_rng(70)
    img = rng.integers(-200, 200, size=(9, 6, 5)).astype(np.int16)
    mask = (rng.random(img.shape) < 0.7).astype(np.uint8)
    for kw in (dict(disc_mode=O.FBN, bin_count=7), dict(disc_mode=O.FBW, bin_width=30.0),
               dict(disc_mode=O.FBW, bin_width=30.0, fbw_anchor=O.ANCHOR_ZERO_FLOOR)):
        lev, ng, lo, hi = O.discretise(O.make_params(img.shape, **kw), img, mask)
        lev2, ng2, _, _ = O.discretise(O.make_params(img.shape, value_range=(lo, hi), **kw),
                                       img, mask)
        assert ng2 == ng and np.array_equal(lev2, lev)
        sub = slice(3, 7)
        lev3, ng3, _, _ = O.discretise(O.make_params(img[sub].shape, value_range=(lo, hi), **kw),
                                       img[sub], mask[sub])
        assert ng3 == ng and np.array_equal(lev3, lev[sub])
    x = np.array([[[0, 10, 15, 20, 25, 30, 99]]], np.int16)
    lev, ng, _, _ = O.discretise(O.make_params(x.shape, disc_mode=O.FBN, bin_count=4,
                                               value_range=(10, 30)), x, np.ones_like(x, np.uint8))
    # g = floor(4 (x - 10) / 20) + 1 on the clamped x, top bin at x = 30
    assert lev.reshape(-1).tolist() == [1, 1, 2, 3, 4, 4, 4] and ng == 4
