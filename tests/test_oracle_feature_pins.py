"""Pins of the oracle's texture-feature formulas by values worked out by hand.

Every expected value below is a literal fraction (or a literal entropy of
literal probabilities) derived on paper from the IBSI definitions that the
paper's backends follow (Introduction; "IBSI compliance tests"), for
matrices whose entries are themselves fixed by hand: a small run-length
matrix with unequal row and column sums, the constant and checkerboard
phantoms (whose runs, zones and dependences follow from counting lattice
lines and neighbours), and a three-level co-occurrence matrix whose second
eigenvalue is found from its trace and determinant.  None of the expected
values is computed by a formula of the oracle's kind, so a misread
definition (GLNU against RLNU normalisation, the mean in RunVariance, the
exponents of the emphasis features, the Ng of Idmn) fails here.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import oracle as O

GLCM, GLRLM, GLSZM, GLDM = slice(18, 42), slice(42, 58), slice(58, 74), slice(74, 88)
L2 = math.log2


def _ent(*ps):
    """-sum p log2 p of literal probabilities."""
    return -sum(float(p) * L2(float(p)) for p in ps if p)


def _check(got, names, expect):
    for name, v in expect.items():
        k = names.index(name)
        assert got[k] == pytest.approx(float(v), rel=1e-12, abs=1e-15), name


RL_NAMES = ["SRE", "LRE", "GLNU", "GLNUN", "RLNU", "RLNUN", "RP", "GLV", "RV", "RE",
            "LGLRE", "HGLRE", "SRLGLE", "SRHGLE", "LRLGLE", "LRHGLE"]
DM_NAMES = ["SDE", "LDE", "GLNU", "DNU", "DNUN", "GLV", "DV", "DE", "LGLE", "HGLE",
            "SDLGLE", "SDHGLE", "LDLGLE", "LDHGLE"]

# ------------------------------------------------------------ a hand matrix
# Rows: gray levels 1, 2; columns: run length (zone size, dependence) 1, 2, 3.
#   level 1: two of length 1, one of length 3;  level 2: three of length 2.
# N = 6; p(1,1) = 1/3, p(1,3) = 1/6, p(2,2) = 1/2; voxels 2 + 3 + 6 = 11.
HAND = np.array([[2.0, 0.0, 1.0], [0.0, 3.0, 0.0]])
HAND_RL = {
    # sum p / j^2 = 1/3 + 1/54 + 1/8
    "SRE": F(103, 216),
    # sum p j^2 = 1/3 + 3/2 + 2
    "LRE": F(23, 6),
    # row sums (3, 3): (9 + 9) / 6 and / 36
    "GLNU": F(3), "GLNUN": F(1, 2),
    # column sums (2, 3, 1): (4 + 9 + 1) / 6 and / 36
    "RLNU": F(7, 3), "RLNUN": F(7, 18),
    "RP": F(6, 11),
    # mean level 3/2, each level a quarter away squared
    "GLV": F(1, 4),
    # mean length 1/3 + 1/2 + 1 = 11/6: (25/36)/3 + (49/36)/6 + (1/36)/2
    "RV": F(17, 36),
    "RE": _ent(F(1, 3), F(1, 6), F(1, 2)),
    # sum p / i^2 = 1/2 + 1/8; sum p i^2 = 1/2 + 2
    "LGLRE": F(5, 8), "HGLRE": F(5, 2),
    # sum p/(i^2 j^2) = 1/3 + 1/54 + 1/32
    "SRLGLE": F(331, 864),
    # sum p i^2 / j^2 = 1/3 + 1/54 + 1/2
    "SRHGLE": F(23, 27),
    # sum p j^2 / i^2 = 1/3 + 3/2 + 1/2
    "LRLGLE": F(7, 3),
    # sum p i^2 j^2 = 1/3 + 3/2 + 8
    "LRHGLE": F(59, 6),
}


def test_run_length_features_of_a_hand_matrix():
    _check(O.glrlm_features(HAND, 11), RL_NAMES, HAND_RL)


def test_size_zone_features_of_a_hand_matrix():
    # the GLSZM features read the same matrix as zones of size 1, 2, 3
    _check(O.glszm_features(HAND, 11), RL_NAMES, HAND_RL)


def test_dependence_features_of_a_hand_matrix():
    expect = {"SDE": HAND_RL["SRE"], "LDE": HAND_RL["LRE"], "GLNU": F(3), "DNU": F(7, 3),
              "DNUN": F(7, 18), "GLV": F(1, 4), "DV": F(17, 36), "DE": HAND_RL["RE"],
              "LGLE": F(5, 8), "HGLE": F(5, 2), "SDLGLE": F(331, 864), "SDHGLE": F(23, 27),
              "LDLGLE": F(7, 3), "LDHGLE": F(59, 6)}
    _check(O.gldm_features(HAND), DM_NAMES, expect)


# ------------------------------------------------------------ phantoms
def _cube(kind, level=3, size=7):
    z, y, x = np.meshgrid(*[np.arange(size)] * 3, indexing="ij")
    if kind == "constant":
        lev = np.full((size,) * 3, level, np.uint8)
    else:
        lev = (1 + (x + y + z) % 2).astype(np.uint8)
    c = size // 2
    return lev, (c * size + c) * size + c


def _matrices(lev, ng, v, r=2):
    p = O.make_params(lev.shape, disc_mode=O.FBN, bin_count=ng, radius=r)
    return O.matrices(p, lev, ng, v)


def _dir_class(d):
    """axis, face-diagonal or body-diagonal direction"""
    nz = sum(1 for t in d if t)
    return {1: "axis", 2: "face", 3: "body"}[nz]


def _constant_run_features(i2):
    """GLRLM features of one direction of the constant 5^3 window at a level
    with i^2 = i2, by direction class.  Runs are the lattice lines:
      axis: 25 lines of length 5;
      face diagonal: per slice the diagonals 1,2,3,4,5,4,3,2,1, so lengths
        1..5 occur 10, 10, 10, 10, 5 times (45 runs);
      body diagonal: a line starts where a coordinate is 0 and has length
        5 - (largest start coordinate): lengths 1..5 occur 24, 18, 12, 6, 1
        times (61 runs = 125 - 64)."""
    i2 = F(i2)
    axis = {"SRE": F(1, 25), "LRE": F(25), "GLNU": F(25), "GLNUN": F(1), "RLNU": F(25),
            "RLNUN": F(1), "RP": F(1, 5), "GLV": F(0), "RV": F(0), "RE": 0.0,
            "SRLGLE": F(1, 25) / i2, "SRHGLE": F(1, 25) * i2, "LRLGLE": F(25) / i2,
            "LRHGLE": F(25) * i2}
    # face: sum c/j^2 = 10 + 5/2 + 10/9 + 5/8 + 1/5 = 5197/360 over 45 runs;
    # sum c j^2 = 425; column sums 10,10,10,10,5 -> 425; mean length 25/9
    sre_f, lre_f = F(5197, 16200), F(85, 9)
    face = {"SRE": sre_f, "LRE": lre_f, "GLNU": F(45), "GLNUN": F(1), "RLNU": F(85, 9),
            "RLNUN": F(17, 81), "RP": F(9, 25), "GLV": F(0), "RV": F(140, 81),
            "RE": _ent(*[F(2, 9)] * 4, F(1, 9)),
            "SRLGLE": sre_f / i2, "SRHGLE": sre_f * i2, "LRLGLE": lre_f / i2,
            "LRHGLE": lre_f * i2}
    # body: sum c/j^2 = 24 + 9/2 + 4/3 + 3/8 + 1/25 = 18149/600 over 61 runs;
    # sum c j^2 = 325; column sums squared 576+324+144+36+1 = 1081;
    # mean length 125/61, so RV = 325/61 - (125/61)^2 = 4200/3721
    sre_b, lre_b = F(18149, 36600), F(325, 61)
    body = {"SRE": sre_b, "LRE": lre_b, "GLNU": F(61), "GLNUN": F(1), "RLNU": F(1081, 61),
            "RLNUN": F(1081, 3721), "RP": F(61, 125), "GLV": F(0), "RV": F(4200, 3721),
            "RE": _ent(F(24, 61), F(18, 61), F(12, 61), F(6, 61), F(1, 61)),
            "SRLGLE": sre_b / i2, "SRHGLE": sre_b * i2, "LRLGLE": lre_b / i2,
            "LRHGLE": lre_b * i2}
    for d in (axis, face, body):
        d["LGLRE"], d["HGLRE"] = 1 / i2, i2
    return {"axis": axis, "face": face, "body": body}


def test_glrlm_constant_window_run_lengths_and_features():
    lev, v = _cube("constant", level=3)
    m = _matrices(lev, 4, v)["glrlm"]
    hist = {"axis": [0, 0, 0, 0, 25], "face": [10, 10, 10, 10, 5], "body": [24, 18, 12, 6, 1]}
    exp = _constant_run_features(9)
    for k, d in enumerate(O.directions()):
        cls = _dir_class(d)
        assert m[k][2].tolist() == hist[cls], d
        assert m[k][[0, 1, 3]].sum() == 0
        _check(O.glrlm_features(m[k], 125), RL_NAMES, exp[cls])


def test_glrlm_checkerboard_axis_and_body_features():
    # axis and body-diagonal steps change x + y + z by an odd amount, so every
    # run has length 1.  The window (coordinates 1..5 of the 7^3 lattice) holds
    # 62 voxels of even coordinate sum (level 1) and 63 of odd sum (level 2):
    # even sums need 0 or 2 odd coordinates, 2^3 + 3 * 3^2 * 2 = 62.
    lev, v = _cube("checker")
    m = _matrices(lev, 2, v)["glrlm"]
    expect = {"SRE": F(1), "LRE": F(1), "GLNU": F(62 ** 2 + 63 ** 2, 125),
              "GLNUN": F(7813, 15625), "RLNU": F(125), "RLNUN": F(1), "RP": F(1),
              "GLV": F(62 * 63, 125 ** 2), "RV": F(0), "RE": _ent(F(62, 125), F(63, 125)),
              "LGLRE": F(311, 500), "HGLRE": F(314, 125), "SRLGLE": F(311, 500),
              "SRHGLE": F(314, 125), "LRLGLE": F(311, 500), "LRHGLE": F(314, 125)}
    for k, d in enumerate(O.directions()):
        if _dir_class(d) == "face":
            continue
        assert m[k][:, 0].tolist() == [62, 63] and m[k][:, 1:].sum() == 0, d
        _check(O.glrlm_features(m[k], 125), RL_NAMES, expect)


def test_glszm_constant_and_checkerboard_features():
    # constant: one zone of 125 voxels at level 3
    lev, v = _cube("constant", level=3)
    z = _matrices(lev, 4, v)["glszm"]
    n = 125
    expect = {"SRE": F(1, n * n), "LRE": F(n * n), "GLNU": F(1), "GLNUN": F(1), "RLNU": F(1),
              "RLNUN": F(1), "RP": F(1, n), "GLV": F(0), "RV": F(0), "RE": 0.0,
              "LGLRE": F(1, 9), "HGLRE": F(9), "SRLGLE": F(1, 9 * n * n),
              "SRHGLE": F(9, n * n), "LRLGLE": F(n * n, 9), "LRHGLE": F(9 * n * n)}
    _check(O.glszm_features(z, 125), RL_NAMES, expect)
    # checkerboard, 26-connected: one zone per level, 62 voxels at level 1
    # and 63 at level 2 (edge neighbours share the parity)
    lev, v = _cube("checker")
    z = _matrices(lev, 2, v)["glszm"]
    assert z[0, 61] == 1 and z[1, 62] == 1 and z.sum() == 2
    a, b = F(1, 62 ** 2), F(1, 63 ** 2)
    expect = {"SRE": (a + b) / 2, "LRE": F(62 ** 2 + 63 ** 2, 2), "GLNU": F(1),
              "GLNUN": F(1, 2), "RLNU": F(1), "RLNUN": F(1, 2), "RP": F(2, 125),
              "GLV": F(1, 4), "RV": F(1, 4), "RE": 1.0, "LGLRE": F(5, 8), "HGLRE": F(5, 2),
              "SRLGLE": (a + b / 4) / 2, "SRHGLE": (a + 4 * b) / 2,
              "LRLGLE": F(62 ** 2 * 4 + 63 ** 2, 8), "LRHGLE": F(62 ** 2 + 4 * 63 ** 2, 2)}
    _check(O.glszm_features(z, 125), RL_NAMES, expect)


def test_gldm_constant_cube_features():
    # full 5^3 cube at level 3: a voxel with b coordinates on the cube's
    # boundary has 3^(3-b) 2^b - 1 equal neighbours, so dependence j = k + 1
    # takes 27, 18, 12, 8 for 27, 54, 36, 8 voxels.
    lev, v = _cube("constant", level=3)
    m = _matrices(lev, 4, v)["gldm"]
    assert {j + 1: int(c) for j, c in enumerate(m[2]) if c} == {27: 27, 18: 54, 12: 36, 8: 8}
    expect = {
        # sum c / j^2 = 1/27 + 1/6 + 1/4 + 1/8 = 125/216, over 125
        "SDE": F(1, 216),
        # sum c j^2 = 19683 + 17496 + 5184 + 512 = 42875 = 125 * 343
        "LDE": F(343),
        "GLNU": F(125),
        # 27^2 + 54^2 + 36^2 + 8^2 = 5005
        "DNU": F(5005, 125), "DNUN": F(5005, 125 ** 2),
        "GLV": F(0),
        # mean dependence 2197/125, second moment 343
        "DV": F(343) - F(2197, 125) ** 2,
        "DE": _ent(F(27, 125), F(54, 125), F(36, 125), F(8, 125)),
        "LGLE": F(1, 9), "HGLE": F(9), "SDLGLE": F(1, 216 * 9), "SDHGLE": F(9, 216),
        "LDLGLE": F(343, 9), "LDHGLE": F(343 * 9),
    }
    _check(O.gldm_features(m), DM_NAMES, expect)


def test_gldm_checkerboard_dependence_counts():
    # Equal neighbours of a checkerboard voxel are its in-window edge
    # neighbours (two of dz, dy, dx nonzero): 12 inside, 8 with one boundary
    # coordinate, 5 with two, 3 at a corner (j = 13, 9, 6, 4).  The window
    # spans lattice coordinates 1..5, whose boundary values 1 and 5 are odd and
    # whose inner values 2, 3, 4 are even, odd, even; the level follows the
    # parity of the coordinate sum, which splits the classes as
    #   inner 27: 14 even (level 1), 13 odd;  one boundary 54: 24 / 30;
    #   two boundary 36: 24 / 12;  corners 8: 0 / 8.
    lev, v = _cube("checker")
    m = _matrices(lev, 2, v)["gldm"]
    got = [{j + 1: int(c) for j, c in enumerate(m[a]) if c} for a in range(2)]
    assert got == [{13: 14, 9: 24, 6: 24}, {13: 13, 9: 30, 6: 12, 4: 8}]


def test_glrlm_glszm_gldm_maps_of_a_constant_volume():
    # the whole chain through the map path: a constant image discretises to
    # level 1; the centre voxel's window is the full 5^3 cube, so its GLRLM
    # maps are the direction means (3 axis, 6 face, 4 body directions) of the
    # class values above, and its GLSZM / GLDM maps the one-matrix values.
    img = np.full((7, 7, 7), 40, np.int16)
    mask = np.ones(img.shape, np.uint8)
    p = O.make_params(img.shape, disc_mode=O.FBN, bin_count=4, radius=2)
    levels, ng, _, _ = O.discretise(p, img, mask)
    assert ng == 4 and np.all(levels == 1)
    out = O.map_voxels(p, img, levels, ng, np.array([(3 * 7 + 3) * 7 + 3]), nthreads=1)[:, 0]
    cls = _constant_run_features(1)
    mean = {}
    for name in RL_NAMES:
        a, f, b = (cls[c][name] for c in ("axis", "face", "body"))
        mean[name] = (3 * a + 6 * f + 4 * b) / 13
    _check(out[GLRLM], RL_NAMES, mean)
    n = 125
    _check(out[GLSZM], RL_NAMES, {"SRE": F(1, n * n), "LRE": F(n * n), "RP": F(1, n),
                                  "LRHGLE": F(n * n), "SRLGLE": F(1, n * n)})
    _check(out[GLDM], DM_NAMES, {"SDE": F(1, 216), "LDE": F(343), "DNU": F(5005, 125),
                                 "LDLGLE": F(343), "SDHGLE": F(1, 216)})


# ------------------------------------------------------------ GLCM by hand
GLCM_NAMES = ["Autocorrelation", "JointAverage", "ClusterProminence", "ClusterShade",
              "ClusterTendency", "Contrast", "Correlation", "DifferenceAverage",
              "DifferenceEntropy", "DifferenceVariance", "JointEnergy", "JointEntropy",
              "Imc1", "Imc2", "Idm", "Idmn", "Id", "Idn", "InverseVariance",
              "MaximumProbability", "SumAverage", "SumEntropy", "SumSquares", "MCC"]


def _three_level(ng):
    # symmetric counts over levels 1..3 (total 12):
    #   p11 = 1/3, p12 = p21 = 1/6, p23 = p32 = 1/12, p33 = 1/6, p22 = 0
    C = np.zeros((ng, ng))
    C[:3, :3] = [[4, 2, 0], [2, 0, 1], [0, 1, 2]]
    return C


def _three_level_expect(ng):
    l3 = L2(3)
    # marginals (1/2, 1/4, 1/4); mean 7/4; variance 9/32 + 1/64 + 25/64 = 11/16;
    # sum i j p = 1/3 + 2/3 + 1 + 3/2 = 7/2, so the covariance is 7/16.
    # With t = i + j - 7/2 the mass sits at t = -3/2 (1/3), -1/2 (1/3),
    # 3/2 (1/6), 5/2 (1/6).
    # HX = 3/2; HXY = log2 3 + 5/6; HXY1 = 2/3 + 1 + 2/3 + 2/3 = 3 (the
    # products p_i p_j are 1/4, 1/8, 1/16, 1/16); HXY2 = HX + HY = 3.
    # S = D^-1/2 P D^-1/2 has eigenvalue 1, trace 4/3 and determinant -2/9, so
    # the other two solve x^2 - x/3 - 2/9 = 0: 2/3 and -1/3.
    return {
        "Autocorrelation": F(7, 2), "JointAverage": F(7, 4),
        # (81/16)/3 + (1/16)/3 + (81/16)/6 + (625/16)/6
        "ClusterProminence": F(145, 16),
        # (-27/8)/3 + (-1/8)/3 + (27/8)/6 + (125/8)/6
        "ClusterShade": F(2),
        "ClusterTendency": F(9, 4),
        "Contrast": F(1, 2),
        "Correlation": F(7, 11),
        # |i - j| = 0 with mass 1/2, 1 with mass 1/2
        "DifferenceAverage": F(1, 2), "DifferenceEntropy": 1.0, "DifferenceVariance": F(1, 4),
        "JointEnergy": F(5, 24),
        "JointEntropy": l3 + 5 / 6,
        "Imc1": (l3 + 5 / 6 - 3) / 1.5,
        "Imc2": math.sqrt(1 - math.exp(-2 * (3 - (l3 + 5 / 6)))),
        "Idm": F(3, 4),
        # 1/2 + (1/2) / (1 + 1/Ng^2)
        "Idmn": F(1, 2) + F(1, 2) / (1 + F(1, ng * ng)),
        "Id": F(3, 4),
        # 1/2 + (1/2) / (1 + 1/Ng)
        "Idn": F(1, 2) + F(1, 2) / (1 + F(1, ng)),
        "InverseVariance": F(1, 2),
        "MaximumProbability": F(1, 3),
        # i + j = 2, 3, 5, 6 with mass 1/3, 1/3, 1/6, 1/6
        "SumAverage": F(7, 2), "SumEntropy": l3 + 1 / 3,
        "SumSquares": F(11, 16),
        "MCC": F(2, 3),
    }


@pytest.mark.parametrize("ng", [3, 5])
def test_glcm_features_of_a_three_level_matrix(ng):
    # ng = 5 leaves levels 4, 5 empty: only Idmn and Idn change (they use the
    # discretisation's Ng, not the count of present levels)
    _check(O.glcm_features(_three_level(ng)), GLCM_NAMES, _three_level_expect(ng))
    assert O.glcm_mcc(_three_level(ng)) == pytest.approx(2 / 3, rel=1e-12)
