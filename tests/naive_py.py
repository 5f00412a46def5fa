"""A second, independently written naive enumerator of the spatial-mapping
features (numpy/scipy), used only to pin the C++ oracle on tiny inputs.

It is deliberately built with different algorithms from the oracle:
GLCM pairs from shifted arrays, runs by walking whole lines and grouping,
zones with scipy.ndimage.label, dependences and neighbourhood sums from
shifted arrays, MCC from the eigenvalues of the literal Q matrix,
percentiles from numpy.percentile and moments from scipy.stats.
"""
import itertools
from fractions import Fraction

import numpy as np
from scipy import ndimage, stats

DIRS = [d for d in itertools.product((-1, 0, 1), repeat=3) if d > (0, 0, 0)]  # (dz, dy, dx)
NEIGH26 = [d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]


def sub_voi(levels, image, voxel_zyx, r):
    """Cube of side 2r+1 around the voxel: levels (0 outside V(v)) and raw."""
    s = 2 * r + 1
    lv = np.zeros((s, s, s), np.int64)
    raw = np.zeros((s, s, s), np.int64)
    z0, y0, x0 = voxel_zyx
    Z, Y, X = levels.shape
    for a in range(s):
        for b in range(s):
            for c in range(s):
                z, y, x = z0 - r + a, y0 - r + b, x0 - r + c
                if 0 <= z < Z and 0 <= y < Y and 0 <= x < X and levels[z, y, x]:
                    lv[a, b, c] = levels[z, y, x]
                    raw[a, b, c] = image[z, y, x] if image is not None else 0
    return lv, raw


def _shift_pairs(lv, d, delta=1):
    """Arrays (a, b) of levels at u and u + delta*d, both inside the cube."""
    s = lv.shape[0]
    sl_a, sl_b = [], []
    for k in d:
        o = k * delta
        if o >= 0:
            sl_a.append(slice(0, s - o))
            sl_b.append(slice(o, s))
        else:
            sl_a.append(slice(-o, s))
            sl_b.append(slice(0, s + o))
    a = lv[tuple(sl_a)].ravel()
    b = lv[tuple(sl_b)].ravel()
    keep = (a > 0) & (b > 0)
    return a[keep], b[keep]


def glcm(lv, ng, delta=1):
    out = np.zeros((13, ng, ng), np.int64)
    for k, d in enumerate(DIRS):
        a, b = _shift_pairs(lv, d, delta)
        np.add.at(out[k], (a - 1, b - 1), 1)
        np.add.at(out[k], (b - 1, a - 1), 1)
    return out


def _lines(s, d):
    """All maximal lines of the cube along direction d, as index lists."""
    lines = []
    for start in itertools.product(range(s), repeat=3):
        prev = tuple(p - q for p, q in zip(start, d))
        if all(0 <= t < s for t in prev):
            continue  # not the first voxel of its line
        line, cur = [], start
        while all(0 <= t < s for t in cur):
            line.append(cur)
            cur = tuple(p + q for p, q in zip(cur, d))
        lines.append(line)
    return lines


def glrlm(lv, ng):
    s = lv.shape[0]
    out = np.zeros((13, ng, s), np.int64)
    for k, d in enumerate(DIRS):
        for line in _lines(s, d):
            vals = [lv[p] for p in line]
            for key, grp in itertools.groupby(vals):
                n = len(list(grp))
                if key:
                    out[k, key - 1, n - 1] += 1
    return out


def glszm(lv, ng):
    s = lv.shape[0]
    out = np.zeros((ng, s ** 3), np.int64)
    structure = np.ones((3, 3, 3), bool)
    for g in range(1, ng + 1):
        lab, n = ndimage.label(lv == g, structure=structure)
        if n == 0:
            continue
        sizes = np.bincount(lab.ravel())[1:]
        for sz in sizes:
            out[g - 1, sz - 1] += 1
    return out


def _neighbour_stats(lv):
    """Per cube voxel: number of equal-level neighbours, number of valid
    neighbours and the sum of their levels (26-neighbourhood within V(v))."""
    s = lv.shape[0]
    pad = np.zeros((s + 2, s + 2, s + 2), np.int64)
    pad[1:-1, 1:-1, 1:-1] = lv
    eq = np.zeros_like(lv)
    cnt = np.zeros_like(lv)
    tot = np.zeros_like(lv)
    for dz, dy, dx in NEIGH26:
        nb = pad[1 + dz:1 + dz + s, 1 + dy:1 + dy + s, 1 + dx:1 + dx + s]
        valid = nb > 0
        eq += valid & (nb == lv)
        cnt += valid
        tot += nb
    return eq, cnt, tot


def gldm(lv, ng):
    eq, _, _ = _neighbour_stats(lv)
    out = np.zeros((ng, 27), np.int64)
    inside = lv > 0
    np.add.at(out, (lv[inside] - 1, eq[inside]), 1)
    return out


def ngtdm_exact(lv, ng):
    """n_i and s_i as exact Fractions."""
    _, cnt, tot = _neighbour_stats(lv)
    n = [0] * ng
    s = [Fraction(0)] * ng
    for idx in zip(*np.nonzero(lv)):
        w = int(cnt[idx])
        if w == 0:
            continue
        i = int(lv[idx])
        n[i - 1] += 1
        s[i - 1] += abs(Fraction(i) - Fraction(int(tot[idx]), w))
    return n, s


# ------------------------------------------------------------------ features

def _ent(p):
    p = p[p > 0]
    return float(-(p * np.log2(p)).sum())


def mcc_literal(P):
    """sqrt of the second-largest eigenvalue of Q(i,j) = sum_k p(i,k)p(j,k) /
    (p_x(i) p_y(k)), on the levels with nonzero marginals."""
    P = np.asarray(P, float)
    P = P / P.sum()
    keep = P.sum(1) > 0
    P = P[np.ix_(keep, keep)]
    if P.shape[0] < 2:
        return float("nan")
    px, py = P.sum(1), P.sum(0)
    Q = (P / px[:, None]) @ (P / py[None, :]).T
    ev = np.sort(np.real(np.linalg.eigvals(Q)))[::-1]
    return float(np.sqrt(max(ev[1], 0.0)))


def glcm_features(C, ng):
    C = np.asarray(C, float)
    T = C.sum()
    if T == 0:
        return np.full(24, np.nan)
    P = C / T
    i = np.arange(1, ng + 1)[:, None] * np.ones((1, ng))
    j = i.T
    px, py = P.sum(1), P.sum(0)
    lv = np.arange(1, ng + 1)
    mux, muy = (lv * px).sum(), (lv * py).sum()
    sx = np.sqrt(((lv - mux) ** 2 * px).sum())
    sy = np.sqrt(((lv - muy) ** 2 * py).sum())
    k_diff = np.abs(i - j).astype(int)
    k_sum = (i + j).astype(int)
    pxmy = np.bincount(k_diff.ravel(), weights=P.ravel(), minlength=ng)
    pxpy = np.bincount(k_sum.ravel(), weights=P.ravel(), minlength=2 * ng + 1)
    kd = np.arange(pxmy.size)
    ks = np.arange(pxpy.size)
    da = (kd * pxmy).sum()
    hx, hy, hxy = _ent(px), _ent(py), _ent(P)
    outer = np.outer(px, py)
    nz = P > 0
    hxy1 = float(-(P[nz] * np.log2(outer[nz])).sum())
    hxy2 = _ent(outer)
    cl = i + j - mux - muy
    f = [
        (i * j * P).sum(), mux, (cl ** 4 * P).sum(), (cl ** 3 * P).sum(),
        (cl ** 2 * P).sum(), ((i - j) ** 2 * P).sum(),
        ((i * j * P).sum() - mux * muy) / (sx * sy) if sx * sy > 0 else np.nan,
        da, _ent(pxmy), ((kd - da) ** 2 * pxmy).sum(), (P ** 2).sum(), hxy,
        (hxy - hxy1) / max(hx, hy) if max(hx, hy) > 0 else np.nan,
        np.sqrt(max(0.0, 1 - np.exp(-2 * (hxy2 - hxy)))),
        (P / (1 + (i - j) ** 2)).sum(), (P / (1 + (i - j) ** 2 / ng ** 2)).sum(),
        (P / (1 + np.abs(i - j))).sum(), (P / (1 + np.abs(i - j) / ng)).sum(),
        (pxmy[1:] / kd[1:] ** 2).sum(), P.max(), (ks * pxpy).sum(), _ent(pxpy),
        ((i - mux) ** 2 * P).sum(), mcc_literal(C),
    ]
    return np.array(f, float)


def rl_features(R, nv):
    R = np.asarray(R, float)
    N = R.sum()
    if N == 0:
        return np.full(16, np.nan)
    P = R / N
    ng, nj = R.shape
    I = np.arange(1, ng + 1)[:, None] * np.ones((1, nj))
    J = np.ones((ng, 1)) * np.arange(1, nj + 1)[None, :]
    mui, muj = (I * P).sum(), (J * P).sum()
    f = [
        (P / J ** 2).sum(), (P * J ** 2).sum(),
        (R.sum(1) ** 2).sum() / N, (R.sum(1) ** 2).sum() / N ** 2,
        (R.sum(0) ** 2).sum() / N, (R.sum(0) ** 2).sum() / N ** 2,
        N / nv, ((I - mui) ** 2 * P).sum(), ((J - muj) ** 2 * P).sum(), _ent(P),
        (P / I ** 2).sum(), (P * I ** 2).sum(), (P / (I ** 2 * J ** 2)).sum(),
        (P * I ** 2 / J ** 2).sum(), (P * J ** 2 / I ** 2).sum(),
        (P * I ** 2 * J ** 2).sum(),
    ]
    return np.array(f, float)


def gldm_features(M):
    M = np.asarray(M, float)
    N = M.sum()
    P = M / N
    ng, nj = M.shape
    I = np.arange(1, ng + 1)[:, None] * np.ones((1, nj))
    J = np.ones((ng, 1)) * np.arange(1, nj + 1)[None, :]
    mui, muj = (I * P).sum(), (J * P).sum()
    f = [
        (P / J ** 2).sum(), (P * J ** 2).sum(), (M.sum(1) ** 2).sum() / N,
        (M.sum(0) ** 2).sum() / N, (M.sum(0) ** 2).sum() / N ** 2,
        ((I - mui) ** 2 * P).sum(), ((J - muj) ** 2 * P).sum(), _ent(P),
        (P / I ** 2).sum(), (P * I ** 2).sum(), (P / (I ** 2 * J ** 2)).sum(),
        (P * I ** 2 / J ** 2).sum(), (P * J ** 2 / I ** 2).sum(),
        (P * I ** 2 * J ** 2).sum(),
    ]
    return np.array(f, float)


def ngtdm_features(n, s):
    n = np.asarray(n, float)
    s = np.asarray([float(v) for v in s])
    Nvp = n.sum()
    if Nvp == 0:
        return np.full(5, np.nan)
    p = n / Nvp
    lv = np.arange(1, n.size + 1)
    pres = p > 0
    ngp = int(pres.sum())
    pi, li, si = p[pres], lv[pres], s[pres]
    Pi, Pj = np.meshgrid(pi, pi, indexing="ij")
    Li, Lj = np.meshgrid(li, li, indexing="ij")
    Si, Sj = np.meshgrid(si, si, indexing="ij")
    sps = (p * s).sum()
    coarse = 1.0 / sps if sps != 0 else np.nan
    if ngp == 1:
        contrast = 0.0
    else:
        contrast = (Pi * Pj * (Li - Lj) ** 2).sum() / (ngp * (ngp - 1)) * s.sum() / Nvp
    bden = np.abs(Li * Pi - Lj * Pj).sum()
    busy = sps / bden if bden != 0 else np.nan
    cplx = (np.abs(Li - Lj) * (Pi * Si + Pj * Sj) / (Pi + Pj)).sum() / Nvp
    strength = ((Pi + Pj) * (Li - Lj) ** 2).sum() / s.sum() if s.sum() != 0 else np.nan
    return np.array([coarse, contrast, busy, cplx, strength], float)


def firstorder_features(x, g, ng, vvox=1.0, excess=True):
    x = np.asarray(x, float)
    N = x.size
    hist = np.bincount(np.asarray(g, int), minlength=ng + 1)[1:] / N
    p10, p25, p50, p75, p90 = np.percentile(x, [10, 25, 50, 75, 90])
    sub = x[(x >= p10) & (x <= p90)]
    var = x.var()
    f = [
        (x ** 2).sum(), vvox * (x ** 2).sum(), _ent(hist), x.min(), p10, p90,
        x.max(), x.mean(), p50, p75 - p25, x.max() - x.min(),
        np.abs(x - x.mean()).mean(), np.abs(sub - sub.mean()).mean(),
        np.sqrt((x ** 2).mean()),
        stats.skew(x, bias=True) if var > 0 else np.nan,
        (stats.kurtosis(x, fisher=excess, bias=True) if var > 0 else np.nan),
        var, (hist ** 2).sum(),
    ]
    return np.array(f, float)


def firstorder_extra(x):
    """IBSI median absolute deviation, coefficient of variation, quartile
    coefficient of dispersion."""
    x = np.asarray(x, float)
    p25, p50, p75 = np.percentile(x, [25, 50, 75])
    m = x.mean()
    cov = np.sqrt(x.var()) / m if m != 0 else np.nan
    qcod = (p75 - p25) / (p75 + p25) if (p75 + p25) != 0 else np.nan
    return np.array([np.abs(x - p50).mean(), cov, qcod], float)


def glcm_extra(C, ng):
    """IBSI sum variance and dissimilarity of one direction's counts."""
    C = np.asarray(C, float)
    T = C.sum()
    if T == 0:
        return np.full(2, np.nan)
    P = C / T
    i = np.arange(1, ng + 1)[:, None] * np.ones((1, ng))
    j = i.T
    ks = (i + j).ravel()
    kd = np.abs(i - j).ravel()
    pp = P.ravel()
    sa = (ks * pp).sum()
    return np.array([((ks - sa) ** 2 * pp).sum(), (kd * pp).sum()], float)


def gldm_extra(M, nv):
    """IBSI grey level non-uniformity normalised, dependence count percentage,
    dependence count energy."""
    M = np.asarray(M, float)
    N = M.sum()
    return np.array([(M.sum(1) ** 2).sum() / N ** 2, N / nv, ((M / N) ** 2).sum()], float)


def _nanmean_rows(a):
    a = np.asarray(a, float)
    out = np.full(a.shape[1], np.nan)
    for k in range(a.shape[1]):
        col = a[:, k]
        col = col[~np.isnan(col)]
        if col.size:
            out[k] = col.mean()
    return out


def features_of_cube(lv, raw, ng, delta=1, vvox=1.0, excess=True, merged=False):
    """All 101 features of one sub-VOI cube (93 benchmark maps, then the 8
    IBSI extras).  merged: GLCM and GLRLM features
    of the sum of the 13 directional matrices (run percentage over 13 N_v)."""
    inside = lv > 0
    nv = int(inside.sum())
    fo = firstorder_features(raw[inside], lv[inside], ng, vvox, excess)
    G = glcm(lv, ng, delta)
    R = glrlm(lv, ng)
    if merged:
        gl = glcm_features(G.sum(axis=0), ng)
        gx = glcm_extra(G.sum(axis=0), ng)
        rl = rl_features(R.sum(axis=0), 13 * nv)
    else:
        gl = _nanmean_rows([glcm_features(G[k], ng) for k in range(13)])
        gx = _nanmean_rows([glcm_extra(G[k], ng) for k in range(13)])
        rl = _nanmean_rows([rl_features(R[k], nv) for k in range(13)])
    sz = rl_features(glszm(lv, ng), nv)
    dm = gldm_features(gldm(lv, ng))
    n, s = ngtdm_exact(lv, ng)
    nt = ngtdm_features(n, s)
    fx = firstorder_extra(raw[inside])
    dx = gldm_extra(gldm(lv, ng), nv)
    return np.concatenate([fo, gl, rl, sz, dm, nt, fx, gx, dx])


def map_voxels(levels, image, ng, voxels, r, delta=1, vvox=1.0, excess=True, merged=False):
    Z, Y, X = levels.shape
    out = []
    for lin in voxels:
        z, y, x = lin // (Y * X), (lin // X) % Y, lin % X
        lv, raw = sub_voi(levels, image, (z, y, x), r)
        out.append(features_of_cube(lv, raw, ng, delta, vvox, excess, merged))
    return np.array(out).T
