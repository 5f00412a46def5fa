"""Comparison of GPU maps with the FP64 oracle.

Tolerance (FP32 maps against the FP64 oracle): a value passes when
|gpu - oracle| <= max(1e-6, 1e-4 |oracle|), the OR form of the paper's
concordance rule ("CPU-CUDA concordance tests") with FP32 limits; the
finite / non-finite patterns must be identical ("Spatial concordance").
"""
import numpy as np

ABS_TOL = 1e-6
REL_TOL = 1e-4


def compare(gpu, ref, names):
    """Returns a list of failure strings (empty when every map passes) and a
    per-map summary (exact count, max abs diff)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    fails, summary = [], {}
    for k, name in enumerate(names):
        g, r = gpu[k], ref[k]
        gn, rn = ~np.isfinite(g), ~np.isfinite(r)
        if not np.array_equal(gn, rn):
            bad = np.flatnonzero(gn != rn)
            fails.append("%s: finite pattern differs at %d columns (first %d: gpu %r oracle %r)"
                         % (name, bad.size, bad[0], g[bad[0]], r[bad[0]]))
            continue
        ok = ~rn
        d = np.abs(g[ok] - r[ok])
        tol = np.maximum(ABS_TOL, REL_TOL * np.abs(r[ok]))
        summary[name] = (int(np.sum(d == 0)), float(d.max()) if d.size else 0.0)
        if np.any(d > tol):
            i = np.argmax(d / tol)
            col = np.flatnonzero(ok)[i]
            fails.append("%s: %d values out of tolerance; worst col %d gpu %.9g oracle %.9g"
                         % (name, int(np.sum(d > tol)), col, g[col], r[col]))
    return fails, summary


def assert_close(gpu, ref, names):
    fails, _ = compare(gpu, ref, names)
    assert not fails, "\n".join(fails[:20])
