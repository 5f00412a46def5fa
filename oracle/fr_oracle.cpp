/*
 * fr_oracle.cpp -- plain FP64 CPU oracle for radiomic spatial mapping.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  See
 * fr_oracle.h for what it computes and where each definition comes from.
 *
 * Structure: one sub-VOI V(v) is copied into a dense cube of side 2r+1
 * (level 0 = not in V(v)); each family builds its dense count matrix from
 * the cube by direct enumeration and evaluates its features in double
 * precision, in the textbook form.  Readings of points the paper leaves
 * open (percentile interpolation, undefined values, NGTDM voxels without
 * neighbours, ...) are stated at the function that applies them.
 */
#include "fr_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kNaN = std::numeric_limits<double>::quiet_NaN();

/* Feature names: PyRadiomics-style class_Feature names of the 93 maps the
 * paper benchmarks (Table 2, spatial benchmark column). */
const char* const kNames[FRO_NUM_SCALAR_FEATURES] = {
    /* first order (18) */
    "firstorder_Energy", "firstorder_TotalEnergy", "firstorder_Entropy",
    "firstorder_Minimum", "firstorder_10Percentile", "firstorder_90Percentile",
    "firstorder_Maximum", "firstorder_Mean", "firstorder_Median",
    "firstorder_InterquartileRange", "firstorder_Range",
    "firstorder_MeanAbsoluteDeviation", "firstorder_RobustMeanAbsoluteDeviation",
    "firstorder_RootMeanSquared", "firstorder_Skewness", "firstorder_Kurtosis",
    "firstorder_Variance", "firstorder_Uniformity",
    /* GLCM (24) */
    "glcm_Autocorrelation", "glcm_JointAverage", "glcm_ClusterProminence",
    "glcm_ClusterShade", "glcm_ClusterTendency", "glcm_Contrast",
    "glcm_Correlation", "glcm_DifferenceAverage", "glcm_DifferenceEntropy",
    "glcm_DifferenceVariance", "glcm_JointEnergy", "glcm_JointEntropy",
    "glcm_Imc1", "glcm_Imc2", "glcm_Idm", "glcm_Idmn", "glcm_Id", "glcm_Idn",
    "glcm_InverseVariance", "glcm_MaximumProbability", "glcm_SumAverage",
    "glcm_SumEntropy", "glcm_SumSquares", "glcm_MCC",
    /* GLRLM (16) */
    "glrlm_ShortRunEmphasis", "glrlm_LongRunEmphasis",
    "glrlm_GrayLevelNonUniformity", "glrlm_GrayLevelNonUniformityNormalized",
    "glrlm_RunLengthNonUniformity", "glrlm_RunLengthNonUniformityNormalized",
    "glrlm_RunPercentage", "glrlm_GrayLevelVariance", "glrlm_RunVariance",
    "glrlm_RunEntropy", "glrlm_LowGrayLevelRunEmphasis",
    "glrlm_HighGrayLevelRunEmphasis", "glrlm_ShortRunLowGrayLevelEmphasis",
    "glrlm_ShortRunHighGrayLevelEmphasis", "glrlm_LongRunLowGrayLevelEmphasis",
    "glrlm_LongRunHighGrayLevelEmphasis",
    /* GLSZM (16) */
    "glszm_SmallAreaEmphasis", "glszm_LargeAreaEmphasis",
    "glszm_GrayLevelNonUniformity", "glszm_GrayLevelNonUniformityNormalized",
    "glszm_SizeZoneNonUniformity", "glszm_SizeZoneNonUniformityNormalized",
    "glszm_ZonePercentage", "glszm_GrayLevelVariance", "glszm_ZoneVariance",
    "glszm_ZoneEntropy", "glszm_LowGrayLevelZoneEmphasis",
    "glszm_HighGrayLevelZoneEmphasis", "glszm_SmallAreaLowGrayLevelEmphasis",
    "glszm_SmallAreaHighGrayLevelEmphasis",
    "glszm_LargeAreaLowGrayLevelEmphasis",
    "glszm_LargeAreaHighGrayLevelEmphasis",
    /* GLDM / NGLDM (14) */
    "gldm_SmallDependenceEmphasis", "gldm_LargeDependenceEmphasis",
    "gldm_GrayLevelNonUniformity", "gldm_DependenceNonUniformity",
    "gldm_DependenceNonUniformityNormalized", "gldm_GrayLevelVariance",
    "gldm_DependenceVariance", "gldm_DependenceEntropy",
    "gldm_LowGrayLevelEmphasis", "gldm_HighGrayLevelEmphasis",
    "gldm_SmallDependenceLowGrayLevelEmphasis",
    "gldm_SmallDependenceHighGrayLevelEmphasis",
    "gldm_LargeDependenceLowGrayLevelEmphasis",
    "gldm_LargeDependenceHighGrayLevelEmphasis",
    /* NGTDM (5) */
    "ngtdm_Coarseness", "ngtdm_Contrast", "ngtdm_Busyness", "ngtdm_Complexity",
    "ngtdm_Strength",
    /* IBSI extras completing the 101-map default set (ids 93..100) */
    "firstorder_MedianAbsoluteDeviation", "firstorder_CoefficientOfVariation",
    "firstorder_QuartileCoefficientOfDispersion", "glcm_SumVariance",
    "glcm_Dissimilarity", "gldm_GrayLevelNonUniformityNormalized",
    "gldm_DependencePercentage", "gldm_DependenceEnergy",
    /* scalar extraction only (id 101) */
    "firstorder_StandardDeviation"
};

/* The 13 directions of 3-D texture analysis: one vector d of every +-d pair
 * of the 26-neighbourhood, taken as the vectors (dz, dy, dx) that are
 * lexicographically greater than (0, 0, 0). */
void make_dirs(int dirs[FRO_NUM_DIRS][3]) {
  int n = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        bool positive = dz > 0 || (dz == 0 && dy > 0) ||
                        (dz == 0 && dy == 0 && dx > 0);
        if (positive) {
          dirs[n][0] = dz;
          dirs[n][1] = dy;
          dirs[n][2] = dx;
          ++n;
        }
      }
}

double safe_div(double a, double b) { return b == 0.0 ? kNaN : a / b; }

/* ---------------------------------------------------------------------- */
/* Sub-VOI V(v) as a dense cube of side s = 2r+1.                           */
/* ---------------------------------------------------------------------- */
struct Cube {
  int s = 0;
  std::vector<int> lev;  /* 0 = not in V(v), else gray level 1..Ng */
  std::vector<int> raw;  /* raw intensity where lev > 0            */

  bool inside(int z, int y, int x) const {
    return z >= 0 && y >= 0 && x >= 0 && z < s && y < s && x < s;
  }
  int at(int z, int y, int x) const { return (z * s + y) * s + x; }
  int level(int z, int y, int x) const {
    return inside(z, y, x) ? lev[at(z, y, x)] : 0;
  }
};

Cube make_cube(const fro_params* p, const int16_t* img, const uint8_t* levels,
               int64_t vox) {
  Cube c;
  const int r = p->radius;
  c.s = 2 * r + 1;
  c.lev.assign((size_t)c.s * c.s * c.s, 0);
  c.raw.assign((size_t)c.s * c.s * c.s, 0);
  const int64_t nx = p->nx, ny = p->ny, nz = p->nz;
  const int64_t vz = vox / (nx * ny), vy = (vox / nx) % ny, vx = vox % nx;
  for (int dz = -r; dz <= r; ++dz)
    for (int dy = -r; dy <= r; ++dy)
      for (int dx = -r; dx <= r; ++dx) {
        int64_t z = vz + dz, y = vy + dy, x = vx + dx;
        if (z < 0 || y < 0 || x < 0 || z >= nz || y >= ny || x >= nx) continue;
        int64_t lin = (z * ny + y) * nx + x;
        if (levels[lin] == 0) continue;
        int k = c.at(dz + r, dy + r, dx + r);
        c.lev[k] = levels[lin];
        c.raw[k] = img ? img[lin] : 0;
      }
  return c;
}

/* The whole volume as one cube of side max(nx, ny, nz) (zeros beyond it):
 * the sub-VOI of a window that covers every VOI voxel. */
Cube make_whole_cube(const fro_params* p, const int16_t* img, const uint8_t* levels) {
  Cube c;
  c.s = std::max(p->nx, std::max(p->ny, p->nz));
  c.lev.assign((size_t)c.s * c.s * c.s, 0);
  c.raw.assign((size_t)c.s * c.s * c.s, 0);
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        const int64_t lin = ((int64_t)z * p->ny + y) * p->nx + x;
        if (!levels[lin]) continue;
        c.lev[c.at(z, y, x)] = levels[lin];
        c.raw[c.at(z, y, x)] = img[lin];
      }
  return c;
}

/* ---------------------------------------------------------------------- */
/* Matrices                                                                 */
/* ---------------------------------------------------------------------- */

/* Symmetric co-occurrence counts of one direction at offset delta*d: every
 * unordered pair of V(v) voxels (u, u + delta*d) adds one to (g_u, g_w) and
 * one to (g_w, g_u). */
void glcm_counts(const Cube& c, const int d[3], int delta, int ng,
                 std::vector<double>& C) {
  C.assign((size_t)ng * ng, 0.0);
  for (int z = 0; z < c.s; ++z)
    for (int y = 0; y < c.s; ++y)
      for (int x = 0; x < c.s; ++x) {
        int a = c.lev[c.at(z, y, x)];
        if (!a) continue;
        int b = c.level(z + delta * d[0], y + delta * d[1], x + delta * d[2]);
        if (!b) continue;
        C[(size_t)(a - 1) * ng + (b - 1)] += 1.0;
        C[(size_t)(b - 1) * ng + (a - 1)] += 1.0;
      }
}

/* Run-length counts of one direction: a run is a maximal chain u, u+d,
 * u+2d, ... of V(v) voxels with one gray level; leaving V(v) ends it.  Run
 * lengths are 1..s (index j-1). */
void glrlm_counts(const Cube& c, const int d[3], int ng,
                  std::vector<double>& R) {
  R.assign((size_t)ng * c.s, 0.0);
  for (int z = 0; z < c.s; ++z)
    for (int y = 0; y < c.s; ++y)
      for (int x = 0; x < c.s; ++x) {
        int a = c.lev[c.at(z, y, x)];
        if (!a) continue;
        if (c.level(z - d[0], y - d[1], x - d[2]) == a) continue; /* not a start */
        int len = 1;
        while (c.level(z + len * d[0], y + len * d[1], x + len * d[2]) == a) ++len;
        R[(size_t)(a - 1) * c.s + (len - 1)] += 1.0;
      }
}

/* Size-zone counts: zones are the 26-connected components of equal gray
 * level inside V(v) (labelled by breadth-first search); sizes 1..s^3. */
void glszm_counts(const Cube& c, int ng, std::vector<double>& Z) {
  const int w = c.s * c.s * c.s;
  Z.assign((size_t)ng * w, 0.0);
  std::vector<char> seen(w, 0);
  std::vector<int> queue;
  for (int start = 0; start < w; ++start) {
    if (!c.lev[start] || seen[start]) continue;
    const int a = c.lev[start];
    queue.clear();
    queue.push_back(start);
    seen[start] = 1;
    for (size_t head = 0; head < queue.size(); ++head) {
      int k = queue[head];
      int z = k / (c.s * c.s), y = (k / c.s) % c.s, x = k % c.s;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dz && !dy && !dx) continue;
            if (!c.inside(z + dz, y + dy, x + dx)) continue;
            int q = c.at(z + dz, y + dy, x + dx);
            if (seen[q] || c.lev[q] != a) continue;
            seen[q] = 1;
            queue.push_back(q);
          }
    }
    Z[(size_t)(a - 1) * w + (queue.size() - 1)] += 1.0;
  }
}

/* The same zones as counts per (level, size) over only the sizes that occur:
 * Z[ng][jv.size()], column k holding zones of size jv[k] (ascending).  Zone
 * sizes reach N_v, so a dense size axis does not fit whole-VOI cubes. */
void glszm_zones(const Cube& c, int ng, std::vector<double>& Z, std::vector<double>& jv) {
  const int w = c.s * c.s * c.s;
  std::vector<char> seen(w, 0);
  std::vector<int> queue;
  std::vector<std::pair<int, int>> zones;  // (level, size)
  for (int start = 0; start < w; ++start) {
    if (!c.lev[start] || seen[start]) continue;
    const int a = c.lev[start];
    queue.clear();
    queue.push_back(start);
    seen[start] = 1;
    for (size_t head = 0; head < queue.size(); ++head) {
      int k = queue[head];
      int z = k / (c.s * c.s), y = (k / c.s) % c.s, x = k % c.s;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dz && !dy && !dx) continue;
            if (!c.inside(z + dz, y + dy, x + dx)) continue;
            int q = c.at(z + dz, y + dy, x + dx);
            if (seen[q] || c.lev[q] != a) continue;
            seen[q] = 1;
            queue.push_back(q);
          }
    }
    zones.push_back({a, (int)queue.size()});
  }
  std::vector<int> sizes;
  for (auto& z : zones) sizes.push_back(z.second);
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  jv.assign(sizes.begin(), sizes.end());
  Z.assign((size_t)ng * sizes.size(), 0.0);
  for (auto& z : zones) {
    const size_t col = std::lower_bound(sizes.begin(), sizes.end(), z.second) - sizes.begin();
    Z[(size_t)(z.first - 1) * sizes.size() + col] += 1.0;
  }
}

/* Dependence counts (alpha = 0, Chebyshev distance 1): a voxel of level i
 * with k equal-level 26-neighbours inside V(v) adds one to (i, k+1). */
void gldm_counts(const Cube& c, int ng, std::vector<double>& M) {
  M.assign((size_t)ng * 27, 0.0);
  for (int z = 0; z < c.s; ++z)
    for (int y = 0; y < c.s; ++y)
      for (int x = 0; x < c.s; ++x) {
        int a = c.lev[c.at(z, y, x)];
        if (!a) continue;
        int k = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dz && !dy && !dx) continue;
              if (c.level(z + dz, y + dy, x + dx) == a) ++k;
            }
        M[(size_t)(a - 1) * 27 + k] += 1.0;
      }
}

/* NGTDM: for each V(v) voxel of level i with W >= 1 neighbours in V(v)
 * (26-neighbourhood, centre excluded), n_i += 1 and s_i += |i - A| with A
 * the mean neighbour level.  Voxels without a neighbour are left out of
 * n_i and s_i.  s_i is accumulated in double and, separately, exactly as
 * s_i * L with L = lcm(1..26) (|i*W - S| * L / W is an integer). */
int64_t lcm_1_to_26() {
  int64_t l = 1;
  for (int64_t k = 2; k <= 26; ++k) l = l / std::gcd(l, k) * k;
  return l;
}

void ngtdm_counts(const Cube& c, int ng, std::vector<double>& n,
                  std::vector<double>& s, std::vector<int64_t>* sl) {
  static const int64_t L = lcm_1_to_26();
  n.assign(ng, 0.0);
  s.assign(ng, 0.0);
  if (sl) sl->assign(ng, 0);
  for (int z = 0; z < c.s; ++z)
    for (int y = 0; y < c.s; ++y)
      for (int x = 0; x < c.s; ++x) {
        int a = c.lev[c.at(z, y, x)];
        if (!a) continue;
        int64_t W = 0, S = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dz && !dy && !dx) continue;
              int b = c.level(z + dz, y + dy, x + dx);
              if (!b) continue;
              ++W;
              S += b;
            }
        if (W == 0) continue;
        double mean = (double)S / (double)W;
        n[a - 1] += 1.0;
        s[a - 1] += std::fabs((double)a - mean);
        if (sl) (*sl)[a - 1] += std::llabs((int64_t)a * W - S) * (L / W);
      }
}

/* ---------------------------------------------------------------------- */
/* Feature functions                                                        */
/* ---------------------------------------------------------------------- */

/* Cyclic Jacobi eigenvalues of a symmetric n x n matrix (row-major). */
std::vector<double> jacobi_eigenvalues(std::vector<double> A, int n) {
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, norm = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
        norm += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * norm || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) /
                   (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < n; ++k) {
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = cs * akp - sn * akq;
          A[(size_t)k * n + q] = sn * akp + cs * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = cs * apk - sn * aqk;
          A[(size_t)q * n + k] = sn * apk + cs * aqk;
        }
      }
  }
  std::vector<double> ev(n);
  for (int i = 0; i < n; ++i) ev[i] = A[(size_t)i * n + i];
  return ev;
}

/* MCC: square root of the second-largest eigenvalue of
 *   Q(i,j) = sum_k p(i,k) p(j,k) / (p_x(i) p_y(k)).
 * For a symmetric P (p_x = p_y), Q = D^-1 P D^-1 P with D = diag(p_x), which
 * is similar to S^2 for S = D^-1/2 P D^-1/2, so the eigenvalues of Q are the
 * squares of those of S and MCC is the second-largest |eigenvalue| of S,
 * over the levels with p_x > 0.  Fewer than two such levels: NaN. */
double mcc_from_counts(const std::vector<double>& C, int ng) {
  double T = 0.0;
  for (double v : C) T += v;
  if (T == 0.0) return kNaN;
  std::vector<double> px(ng, 0.0);
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < ng; ++j) px[i] += C[(size_t)i * ng + j] / T;
  std::vector<int> present;
  for (int i = 0; i < ng; ++i)
    if (px[i] > 0.0) present.push_back(i);
  const int n = (int)present.size();
  if (n < 2) return kNaN;
  std::vector<double> S((size_t)n * n);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      int i = present[a], j = present[b];
      S[(size_t)a * n + b] =
          (C[(size_t)i * ng + j] / T) / std::sqrt(px[i] * px[j]);
    }
  std::vector<double> ev = jacobi_eigenvalues(S, n);
  for (double& e : ev) e = std::fabs(e);
  std::sort(ev.begin(), ev.end(), [](double x, double y) { return x > y; });
  return ev[1];
}

/* GLCM features of one direction (IBSI definitions; i, j are gray levels
 * 1..Ng, p = counts / total).  Ng in Idmn and Idn is the number of gray
 * levels of the discretisation.  Empty matrix: all NaN. */
void glcm_features(const std::vector<double>& C, int ng, double* f) {
  double T = 0.0;
  for (double v : C) T += v;
  if (T == 0.0) {
    for (int k = 0; k < 24; ++k) f[k] = kNaN;
    return;
  }
  std::vector<double> px(ng, 0.0), py(ng, 0.0), pxmy(ng, 0.0),
      pxpy(2 * ng + 1, 0.0);
  for (int i = 1; i <= ng; ++i)
    for (int j = 1; j <= ng; ++j) {
      double p = C[(size_t)(i - 1) * ng + (j - 1)] / T;
      px[i - 1] += p;
      py[j - 1] += p;
      pxmy[std::abs(i - j)] += p;
      pxpy[i + j] += p;
    }
  double mux = 0, muy = 0;
  for (int i = 1; i <= ng; ++i) {
    mux += i * px[i - 1];
    muy += i * py[i - 1];
  }
  double sx2 = 0, sy2 = 0;
  for (int i = 1; i <= ng; ++i) {
    sx2 += (i - mux) * (i - mux) * px[i - 1];
    sy2 += (i - muy) * (i - muy) * py[i - 1];
  }
  double autoc = 0, cp = 0, cs = 0, ct = 0, contrast = 0, je = 0, jent = 0;
  double hxy1 = 0, hxy2 = 0, idm = 0, idmn = 0, id = 0, idn = 0, iv = 0,
         maxp = 0, ss = 0;
  for (int i = 1; i <= ng; ++i)
    for (int j = 1; j <= ng; ++j) {
      double p = C[(size_t)(i - 1) * ng + (j - 1)] / T;
      double pxy = px[i - 1] * py[j - 1];
      if (pxy > 0) hxy2 -= pxy * std::log2(pxy);
      if (p == 0.0) continue;
      double t = i + j - mux - muy;
      autoc += i * j * p;
      cp += t * t * t * t * p;
      cs += t * t * t * p;
      ct += t * t * p;
      contrast += (double)(i - j) * (i - j) * p;
      je += p * p;
      jent -= p * std::log2(p);
      hxy1 -= p * std::log2(pxy);
      double dd = std::fabs((double)(i - j));
      idm += p / (1.0 + dd * dd);
      idmn += p / (1.0 + dd * dd / ((double)ng * ng));
      id += p / (1.0 + dd);
      idn += p / (1.0 + dd / ng);
      if (i != j) iv += p / (dd * dd);
      maxp = std::max(maxp, p);
      ss += (i - mux) * (i - mux) * p;
    }
  double hx = 0, hy = 0;
  for (int i = 0; i < ng; ++i) {
    if (px[i] > 0) hx -= px[i] * std::log2(px[i]);
    if (py[i] > 0) hy -= py[i] * std::log2(py[i]);
  }
  double da = 0, de = 0, dv = 0;
  for (int k = 0; k < ng; ++k) {
    da += k * pxmy[k];
    if (pxmy[k] > 0) de -= pxmy[k] * std::log2(pxmy[k]);
  }
  for (int k = 0; k < ng; ++k) dv += (k - da) * (k - da) * pxmy[k];
  double sa = 0, se = 0;
  for (int k = 2; k <= 2 * ng; ++k) {
    sa += k * pxpy[k];
    if (pxpy[k] > 0) se -= pxpy[k] * std::log2(pxpy[k]);
  }
  double sxy = std::sqrt(sx2) * std::sqrt(sy2);
  f[0] = autoc;
  f[1] = mux;
  f[2] = cp;
  f[3] = cs;
  f[4] = ct;
  f[5] = contrast;
  f[6] = safe_div(autoc - mux * muy, sxy);
  f[7] = da;
  f[8] = de;
  f[9] = dv;
  f[10] = je;
  f[11] = jent;
  f[12] = safe_div(jent - hxy1, std::max(hx, hy));
  /* 1 - exp(-2 (HXY2 - HXY)) >= 0 exactly (HXY2 - HXY is a mutual
   * information); the clamp only removes rounding below zero. */
  f[13] = std::sqrt(std::max(0.0, 1.0 - std::exp(-2.0 * (hxy2 - jent))));
  f[14] = idm;
  f[15] = idmn;
  f[16] = id;
  f[17] = idn;
  f[18] = iv;
  f[19] = maxp;
  f[20] = sa;
  f[21] = se;
  f[22] = ss;
  f[23] = mcc_from_counts(C, ng);
}

/* Run-length-type features of a [ng][nj] count matrix, with i the gray level
 * (1..ng) and j = column + 1 the run length, zone size or dependence.  The
 * 16 GLRLM and the 16 GLSZM features share these formulas; nv is the number
 * of voxels (the denominator of run/zone percentage). */
/* Run-length / size-zone features of R[ng][nj] whose column j counts runs
 * (zones) of length (size) jv[j]. */
void rl_features_j(const std::vector<double>& R, int ng, const std::vector<double>& jv,
                   double nv, double* f) {
  const int nj = (int)jv.size();
  double N = 0;
  for (double v : R) N += v;
  if (N == 0) {
    for (int k = 0; k < 16; ++k) f[k] = kNaN;
    return;
  }
  std::vector<double> pi(ng, 0.0), pj(nj, 0.0);
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < nj; ++j) {
      pi[i] += R[(size_t)i * nj + j];
      pj[j] += R[(size_t)i * nj + j];
    }
  double mui = 0, muj = 0;
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < nj; ++j) {
      double p = R[(size_t)i * nj + j] / N;
      mui += (i + 1) * p;
      muj += jv[j] * p;
    }
  double sre = 0, lre = 0, glv = 0, rv = 0, ent = 0, lgl = 0, hgl = 0, srl = 0,
         srh = 0, lrl = 0, lrh = 0;
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < nj; ++j) {
      double p = R[(size_t)i * nj + j] / N;
      if (p == 0) continue;
      double I = i + 1, J = jv[j];
      sre += p / (J * J);
      lre += p * J * J;
      glv += (I - mui) * (I - mui) * p;
      rv += (J - muj) * (J - muj) * p;
      ent -= p * std::log2(p);
      lgl += p / (I * I);
      hgl += p * I * I;
      srl += p / (I * I * J * J);
      srh += p * I * I / (J * J);
      lrl += p * J * J / (I * I);
      lrh += p * I * I * J * J;
    }
  double glnu = 0, rlnu = 0;
  for (double v : pi) glnu += v * v;
  for (double v : pj) rlnu += v * v;
  f[0] = sre;
  f[1] = lre;
  f[2] = glnu / N;
  f[3] = glnu / (N * N);
  f[4] = rlnu / N;
  f[5] = rlnu / (N * N);
  f[6] = N / nv;
  f[7] = glv;
  f[8] = rv;
  f[9] = ent;
  f[10] = lgl;
  f[11] = hgl;
  f[12] = srl;
  f[13] = srh;
  f[14] = lrl;
  f[15] = lrh;
}

/* The same with column j holding length (size) j + 1. */
void rl_features(const std::vector<double>& R, int ng, int nj, double nv, double* f) {
  std::vector<double> jv(nj);
  for (int j = 0; j < nj; ++j) jv[j] = j + 1;
  rl_features_j(R, ng, jv, nv, f);
}

/* GLDM features of a [ng][nj] dependence count matrix (j = column + 1). */
void gldm_features(const std::vector<double>& M, int ng, int nj, double* f) {
  double N = 0;
  for (double v : M) N += v;
  if (N == 0) {
    for (int k = 0; k < 14; ++k) f[k] = kNaN;
    return;
  }
  std::vector<double> pi(ng, 0.0), pj(nj, 0.0);
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < nj; ++j) {
      pi[i] += M[(size_t)i * nj + j];
      pj[j] += M[(size_t)i * nj + j];
    }
  double mui = 0, muj = 0;
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < nj; ++j) {
      double p = M[(size_t)i * nj + j] / N;
      mui += (i + 1) * p;
      muj += (j + 1) * p;
    }
  double sde = 0, lde = 0, glv = 0, dv = 0, ent = 0, lgl = 0, hgl = 0, sdl = 0,
         sdh = 0, ldl = 0, ldh = 0;
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < nj; ++j) {
      double p = M[(size_t)i * nj + j] / N;
      if (p == 0) continue;
      double I = i + 1, J = j + 1;
      sde += p / (J * J);
      lde += p * J * J;
      glv += (I - mui) * (I - mui) * p;
      dv += (J - muj) * (J - muj) * p;
      ent -= p * std::log2(p);
      lgl += p / (I * I);
      hgl += p * I * I;
      sdl += p / (I * I * J * J);
      sdh += p * I * I / (J * J);
      ldl += p * J * J / (I * I);
      ldh += p * I * I * J * J;
    }
  double glnu = 0, dnu = 0;
  for (double v : pi) glnu += v * v;
  for (double v : pj) dnu += v * v;
  f[0] = sde;
  f[1] = lde;
  f[2] = glnu / N;
  f[3] = dnu / N;
  f[4] = dnu / (N * N);
  f[5] = glv;
  f[6] = dv;
  f[7] = ent;
  f[8] = lgl;
  f[9] = hgl;
  f[10] = sdl;
  f[11] = sdh;
  f[12] = ldl;
  f[13] = ldh;
}

/* IBSI statistics beyond the benchmark set, raw intensities x:
 * median absolute deviation (1/N) sum |x - median|, coefficient of variation
 * sigma / mean (population sigma; NaN for a zero mean), quartile coefficient
 * of dispersion (P75 - P25) / (P75 + P25) (NaN for a zero denominator), with
 * the percentiles of firstorder_features. */
void firstorder_extra(std::vector<int> x, double* f) {
  const int64_t n = (int64_t)x.size();
  if (n == 0) {
    for (int k = 0; k < 3; ++k) f[k] = kNaN;
    return;
  }
  std::sort(x.begin(), x.end());
  auto pct = [&](int q) {
    const int64_t num = (n - 1) * q, k = num / 100, rem = num % 100;
    if (rem == 0) return (double)x[k];
    return x[k] + (rem / 100.0) * (double)(x[k + 1] - x[k]);
  };
  const double N = (double)n, med = pct(50);
  double sum = 0, medad = 0;
  for (int v : x) {
    sum += v;
    medad += std::fabs(v - med);
  }
  const double mean = sum / N;
  double m2 = 0;
  for (int v : x) m2 += (v - mean) * (v - mean);
  m2 /= N;
  const double p25 = pct(25), p75 = pct(75);
  f[0] = medad / N;
  f[1] = safe_div(std::sqrt(m2), mean);
  f[2] = safe_div(p75 - p25, p75 + p25);
}

/* GLCM sum variance sum_k (k - SA)^2 p_{x+y}(k), SA = sum_k k p_{x+y}(k), and
 * dissimilarity sum_k k p_{x-y}(k) (IBSI) of one symmetric count matrix. */
void glcm_extra(const std::vector<double>& C, int ng, double* f) {
  double T = 0.0;
  for (double v : C) T += v;
  if (T == 0.0) {
    f[0] = f[1] = kNaN;
    return;
  }
  std::vector<double> pxpy(2 * ng + 1, 0.0), pxmy(ng, 0.0);
  for (int i = 1; i <= ng; ++i)
    for (int j = 1; j <= ng; ++j) {
      const double p = C[(size_t)(i - 1) * ng + (j - 1)] / T;
      pxpy[i + j] += p;
      pxmy[std::abs(i - j)] += p;
    }
  double sa = 0, sv = 0, dis = 0;
  for (int k = 2; k <= 2 * ng; ++k) sa += k * pxpy[k];
  for (int k = 2; k <= 2 * ng; ++k) sv += (k - sa) * (k - sa) * pxpy[k];
  for (int k = 0; k < ng; ++k) dis += k * pxmy[k];
  f[0] = sv;
  f[1] = dis;
}

/* NGLDM extras (IBSI) of a dependence count matrix [ng][nj]: grey level
 * non-uniformity normalised sum_i (sum_j s_ij)^2 / N_s^2, dependence count
 * percentage N_s / N_v, dependence count energy sum_ij p_ij^2. */
void gldm_extra(const std::vector<double>& M, int ng, int nj, double nv, double* f) {
  double N = 0;
  for (double v : M) N += v;
  if (N == 0) {
    for (int k = 0; k < 3; ++k) f[k] = kNaN;
    return;
  }
  double glnu = 0, energy = 0;
  for (int i = 0; i < ng; ++i) {
    double row = 0;
    for (int j = 0; j < nj; ++j) {
      const double p = M[(size_t)i * nj + j] / N;
      row += M[(size_t)i * nj + j];
      energy += p * p;
    }
    glnu += row * row;
  }
  f[0] = glnu / (N * N);
  f[1] = N / nv;
  f[2] = energy;
}

/* NGTDM features (IBSI).  N_vp = sum n_i, p_i = n_i / N_vp, N_gp = number of
 * levels with p_i > 0; sums over i, j run over those levels.
 * Undefined values: N_vp = 0 -> all NaN; a zero denominator -> NaN, except
 * Contrast, which is 0 when only one level occurs (its double sum and its
 * sum of s_i are then both 0). */
void ngtdm_features(const std::vector<double>& n, const std::vector<double>& s,
                    int ng, double* f) {
  double Nvp = 0;
  for (double v : n) Nvp += v;
  if (Nvp == 0) {
    for (int k = 0; k < 5; ++k) f[k] = kNaN;
    return;
  }
  std::vector<double> p(ng);
  int ngp = 0;
  for (int i = 0; i < ng; ++i) {
    p[i] = n[i] / Nvp;
    if (p[i] > 0) ++ngp;
  }
  double sum_ps = 0, sum_s = 0;
  for (int i = 0; i < ng; ++i) {
    sum_ps += p[i] * s[i];
    sum_s += s[i];
  }
  double c1 = 0, busy_den = 0, cplx = 0, str = 0;
  for (int i = 1; i <= ng; ++i) {
    if (p[i - 1] == 0) continue;
    for (int j = 1; j <= ng; ++j) {
      if (p[j - 1] == 0) continue;
      double pi_ = p[i - 1], pj_ = p[j - 1];
      double d = (double)(i - j);
      c1 += pi_ * pj_ * d * d;
      /* |i p_i - j p_j| from the integer counts, so that a difference that
       * vanishes exactly (i n_i = j n_j) is exactly zero */
      busy_den += std::fabs((double)i * n[i - 1] - (double)j * n[j - 1]) / Nvp;
      cplx += std::fabs(d) * (pi_ * s[i - 1] + pj_ * s[j - 1]) / (pi_ + pj_);
      str += (pi_ + pj_) * d * d;
    }
  }
  f[0] = safe_div(1.0, sum_ps);
  f[1] = ngp == 1 ? 0.0
                  : (c1 / ((double)ngp * (ngp - 1))) * (sum_s / Nvp);
  f[2] = safe_div(sum_ps, busy_den);
  f[3] = cplx / Nvp;
  f[4] = safe_div(str, sum_s);
}

/* First-order features (IBSI).  Raw intensities x, except Entropy and
 * Uniformity, which use the discretised histogram.  Variance and the
 * moments are population moments (divide by N).  Kurtosis is the excess
 * kurtosis m4/m2^2 - 3 unless kurtosis_excess == 0 (the paper's kurtosis
 * check: reference values are excess kurtosis).  Percentiles interpolate
 * linearly at rank h = (N-1) q / 100 (q in percent), taken as an exact
 * rational; RobustMeanAbsoluteDeviation uses the x with P10 <= x <= P90,
 * around their own mean.  Zero variance makes skewness and kurtosis NaN. */
void firstorder_features(std::vector<int> x, const std::vector<int>& g, int ng,
                         double vvox, int excess, double* f) {
  const int64_t n = (int64_t)x.size();
  if (n == 0) {
    for (int k = 0; k < 18; ++k) f[k] = kNaN;
    return;
  }
  std::sort(x.begin(), x.end());
  double sum = 0, sum2 = 0;
  for (int v : x) {
    sum += v;
    sum2 += (double)v * v;
  }
  const double N = (double)n, mean = sum / N;
  double m2 = 0, m3 = 0, m4 = 0, mad = 0;
  for (int v : x) {
    double d = v - mean;
    m2 += d * d;
    m3 += d * d * d;
    m4 += d * d * d * d;
    mad += std::fabs(d);
  }
  m2 /= N;
  m3 /= N;
  m4 /= N;
  mad /= N;
  /* percentile q as the exact rational x_k + rem/100 * (x_{k+1} - x_k):
   * returns k and rem with (n-1)*q = 100*k + rem. */
  auto rank = [&](int q, int64_t* k, int64_t* rem) {
    int64_t num = (n - 1) * q;
    *k = num / 100;
    *rem = num % 100;
  };
  auto pct = [&](int q) {
    int64_t k, rem;
    rank(q, &k, &rem);
    if (rem == 0) return (double)x[k];
    return x[k] + (rem / 100.0) * (double)(x[k + 1] - x[k]);
  };
  /* 100 * x >= 100 * P_q, exactly */
  auto ge_pct = [&](int v, int q) {
    int64_t k, rem;
    rank(q, &k, &rem);
    int64_t lhs = 100 * (int64_t)v;
    int64_t rhs = 100 * (int64_t)x[k] + (rem ? rem * (int64_t)(x[k + 1] - x[k]) : 0);
    return lhs >= rhs;
  };
  auto le_pct = [&](int v, int q) {
    int64_t k, rem;
    rank(q, &k, &rem);
    int64_t lhs = 100 * (int64_t)v;
    int64_t rhs = 100 * (int64_t)x[k] + (rem ? rem * (int64_t)(x[k + 1] - x[k]) : 0);
    return lhs <= rhs;
  };
  double rsum = 0;
  int64_t rn = 0;
  for (int v : x)
    if (ge_pct(v, 10) && le_pct(v, 90)) {
      rsum += v;
      ++rn;
    }
  double rmean = rsum / (double)rn, rmad = 0;
  for (int v : x)
    if (ge_pct(v, 10) && le_pct(v, 90)) rmad += std::fabs(v - rmean);
  rmad /= (double)rn;
  std::vector<double> h(ng + 1, 0.0);
  for (int lv : g) h[lv] += 1.0;
  double ent = 0, uni = 0;
  for (int i = 1; i <= ng; ++i) {
    if (h[i] == 0) continue;
    double p = h[i] / N;
    ent -= p * std::log2(p);
    uni += p * p;
  }
  f[0] = sum2;
  f[1] = vvox * sum2;
  f[2] = ent;
  f[3] = x.front();
  f[4] = pct(10);
  f[5] = pct(90);
  f[6] = x.back();
  f[7] = mean;
  f[8] = pct(50);
  f[9] = pct(75) - pct(25);
  f[10] = (double)x.back() - x.front();
  f[11] = mad;
  f[12] = rmad;
  f[13] = std::sqrt(sum2 / N);
  f[14] = m2 == 0 ? kNaN : m3 / std::pow(m2, 1.5);
  f[15] = m2 == 0 ? kNaN : m4 / (m2 * m2) - (excess ? 3.0 : 0.0);
  f[16] = m2;
  f[17] = uni;
}

/* Mean over directions, skipping NaN (the IBSI "average over directions"
 * of per-direction features; a direction whose matrix is empty yields NaN
 * for every feature and so drops out).  All NaN -> NaN. */
void average_dirs(const std::vector<double>& per_dir, int ndir, int nf,
                  double* out) {
  for (int k = 0; k < nf; ++k) {
    double s = 0;
    int c = 0;
    for (int d = 0; d < ndir; ++d) {
      double v = per_dir[(size_t)d * nf + k];
      if (std::isnan(v)) continue;
      s += v;
      ++c;
    }
    out[k] = c ? s / c : kNaN;
  }
}

/* All 93 features of one sub-VOI. */
void map_one(const fro_params* p, const Cube& c, int ng, double* f) {
  int dirs[FRO_NUM_DIRS][3];
  make_dirs(dirs);
  std::vector<int> x, g;
  for (size_t k = 0; k < c.lev.size(); ++k)
    if (c.lev[k]) {
      x.push_back(c.raw[k]);
      g.push_back(c.lev[k]);
    }
  const double nv = (double)x.size();
  const double vvox = p->spacing[0] * p->spacing[1] * p->spacing[2];
  firstorder_features(x, g, ng, vvox, p->kurtosis_excess, f + 0);
  firstorder_extra(x, f + 93);

  std::vector<double> M, per((size_t)FRO_NUM_DIRS * 24), perx((size_t)FRO_NUM_DIRS * 2);
  if (p->aggregation == FRO_AGG_MERGED) {
    /* one matrix: the sum of the 13 directional matrices */
    std::vector<double> sum((size_t)ng * ng, 0.0);
    for (int d = 0; d < FRO_NUM_DIRS; ++d) {
      glcm_counts(c, dirs[d], p->distance, ng, M);
      for (size_t k = 0; k < sum.size(); ++k) sum[k] += M[k];
    }
    glcm_features(sum, ng, f + 18);
    glcm_extra(sum, ng, f + 96);
    std::vector<double> rsum((size_t)ng * c.s, 0.0);
    for (int d = 0; d < FRO_NUM_DIRS; ++d) {
      glrlm_counts(c, dirs[d], ng, M);
      for (size_t k = 0; k < rsum.size(); ++k) rsum[k] += M[k];
    }
    rl_features(rsum, ng, c.s, FRO_NUM_DIRS * nv, f + 42);
  } else {
    for (int d = 0; d < FRO_NUM_DIRS; ++d) {
      glcm_counts(c, dirs[d], p->distance, ng, M);
      glcm_features(M, ng, &per[(size_t)d * 24]);
      glcm_extra(M, ng, &perx[(size_t)d * 2]);
    }
    average_dirs(per, FRO_NUM_DIRS, 24, f + 18);
    average_dirs(perx, FRO_NUM_DIRS, 2, f + 96);

    per.assign((size_t)FRO_NUM_DIRS * 16, 0.0);
    for (int d = 0; d < FRO_NUM_DIRS; ++d) {
      glrlm_counts(c, dirs[d], ng, M);
      rl_features(M, ng, c.s, nv, &per[(size_t)d * 16]);
    }
    average_dirs(per, FRO_NUM_DIRS, 16, f + 42);
  }

  std::vector<double> jv;
  glszm_zones(c, ng, M, jv);
  rl_features_j(M, ng, jv, nv, f + 58);

  gldm_counts(c, ng, M);
  gldm_features(M, ng, 27, f + 74);
  gldm_extra(M, ng, 27, nv, f + 98);

  std::vector<double> n, s;
  ngtdm_counts(c, ng, n, s, nullptr);
  ngtdm_features(n, s, ng, f + 88);
}

bool params_ok(const fro_params* p) {
  if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return false;
  if (p->radius < 1 || p->radius > 7 || p->distance < 1) return false;
  if (p->disc_mode == FRO_FBN && p->bin_count < 1) return false;
  if (p->disc_mode == FRO_FBW && !(p->bin_width > 0)) return false;
  if (p->disc_mode != FRO_FBN && p->disc_mode != FRO_FBW) return false;
  if (p->aggregation != FRO_AGG_AVERAGE && p->aggregation != FRO_AGG_MERGED) return false;
  if (p->range_given && p->range_min > p->range_max) return false;
  return true;
}

}  // namespace

extern "C" {

int32_t fro_feature_count(void) { return FRO_NUM_FEATURES; }

const char* fro_feature_name(int32_t id) {
  return (id >= 0 && id < FRO_NUM_SCALAR_FEATURES) ? kNames[id] : nullptr;
}

void fro_direction(int32_t i, int32_t* dz, int32_t* dy, int32_t* dx) {
  int dirs[FRO_NUM_DIRS][3];
  make_dirs(dirs);
  if (i < 0 || i >= FRO_NUM_DIRS) return;
  *dz = dirs[i][0];
  *dy = dirs[i][1];
  *dx = dirs[i][2];
}

/* Discretisation (IBSI), over the whole VOI:
 *   FBN: g = floor(Ng (x - xmin) / (xmax - xmin)) + 1, x = xmax -> Ng,
 *        all ones when xmax == xmin (exact integer arithmetic);
 *   FBW: g = floor((x - a) / w) + 1 in double precision, with anchor
 *        a = xmin (VOI minimum) or a = floor(xmin / w) * w (zero floor);
 *        Ng = floor((xmax - a) / w) + 1. */
int32_t fro_discretise(const fro_params* p, const int16_t* img,
                       const uint8_t* mask, uint8_t* levels, int32_t* ng_out,
                       int32_t* xmin_out, int32_t* xmax_out) {
  if (!params_ok(p)) return 3;
  const int64_t nvox = (int64_t)p->nx * p->ny * p->nz;
  int xmin = std::numeric_limits<int>::max(), xmax = std::numeric_limits<int>::min();
  int64_t count = 0;
  for (int64_t i = 0; i < nvox; ++i)
    if (mask[i]) {
      xmin = std::min(xmin, (int)img[i]);
      xmax = std::max(xmax, (int)img[i]);
      ++count;
    }
  if (count == 0) return 1;
  if (p->range_given) {
    xmin = p->range_min;
    xmax = p->range_max;
  }
  int ng;
  double anchor = xmin;
  if (p->disc_mode == FRO_FBN) {
    ng = p->bin_count;
  } else {
    if (p->fbw_anchor == FRO_ANCHOR_ZERO_FLOOR)
      anchor = std::floor((double)xmin / p->bin_width) * p->bin_width;
    ng = (int)std::floor(((double)xmax - anchor) / p->bin_width) + 1;
  }
  if (ng > 255) return 2;
  for (int64_t i = 0; i < nvox; ++i) {
    if (!mask[i]) {
      levels[i] = 0;
      continue;
    }
    int g;
    /* a given range: the intensity clamped to it */
    const int x = p->range_given ? std::min(std::max((int)img[i], xmin), xmax) : (int)img[i];
    if (p->disc_mode == FRO_FBN) {
      if (xmax == xmin) {
        g = 1;
      } else {
        g = (int)(((int64_t)ng * (x - xmin)) / (xmax - xmin)) + 1;
        if (g > ng) g = ng;
      }
    } else {
      g = (int)std::floor(((double)x - anchor) / p->bin_width) + 1;
    }
    levels[i] = (uint8_t)g;
  }
  *ng_out = ng;
  if (xmin_out) *xmin_out = xmin;
  if (xmax_out) *xmax_out = xmax;
  return 0;
}

int32_t fro_map_voxels(const fro_params* p, const int16_t* img,
                       const uint8_t* levels, int32_t ng, const int64_t* vox,
                       int64_t n, double* out, int32_t nthreads) {
  if (!params_ok(p)) return 3;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
  for (int64_t k = 0; k < n; ++k) {
    double f[FRO_NUM_FEATURES];
    Cube c = make_cube(p, img, levels, vox[k]);
    map_one(p, c, ng, f);
    for (int q = 0; q < FRO_NUM_FEATURES; ++q) out[(size_t)q * n + k] = f[q];
  }
  (void)nthreads;
  return 0;
}

int32_t fro_scalar(const fro_params* p, const int16_t* img, const uint8_t* levels,
                   int32_t ng, double* out) {
  if (!p) return 3;
  fro_params q = *p;
  q.radius = 1;  /* the window is the whole volume; radius plays no part */
  if (!params_ok(&q)) return 3;
  bool any = false;
  const int64_t nvox = (int64_t)p->nx * p->ny * p->nz;
  for (int64_t k = 0; k < nvox && !any; ++k) any = levels[k] != 0;
  if (!any) return 1;
  Cube c = make_whole_cube(p, img, levels);
  map_one(&q, c, ng, out);
  /* standard deviation: sqrt((1/N) sum (x - mean)^2) over the raw
   * intensities of the VOI (population form, as firstorder_Variance) */
  double sum = 0.0, n = 0.0;
  for (size_t k = 0; k < c.lev.size(); ++k)
    if (c.lev[k]) {
      sum += c.raw[k];
      n += 1.0;
    }
  const double mean = sum / n;
  double ss = 0.0;
  for (size_t k = 0; k < c.lev.size(); ++k)
    if (c.lev[k]) ss += (c.raw[k] - mean) * (c.raw[k] - mean);
  out[101] = std::sqrt(ss / n);
  return 0;
}

int32_t fro_matrices(const fro_params* p, const uint8_t* levels, int32_t ng,
                     int64_t vox, int32_t* glcm, int32_t* glrlm,
                     int32_t* glszm, int32_t* gldm, int32_t* ngtdm_n,
                     int64_t* ngtdm_sl, int32_t* hist) {
  if (!params_ok(p)) return 3;
  Cube c = make_cube(p, nullptr, levels, vox);
  int dirs[FRO_NUM_DIRS][3];
  make_dirs(dirs);
  std::vector<double> M;
  if (glcm)
    for (int d = 0; d < FRO_NUM_DIRS; ++d) {
      glcm_counts(c, dirs[d], p->distance, ng, M);
      for (size_t k = 0; k < M.size(); ++k)
        glcm[(size_t)d * ng * ng + k] = (int32_t)M[k];
    }
  if (glrlm)
    for (int d = 0; d < FRO_NUM_DIRS; ++d) {
      glrlm_counts(c, dirs[d], ng, M);
      for (size_t k = 0; k < M.size(); ++k)
        glrlm[(size_t)d * ng * c.s + k] = (int32_t)M[k];
    }
  if (glszm) {
    glszm_counts(c, ng, M);
    for (size_t k = 0; k < M.size(); ++k) glszm[k] = (int32_t)M[k];
  }
  if (gldm) {
    gldm_counts(c, ng, M);
    for (size_t k = 0; k < M.size(); ++k) gldm[k] = (int32_t)M[k];
  }
  if (ngtdm_n || ngtdm_sl) {
    std::vector<double> n, s;
    std::vector<int64_t> sl;
    ngtdm_counts(c, ng, n, s, &sl);
    for (int i = 0; i < ng; ++i) {
      if (ngtdm_n) ngtdm_n[i] = (int32_t)n[i];
      if (ngtdm_sl) ngtdm_sl[i] = sl[i];
    }
  }
  if (hist) {
    for (int i = 0; i < ng; ++i) hist[i] = 0;
    for (int v : c.lev)
      if (v) hist[v - 1] += 1;
  }
  return 0;
}

void fro_glcm_features(const double* counts, int32_t ng, double* out24) {
  std::vector<double> C(counts, counts + (size_t)ng * ng);
  glcm_features(C, ng, out24);
}

void fro_glrlm_features(const double* counts, int32_t ng, int32_t nj,
                        double n_vox, double* out16) {
  std::vector<double> R(counts, counts + (size_t)ng * nj);
  rl_features(R, ng, nj, n_vox, out16);
}

void fro_glszm_features(const double* counts, int32_t ng, int32_t nj,
                        double n_vox, double* out16) {
  std::vector<double> R(counts, counts + (size_t)ng * nj);
  rl_features(R, ng, nj, n_vox, out16);
}

void fro_gldm_features(const double* counts, int32_t ng, int32_t nj,
                       double* out14) {
  std::vector<double> M(counts, counts + (size_t)ng * nj);
  gldm_features(M, ng, nj, out14);
}

void fro_ngtdm_features(const double* n, const double* s, int32_t ng,
                        double* out5) {
  std::vector<double> nn(n, n + ng), ss(s, s + ng);
  ngtdm_features(nn, ss, ng, out5);
}

void fro_firstorder_features(const int32_t* x, const int32_t* g, int64_t n,
                             int32_t ng, double voxel_volume,
                             int32_t kurtosis_excess, double* out18) {
  std::vector<int> xv(x, x + n), gv(g, g + n);
  firstorder_features(xv, gv, ng, voxel_volume, kurtosis_excess, out18);
}

double fro_glcm_mcc(const double* counts, int32_t ng) {
  std::vector<double> C(counts, counts + (size_t)ng * ng);
  return mcc_from_counts(C, ng);
}

}  // extern "C"
