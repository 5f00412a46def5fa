/*
 * fr_oracle.h -- plain FP64 CPU oracle for radiomic spatial mapping.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this library: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library under paper_2609_19190_gb300/csrc.
 *
 * What it computes (paper: Introduction and "Software design and extraction
 * modes"): spatial mapping evaluates, for every voxel v of the VOI, the
 * scalar feature of the image restricted to the local neighbourhood of v.
 * Here that neighbourhood is V(v) = { u : |u - v|_inf <= r } intersected
 * with the image and the VOI, and map_f(v) = feature_f(V(v)).  Gray levels
 * come from one discretisation of the whole VOI (paper: "Hybrid CUDA backend
 * implementation" -- discretisation is a preprocessing step over the VOI).
 * Feature families and counts follow Table 2: ids 0..92 are the spatial
 * benchmark column (statistics 18, GLCM 24, GLRLM 16, GLSZM 16, NGLDM 14,
 * NGTDM 5 = 93); ids 93..100 complete the default spatial column (101: +3
 * statistics, +2 GLCM, +3 NGLDM), read as the IBSI features the benchmark's
 * PyRadiomics-named classes lack: median absolute deviation, coefficient of
 * variation, quartile coefficient of dispersion; GLCM sum variance and
 * dissimilarity; NGLDM grey level non-uniformity normalised, dependence
 * count percentage and dependence count energy.
 * The paper prints no formula; the definitions used are the IBSI ones the
 * paper says both of its backends follow (Introduction; "IBSI compliance
 * tests"), written out in fr_oracle.cpp next to each feature.
 *
 * Every value is computed from dense matrices in double precision, feature
 * by feature, in the textbook form.  Nothing is fused, reordered or made
 * exact beyond what the definitions themselves state.
 */
#ifndef FR_ORACLE_H
#define FR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { FRO_FBN = 0, FRO_FBW = 1 };
enum { FRO_ANCHOR_VOI_MIN = 0, FRO_ANCHOR_ZERO_FLOOR = 1 };
/* Aggregation of the direction-dependent families (GLCM, GLRLM) over the
 * 13 directions: AVERAGE takes features per direction and averages them;
 * MERGED sums the 13 matrices and takes the features once (IBSI 3D:avg and
 * 3D:mrg; the IBSI configurations of the paper's compliance tests name one
 * per family).  Merged GLRLM run percentage divides by 13 N_v. */
enum { FRO_AGG_AVERAGE = 0, FRO_AGG_MERGED = 1 };

#define FRO_NUM_FEATURES 101
/* Scalar extraction adds the one statistic of Table 2's scalar column that
 * has no map (statistics 22 there against 21 in the default spatial column):
 * id 101, the standard deviation (population) of the raw intensities. */
#define FRO_NUM_SCALAR_FEATURES 102
#define FRO_NUM_BENCH 93
#define FRO_NUM_DIRS 13

typedef struct fro_params {
  int32_t nx, ny, nz;        /* volume extents; arrays are [nz][ny][nx]      */
  double spacing[3];         /* voxel spacing in mm (x, y, z)               */
  int32_t disc_mode;         /* FRO_FBN or FRO_FBW                           */
  int32_t bin_count;         /* FBN: number of bins                          */
  double bin_width;          /* FBW: bin width (> 0)                         */
  int32_t fbw_anchor;        /* FRO_ANCHOR_*                                 */
  int32_t radius;            /* window radius r (Chebyshev), 1..7            */
  int32_t distance;          /* GLCM offset distance delta (>= 1)            */
  int32_t kurtosis_excess;   /* 1: m4/m2^2 - 3 ; 0: m4/m2^2                  */
  int32_t aggregation;       /* FRO_AGG_AVERAGE or FRO_AGG_MERGED            */
  int32_t range_given;       /* 1: discretise over [range_min, range_max],   */
  int32_t range_min;         /*    each intensity clamped to it (a z-slab of */
  int32_t range_max;         /*    one volume, discretised as the whole VOI) */
} fro_params;

/* Number of features and the name of feature id (0..92). */
int32_t fro_feature_count(void);
const char* fro_feature_name(int32_t id);

/* The 13 direction vectors (dz, dy, dx), lexicographically positive. */
void fro_direction(int32_t i, int32_t* dz, int32_t* dy, int32_t* dx);

/* Discretise the VOI.  levels[nz*ny*nx] receives 1..Ng inside the VOI, 0
 * outside.  Returns 0 on success, 1 for an empty mask, 2 for Ng > 255,
 * 3 for invalid parameters. */
int32_t fro_discretise(const fro_params* p, const int16_t* img,
                       const uint8_t* mask, uint8_t* levels, int32_t* ng,
                       int32_t* xmin, int32_t* xmax);

/* Feature maps at the listed voxels (linear indices (z*ny + y)*nx + x, each
 * inside the VOI).  out is [101][n] (feature-major).  nthreads <= 0 uses the
 * OpenMP default.  Returns 0 on success. */
int32_t fro_map_voxels(const fro_params* p, const int16_t* img,
                       const uint8_t* levels, int32_t ng, const int64_t* vox,
                       int64_t n, double* out, int32_t nthreads);

/* Scalar extraction: the 102 features of the whole VOI (the paper's other
 * extraction mode; ids 0..100 equal the map value at v whenever the window
 * around v covers the VOI, id 101 is the scalar-only standard deviation).
 * levels from fro_discretise; p->radius is ignored.  Returns 0, 1 for an
 * empty VOI, 3 for invalid parameters. */
int32_t fro_scalar(const fro_params* p, const int16_t* img, const uint8_t* levels,
                   int32_t ng, double* out102);

/* Dense texture matrices of one voxel's sub-VOI V(v) (bit-exact integers).
 * glcm  : [13][ng][ng]  symmetric co-occurrence counts (levels 1..ng at 0..ng-1)
 * glrlm : [13][ng][s]   runs of level i and length j+1, s = 2r+1
 * glszm : [ng][w]       zones of level i and size j+1, w = s^3
 * gldm  : [ng][27]      voxels of level i with j equal 26-neighbours
 * ngtdm_n  : [ng]       voxels of level i with >= 1 neighbour
 * ngtdm_sl : [ng]       s_i * lcm(1..26), exact
 * hist  : [ng]          voxels of level i in V(v)
 * Any pointer may be NULL to skip that family. */
int32_t fro_matrices(const fro_params* p, const uint8_t* levels, int32_t ng,
                     int64_t vox, int32_t* glcm, int32_t* glrlm,
                     int32_t* glszm, int32_t* gldm, int32_t* ngtdm_n,
                     int64_t* ngtdm_sl, int32_t* hist);

/* Feature functions of one matrix, for pins on hand-made matrices.
 * glcm_dir : counts [ng][ng] of ONE direction -> 24 values (NaN if empty)
 * rl       : counts [ng][nj] (one direction / zones / dependences) -> 16 or 14
 * ngtdm    : n[ng], s[ng] (s_i as real numbers) -> 5 values
 * firstorder: raw values x[n] and levels g[n] -> 18 values */
void fro_glcm_features(const double* counts, int32_t ng, double* out24);
void fro_glrlm_features(const double* counts, int32_t ng, int32_t nj,
                        double n_vox, double* out16);
void fro_glszm_features(const double* counts, int32_t ng, int32_t nj,
                        double n_vox, double* out16);
void fro_gldm_features(const double* counts, int32_t ng, int32_t nj,
                       double* out14);
void fro_ngtdm_features(const double* n, const double* s, int32_t ng,
                        double* out5);
void fro_firstorder_features(const int32_t* x, const int32_t* g, int64_t n,
                             int32_t ng, double voxel_volume,
                             int32_t kurtosis_excess, double* out18);

/* Second-largest |eigenvalue| of S = D^-1/2 P D^-1/2 (GLCM MCC) of one
 * direction's counts [ng][ng]; NaN when fewer than two levels occur. */
double fro_glcm_mcc(const double* counts, int32_t ng);

#ifdef __cplusplus
}
#endif
#endif
