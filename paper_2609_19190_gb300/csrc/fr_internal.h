// fr_internal.h -- structures shared by the host plan code and the kernels.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <vector_types.h>

namespace fr {

// Feature ids: 0..92 the 93-map benchmark set, 93..100 the IBSI extras that
// complete the 101-map default set (3 statistics, 2 GLCM, 3 NGLDM).
constexpr int kNumFeatures = 101;
constexpr int kNumBench = 93;
constexpr int kFirstExtra = 93;  // median abs. deviation, CoV, QCoD
constexpr int kGlcmExtra = 96;   // sum variance, dissimilarity
constexpr int kGldmExtra = 98;   // GLNUN, dependence count percentage, energy
// Scalar extraction adds one statistic that has no map: the standard
// deviation (Table 2: statistics 22 in the scalar benchmark column, 21 in
// the default spatial column), id 101.
constexpr int kScalarStd = 101;
constexpr int kNumScalarFeatures = 102;
constexpr int kRowOf = 104;      // row_of entries (>= kNumScalarFeatures)
constexpr int kScalarDirF = 42;  // per-direction values of the scalar path
constexpr int kNumDirs = 13;
constexpr int kMaxRadius = 7;
// Present-level count and level-range limits of the per-warp shared-memory
// arena; a voxel whose window exceeds either uses the warp's global slab.
constexpr int kMCap = 24;
constexpr int kBinCap = 64;
// GLCM MCC: directions whose present-level count is at most kCapL are solved
// after the 13-direction loop, one lane per direction, from packed matrices
// kept in per-direction slots of kSlot floats (packed upper triangle of
// kCapL levels, zero beyond the direction's own levels).
constexpr int kCapL = 12;
constexpr int kSlot = kCapL * (kCapL + 1) / 2 + 1;  // odd: lanes hit distinct banks
constexpr int kMaxConsumerWarps = 16;
// Padded window of the GLDM / NGTDM neighbour pass: sides up to 7 (r <= 3)
// with a one-voxel zero border.
constexpr int kPadMaxSide = 7;
constexpr int kPadCells = (kPadMaxSide + 2) * (kPadMaxSide + 2) * (kPadMaxSide + 2);
constexpr int kMaxStages = 4;
// CTA pool of many-level MCC solves: at most one per direction per warp;
// each direction's S - u u^T is the packed upper triangle of its m x m
// matrix (m (m + 1) / 2 contiguous floats, each written once) in the warp's
// global scratch (kFbDir floats per direction)
constexpr int kFbTasks = kMaxConsumerWarps * kNumDirs;
constexpr int kFbDir = kMCap * kMCap;

// Feature families (bits of FrJob::families).
enum : uint32_t {
  kFamFO = 1u << 0,
  kFamGLCM = 1u << 1,
  kFamMCC = 1u << 2,  // GLCM MCC (the eigenvalue part) requested
  kFamGLRLM = 1u << 3,
  kFamGLSZM = 1u << 4,
  kFamGLDM = 1u << 5,
  kFamNGTDM = 1u << 6,
};

// Run-time state of a job, written by the preparation kernels.
struct FrJobState {
  int32_t xmin, xmax;  // VOI intensity range
  int32_t ng;          // gray levels of the discretisation
  int32_t status;      // fr_status of the job (0 = ok)
};

// One VOI to map (device-resident; 128-byte aligned for the tensor map).
struct alignas(128) FrJob {
  CUtensorMap tmap;      // 3-D tiled map over `packed` (uint32, [nz][ny][px])
  uint32_t* packed;      // ((raw + 32768) << 8) | level, 0 outside the VOI
  const int32_t* voi;    // linear voxel index per output column
  const int32_t* bcols;  // output columns the mapping kernel reads, by brick
  FrJobState* state;
  // Run-time order of the columns inside each brick (fr_order_kernel): by
  // the number of distinct levels in each voxel's window, so that the
  // voxels a CTA maps side by side cost alike.  bcols_brick is the plan's
  // brick order, bseg its non-empty brick segments (offset, count); bcols
  // is written by the ordering (== bcols_brick when there is none).
  const int32_t* bcols_brick;
  const int2* bseg;
  int32_t nbseg;
  int32_t order;  // 1: bcols is reordered per run
  int64_t n_voi;
  int32_t nx, ny, nz, px;
  int32_t r, delta;
  int32_t hx;  // x halo of the TMA box (multiple of 4, >= r)
  int32_t box_x, box_y, box_z;
  int32_t disc_mode, bin_count, anchor_zero_floor;
  int32_t range_given, range_min, range_max;  // given discretisation range
  int32_t kurt_excess;
  int32_t agg;  // FR_AGG_AVERAGE / FR_AGG_MERGED
  int32_t nf;  // output rows
  uint32_t families;
  double bin_width;
  double voxel_volume;
  int16_t row_of[kRowOf];  // output row of each feature id, -1 if not selected
};

// One work-queue entry: up to `n` voxels of one brick of one job.
struct FrItem {
  int32_t job;
  int32_t bx, by, bz;  // brick origin (voxels)
  int32_t j0, n;       // range in the job's brick-ordered column list
};

// Byte offsets of one warp's shared-memory arena.
struct FrArena {
  int32_t bytes;      // arena size (multiple of 16)
  int32_t off_kb;     // uint32[p_max]   sort keys / zone keys
  int32_t off_lvl;    // uint8[w_max]    compact level + 1 per window position
  int32_t off_lut;    // uint8[256]      level -> compact index
  int32_t off_lev;    // uint8[256]      compact index -> level
  int32_t off_st;     // uint16[264]     start of each level run in the sorted keys
  int32_t off_fv;     // float[96]       features of the current voxel
  int32_t off_acc;    // float[32] + int32[32]  per-direction accumulators
  int32_t off_tmp;    // float[64]       compensation terms of the direction sums
  int32_t off_big;    // family matrices (layout from (mc, bc, w))
  int32_t big_bytes;  // size of the shared big region
  int32_t p_max, w_max;
};

// Per-run pointers of job j: run_ptrs[2j] = image (int16), run_ptrs[2j+1] =
// output (float32 [nf][n_voi]).
struct FrMapArgs {
  const FrJob* jobs;
  void* const* run_ptrs;
  const FrItem* items;
  int32_t n_items;
  int32_t consumer_warps;
  int32_t stages;
  int32_t tile_bytes;  // per stage, multiple of 128
  uint32_t* queue;     // work-queue head (reset per run)
  int32_t* status;     // launch-wide status word (timeouts)
  char* slab;          // global big regions, one per resident warp
  int64_t slab_stride; // bytes per warp
  int32_t slab_ngc;    // level cap the slab is laid out for
  FrArena arena;
  float* fb;           // per-warp matrices of many-level MCC solves (kNumDirs x
  int64_t fb_stride;   // kFbDir floats each) handed to the CTA's pool; null: inline
  int32_t* dbg;        // debug records (DUMP kernel only)
  int64_t dbg_stride;  // int32 per record
  int64_t timeout_ns;  // bound of every device wait
  int32_t withhold_item;  // testing: the feeder leaves this item's buffer unfilled (-1: none)
};

// Scalar extraction (the whole VOI as one region): device buffers and sizes.
// Counts are exact integers; features are taken in FP64 (MCC in FP32).
struct FrScalarArgs {
  const uint32_t* packed;      // ((raw + 32768) << 8) | level, 0 outside the VOI
  const int32_t* voi;          // linear index of each VOI voxel
  const FrJobState* state;     // xmin, xmax, ng, status of the discretisation
  int64_t n_voi;
  int32_t nx, ny, nz, px;
  int32_t ngc;                 // level cap of the count buffers (<= 255)
  int32_t lmax;                // longest possible run: max(nx, ny, nz)
  int32_t delta, agg, kurt_excess;
  double voxel_volume;
  uint32_t* hraw;              // [65536] raw-intensity histogram
  uint32_t* hlev;              // [256] level histogram
  uint32_t* gldm;              // [256][27] dependence counts
  uint32_t* ngn;               // [256] NGTDM n_i
  unsigned long long* ngacc;   // [256][27] sum |i k - sum of neighbours| by k
  uint32_t* glcm;              // [13][ngc (ngc + 1) / 2] packed upper-triangle pair counts
  uint32_t* glrlm;             // [13][ngc][lmax] run counts
  int32_t* parent;             // [nvox] union-find forest over VOI voxels
  int32_t* zsize;              // [nvox] zone size at each root
  uint32_t* zrow;              // [256] zones per level
  uint32_t* zcol;              // [n_voi + 1] zones per size
  unsigned long long* hkey;    // [hcap] (level << 32 | size) keys, ~0 = empty
  uint32_t* hcnt;              // [hcap] zones per key
  int64_t hcap;                // power of two >= 2 n_voi
  float* mcc_s;                // [13][ngc][ngc] deflated S matrices
  float* mcc_v;                // [13][4][ngc] solver vectors
  double* dirf;                // [13][kScalarDirF]: GLCM (24), GLRLM (16), GLCM extras (2)
  double* out;                 // [kRowOf] feature values (written by the final kernel)
  int32_t* status;             // run status word
};

// Big-region layout for caps (mc, bc) and window size w.
struct BigLayout {
  int32_t cnt, marg, prank, sbin, dbin, vec;  // GLCM (vec: 4 float vectors of mc)
  int32_t mn, mres, slots;                    // GLCM MCC: n per direction, results, slots
  int32_t csn, cst;                           // GLCM ClusterShade numerators (f64), totals
  int32_t rhist, rlv, rlen;                  // GLRLM
  int32_t parent, zsz, zlv;                  // GLSZM
  int32_t ghist, gj, ngn, ngs;               // GLDM / NGTDM
  int32_t ngacc, pad;                        // NGTDM [level][neighbours], padded window
  int32_t bytes;
};

__host__ __device__ inline int32_t fr_align(int32_t v, int32_t a) {
  return (v + a - 1) / a * a;
}

__host__ __device__ inline BigLayout fr_big_layout(int32_t mc, int32_t bc,
                                                   int32_t w) {
  BigLayout L;
  // GLCM
  L.cnt = 0;
  L.marg = L.cnt + mc * mc * 4;
  L.prank = L.marg + mc * 4;
  L.sbin = L.prank + mc * 4;
  L.dbin = L.sbin + 2 * bc * 4;
  L.vec = L.dbin + bc * 4;
  L.mn = L.vec + 4 * mc * 4;
  L.mres = L.mn + 16 * 4;
  L.slots = L.mres + 16 * 4;
  L.csn = fr_align(L.slots + kNumDirs * kSlot * 4, 8);
  L.cst = L.csn + 16 * 8;
  int32_t glcm_end = L.cst + 16 * 4;
  // GLRLM
  L.rhist = 0;
  L.rlv = L.rhist + mc * 16 * 4;
  L.rlen = L.rlv + mc * 4;
  int32_t glrlm_end = L.rlen + 16 * 4;
  // GLSZM
  L.parent = 0;
  L.zsz = L.parent + w * 4;
  L.zlv = L.zsz + w * 4;
  int32_t glszm_end = L.zlv + mc * 4;
  // GLDM + NGTDM
  L.ghist = 0;
  L.gj = L.ghist + mc * 28 * 4;
  L.ngn = L.gj + 28 * 4;
  L.ngs = fr_align(L.ngn + mc * 4, 8);
  L.ngacc = L.ngs + mc * 8;
  L.pad = L.ngacc + mc * 27 * 4;
  int32_t gldm_end = L.pad + fr_align(kPadCells * 2, 16);
  int32_t m = glcm_end;
  if (glrlm_end > m) m = glrlm_end;
  if (glszm_end > m) m = glszm_end;
  if (gldm_end > m) m = gldm_end;
  L.bytes = fr_align(m, 16);
  return L;
}

inline int32_t fr_next_pow2(int32_t v) {
  int32_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Arena layout for windows up to radius r_max.
inline FrArena fr_make_arena(int32_t r_max) {
  FrArena a;
  const int32_t s = 2 * r_max + 1;
  a.w_max = s * s * s;
  a.p_max = fr_next_pow2(a.w_max);
  int32_t o = 0;
  a.off_kb = o;
  o += a.p_max * 4;
  a.off_lvl = o;
  o += fr_align(a.w_max, 16);
  a.off_lut = o;
  o += 256;
  a.off_lev = o;
  o += 256;
  a.off_st = o;
  o += 264 * 2;
  a.off_fv = o;
  o += kRowOf * 4;
  a.off_acc = o;
  o += 64 * 4;
  a.off_tmp = o;
  o += 64 * 4;
  a.off_big = fr_align(o, 16);
  BigLayout L = fr_big_layout(kMCap, kBinCap, a.w_max);
  a.big_bytes = L.bytes;
  a.bytes = fr_align(a.off_big + a.big_bytes, 16);
  return a;
}

}  // namespace fr
