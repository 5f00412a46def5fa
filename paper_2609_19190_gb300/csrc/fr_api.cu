// fr_api.cu -- host side of the C ABI (include/flashmap.h): parameter
// checks, plans (VOI list, brick schedule, work items, tensor maps, scratch),
// runs, batches with CUDA-graph launch, and the debug / export calls.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/flashmap.h"
#include "fr_internal.h"

namespace fr {
// fr_map_kernel.cu
int fr_map_smem_bytes(int stages, int tile_bytes, int nw, int arena_bytes);
cudaError_t fr_map_configure(bool dump, int smem_bytes);
cudaError_t fr_map_occupancy(bool dump, int threads, int smem_bytes, int* blocks);
cudaError_t fr_map_launch(bool dump, const FrMapArgs& args, int grid, int smem_bytes,
                          cudaStream_t s);
// fr_scalar.cu
cudaError_t fr_scalar_configure(int ngc);
cudaError_t fr_scalar_launch(const FrScalarArgs& a, double* user_out, const int16_t* row_of_dev,
                             int sms, cudaStream_t s);
// fr_prep.cu
cudaError_t fr_launch_prepare(const FrJob* jobs, int njobs, int64_t max_voi,
                              void* const* run_ptrs, uint32_t* queue, int32_t* status,
                              int sms, cudaStream_t s);
cudaError_t fr_launch_order(const FrJob* jobs, int njobs, int max_segments, int sms,
                            cudaStream_t s);
cudaError_t fr_launch_row_count(const uint8_t* mask, int nx, int rows, int32_t* rowcnt,
                                cudaStream_t s);
cudaError_t fr_launch_scan(const int32_t* in, int32_t* out, int n, long long* tot,
                           cudaStream_t s);
cudaError_t fr_launch_voi_fill(const uint8_t* mask, int nx, int rows, const int32_t* rowoff,
                               int32_t* voi, cudaStream_t s);
cudaError_t fr_launch_bricks(const int32_t* voi, int64_t n, int nx, int ny, int bx, int by,
                             int bz, int nbx, int nby, int32_t* bcount, cudaStream_t s);
cudaError_t fr_launch_brick_fill(const int32_t* voi, int64_t n, int nx, int ny, int bx, int by,
                                 int bz, int nbx, int nby, const int32_t* boff,
                                 int32_t* bfill, int32_t* bcols, cudaStream_t s);
cudaError_t fr_launch_scatter(const int32_t* voi, int64_t n, int nf, int64_t nvox,
                              const float* out, float* dense, cudaStream_t s);
cudaError_t fr_launch_levels(const uint32_t* packed, int nx, int rows, int px,
                             uint8_t* levels, cudaStream_t s);
}  // namespace fr

using namespace fr;

namespace {

// Feature names: PyRadiomics-style class_Feature names of the 93 spatial
// benchmark maps (Table 2), in feature-id order.
const char* const kFeatureNames[kNumScalarFeatures] = {
    "firstorder_Energy", "firstorder_TotalEnergy", "firstorder_Entropy",
    "firstorder_Minimum", "firstorder_10Percentile", "firstorder_90Percentile",
    "firstorder_Maximum", "firstorder_Mean", "firstorder_Median",
    "firstorder_InterquartileRange", "firstorder_Range",
    "firstorder_MeanAbsoluteDeviation", "firstorder_RobustMeanAbsoluteDeviation",
    "firstorder_RootMeanSquared", "firstorder_Skewness", "firstorder_Kurtosis",
    "firstorder_Variance", "firstorder_Uniformity",
    "glcm_Autocorrelation", "glcm_JointAverage", "glcm_ClusterProminence",
    "glcm_ClusterShade", "glcm_ClusterTendency", "glcm_Contrast",
    "glcm_Correlation", "glcm_DifferenceAverage", "glcm_DifferenceEntropy",
    "glcm_DifferenceVariance", "glcm_JointEnergy", "glcm_JointEntropy",
    "glcm_Imc1", "glcm_Imc2", "glcm_Idm", "glcm_Idmn", "glcm_Id", "glcm_Idn",
    "glcm_InverseVariance", "glcm_MaximumProbability", "glcm_SumAverage",
    "glcm_SumEntropy", "glcm_SumSquares", "glcm_MCC",
    "glrlm_ShortRunEmphasis", "glrlm_LongRunEmphasis",
    "glrlm_GrayLevelNonUniformity", "glrlm_GrayLevelNonUniformityNormalized",
    "glrlm_RunLengthNonUniformity", "glrlm_RunLengthNonUniformityNormalized",
    "glrlm_RunPercentage", "glrlm_GrayLevelVariance", "glrlm_RunVariance",
    "glrlm_RunEntropy", "glrlm_LowGrayLevelRunEmphasis",
    "glrlm_HighGrayLevelRunEmphasis", "glrlm_ShortRunLowGrayLevelEmphasis",
    "glrlm_ShortRunHighGrayLevelEmphasis", "glrlm_LongRunLowGrayLevelEmphasis",
    "glrlm_LongRunHighGrayLevelEmphasis",
    "glszm_SmallAreaEmphasis", "glszm_LargeAreaEmphasis",
    "glszm_GrayLevelNonUniformity", "glszm_GrayLevelNonUniformityNormalized",
    "glszm_SizeZoneNonUniformity", "glszm_SizeZoneNonUniformityNormalized",
    "glszm_ZonePercentage", "glszm_GrayLevelVariance", "glszm_ZoneVariance",
    "glszm_ZoneEntropy", "glszm_LowGrayLevelZoneEmphasis",
    "glszm_HighGrayLevelZoneEmphasis", "glszm_SmallAreaLowGrayLevelEmphasis",
    "glszm_SmallAreaHighGrayLevelEmphasis", "glszm_LargeAreaLowGrayLevelEmphasis",
    "glszm_LargeAreaHighGrayLevelEmphasis",
    "gldm_SmallDependenceEmphasis", "gldm_LargeDependenceEmphasis",
    "gldm_GrayLevelNonUniformity", "gldm_DependenceNonUniformity",
    "gldm_DependenceNonUniformityNormalized", "gldm_GrayLevelVariance",
    "gldm_DependenceVariance", "gldm_DependenceEntropy",
    "gldm_LowGrayLevelEmphasis", "gldm_HighGrayLevelEmphasis",
    "gldm_SmallDependenceLowGrayLevelEmphasis",
    "gldm_SmallDependenceHighGrayLevelEmphasis",
    "gldm_LargeDependenceLowGrayLevelEmphasis",
    "gldm_LargeDependenceHighGrayLevelEmphasis",
    "ngtdm_Coarseness", "ngtdm_Contrast", "ngtdm_Busyness", "ngtdm_Complexity",
    "ngtdm_Strength",
    // IBSI extras completing the 101-map default set
    "firstorder_MedianAbsoluteDeviation", "firstorder_CoefficientOfVariation",
    "firstorder_QuartileCoefficientOfDispersion", "glcm_SumVariance", "glcm_Dissimilarity",
    "gldm_GrayLevelNonUniformityNormalized", "gldm_DependencePercentage",
    "gldm_DependenceEnergy",
    // scalar extraction only (no map)
    "firstorder_StandardDeviation"
};

// Directions (dz, dy, dx) in the documented order.
const int kDirs[kNumDirs][3] = {{0, 0, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1},
                                {1, -1, -1}, {1, -1, 0}, {1, -1, 1}, {1, 0, -1},
                                {1, 0, 0},  {1, 0, 1},  {1, 1, -1}, {1, 1, 0},
                                {1, 1, 1}};

constexpr long long kTimeoutNs = 10LL * 1000 * 1000 * 1000;  // 10 s per device wait

struct CudaFail {
  fr_status st;
};

#define FR_TRY(expr)                                                     \
  do {                                                                   \
    cudaError_t e__ = (expr);                                            \
    if (e__ != cudaSuccess) {                                            \
      throw CudaFail{e__ == cudaErrorMemoryAllocation ? FR_ERR_OOM        \
                                                      : FR_ERR_CUDA};    \
    }                                                                    \
  } while (0)

template <class T>
T* dev_alloc(size_t count, size_t* acct) {
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) throw CudaFail{FR_ERR_OOM};
  if (acct) *acct += count * sizeof(T);
  return (T*)p;
}

// Allocation from a stream-ordered memory pool on stream s (no device-wide
// synchronisation, unlike cudaMalloc / cudaFree), or plain cudaMalloc when
// pool is null.
template <class T>
T* dev_alloc_on(size_t count, size_t* acct, cudaMemPool_t pool, cudaStream_t s) {
  if (!pool) return dev_alloc<T>(count, acct);
  void* p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMallocFromPoolAsync(&p, count * sizeof(T), pool, s);
  if (e != cudaSuccess) throw CudaFail{FR_ERR_OOM};
  if (acct) *acct += count * sizeof(T);
  return (T*)p;
}

void dev_free_on(void* p, cudaMemPool_t pool, cudaStream_t s) {
  if (!p) return;
  if (pool)
    cudaFreeAsync(p, s);
  else
    cudaFree(p);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// nfeat: ids below it may be selected (maps: kNumFeatures; scalar
// extraction: kNumScalarFeatures).
bool valid_params(const fr_map_params* p, int nfeat = kNumFeatures) {
  if (!p) return false;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return false;
  if (p->kernel_radius < 1 || p->kernel_radius > kMaxRadius) return false;
  if (p->glcm_distance < 1 || p->glcm_distance > 2 * kMaxRadius) return false;
  if (p->disc_mode == FR_FBN) {
    if (p->bin_count < 1 || p->bin_count > 255) return false;
  } else if (p->disc_mode == FR_FBW) {
    if (!(p->bin_width > 0.0)) return false;
    if (p->fbw_anchor != FR_ANCHOR_VOI_MIN && p->fbw_anchor != FR_ANCHOR_ZERO_FLOOR)
      return false;
  } else {
    return false;
  }
  if (!(p->spacing[0] > 0 && p->spacing[1] > 0 && p->spacing[2] > 0)) return false;
  if (p->aggregation != FR_AGG_AVERAGE && p->aggregation != FR_AGG_MERGED) return false;
  if (p->range_given != 0 && p->range_given != 1) return false;
  if (p->range_given && (p->range_min < -32768 || p->range_max > 32767 ||
                         p->range_min > p->range_max))
    return false;
  bool any = false;
  for (int f = 0; f < nfeat; ++f)
    if ((p->feature_mask[f >> 6] >> (f & 63)) & 1ull) any = true;
  if (!any) return false;
  if ((p->feature_mask[1] >> (nfeat - 64)) != 0ull) return false;
  return true;
}

// Built-in launch shape for windows up to radius r_max over about n_voxels
// VOI voxels.  Bricks of 1,024 voxels for launches of at least 100k voxels
// up to r = 3: the per-run voxel order sorts each brick's columns by window
// level count, and larger bricks give it more voxels to group into even
// rounds (C3: 162.1 -> 158.7 ms, C2: 7.23 -> 6.95 ms against 8 x 4 x 4).
// In smaller launches each CTA gets a few items, and grouping the heavy
// windows into the same items lengthens the slowest one (256 VOIs of 4k-20k
// voxels mapped one by one: 150 -> 179 ms); beyond r = 3 the larger halo
// tile would cost consumer warps.
constexpr int64_t kBigBrickVoxels = 100000;
fr_tune default_tune(const fr_tune* t, int r_max, int64_t n_voxels) {
  fr_tune d;
  const bool big = r_max <= 3 && n_voxels >= kBigBrickVoxels;
  d.brick_x = big ? 16 : 8;
  d.brick_y = big ? 8 : 4;
  d.brick_z = big ? 8 : 4;
  d.voxels_per_item = 16;
  d.consumer_warps = 16;
  d.stages = 1;
  d.ctas_per_sm = 0;
  if (t) {
    if (t->brick_x) d.brick_x = t->brick_x;
    if (t->brick_y) d.brick_y = t->brick_y;
    if (t->brick_z) d.brick_z = t->brick_z;
    if (t->voxels_per_item) d.voxels_per_item = t->voxels_per_item;
    if (t->consumer_warps) d.consumer_warps = t->consumer_warps;
    if (t->stages) d.stages = t->stages;
    if (t->ctas_per_sm) d.ctas_per_sm = t->ctas_per_sm;
  }
  return d;
}

// Nonzero bytes of a host buffer, eight at a time.
int64_t count_nonzero(const uint8_t* m, int64_t n) {
  int64_t c = 0, i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, m + i, 8);
    // high bit of each byte set where the byte is nonzero
    const uint64_t lo7 = 0x7F7F7F7F7F7F7F7Full;
    const uint64_t nz = (((w & lo7) + lo7) | w) & ~lo7;
    c += __builtin_popcountll(nz);
  }
  for (; i < n; ++i) c += m[i] != 0;
  return c;
}

bool valid_tune(const fr_tune& t) {
  return t.brick_x >= 4 && t.brick_x % 4 == 0 && t.brick_x <= 64 && t.brick_y >= 1 &&
         t.brick_y <= 64 && t.brick_z >= 1 && t.brick_z <= 64 && t.voxels_per_item >= 1 &&
         t.voxels_per_item <= 1024 && t.consumer_warps >= 1 &&
         t.consumer_warps <= kMaxConsumerWarps && t.stages >= 1 && t.stages <= kMaxStages &&
         t.ctas_per_sm >= 0;
}

// Device resources of one VOI.
struct JobRes {
  fr_map_params p;
  int64_t n_voi = 0;
  int32_t nf = 0;
  int16_t row_of[kRowOf];
  uint32_t families = 0;
  int32_t px = 0;
  int32_t ngc = 0;  // level cap of this job
  uint32_t* packed = nullptr;
  int32_t* voi = nullptr;
  int32_t* bcols = nullptr;      // columns in brick order (plan)
  int32_t* bcols_run = nullptr;  // the same, reordered within bricks per run
  int2* bseg = nullptr;          // non-empty brick segments (offset, count)
  int32_t nbseg = 0;
  FrJobState* state = nullptr;
  std::vector<FrItem> items;  // job field = 0
  size_t bytes = 0;

  // Stream-ordered release (buffers from a memory pool): freed once the work
  // already queued on s has finished; the host does not wait.
  void release_async(cudaStream_t s) {
    cudaFreeAsync(packed, s);
    cudaFreeAsync(voi, s);
    cudaFreeAsync(bcols, s);
    cudaFreeAsync(bcols_run, s);
    cudaFreeAsync(bseg, s);
    cudaFreeAsync(state, s);
    packed = nullptr;
    voi = bcols = bcols_run = nullptr;
    bseg = nullptr;
    state = nullptr;
  }

  void release() {
    cudaFree(packed);
    cudaFree(voi);
    cudaFree(bcols);
    cudaFree(bcols_run);
    cudaFree(bseg);
    cudaFree(state);
    packed = nullptr;
    voi = bcols = bcols_run = nullptr;
    bseg = nullptr;
    state = nullptr;
  }
};

void select_features(JobRes& j, int nfeat) {
  int row = 0;
  j.families = kFamFO;
  for (int f = 0; f < nfeat; ++f) {
    bool on = (j.p.feature_mask[f >> 6] >> (f & 63)) & 1ull;
    j.row_of[f] = on ? (int16_t)row++ : (int16_t)-1;
    if (!on) continue;
    if (f >= FR_GLCM_BEGIN && f < FR_GLRLM_BEGIN) j.families |= kFamGLCM;
    if (f == FR_GLRLM_BEGIN - 1) j.families |= kFamMCC;
    if (f >= FR_GLRLM_BEGIN && f < FR_GLSZM_BEGIN) j.families |= kFamGLRLM;
    if (f >= FR_GLSZM_BEGIN && f < FR_GLDM_BEGIN) j.families |= kFamGLSZM;
    if (f >= FR_GLDM_BEGIN && f < FR_NGTDM_BEGIN) j.families |= kFamGLDM;
    if (f >= FR_NGTDM_BEGIN && f < FR_EXTRAS_BEGIN) j.families |= kFamNGTDM;
    if (f >= kGlcmExtra && f < kGldmExtra) j.families |= kFamGLCM;
    if (f >= kGldmExtra && f < kNumFeatures) j.families |= kFamGLDM;
  }
  for (int f = nfeat; f < kRowOf; ++f) j.row_of[f] = -1;
  j.nf = row;
  j.ngc = j.p.disc_mode == FR_FBN ? j.p.bin_count : 255;
}

// Build the VOI list, brick schedule and items of one mask (synchronous).
// pool: allocate from this stream-ordered pool on s (the server's requests:
// planning never synchronises the device); null: cudaMalloc.
fr_status build_job(const fr_map_params* p, const uint8_t* mask, const fr_tune& tune,
                    JobRes& j, cudaStream_t s, int nfeat = kNumFeatures,
                    cudaMemPool_t pool = nullptr) {
  j.p = *p;
  select_features(j, nfeat);
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const int rows = ny * nz;
  const int64_t nvox = (int64_t)nx * ny * nz;
  uint8_t* dmask = nullptr;
  int32_t *rowcnt = nullptr, *rowoff = nullptr, *bcount = nullptr, *boff = nullptr,
          *bfill = nullptr;
  long long* tot = nullptr;
  fr_status st = FR_OK;
  try {
    const uint8_t* m = mask;
    if (!p->mask_on_device) {
      dmask = dev_alloc_on<uint8_t>(nvox, nullptr, pool, s);
      FR_TRY(cudaMemcpyAsync(dmask, mask, nvox, cudaMemcpyHostToDevice, s));
      m = dmask;
    }
    rowcnt = dev_alloc_on<int32_t>(rows, nullptr, pool, s);
    rowoff = dev_alloc_on<int32_t>(rows, nullptr, pool, s);
    tot = dev_alloc_on<long long>(1, nullptr, pool, s);
    FR_TRY(fr_launch_row_count(m, nx, rows, rowcnt, s));
    FR_TRY(fr_launch_scan(rowcnt, rowoff, rows, tot, s));
    long long n = 0;
    FR_TRY(cudaMemcpyAsync(&n, tot, sizeof(n), cudaMemcpyDeviceToHost, s));
    FR_TRY(cudaStreamSynchronize(s));
    if (n == 0) throw CudaFail{FR_ERR_EMPTY_MASK};
    j.n_voi = n;
    j.voi = dev_alloc_on<int32_t>(n, &j.bytes, pool, s);
    FR_TRY(fr_launch_voi_fill(m, nx, rows, rowoff, j.voi, s));
    const int bx = tune.brick_x, by = tune.brick_y, bz = tune.brick_z;
    const int nbx = (nx + bx - 1) / bx, nby = (ny + by - 1) / by, nbz = (nz + bz - 1) / bz;
    const int nb = nbx * nby * nbz;
    bcount = dev_alloc_on<int32_t>(nb, nullptr, pool, s);
    boff = dev_alloc_on<int32_t>(nb, nullptr, pool, s);
    bfill = dev_alloc_on<int32_t>(nb, nullptr, pool, s);
    FR_TRY(cudaMemsetAsync(bcount, 0, nb * sizeof(int32_t), s));
    FR_TRY(cudaMemsetAsync(bfill, 0, nb * sizeof(int32_t), s));
    FR_TRY(fr_launch_bricks(j.voi, n, nx, ny, bx, by, bz, nbx, nby, bcount, s));
    FR_TRY(fr_launch_scan(bcount, boff, nb, tot, s));
    j.bcols = dev_alloc_on<int32_t>(n, &j.bytes, pool, s);
    FR_TRY(fr_launch_brick_fill(j.voi, n, nx, ny, bx, by, bz, nbx, nby, boff, bfill, j.bcols,
                                s));
    std::vector<int32_t> hc(nb), ho(nb);
    FR_TRY(cudaMemcpyAsync(hc.data(), bcount, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FR_TRY(cudaMemcpyAsync(ho.data(), boff, nb * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FR_TRY(cudaStreamSynchronize(s));
    const int iv = tune.voxels_per_item;
    std::vector<int2> segs;
    for (int b = 0; b < nb; ++b)
      if (hc[b]) segs.push_back(make_int2(ho[b], hc[b]));
    j.nbseg = (int32_t)segs.size();
    j.bseg = dev_alloc_on<int2>(segs.size(), &j.bytes, pool, s);
    FR_TRY(cudaMemcpyAsync(j.bseg, segs.data(), segs.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, s));
    j.bcols_run = dev_alloc_on<int32_t>(n, &j.bytes, pool, s);
    FR_TRY(cudaMemcpyAsync(j.bcols_run, j.bcols, n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                           s));
    for (int b = 0; b < nb; ++b) {
      if (!hc[b]) continue;
      const int ix = b % nbx, iy = (b / nbx) % nby, iz = b / (nbx * nby);
      for (int t = 0; t < hc[b]; t += iv) {
        FrItem it;
        it.job = 0;
        it.bx = ix * bx;
        it.by = iy * by;
        it.bz = iz * bz;
        it.j0 = ho[b] + t;
        it.n = std::min(iv, hc[b] - t);
        j.items.push_back(it);
      }
    }
    j.px = (nx + 3) / 4 * 4;
    const size_t packed_n = (size_t)j.px * ny * nz;
    j.packed = dev_alloc_on<uint32_t>(packed_n, &j.bytes, pool, s);
    FR_TRY(cudaMemsetAsync(j.packed, 0, packed_n * sizeof(uint32_t), s));
    j.state = dev_alloc_on<FrJobState>(1, &j.bytes, pool, s);
    FR_TRY(cudaMemsetAsync(j.state, 0, sizeof(FrJobState), s));
    FR_TRY(cudaStreamSynchronize(s));
  } catch (CudaFail& f) {
    st = f.st;
    cudaStreamSynchronize(s);
    j.release();
  }
  dev_free_on(dmask, pool, s);
  dev_free_on(rowcnt, pool, s);
  dev_free_on(rowoff, pool, s);
  dev_free_on(bcount, pool, s);
  dev_free_on(boff, pool, s);
  dev_free_on(bfill, pool, s);
  dev_free_on(tot, pool, s);
  return st;
}

// A set of jobs sharing one persistent launch.
struct Engine {
  int device = 0, sms = 0;
  std::vector<JobRes> jobs;
  std::vector<FrJob> hjobs;
  FrJob* jobs_dev = nullptr;
  void** run_ptrs_dev = nullptr;
  FrItem* items_dev = nullptr;
  int n_items = 0;
  int64_t timeout_ns = kTimeoutNs;  // bound of every device wait
  int32_t withhold_item = -1;       // testing hook (fr_debug_wait_fault)
  uint32_t* queue = nullptr;
  int32_t* status = nullptr;
  char* slab = nullptr;
  int64_t slab_stride = 0;
  int slab_ngc = 0;
  float* fb = nullptr;  // many-level MCC matrices handed to the CTA pool
  int64_t fb_stride = 0;
  FrArena arena{};
  fr_tune tune{};
  int nw = 0, stages = 0, tile_bytes = 0, smem = 0, grid = 0;
  int64_t max_voi = 0;
  int max_nbseg = 0;  // brick segments of the largest job (voxel ordering)
  size_t bytes = 0;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t private_stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t k_begin = nullptr, k_end = nullptr;  // around the mapping kernel
  bool ran = false;

  void release() {
    if (done) cudaEventSynchronize(done);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (private_stream) cudaStreamDestroy(private_stream);
    if (done) cudaEventDestroy(done);
    if (k_begin) cudaEventDestroy(k_begin);
    if (k_end) cudaEventDestroy(k_end);
    k_begin = k_end = nullptr;
    for (auto& j : jobs) j.release();
    cudaFree(jobs_dev);
    cudaFree(run_ptrs_dev);
    cudaFree(items_dev);
    cudaFree(queue);
    cudaFree(status);
    cudaFree(slab);
    cudaFree(fb);
    fb = nullptr;
    gexec = nullptr;
    private_stream = nullptr;
    done = nullptr;
    jobs_dev = nullptr;
    run_ptrs_dev = nullptr;
    items_dev = nullptr;
    queue = nullptr;
    status = nullptr;
    slab = nullptr;
  }

  FrMapArgs args(bool dump) const {
    FrMapArgs a{};
    a.jobs = jobs_dev;
    a.run_ptrs = run_ptrs_dev;
    a.items = items_dev;
    a.n_items = n_items;
    a.consumer_warps = nw;
    a.stages = stages;
    a.tile_bytes = tile_bytes;
    a.queue = queue;
    a.status = status;
    a.slab = slab;
    a.slab_stride = slab_stride;
    a.slab_ngc = slab_ngc;
    a.fb = fb;
    a.fb_stride = fb_stride;
    a.arena = arena;
    a.dbg = nullptr;
    a.dbg_stride = 0;
    a.timeout_ns = timeout_ns;
    a.withhold_item = withhold_item;
    (void)dump;
    return a;
  }

  // Everything after the jobs are built: launch shape, scratch, tensor maps.
  fr_status finalize(cudaStream_t s) {
    try {
      int r_max = 1;
      for (auto& j : jobs) {
        r_max = std::max(r_max, j.p.kernel_radius);
        max_voi = std::max(max_voi, j.n_voi);
        max_nbseg = std::max(max_nbseg, (int)j.nbseg);
      }
      arena = fr_make_arena(r_max);
      tile_bytes = 0;
      for (auto& j : jobs) {
        const int r = j.p.kernel_radius, hx = (r + 3) / 4 * 4;
        const int b = (tune.brick_x + 2 * hx) * (tune.brick_y + 2 * r) * (tune.brick_z + 2 * r) * 4;
        tile_bytes = std::max(tile_bytes, b);
      }
      tile_bytes = fr_align(tile_bytes, 128);
      stages = tune.stages;
      nw = tune.consumer_warps;
      int max_smem = 0;
      FR_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
      while (nw > 1 && fr_map_smem_bytes(stages, tile_bytes, nw, arena.bytes) > max_smem) --nw;
      smem = fr_map_smem_bytes(stages, tile_bytes, nw, arena.bytes);
      if (smem > max_smem) throw CudaFail{FR_ERR_UNSUPPORTED};
      // the attribute is global to the kernel: raise it to the device's
      // limit, so plans of different sizes can all launch
      FR_TRY(fr_map_configure(false, max_smem));
      FR_TRY(fr_map_configure(true, max_smem));
      int blocks = 0;
      FR_TRY(fr_map_occupancy(false, 32 * nw, smem, &blocks));
      if (blocks < 1) throw CudaFail{FR_ERR_UNSUPPORTED};
      if (tune.ctas_per_sm > 0) blocks = std::min(blocks, tune.ctas_per_sm);
      grid = sms * blocks;
      slab_ngc = 0;
      for (auto& j : jobs) slab_ngc = std::max(slab_ngc, j.ngc);
      if (slab_ngc > kMCap) {
        slab_stride = fr_align(fr_big_layout(slab_ngc, slab_ngc, arena.w_max).bytes, 256);
        slab = dev_alloc<char>((size_t)grid * nw * slab_stride, &bytes);
        FR_TRY(cudaMemsetAsync(slab, 0, (size_t)grid * nw * slab_stride, s));
      } else {
        slab_stride = 0;
      }
      fb_stride = (int64_t)kNumDirs * kFbDir;
      fb = dev_alloc<float>((size_t)grid * nw * fb_stride, &bytes);
      // device job table with tensor maps
      PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
      if (!enc) throw CudaFail{FR_ERR_CUDA};
      hjobs.resize(jobs.size());
      for (size_t i = 0; i < jobs.size(); ++i) {
        JobRes& j = jobs[i];
        FrJob& h = hjobs[i];
        memset((void*)&h, 0, sizeof(FrJob));
        h.packed = j.packed;
        h.voi = j.voi;
        h.bcols = j.bcols_run;
        h.bcols_brick = j.bcols;
        h.bseg = j.bseg;
        h.nbseg = j.nbseg;
        h.order = 1;
        h.state = j.state;
        h.n_voi = j.n_voi;
        h.nx = j.p.nx;
        h.ny = j.p.ny;
        h.nz = j.p.nz;
        h.px = j.px;
        h.r = j.p.kernel_radius;
        h.delta = j.p.glcm_distance;
        h.agg = j.p.aggregation;
        h.hx = (h.r + 3) / 4 * 4;
        h.box_x = tune.brick_x + 2 * h.hx;
        h.box_y = tune.brick_y + 2 * h.r;
        h.box_z = tune.brick_z + 2 * h.r;
        h.disc_mode = j.p.disc_mode;
        h.bin_count = j.p.bin_count;
        h.anchor_zero_floor = j.p.fbw_anchor == FR_ANCHOR_ZERO_FLOOR;
        h.range_given = j.p.range_given ? 1 : 0;
        h.range_min = j.p.range_min;
        h.range_max = j.p.range_max;
        h.kurt_excess = j.p.kurtosis_excess ? 1 : 0;
        h.nf = j.nf;
        h.families = j.families;
        h.bin_width = j.p.bin_width;
        h.voxel_volume = j.p.spacing[0] * j.p.spacing[1] * j.p.spacing[2];
        memcpy(h.row_of, j.row_of, sizeof(h.row_of));
        cuuint64_t gdim[3] = {(cuuint64_t)j.px, (cuuint64_t)j.p.ny, (cuuint64_t)j.p.nz};
        cuuint64_t gstride[2] = {(cuuint64_t)j.px * 4, (cuuint64_t)j.px * j.p.ny * 4};
        cuuint32_t box[3] = {(cuuint32_t)h.box_x, (cuuint32_t)h.box_y, (cuuint32_t)h.box_z};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult cr = enc(&h.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, (void*)j.packed, gdim,
                          gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) throw CudaFail{FR_ERR_UNSUPPORTED};
      }
      jobs_dev = dev_alloc<FrJob>(jobs.size(), &bytes);
      FR_TRY(cudaMemcpyAsync(jobs_dev, hjobs.data(), jobs.size() * sizeof(FrJob),
                             cudaMemcpyHostToDevice, s));
      // items: most expensive windows first, then job, then brick order
      std::vector<FrItem> all;
      std::vector<int> order(jobs.size());
      for (size_t i = 0; i < jobs.size(); ++i) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return jobs[a].p.kernel_radius > jobs[b].p.kernel_radius;
      });
      for (int i : order)
        for (FrItem it : jobs[i].items) {
          it.job = i;
          all.push_back(it);
        }
      n_items = (int)all.size();
      items_dev = dev_alloc<FrItem>(all.size(), &bytes);
      FR_TRY(cudaMemcpyAsync(items_dev, all.data(), all.size() * sizeof(FrItem),
                             cudaMemcpyHostToDevice, s));
      run_ptrs_dev = dev_alloc<void*>(2 * jobs.size(), &bytes);
      queue = dev_alloc<uint32_t>(1, &bytes);
      status = dev_alloc<int32_t>(1, &bytes);
      FR_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
      FR_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
      FR_TRY(cudaEventCreate(&k_begin));
      FR_TRY(cudaEventCreate(&k_end));
      FR_TRY(cudaStreamSynchronize(s));
      for (auto& j : jobs) bytes += j.bytes;
    } catch (CudaFail& f) {
      cudaStreamSynchronize(s);
      return f.st;
    }
    return FR_OK;
  }

  cudaError_t enqueue(cudaStream_t s) {
    cudaError_t e = fr_launch_prepare(jobs_dev, (int)jobs.size(), max_voi, run_ptrs_dev, queue,
                                      status, sms, s);
    if (e != cudaSuccess) return e;
    if ((e = fr_launch_order(jobs_dev, (int)jobs.size(), max_nbseg, sms, s)) != cudaSuccess)
      return e;
    // while capturing, external records stay timing records in the graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cap)) != cudaSuccess) return e;
    const unsigned flags =
        cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if ((e = cudaEventRecordWithFlags(k_begin, s, flags)) != cudaSuccess) return e;
    if ((e = fr_map_launch(false, args(false), grid, smem, s)) != cudaSuccess) return e;
    return cudaEventRecordWithFlags(k_end, s, flags);
  }

  fr_status kernel_ms(float* ms) {
    if (!ms) return FR_ERR_INVALID_ARG;
    if (!ran) return FR_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
    if (cudaEventSynchronize(k_end) != cudaSuccess) return FR_ERR_CUDA;
    return cudaEventElapsedTime(ms, k_begin, k_end) == cudaSuccess ? FR_OK : FR_ERR_CUDA;
  }

  fr_status capture_graph() {
    if (gexec) return FR_OK;
    if (!private_stream &&
        cudaStreamCreateWithFlags(&private_stream, cudaStreamNonBlocking) != cudaSuccess)
      return FR_ERR_CUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(private_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return FR_ERR_CUDA;
    cudaError_t e = enqueue(private_stream);
    cudaError_t e2 = cudaStreamEndCapture(private_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return FR_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? FR_OK : FR_ERR_CUDA;
  }

  fr_status run(void* const* ptrs, cudaStream_t s, bool graph) {
    if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
    if (cudaMemcpyAsync(run_ptrs_dev, ptrs, 2 * jobs.size() * sizeof(void*),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return FR_ERR_CUDA;
    if (graph) {
      fr_status st = capture_graph();
      if (st != FR_OK) return st;
      if (cudaGraphLaunch(gexec, s) != cudaSuccess) return FR_ERR_CUDA;
    } else {
      if (enqueue(s) != cudaSuccess) return FR_ERR_CUDA;
    }
    if (cudaEventRecord(done, s) != cudaSuccess) return FR_ERR_CUDA;
    ran = true;
    return FR_OK;
  }

  fr_status sync_status() {
    if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
    if (ran && cudaEventSynchronize(done) != cudaSuccess) return FR_ERR_CUDA;
    int32_t st = 0;
    if (cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
      return FR_ERR_CUDA;
    if (st) return (fr_status)st;
    for (auto& j : jobs) {
      FrJobState js;
      if (cudaMemcpy(&js, j.state, sizeof(js), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FR_ERR_CUDA;
      if (js.status) return (fr_status)js.status;
    }
    return FR_OK;
  }
};

fr_status engine_open(Engine& E, const fr_map_params* ps, const uint8_t* const* masks, int n,
                      const fr_tune* tune) {
  for (int i = 0; i < n; ++i) {
    if (!valid_params(&ps[i]) || !masks[i]) return FR_ERR_INVALID_ARG;
    if (ps[i].device != ps[0].device) return FR_ERR_INVALID_ARG;
  }
  int r_max = 1;
  int64_t nvoi = 0;  // host masks: VOI voxels; device masks: volume voxels
  for (int i = 0; i < n; ++i) {
    r_max = std::max(r_max, (int)ps[i].kernel_radius);
    nvoi += ps[i].mask_on_device ? (int64_t)ps[i].nx * ps[i].ny * ps[i].nz
                                 : count_nonzero(masks[i], (int64_t)ps[i].nx * ps[i].ny * ps[i].nz);
  }
  E.tune = default_tune(tune, r_max, nvoi);
  if (!valid_tune(E.tune)) return FR_ERR_INVALID_ARG;
  E.device = ps[0].device;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || E.device < 0 || E.device >= ndev)
    return FR_ERR_UNSUPPORTED;
  if (cudaSetDevice(E.device) != cudaSuccess) return FR_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, E.device) != cudaSuccess) return FR_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return FR_ERR_UNSUPPORTED;
  E.sms = prop.multiProcessorCount;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FR_ERR_CUDA;
  fr_status st = FR_OK;
  E.jobs.resize(n);
  for (int i = 0; i < n && st == FR_OK; ++i) st = build_job(&ps[i], masks[i], E.tune, E.jobs[i], s);
  if (st == FR_OK) st = E.finalize(s);
  cudaStreamDestroy(s);
  if (st != FR_OK) E.release();
  return st;
}


// ---------------------------------------------------------------------------
// Server: iteration-level continuous batching.  Requests own their device
// resources (a planned job); the server owns a job table of `max_slots`
// entries, a launch configuration for windows up to `max_radius`, and a
// stream.  Each step launches the persistent mapping kernel once over a
// bounded number of voxels taken round-robin from every active request, so a
// request that arrives while others are mapped joins the very next step and
// its work shares the launches of the long-running ones.
struct ServerReq {
  JobRes job;
  int64_t id = 0;
  int slot = -1;
  size_t issued = 0;     // items handed to launched steps
  size_t completed = 0;  // items of completed steps
  bool prepared = false;
  bool done = false;
  const int16_t* image = nullptr;
  float* out = nullptr;
};

struct ServerStep {
  cudaEvent_t ev = nullptr;
  std::vector<std::pair<int, size_t>> advance;  // (slot, items) finished by this step
  bool busy = false;
};

}  // namespace

struct fr_server {
  int device = 0, sms = 0, max_radius = 3, max_slots = 0;
  fr_tune tune{};
  FrArena arena{};
  int nw = 0, stages = 0, tile_bytes = 0, smem = 0, grid = 0;
  FrJob* jobs_dev = nullptr;
  void** run_ptrs_dev = nullptr;
  FrItem* items_dev[2] = {nullptr, nullptr};
  int max_items = 0;
  uint32_t* queue = nullptr;
  int32_t* status = nullptr;
  char* slab = nullptr;
  int64_t slab_stride = 0;
  float* fb = nullptr;
  int64_t fb_stride = 0;
  int slab_ngc = 255;
  cudaStream_t stream = nullptr;       // steps
  cudaStream_t plan_stream = nullptr;  // request planning
  cudaMemPool_t pool = nullptr;        // stream-ordered pool of request buffers
  uint32_t* prep_queue = nullptr;      // words the discretisation kernels reset,
  int32_t* prep_status = nullptr;      // kept apart from the steps' queue/status
  ServerStep steps[2];
  int next_step = 0;
  std::vector<ServerReq*> slots;
  int64_t next_id = 1;
  size_t bytes = 0;
  std::vector<FrItem> host_items;
};

namespace {

void server_release_all(fr_server* S) {
  if (S->stream) cudaStreamSynchronize(S->stream);
  for (auto*& r : S->slots)
    if (r) {
      r->job.release();
      delete r;
      r = nullptr;
    }
  for (auto& st : S->steps)
    if (st.ev) cudaEventDestroy(st.ev);
  cudaFree(S->jobs_dev);
  cudaFree(S->run_ptrs_dev);
  cudaFree(S->items_dev[0]);
  cudaFree(S->items_dev[1]);
  cudaFree(S->queue);
  cudaFree(S->status);
  cudaFree(S->slab);
  cudaFree(S->fb);
  cudaFree(S->prep_queue);
  cudaFree(S->prep_status);
  if (S->stream) cudaStreamDestroy(S->stream);
  if (S->plan_stream) cudaStreamDestroy(S->plan_stream);
  if (S->pool) {
    cudaDeviceSynchronize();
    cudaMemPoolDestroy(S->pool);
  }
}

// Complete the oldest busy step if it has finished (or wait for it).
fr_status server_complete(fr_server* S, ServerStep& st, bool wait) {
  if (!st.busy) return FR_OK;
  cudaError_t e = wait ? cudaEventSynchronize(st.ev) : cudaEventQuery(st.ev);
  if (e == cudaErrorNotReady) return FR_OK;
  if (e != cudaSuccess) return FR_ERR_CUDA;
  for (auto& a : st.advance) {
    ServerReq* r = S->slots[a.first];
    if (r) r->completed += a.second;
  }
  st.advance.clear();
  st.busy = false;
  return FR_OK;
}

}  // namespace

struct fr_plan {
  Engine E;
  int16_t* img_stage = nullptr;
  float* out_stage = nullptr;
  size_t stage_bytes = 0;
};

struct fr_batch {
  Engine E;
};

// Scalar extraction: the discretised VOI (a planned job without bricks) and
// the count buffers of the whole-VOI matrices, in one allocation.
struct fr_scalar {
  JobRes j;
  int device = 0, sms = 0;
  FrJob* d_job = nullptr;
  void** d_run = nullptr;
  uint32_t* d_queue = nullptr;
  int32_t* d_status = nullptr;
  int16_t* d_row_of = nullptr;
  char* scratch = nullptr;
  size_t zero_bytes = 0;  // counts at the start of scratch, cleared per run
  size_t key_off = 0, key_bytes = 0;  // hash keys, set to ~0 per run
  size_t bytes = 0;
  FrScalarArgs A;
  cudaEvent_t done = nullptr;
  bool ran = false;

  void release() {
    j.release();
    cudaFree(d_job);
    cudaFree(d_run);
    cudaFree(d_queue);
    cudaFree(d_status);
    cudaFree(d_row_of);
    cudaFree(scratch);
    if (done) cudaEventDestroy(done);
    d_job = nullptr;
    d_run = nullptr;
    d_queue = nullptr;
    d_status = nullptr;
    d_row_of = nullptr;
    scratch = nullptr;
    done = nullptr;
  }
};

namespace {

fr_status scalar_open(fr_scalar& S, const fr_map_params* p, const uint8_t* mask) {
  if (!valid_params(p, kNumScalarFeatures) || !mask) return FR_ERR_INVALID_ARG;
  S.device = p->device;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || S.device < 0 || S.device >= ndev)
    return FR_ERR_UNSUPPORTED;
  if (cudaSetDevice(S.device) != cudaSuccess) return FR_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, S.device) != cudaSuccess) return FR_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return FR_ERR_UNSUPPORTED;
  S.sms = prop.multiProcessorCount;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FR_ERR_CUDA;
  fr_status st = build_job(p, mask, default_tune(nullptr, p->kernel_radius, 0), S.j, s,
                           kNumScalarFeatures);
  if (st != FR_OK) {
    cudaStreamDestroy(s);
    return st;
  }
  try {
    JobRes& j = S.j;
    FrJob h;
    memset((void*)&h, 0, sizeof(FrJob));
    h.packed = j.packed;
    h.voi = j.voi;
    h.bcols = j.bcols;
    h.bcols_brick = j.bcols;
    h.order = 0;  // scalar extraction has no mapping kernel
    h.state = j.state;
    h.n_voi = j.n_voi;
    h.nx = p->nx;
    h.ny = p->ny;
    h.nz = p->nz;
    h.px = j.px;
    h.r = p->kernel_radius;
    h.delta = p->glcm_distance;
    h.agg = p->aggregation;
    h.disc_mode = p->disc_mode;
    h.bin_count = p->bin_count;
    h.anchor_zero_floor = p->fbw_anchor == FR_ANCHOR_ZERO_FLOOR;
    h.range_given = p->range_given ? 1 : 0;
    h.range_min = p->range_min;
    h.range_max = p->range_max;
    h.kurt_excess = p->kurtosis_excess ? 1 : 0;
    h.nf = j.nf;
    h.families = j.families;
    h.bin_width = p->bin_width;
    h.voxel_volume = p->spacing[0] * p->spacing[1] * p->spacing[2];
    memcpy(h.row_of, j.row_of, sizeof(h.row_of));
    S.d_job = dev_alloc<FrJob>(1, &S.bytes);
    FR_TRY(cudaMemcpyAsync(S.d_job, &h, sizeof(FrJob), cudaMemcpyHostToDevice, s));
    S.d_run = dev_alloc<void*>(2, &S.bytes);
    S.d_queue = dev_alloc<uint32_t>(1, &S.bytes);
    S.d_status = dev_alloc<int32_t>(1, &S.bytes);
    S.d_row_of = dev_alloc<int16_t>(kRowOf, &S.bytes);
    FR_TRY(cudaMemcpyAsync(S.d_row_of, j.row_of, sizeof(j.row_of), cudaMemcpyHostToDevice, s));
    // count buffers (cleared per run) first, then the rest
    const int ngc = j.ngc;
    const int64_t nvox = (int64_t)p->nx * p->ny * p->nz;
    const int lmax = std::max(p->nx, std::max(p->ny, p->nz));
    int64_t hcap = 1024;
    while (hcap < 2 * j.n_voi) hcap <<= 1;
    size_t off = 0;
    auto take = [&](size_t b) {
      const size_t o = off;
      off = (off + b + 255) / 256 * 256;
      return o;
    };
    const size_t o_hraw = take(65536 * 4), o_hlev = take(256 * 4), o_gldm = take(256 * 27 * 4),
                 o_ngn = take(256 * 4), o_ngacc = take(256 * 27 * 8),
                 o_glcm = take((size_t)kNumDirs * (ngc * (ngc + 1) / 2) * 4),
                 o_glrlm = take((size_t)kNumDirs * ngc * lmax * 4), o_zsize = take((size_t)nvox * 4),
                 o_zrow = take(256 * 4), o_zcol = take((size_t)(j.n_voi + 1) * 4),
                 o_hcnt = take((size_t)hcap * 4);
    S.zero_bytes = off;
    const size_t o_hkey = take((size_t)hcap * 8);
    S.key_off = o_hkey;
    S.key_bytes = (size_t)hcap * 8;
    const size_t o_parent = take((size_t)nvox * 4),
                 o_mccs = take((size_t)kNumDirs * ngc * ngc * 4),
                 o_mccv = take((size_t)kNumDirs * 4 * ngc * 4), o_dirf = take(kNumDirs * kScalarDirF * 8),
                 o_out = take(kRowOf * 8);
    S.scratch = dev_alloc<char>(off, &S.bytes);
    FrScalarArgs& A = S.A;
    memset((void*)&A, 0, sizeof(A));
    A.packed = j.packed;
    A.voi = j.voi;
    A.state = j.state;
    A.n_voi = j.n_voi;
    A.nx = p->nx;
    A.ny = p->ny;
    A.nz = p->nz;
    A.px = j.px;
    A.ngc = ngc;
    A.lmax = lmax;
    A.delta = p->glcm_distance;
    A.agg = p->aggregation;
    A.kurt_excess = p->kurtosis_excess ? 1 : 0;
    A.voxel_volume = h.voxel_volume;
    A.hraw = (uint32_t*)(S.scratch + o_hraw);
    A.hlev = (uint32_t*)(S.scratch + o_hlev);
    A.gldm = (uint32_t*)(S.scratch + o_gldm);
    A.ngn = (uint32_t*)(S.scratch + o_ngn);
    A.ngacc = (unsigned long long*)(S.scratch + o_ngacc);
    A.glcm = (uint32_t*)(S.scratch + o_glcm);
    A.glrlm = (uint32_t*)(S.scratch + o_glrlm);
    A.zsize = (int32_t*)(S.scratch + o_zsize);
    A.zrow = (uint32_t*)(S.scratch + o_zrow);
    A.zcol = (uint32_t*)(S.scratch + o_zcol);
    A.hcnt = (uint32_t*)(S.scratch + o_hcnt);
    A.hkey = (unsigned long long*)(S.scratch + o_hkey);
    A.hcap = hcap;
    A.parent = (int32_t*)(S.scratch + o_parent);
    A.mcc_s = (float*)(S.scratch + o_mccs);
    A.mcc_v = (float*)(S.scratch + o_mccv);
    A.dirf = (double*)(S.scratch + o_dirf);
    A.out = (double*)(S.scratch + o_out);
    A.status = S.d_status;
    FR_TRY(fr_scalar_configure(ngc));
    FR_TRY(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
    FR_TRY(cudaStreamSynchronize(s));
  } catch (CudaFail& f) {
    st = f.st;
  }
  cudaStreamDestroy(s);
  return st;
}

}  // namespace

extern "C" {

void fr_map_params_init(fr_map_params* p, int32_t nx, int32_t ny, int32_t nz) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->spacing[0] = p->spacing[1] = p->spacing[2] = 1.0;
  p->disc_mode = FR_FBN;
  p->bin_count = 16;
  p->bin_width = 25.0;
  p->fbw_anchor = FR_ANCHOR_VOI_MIN;
  p->kernel_radius = 1;
  p->glcm_distance = 1;
  p->feature_mask[0] = ~0ull;
  p->feature_mask[1] = (1ull << (kNumBench - 64)) - 1ull;  // the 93-map benchmark set
  p->kurtosis_excess = 1;
  p->device = 0;
  p->mask_on_device = 0;
  p->aggregation = FR_AGG_AVERAGE;
}

fr_status fr_map_plan(const fr_map_params* p, const uint8_t* mask, const fr_tune* tune,
                      fr_plan** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p || !mask) return FR_ERR_INVALID_ARG;
  fr_plan* plan = new (std::nothrow) fr_plan();
  if (!plan) return FR_ERR_OOM;
  const uint8_t* masks[1] = {mask};
  fr_status st = engine_open(plan->E, p, masks, 1, tune);
  if (st != FR_OK) {
    delete plan;
    return st;
  }
  *out = plan;
  return FR_OK;
}

fr_status fr_map_run(fr_plan* plan, const int16_t* image, float* out, fr_stream_t s) {
  if (!plan || !image || !out) return FR_ERR_INVALID_ARG;
  void* ptrs[2] = {(void*)image, (void*)out};
  return plan->E.run(ptrs, (cudaStream_t)s, false);
}

fr_status fr_map_run_host(fr_plan* plan, const int16_t* image_host, float* out_host,
                          fr_stream_t s) {
  if (!plan || !image_host || !out_host) return FR_ERR_INVALID_ARG;
  Engine& E = plan->E;
  JobRes& j = E.jobs[0];
  const size_t img_bytes = (size_t)j.p.nx * j.p.ny * j.p.nz * sizeof(int16_t);
  const size_t out_bytes = (size_t)j.nf * j.n_voi * sizeof(float);
  if (cudaSetDevice(E.device) != cudaSuccess) return FR_ERR_CUDA;
  if (!plan->img_stage) {
    if (cudaMalloc(&plan->img_stage, img_bytes) != cudaSuccess) return FR_ERR_OOM;
    if (cudaMalloc(&plan->out_stage, out_bytes) != cudaSuccess) return FR_ERR_OOM;
    plan->stage_bytes = img_bytes + out_bytes;
  }
  cudaStream_t cs = (cudaStream_t)s;
  if (cudaMemcpyAsync(plan->img_stage, image_host, img_bytes, cudaMemcpyHostToDevice, cs) !=
      cudaSuccess)
    return FR_ERR_CUDA;
  void* ptrs[2] = {(void*)plan->img_stage, (void*)plan->out_stage};
  fr_status st = E.run(ptrs, cs, false);
  if (st != FR_OK) return st;
  if (cudaMemcpyAsync(out_host, plan->out_stage, out_bytes, cudaMemcpyDeviceToHost, cs) !=
      cudaSuccess)
    return FR_ERR_CUDA;
  if (cudaStreamSynchronize(cs) != cudaSuccess) return FR_ERR_CUDA;
  return E.sync_status();
}

fr_status fr_debug_wait_fault(fr_plan* plan, int32_t item, int64_t wait_limit_ns) {
  if (!plan || item < -1 || item >= plan->E.n_items || wait_limit_ns < 0)
    return FR_ERR_INVALID_ARG;
  plan->E.withhold_item = item;
  plan->E.timeout_ns = wait_limit_ns > 0 ? wait_limit_ns : kTimeoutNs;
  return FR_OK;
}

fr_status fr_map_sync_status(fr_plan* plan) {
  if (!plan) return FR_ERR_INVALID_ARG;
  return plan->E.sync_status();
}

fr_status fr_plan_query(const fr_plan* plan, int64_t* n_voi, int32_t* n_rows,
                        size_t* device_bytes) {
  if (!plan) return FR_ERR_INVALID_ARG;
  if (n_voi) *n_voi = plan->E.jobs[0].n_voi;
  if (n_rows) *n_rows = plan->E.jobs[0].nf;
  if (device_bytes) *device_bytes = plan->E.bytes + plan->stage_bytes;
  return FR_OK;
}

fr_status fr_plan_voxel_index(const fr_plan* plan, int32_t* idx, fr_stream_t s) {
  if (!plan || !idx) return FR_ERR_INVALID_ARG;
  const JobRes& j = plan->E.jobs[0];
  if (cudaSetDevice(plan->E.device) != cudaSuccess) return FR_ERR_CUDA;
  return cudaMemcpyAsync(idx, j.voi, j.n_voi * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                         (cudaStream_t)s) == cudaSuccess
             ? FR_OK
             : FR_ERR_CUDA;
}

fr_status fr_plan_levels(fr_plan* plan, uint8_t* levels, int32_t* ng, int32_t* xmin,
                         int32_t* xmax) {
  if (!plan) return FR_ERR_INVALID_ARG;
  Engine& E = plan->E;
  const JobRes& j = E.jobs[0];
  if (cudaSetDevice(E.device) != cudaSuccess) return FR_ERR_CUDA;
  if (E.ran && cudaEventSynchronize(E.done) != cudaSuccess) return FR_ERR_CUDA;
  if (levels) {
    if (fr_launch_levels(j.packed, j.p.nx, j.p.ny * j.p.nz, j.px, levels, 0) != cudaSuccess)
      return FR_ERR_CUDA;
    if (cudaStreamSynchronize(0) != cudaSuccess) return FR_ERR_CUDA;
  }
  FrJobState js;
  if (cudaMemcpy(&js, j.state, sizeof(js), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FR_ERR_CUDA;
  if (ng) *ng = js.ng;
  if (xmin) *xmin = js.xmin;
  if (xmax) *xmax = js.xmax;
  return FR_OK;
}

fr_status fr_scatter_dense(const fr_plan* plan, const float* out, float* dense, fr_stream_t s) {
  if (!plan || !out || !dense) return FR_ERR_INVALID_ARG;
  const JobRes& j = plan->E.jobs[0];
  if (cudaSetDevice(plan->E.device) != cudaSuccess) return FR_ERR_CUDA;
  const int64_t nvox = (int64_t)j.p.nx * j.p.ny * j.p.nz;
  return fr_launch_scatter(j.voi, j.n_voi, j.nf, nvox, out, dense, (cudaStream_t)s) ==
                 cudaSuccess
             ? FR_OK
             : FR_ERR_CUDA;
}

int64_t fr_debug_record_ints(const fr_plan* plan, int32_t ng) {
  if (!plan || ng < 1 || ng > 255) return 0;
  const int s = 2 * plan->E.jobs[0].p.kernel_radius + 1;
  const int64_t w = (int64_t)s * s * s;
  int64_t n = 4 + ng + (int64_t)kNumDirs * ng * ng + (int64_t)kNumDirs * ng * s + ng * w +
              (int64_t)ng * 27 + ng;
  n = (n + 1) & ~1LL;
  return n + 2LL * ng;
}

fr_status fr_debug_matrices(fr_plan* plan, const int16_t* image, const int32_t* cols,
                            int32_t n, int32_t ng, int32_t* rec, fr_stream_t s) {
  if (!plan || !image || !cols || n < 1 || !rec) return FR_ERR_INVALID_ARG;
  Engine& E = plan->E;
  JobRes& j = E.jobs[0];
  for (int i = 0; i < n; ++i)
    if (cols[i] < 0 || cols[i] >= j.n_voi) return FR_ERR_INVALID_ARG;
  const int64_t stride = fr_debug_record_ints(plan, ng);
  if (stride == 0) return FR_ERR_INVALID_ARG;
  cudaStream_t cs = (cudaStream_t)s;
  if (cudaSetDevice(E.device) != cudaSuccess) return FR_ERR_CUDA;
  // discretise this image, then check its level count
  void* ptrs[2] = {(void*)image, nullptr};
  if (cudaMemcpyAsync(E.run_ptrs_dev, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, cs) !=
      cudaSuccess)
    return FR_ERR_CUDA;
  if (fr_launch_prepare(E.jobs_dev, 1, E.max_voi, E.run_ptrs_dev, E.queue, E.status, E.sms,
                        cs) != cudaSuccess)
    return FR_ERR_CUDA;
  FrJobState js;
  if (cudaMemcpyAsync(&js, j.state, sizeof(js), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return FR_ERR_CUDA;
  if (js.status) return (fr_status)js.status;
  if (js.ng != ng) return FR_ERR_MISMATCH;
  // one item per requested column, in a job copy whose column list is cols
  std::vector<int32_t> voi(j.n_voi);
  if (cudaMemcpy(voi.data(), j.voi, j.n_voi * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return FR_ERR_CUDA;
  std::vector<FrItem> items(n);
  for (int i = 0; i < n; ++i) {
    const int lin = voi[cols[i]];
    const int x = lin % j.p.nx, y = (lin / j.p.nx) % j.p.ny, z = lin / (j.p.nx * j.p.ny);
    items[i].job = 0;
    items[i].bx = x / E.tune.brick_x * E.tune.brick_x;
    items[i].by = y / E.tune.brick_y * E.tune.brick_y;
    items[i].bz = z / E.tune.brick_z * E.tune.brick_z;
    items[i].j0 = i;
    items[i].n = 1;
  }
  FrJob hj = E.hjobs[0];
  hj.order = 0;
  FrJob* djob = nullptr;
  FrItem* ditems = nullptr;
  int32_t* dcols = nullptr;
  fr_status st = FR_OK;
  do {
    if (cudaMalloc(&djob, sizeof(FrJob)) != cudaSuccess ||
        cudaMalloc(&ditems, n * sizeof(FrItem)) != cudaSuccess ||
        cudaMalloc(&dcols, n * sizeof(int32_t)) != cudaSuccess) {
      st = FR_ERR_OOM;
      break;
    }
    hj.bcols = dcols;
    if (cudaMemcpyAsync(djob, &hj, sizeof(FrJob), cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaMemcpyAsync(ditems, items.data(), n * sizeof(FrItem), cudaMemcpyHostToDevice, cs) !=
            cudaSuccess ||
        cudaMemcpyAsync(dcols, cols, n * sizeof(int32_t), cudaMemcpyHostToDevice, cs) !=
            cudaSuccess ||
        cudaMemsetAsync(rec, 0, (size_t)n * stride * sizeof(int32_t), cs) != cudaSuccess ||
        cudaMemsetAsync(E.queue, 0, sizeof(uint32_t), cs) != cudaSuccess) {
      st = FR_ERR_CUDA;
      break;
    }
    // the output pointer of the debug run is a scratch buffer
    float* scratch = nullptr;
    if (cudaMalloc(&scratch, (size_t)j.nf * j.n_voi * sizeof(float)) != cudaSuccess) {
      st = FR_ERR_OOM;
      break;
    }
    void* ptrs2[2] = {(void*)image, (void*)scratch};
    FrMapArgs a = E.args(true);
    a.jobs = djob;
    a.items = ditems;
    a.n_items = n;
    a.dbg = rec;
    a.dbg_stride = stride;
    if (cudaMemcpyAsync(E.run_ptrs_dev, ptrs2, sizeof(ptrs2), cudaMemcpyHostToDevice, cs) !=
            cudaSuccess ||
        fr_map_launch(true, a, std::min(E.grid, n), E.smem, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
      st = FR_ERR_CUDA;
    cudaFree(scratch);
  } while (0);
  cudaFree(djob);
  cudaFree(ditems);
  cudaFree(dcols);
  if (st != FR_OK) return st;
  int32_t dst = 0;
  if (cudaMemcpy(&dst, E.status, sizeof(dst), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FR_ERR_CUDA;
  return (fr_status)dst;
}

fr_status fr_plan_last_kernel_ms(fr_plan* plan, float* ms) {
  if (!plan) return FR_ERR_INVALID_ARG;
  return plan->E.kernel_ms(ms);
}

fr_status fr_batch_last_kernel_ms(fr_batch* b, float* ms) {
  if (!b) return FR_ERR_INVALID_ARG;
  return b->E.kernel_ms(ms);
}

void fr_map_destroy(fr_plan* plan) {
  if (!plan) return;
  cudaSetDevice(plan->E.device);
  plan->E.release();
  cudaFree(plan->img_stage);
  cudaFree(plan->out_stage);
  delete plan;
}

fr_status fr_batch_plan(const fr_map_params* params, const uint8_t* const* masks, int32_t n,
                        const fr_tune* tune, fr_batch** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params || !masks || n < 1) return FR_ERR_INVALID_ARG;
  fr_batch* b = new (std::nothrow) fr_batch();
  if (!b) return FR_ERR_OOM;
  fr_status st = engine_open(b->E, params, masks, n, tune);
  if (st != FR_OK) {
    delete b;
    return st;
  }
  *out = b;
  return FR_OK;
}

fr_status fr_batch_query(const fr_batch* b, int32_t i, int64_t* n_voi, int32_t* n_rows) {
  if (!b || i < 0 || i >= (int32_t)b->E.jobs.size()) return FR_ERR_INVALID_ARG;
  if (n_voi) *n_voi = b->E.jobs[i].n_voi;
  if (n_rows) *n_rows = b->E.jobs[i].nf;
  return FR_OK;
}

fr_status fr_batch_run(fr_batch* b, const int16_t* const* images, float* const* outs,
                       fr_stream_t s) {
  if (!b || !images || !outs) return FR_ERR_INVALID_ARG;
  const size_t n = b->E.jobs.size();
  std::vector<void*> ptrs(2 * n);
  for (size_t i = 0; i < n; ++i) {
    if (!images[i] || !outs[i]) return FR_ERR_INVALID_ARG;
    ptrs[2 * i] = (void*)images[i];
    ptrs[2 * i + 1] = (void*)outs[i];
  }
  return b->E.run(ptrs.data(), (cudaStream_t)s, true);
}

fr_status fr_batch_sync_status(fr_batch* b) {
  if (!b) return FR_ERR_INVALID_ARG;
  return b->E.sync_status();
}

void fr_batch_destroy(fr_batch* b) {
  if (!b) return;
  cudaSetDevice(b->E.device);
  b->E.release();
  delete b;
}


fr_status fr_server_create(int32_t device, int32_t max_radius, int32_t max_slots,
                           const fr_tune* tune, fr_server** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_radius < 1 || max_radius > kMaxRadius || max_slots < 1 || max_slots > 4096)
    return FR_ERR_INVALID_ARG;
  fr_server* S = new (std::nothrow) fr_server();
  if (!S) return FR_ERR_OOM;
  // one step maps up to the voxel budget of the continuous batch
  S->tune = default_tune(tune, max_radius, kBigBrickVoxels);
  S->max_radius = max_radius;
  S->max_slots = max_slots;
  S->device = device;
  fr_status st = FR_OK;
  try {
    if (!valid_tune(S->tune)) throw CudaFail{FR_ERR_INVALID_ARG};
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
      throw CudaFail{FR_ERR_UNSUPPORTED};
    FR_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    FR_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3) throw CudaFail{FR_ERR_UNSUPPORTED};
    S->sms = prop.multiProcessorCount;
    S->arena = fr_make_arena(max_radius);
    const int hx = (max_radius + 3) / 4 * 4;
    S->tile_bytes = fr_align((S->tune.brick_x + 2 * hx) * (S->tune.brick_y + 2 * max_radius) *
                                 (S->tune.brick_z + 2 * max_radius) * 4,
                             128);
    S->stages = S->tune.stages;
    S->nw = S->tune.consumer_warps;
    int max_smem = 0;
    FR_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    while (S->nw > 1 && fr_map_smem_bytes(S->stages, S->tile_bytes, S->nw, S->arena.bytes) > max_smem)
      --S->nw;
    S->smem = fr_map_smem_bytes(S->stages, S->tile_bytes, S->nw, S->arena.bytes);
    if (S->smem > max_smem) throw CudaFail{FR_ERR_UNSUPPORTED};
    FR_TRY(fr_map_configure(false, max_smem));
    FR_TRY(fr_map_configure(true, max_smem));
    int blocks = 0;
    FR_TRY(fr_map_occupancy(false, 32 * S->nw, S->smem, &blocks));
    if (blocks < 1) throw CudaFail{FR_ERR_UNSUPPORTED};
    if (S->tune.ctas_per_sm > 0) blocks = std::min(blocks, S->tune.ctas_per_sm);
    S->grid = S->sms * blocks;
    FR_TRY(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
    FR_TRY(cudaStreamCreateWithFlags(&S->plan_stream, cudaStreamNonBlocking));
    // request buffers come from a pool of the server's own: planning and
    // release order their allocations on streams and never wait for the
    // device (cudaMalloc / cudaFree would drain the steps in flight); freed
    // memory stays in the pool for the next requests
    {
      cudaMemPoolProps props;
      memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      FR_TRY(cudaMemPoolCreate(&S->pool, &props));
      uint64_t keep = ~0ull;
      FR_TRY(cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    S->prep_queue = dev_alloc<uint32_t>(1, &S->bytes);
    S->prep_status = dev_alloc<int32_t>(1, &S->bytes);
    S->slab_stride = fr_align(fr_big_layout(S->slab_ngc, S->slab_ngc, S->arena.w_max).bytes, 256);
    S->slab = dev_alloc<char>((size_t)S->grid * S->nw * S->slab_stride, &S->bytes);
    FR_TRY(cudaMemsetAsync(S->slab, 0, (size_t)S->grid * S->nw * S->slab_stride, S->stream));
    S->fb_stride = (int64_t)kNumDirs * kFbDir;
    S->fb = dev_alloc<float>((size_t)S->grid * S->nw * S->fb_stride, &S->bytes);
    S->jobs_dev = dev_alloc<FrJob>(max_slots, &S->bytes);
    S->run_ptrs_dev = dev_alloc<void*>(2 * (size_t)max_slots, &S->bytes);
    S->max_items = 1 << 16;
    S->items_dev[0] = dev_alloc<FrItem>(S->max_items, &S->bytes);
    S->items_dev[1] = dev_alloc<FrItem>(S->max_items, &S->bytes);
    S->queue = dev_alloc<uint32_t>(1, &S->bytes);
    S->status = dev_alloc<int32_t>(1, &S->bytes);
    FR_TRY(cudaMemsetAsync(S->status, 0, sizeof(int32_t), S->stream));
    for (auto& stp : S->steps) FR_TRY(cudaEventCreateWithFlags(&stp.ev, cudaEventDisableTiming));
    S->slots.assign(max_slots, nullptr);
    FR_TRY(cudaStreamSynchronize(S->stream));
  } catch (CudaFail& f) {
    st = f.st;
  }
  if (st != FR_OK) {
    server_release_all(S);
    delete S;
    return st;
  }
  *out = S;
  return FR_OK;
}

fr_status fr_server_add(fr_server* S, const fr_map_params* p, const uint8_t* mask,
                        const int16_t* image, float* out, int64_t* id) {
  if (!S || !p || !mask || !image || !out || !id) return FR_ERR_INVALID_ARG;
  if (!valid_params(p) || p->device != S->device) return FR_ERR_INVALID_ARG;
  if (p->kernel_radius > S->max_radius) return FR_ERR_UNSUPPORTED;
  int slot = -1;
  for (int i = 0; i < S->max_slots; ++i)
    if (!S->slots[i]) {
      slot = i;
      break;
    }
  if (slot < 0) return FR_ERR_UNSUPPORTED;
  if (cudaSetDevice(S->device) != cudaSuccess) return FR_ERR_CUDA;
  ServerReq* r = new (std::nothrow) ServerReq();
  if (!r) return FR_ERR_OOM;
  fr_status st = build_job(p, mask, S->tune, r->job, S->plan_stream, kNumFeatures, S->pool);
  if (st != FR_OK) {
    delete r;
    return st;
  }
  try {
    FrJob h;
    memset((void*)&h, 0, sizeof(FrJob));
    JobRes& j = r->job;
    h.packed = j.packed;
    h.voi = j.voi;
    h.bcols = j.bcols_run;
    h.bcols_brick = j.bcols;
    h.bseg = j.bseg;
    h.nbseg = j.nbseg;
    h.order = 1;
    h.state = j.state;
    h.n_voi = j.n_voi;
    h.nx = j.p.nx;
    h.ny = j.p.ny;
    h.nz = j.p.nz;
    h.px = j.px;
    h.r = j.p.kernel_radius;
    h.delta = j.p.glcm_distance;
    h.agg = j.p.aggregation;
    h.hx = (h.r + 3) / 4 * 4;
    h.box_x = S->tune.brick_x + 2 * h.hx;
    h.box_y = S->tune.brick_y + 2 * h.r;
    h.box_z = S->tune.brick_z + 2 * h.r;
    h.disc_mode = j.p.disc_mode;
    h.bin_count = j.p.bin_count;
    h.anchor_zero_floor = j.p.fbw_anchor == FR_ANCHOR_ZERO_FLOOR;
    h.range_given = j.p.range_given ? 1 : 0;
    h.range_min = j.p.range_min;
    h.range_max = j.p.range_max;
    h.kurt_excess = j.p.kurtosis_excess ? 1 : 0;
    h.nf = j.nf;
    h.families = j.families;
    h.bin_width = j.p.bin_width;
    h.voxel_volume = j.p.spacing[0] * j.p.spacing[1] * j.p.spacing[2];
    memcpy(h.row_of, j.row_of, sizeof(h.row_of));
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) throw CudaFail{FR_ERR_CUDA};
    cuuint64_t gdim[3] = {(cuuint64_t)j.px, (cuuint64_t)j.p.ny, (cuuint64_t)j.p.nz};
    cuuint64_t gstride[2] = {(cuuint64_t)j.px * 4, (cuuint64_t)j.px * j.p.ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)h.box_x, (cuuint32_t)h.box_y, (cuuint32_t)h.box_z};
    cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&h.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, (void*)j.packed, gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      throw CudaFail{FR_ERR_UNSUPPORTED};
    void* ptrs[2] = {(void*)image, (void*)out};
    FR_TRY(cudaMemcpyAsync(S->jobs_dev + slot, &h, sizeof(FrJob), cudaMemcpyHostToDevice,
                           S->plan_stream));
    FR_TRY(cudaMemcpyAsync(S->run_ptrs_dev + 2 * slot, ptrs, sizeof(ptrs),
                           cudaMemcpyHostToDevice, S->plan_stream));
    FR_TRY(cudaStreamSynchronize(S->plan_stream));
  } catch (CudaFail& f) {
    r->job.release();
    delete r;
    return f.st;
  }
  r->slot = slot;
  r->id = S->next_id++;
  r->image = image;
  r->out = out;
  S->slots[slot] = r;
  *id = r->id;
  return FR_OK;
}

fr_status fr_server_step(fr_server* S, int64_t voxel_budget, int32_t* n_active) {
  if (!S || voxel_budget < 1) return FR_ERR_INVALID_ARG;
  if (cudaSetDevice(S->device) != cudaSuccess) return FR_ERR_CUDA;
  ServerStep& st = S->steps[S->next_step];
  fr_status cs = server_complete(S, st, true);
  if (cs != FR_OK) return cs;
  // discretise and pack requests that joined since the last step
  for (ServerReq* r : S->slots) {
    if (!r || r->prepared) continue;
    if (fr_launch_prepare(S->jobs_dev + r->slot, 1, r->job.n_voi, S->run_ptrs_dev + 2 * r->slot,
                          S->prep_queue, S->prep_status, S->sms, S->stream) != cudaSuccess ||
        fr_launch_order(S->jobs_dev + r->slot, 1, r->job.nbseg, S->sms, S->stream) != cudaSuccess)
      return FR_ERR_CUDA;
    r->prepared = true;
  }
  // round-robin share of the voxel budget over the requests with work left
  std::vector<ServerReq*> act;
  for (ServerReq* r : S->slots)
    if (r && r->issued < r->job.items.size()) act.push_back(r);
  if (n_active) *n_active = (int32_t)act.size();
  if (act.empty()) return FR_OK;
  S->host_items.clear();
  st.advance.clear();
  int64_t left = voxel_budget;
  std::vector<size_t> took(act.size(), 0);
  bool progress = true;
  while (left > 0 && progress && (int)S->host_items.size() < S->max_items) {
    progress = false;
    for (size_t k = 0; k < act.size() && left > 0; ++k) {
      ServerReq* r = act[k];
      const size_t at = r->issued + took[k];
      if (at >= r->job.items.size() || (int)S->host_items.size() >= S->max_items) continue;
      FrItem it = r->job.items[at];
      it.job = r->slot;
      S->host_items.push_back(it);
      left -= it.n;
      ++took[k];
      progress = true;
    }
  }
  for (size_t k = 0; k < act.size(); ++k) {
    if (!took[k]) continue;
    act[k]->issued += took[k];
    st.advance.push_back({act[k]->slot, took[k]});
  }
  FrItem* items = S->items_dev[S->next_step];
  if (cudaMemcpyAsync(items, S->host_items.data(), S->host_items.size() * sizeof(FrItem),
                      cudaMemcpyHostToDevice, S->stream) != cudaSuccess ||
      cudaMemsetAsync(S->queue, 0, sizeof(uint32_t), S->stream) != cudaSuccess)
    return FR_ERR_CUDA;
  FrMapArgs a{};
  a.jobs = S->jobs_dev;
  a.run_ptrs = S->run_ptrs_dev;
  a.items = items;
  a.n_items = (int32_t)S->host_items.size();
  a.consumer_warps = S->nw;
  a.stages = S->stages;
  a.tile_bytes = S->tile_bytes;
  a.queue = S->queue;
  a.status = S->status;
  a.slab = S->slab;
  a.slab_stride = S->slab_stride;
  a.slab_ngc = S->slab_ngc;
  a.fb = S->fb;
  a.fb_stride = S->fb_stride;
  a.arena = S->arena;
  a.timeout_ns = kTimeoutNs;
  a.withhold_item = -1;
  const int grid = std::min(S->grid, a.n_items);
  if (fr_map_launch(false, a, grid, S->smem, S->stream) != cudaSuccess) return FR_ERR_CUDA;
  if (cudaEventRecord(st.ev, S->stream) != cudaSuccess) return FR_ERR_CUDA;
  st.busy = true;
  S->next_step ^= 1;
  return FR_OK;
}

fr_status fr_server_poll(fr_server* S, int32_t wait, int64_t* done_ids, int32_t* done_status,
                         int32_t cap, int32_t* n_done) {
  if (!S || !n_done || cap < 0 || (cap > 0 && (!done_ids || !done_status)))
    return FR_ERR_INVALID_ARG;
  if (cudaSetDevice(S->device) != cudaSuccess) return FR_ERR_CUDA;
  *n_done = 0;
  // steps complete in launch order
  for (int k = 0; k < 2; ++k) {
    ServerStep& st = S->steps[(S->next_step + k) & 1];
    fr_status cs = server_complete(S, st, wait != 0);
    if (cs != FR_OK) return cs;
    if (st.busy) break;
  }
  int32_t dev_status = 0;
  bool status_read = false;
  for (ServerReq* r : S->slots) {
    if (!r || r->done || !r->prepared || r->completed < r->job.items.size()) continue;
    if (*n_done >= cap) break;
    if (!status_read) {
      if (cudaMemcpy(&dev_status, S->status, sizeof(dev_status), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
        return FR_ERR_CUDA;
      status_read = true;
    }
    FrJobState js;
    if (cudaMemcpy(&js, r->job.state, sizeof(js), cudaMemcpyDeviceToHost) != cudaSuccess)
      return FR_ERR_CUDA;
    r->done = true;
    done_ids[*n_done] = r->id;
    done_status[*n_done] = js.status ? js.status : dev_status;
    ++*n_done;
  }
  return FR_OK;
}

fr_status fr_server_release(fr_server* S, int64_t id) {
  if (!S) return FR_ERR_INVALID_ARG;
  for (auto*& r : S->slots) {
    if (!r || r->id != id) continue;
    if (!r->done) return FR_ERR_INVALID_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return FR_ERR_CUDA;
    // freed after the work queued on the step stream, without waiting
    r->job.release_async(S->stream);
    delete r;
    r = nullptr;
    return FR_OK;
  }
  return FR_ERR_INVALID_ARG;
}

fr_status fr_server_query(const fr_server* S, int32_t* active, int32_t* inflight,
                          size_t* device_bytes) {
  if (!S) return FR_ERR_INVALID_ARG;
  int32_t a = 0;
  size_t b = S->bytes;
  for (ServerReq* r : S->slots)
    if (r) {
      ++a;
      b += r->job.bytes;
    }
  if (active) *active = a;
  if (inflight) *inflight = (S->steps[0].busy ? 1 : 0) + (S->steps[1].busy ? 1 : 0);
  if (device_bytes) *device_bytes = b;
  return FR_OK;
}

void fr_server_destroy(fr_server* S) {
  if (!S) return;
  cudaSetDevice(S->device);
  server_release_all(S);
  delete S;
}

int32_t fr_feature_count(void) { return kNumFeatures; }

int32_t fr_scalar_feature_count(void) { return kNumScalarFeatures; }

const char* fr_feature_name(int32_t id) {
  return (id >= 0 && id < kNumScalarFeatures) ? kFeatureNames[id] : nullptr;
}

const char* fr_status_string(fr_status s) {
  switch (s) {
    case FR_OK: return "ok";
    case FR_ERR_INVALID_ARG: return "invalid argument";
    case FR_ERR_EMPTY_MASK: return "empty mask";
    case FR_ERR_TOO_MANY_LEVELS: return "more than 255 gray levels";
    case FR_ERR_OOM: return "out of memory";
    case FR_ERR_CUDA: return "CUDA error";
    case FR_ERR_TIMEOUT: return "device wait timed out";
    case FR_ERR_UNSUPPORTED: return "unsupported device or size";
    case FR_ERR_MISMATCH: return "arguments disagree with the plan";
    case FR_ERR_IO: return "file could not be written";
  }
  return "unknown status";
}

fr_status fr_direction(int32_t i, int32_t* dz, int32_t* dy, int32_t* dx) {
  if (i < 0 || i >= kNumDirs || !dz || !dy || !dx) return FR_ERR_INVALID_ARG;
  *dz = kDirs[i][0];
  *dy = kDirs[i][1];
  *dx = kDirs[i][2];
  return FR_OK;
}

fr_status fr_scalar_plan(const fr_map_params* p, const uint8_t* mask, fr_scalar** out) {
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p || !mask) return FR_ERR_INVALID_ARG;
  fr_scalar* S = new (std::nothrow) fr_scalar();
  if (!S) return FR_ERR_OOM;
  fr_status st = scalar_open(*S, p, mask);
  if (st != FR_OK) {
    S->release();
    delete S;
    return st;
  }
  *out = S;
  return FR_OK;
}

fr_status fr_scalar_run(fr_scalar* S, const int16_t* image, double* out, fr_stream_t stream) {
  if (!S || !image || !out) return FR_ERR_INVALID_ARG;
  if (cudaSetDevice(S->device) != cudaSuccess) return FR_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  void* ptrs[2] = {(void*)image, (void*)out};
  if (cudaMemcpyAsync(S->d_run, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FR_ERR_CUDA;
  if (fr_launch_prepare(S->d_job, 1, S->j.n_voi, S->d_run, S->d_queue, S->d_status, S->sms, s) !=
      cudaSuccess)
    return FR_ERR_CUDA;
  if (cudaMemsetAsync(S->scratch, 0, S->zero_bytes, s) != cudaSuccess ||
      cudaMemsetAsync(S->scratch + S->key_off, 0xFF, S->key_bytes, s) != cudaSuccess)
    return FR_ERR_CUDA;
  if (fr_scalar_launch(S->A, out, S->d_row_of, S->sms, s) != cudaSuccess) return FR_ERR_CUDA;
  if (cudaEventRecord(S->done, s) != cudaSuccess) return FR_ERR_CUDA;
  S->ran = true;
  return FR_OK;
}

fr_status fr_scalar_sync_status(fr_scalar* S) {
  if (!S) return FR_ERR_INVALID_ARG;
  if (cudaSetDevice(S->device) != cudaSuccess) return FR_ERR_CUDA;
  if (S->ran && cudaEventSynchronize(S->done) != cudaSuccess) return FR_ERR_CUDA;
  int32_t st = 0;
  if (cudaMemcpy(&st, S->d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FR_ERR_CUDA;
  if (st) return (fr_status)st;
  FrJobState js;
  if (cudaMemcpy(&js, S->j.state, sizeof(js), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FR_ERR_CUDA;
  return (fr_status)js.status;
}

fr_status fr_scalar_query(const fr_scalar* S, int64_t* n_voi, int32_t* n_features,
                          size_t* device_bytes) {
  if (!S) return FR_ERR_INVALID_ARG;
  if (n_voi) *n_voi = S->j.n_voi;
  if (n_features) *n_features = S->j.nf;
  if (device_bytes) *device_bytes = S->bytes + S->j.bytes;
  return FR_OK;
}

void fr_scalar_destroy(fr_scalar* S) {
  if (!S) return;
  cudaSetDevice(S->device);
  S->release();
  delete S;
}

}  // extern "C"
