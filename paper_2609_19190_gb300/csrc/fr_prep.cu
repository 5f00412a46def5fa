// fr_prep.cu -- discretisation and packing (per run) and the VOI list /
// brick schedule (per plan), plus the small export kernels.
//
// Discretisation (IBSI; paper: discretisation is a preprocessing step over
// the whole VOI):
//   FBN: g = floor(Ng (x - xmin) / (xmax - xmin)) + 1, x = xmax -> Ng, and
//        g = 1 when xmax == xmin; exact in 64-bit integers.
//   FBW: g = floor((x - a) / w) + 1 in IEEE double with a = xmin, or
//        a = floor(xmin / w) * w (zero-floor anchor); Ng = floor((xmax - a)
//        / w) + 1.  Explicit round-to-nearest intrinsics keep the compiler
//        from contracting these into FMAs.
// With a given range (a z-slab of one volume discretised as the whole VOI),
// xmin / xmax are the given bounds and each intensity is clamped to them
// before its level is taken; the packed word keeps the raw intensity.
#include <climits>
#include <cstdint>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

constexpr int kStatusTooManyLevels = 3;  // FR_ERR_TOO_MANY_LEVELS

__global__ void fr_reset_kernel(const FrJob* jobs, int njobs, uint32_t* queue,
                                int32_t* status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < njobs) {
    FrJobState* st = jobs[j].state;
    const bool given = jobs[j].range_given != 0;
    st->xmin = given ? jobs[j].range_min : INT_MAX;
    st->xmax = given ? jobs[j].range_max : INT_MIN;
    st->ng = 0;
    st->status = 0;
  }
  if (j == 0) {
    *queue = 0u;
    *status = 0;
  }
}

// VOI intensity range: grid (blocks per job, jobs).
__global__ void fr_minmax_kernel(const FrJob* jobs, void* const* run_ptrs) {
  const FrJob& job = jobs[blockIdx.y];
  if (job.range_given) return;
  const int16_t* img = (const int16_t*)run_ptrs[2 * blockIdx.y];
  int lo = INT_MAX, hi = INT_MIN;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < job.n_voi;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int v = img[job.voi[k]];
    lo = min(lo, v);
    hi = max(hi, v);
  }
  lo = __reduce_min_sync(kFull, lo);
  hi = __reduce_max_sync(kFull, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&job.state->xmin, lo);
    atomicMax(&job.state->xmax, hi);
  }
}

__device__ __forceinline__ double fbw_anchor(const FrJob& job, int xmin) {
  if (!job.anchor_zero_floor) return (double)xmin;
  return __dmul_rn(floor(__ddiv_rn((double)xmin, job.bin_width)), job.bin_width);
}

__device__ __forceinline__ int fr_num_levels(const FrJob& job, int xmin, int xmax) {
  if (job.disc_mode == 0) return job.bin_count;
  const double a = fbw_anchor(job, xmin);
  return (int)floor(__ddiv_rn(__dsub_rn((double)xmax, a), job.bin_width)) + 1;
}

// Levels and packed words: grid (blocks per job, jobs).
__global__ void fr_pack_kernel(const FrJob* jobs, void* const* run_ptrs) {
  const FrJob& job = jobs[blockIdx.y];
  const int16_t* img = (const int16_t*)run_ptrs[2 * blockIdx.y];
  const int xmin = job.state->xmin, xmax = job.state->xmax;
  const int ng = fr_num_levels(job, xmin, xmax);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    job.state->ng = ng;
    if (ng > 255 || ng < 1) job.state->status = kStatusTooManyLevels;
  }
  if (ng > 255 || ng < 1) return;
  const double a = job.disc_mode == 1 ? fbw_anchor(job, xmin) : 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < job.n_voi;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int lin = job.voi[k];
    const int raw = img[lin];
    const int v = job.range_given ? min(max(raw, xmin), xmax) : raw;
    int g;
    if (job.disc_mode == 0) {
      if (xmax == xmin) {
        g = 1;
      } else {
        g = (int)(((long long)ng * (v - xmin)) / (long long)(xmax - xmin)) + 1;
        if (g > ng) g = ng;
      }
    } else {
      g = (int)floor(__ddiv_rn(__dsub_rn((double)v, a), job.bin_width)) + 1;
    }
    const int x = lin % job.nx;
    const int rest = lin / job.nx;  // z * ny + y
    job.packed[(size_t)rest * job.px + x] =
        ((uint32_t)(raw + 32768) << 8) | (uint32_t)g;
  }
}

// ------------------------------------------------------------------ voxel order
// Distinct gray levels in the window of the VOI voxel at linear index lin
// (levels taken mod 64, so the count is exact up to 64 levels), from the
// packed volume (level 0 = outside the VOI).
__device__ int fr_window_levels(const FrJob& job, int lin) {
  const int x = lin % job.nx, y = (lin / job.nx) % job.ny, z = lin / (job.nx * job.ny);
  const int r = job.r;
  const int x0 = max(0, x - r), x1 = min(job.nx - 1, x + r);
  const int y0 = max(0, y - r), y1 = min(job.ny - 1, y + r);
  const int z0 = max(0, z - r), z1 = min(job.nz - 1, z + r);
  unsigned long long set = 0ull;
  for (int zz = z0; zz <= z1; ++zz)
    for (int yy = y0; yy <= y1; ++yy) {
      const uint32_t* row = job.packed + ((size_t)zz * job.ny + yy) * job.px;
      for (int xx = x0; xx <= x1; ++xx) {
        const uint32_t g = row[xx] & 0xFFu;
        if (g) set |= 1ull << ((g - 1u) & 63u);
      }
    }
  return __popcll(set);
}

// Columns of every brick segment of every job, reordered by the window's
// level count (counting sort, one warp per segment): the voxels of one work
// item then cost alike and take the same code paths, so the CTA's warps
// wait less at the family barriers.  The maps do not depend on the order.
// Grid (blocks, jobs); segments longer than kOrderMax keep the plan order.
constexpr int kOrderWarps = 8;
constexpr int kOrderMax = 1024;
__global__ void __launch_bounds__(32 * kOrderWarps) fr_order_kernel(const FrJob* jobs) {
  __shared__ uint8_t s_m[kOrderWarps][kOrderMax];
  __shared__ int s_hist[kOrderWarps][66];
  const FrJob& job = jobs[blockIdx.y];
  if (!job.order || job.state->status != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* out = const_cast<int32_t*>(job.bcols);
  for (int seg = blockIdx.x * kOrderWarps + warp; seg < job.nbseg;
       seg += gridDim.x * kOrderWarps) {
    const int2 sg = job.bseg[seg];
    const int off = sg.x, cnt = sg.y;
    if (cnt > kOrderMax) {
      for (int i = lane; i < cnt; i += 32) out[off + i] = job.bcols_brick[off + i];
      continue;
    }
    for (int b = lane; b < 66; b += 32) s_hist[warp][b] = 0;
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const int m = fr_window_levels(job, job.voi[job.bcols_brick[off + i]]);
      s_m[warp][i] = (uint8_t)m;
      atomicAdd(&s_hist[warp][m + 1], 1);
    }
    __syncwarp();
    if (lane == 0) {  // exclusive starts of the 65 counts
      int acc = 0;
      for (int b = 0; b < 66; ++b) {
        const int c = s_hist[warp][b];
        s_hist[warp][b] = acc;
        acc += c;
      }
    }
    __syncwarp();
    for (int i = lane; i < cnt; i += 32) {
      const int pos = atomicAdd(&s_hist[warp][s_m[warp][i] + 1], 1);
      out[off + pos] = job.bcols_brick[off + i];
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ plan
// Mask voxels per row (z, y): one warp per row.
__global__ void fr_row_count_kernel(const uint8_t* mask, int nx, int rows,
                                    int32_t* rowcnt) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  int c = 0;
  for (int x = lane; x < nx; x += 32) c += mask[(size_t)row * nx + x] != 0;
  c = __reduce_add_sync(kFull, c);
  if (lane == 0) rowcnt[row] = c;
}

// Exclusive prefix sum of n int32 by one CTA of 1024 threads; total -> *tot.
__global__ void fr_scan_kernel(const int32_t* in, int32_t* out, int n,
                               long long* tot) {
  __shared__ int32_t wsum[32];
  __shared__ long long carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + tid;
    const int v = i < n ? in[i] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int ws = wsum[lane];
      int wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += t;
      }
      wsum[lane] = wi - ws;  // exclusive warp offsets
    }
    __syncthreads();
    const long long c = carry;
    if (i < n) out[i] = (int32_t)(c + wsum[wid] + incl - v);
    __syncthreads();
    if (tid == 1023) carry = c + wsum[wid] + incl;
    __syncthreads();
  }
  if (tid == 0) *tot = carry;
}

// VOI list in z-major order: one warp per row.
__global__ void fr_voi_fill_kernel(const uint8_t* mask, int nx, int rows,
                                   const int32_t* rowoff, int32_t* voi) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  int base = rowoff[row];
  for (int x0 = 0; x0 < nx; x0 += 32) {
    const int x = x0 + lane;
    const bool in = x < nx && mask[(size_t)row * nx + x] != 0;
    const unsigned b = __ballot_sync(kFull, in);
    if (in) voi[base + __popc(b & lanemask_lt())] = row * nx + x;
    base += __popc(b);
  }
}

__device__ __forceinline__ int fr_brick_of(int lin, int nx, int ny, int bx, int by,
                                           int bz, int nbx, int nby) {
  const int x = lin % nx, y = (lin / nx) % ny, z = lin / (nx * ny);
  return ((z / bz) * nby + (y / by)) * nbx + (x / bx);
}

__global__ void fr_brick_count_kernel(const int32_t* voi, int64_t n, int nx, int ny,
                                      int bx, int by, int bz, int nbx, int nby,
                                      int32_t* bcount) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&bcount[fr_brick_of(voi[k], nx, ny, bx, by, bz, nbx, nby)], 1);
}

// Columns grouped by brick; within a brick in increasing column order (one
// warp per brick walks its columns).
__global__ void fr_brick_fill_kernel(const int32_t* voi, int64_t n, int nx, int ny,
                                     int bx, int by, int bz, int nbx, int nby,
                                     const int32_t* boff, int32_t* bfill,
                                     int32_t* bcols) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int b = fr_brick_of(voi[k], nx, ny, bx, by, bz, nbx, nby);
    bcols[boff[b] + atomicAdd(&bfill[b], 1)] = (int32_t)k;
  }
}

// ------------------------------------------------------------------ exports
__global__ void fr_scatter_kernel(const int32_t* voi, int64_t n, int nf,
                                  int64_t nvox, const float* out, float* dense) {
  const float nanv = __int_as_float(0x7fc00000);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nf * nvox;
       t += (int64_t)gridDim.x * blockDim.x)
    dense[t] = nanv;
}

__global__ void fr_scatter_vals_kernel(const int32_t* voi, int64_t n, int nf,
                                       int64_t nvox, const float* out, float* dense) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nf * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = t / n, k = t - f * n;
    dense[f * nvox + voi[k]] = out[t];
  }
}

__global__ void fr_levels_kernel(const uint32_t* packed, int nx, int rows, int px,
                                 uint8_t* levels) {
  const int64_t total = (int64_t)rows * nx;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = t / nx, x = t - row * nx;
    levels[t] = (uint8_t)(packed[row * px + x] & 0xffu);
  }
}

// ------------------------------------------------------------------ host launchers
static int fr_grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

cudaError_t fr_launch_prepare(const FrJob* jobs, int njobs, int64_t max_voi,
                              void* const* run_ptrs, uint32_t* queue, int32_t* status,
                              int sms, cudaStream_t s) {
  fr_reset_kernel<<<(njobs + 127) / 128, 128, 0, s>>>(jobs, njobs, queue, status);
  const int per_job = fr_grid_for(max_voi, 256, 4 * sms);
  dim3 grid(per_job, njobs);
  fr_minmax_kernel<<<grid, 256, 0, s>>>(jobs, run_ptrs);
  fr_pack_kernel<<<grid, 256, 0, s>>>(jobs, run_ptrs);
  return cudaGetLastError();
}

cudaError_t fr_launch_order(const FrJob* jobs, int njobs, int max_segments, int sms,
                            cudaStream_t s) {
  if (max_segments < 1) return cudaSuccess;
  const int blocks = fr_grid_for(max_segments, kOrderWarps, 4 * sms);
  fr_order_kernel<<<dim3(blocks, njobs), 32 * kOrderWarps, 0, s>>>(jobs);
  return cudaGetLastError();
}

cudaError_t fr_launch_row_count(const uint8_t* mask, int nx, int rows, int32_t* rowcnt,
                                cudaStream_t s) {
  const int warps_per_block = 8;
  fr_row_count_kernel<<<(rows + warps_per_block - 1) / warps_per_block, 32 * warps_per_block,
                        0, s>>>(mask, nx, rows, rowcnt);
  return cudaGetLastError();
}

cudaError_t fr_launch_scan(const int32_t* in, int32_t* out, int n, long long* tot,
                           cudaStream_t s) {
  fr_scan_kernel<<<1, 1024, 0, s>>>(in, out, n, tot);
  return cudaGetLastError();
}

cudaError_t fr_launch_voi_fill(const uint8_t* mask, int nx, int rows, const int32_t* rowoff,
                               int32_t* voi, cudaStream_t s) {
  const int warps_per_block = 8;
  fr_voi_fill_kernel<<<(rows + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0,
                       s>>>(mask, nx, rows, rowoff, voi);
  return cudaGetLastError();
}

cudaError_t fr_launch_bricks(const int32_t* voi, int64_t n, int nx, int ny, int bx, int by,
                             int bz, int nbx, int nby, int32_t* bcount, cudaStream_t s) {
  fr_brick_count_kernel<<<fr_grid_for(n, 256, 65535), 256, 0, s>>>(voi, n, nx, ny, bx, by, bz,
                                                                    nbx, nby, bcount);
  return cudaGetLastError();
}

cudaError_t fr_launch_brick_fill(const int32_t* voi, int64_t n, int nx, int ny, int bx, int by,
                                 int bz, int nbx, int nby, const int32_t* boff,
                                 int32_t* bfill, int32_t* bcols, cudaStream_t s) {
  fr_brick_fill_kernel<<<fr_grid_for(n, 256, 65535), 256, 0, s>>>(
      voi, n, nx, ny, bx, by, bz, nbx, nby, boff, bfill, bcols);
  return cudaGetLastError();
}

cudaError_t fr_launch_scatter(const int32_t* voi, int64_t n, int nf, int64_t nvox,
                              const float* out, float* dense, cudaStream_t s) {
  fr_scatter_kernel<<<fr_grid_for((int64_t)nf * nvox, 256, 65535), 256, 0, s>>>(
      voi, n, nf, nvox, out, dense);
  fr_scatter_vals_kernel<<<fr_grid_for((int64_t)nf * n, 256, 65535), 256, 0, s>>>(
      voi, n, nf, nvox, out, dense);
  return cudaGetLastError();
}

cudaError_t fr_launch_levels(const uint32_t* packed, int nx, int rows, int px,
                             uint8_t* levels, cudaStream_t s) {
  fr_levels_kernel<<<fr_grid_for((int64_t)rows * nx, 256, 65535), 256, 0, s>>>(
      packed, nx, rows, px, levels);
  return cudaGetLastError();
}

}  // namespace fr
