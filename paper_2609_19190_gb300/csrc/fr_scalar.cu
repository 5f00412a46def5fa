// fr_scalar.cu -- scalar extraction: the 93 features of the whole VOI (the
// paper's other extraction mode, "Software design and extraction modes"; a
// map value equals it wherever the window covers the VOI).
//
// The whole VOI is one region, so the work is a set of grid-wide counts
// instead of per-voxel windows: histograms, co-occurrence and run-length
// counts per direction (privatised in shared memory where they fit), the
// 26-connected zones by a lock-free union-find over the volume, zone (level,
// size) pairs in an open-addressing hash table.  Counts are exact integers;
// the features are then taken in FP64 by a few small kernels (MCC in FP32 by
// the warp eigen-solver of the map path), one block per direction.
#include <cfloat>
#include <climits>
#include <cstdint>

#include "fr_device.cuh"
#include "fr_internal.h"
#include "fr_voxel.cuh"

namespace fr {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kScThreads = 256;
constexpr int kMiscThreads = 1024;
// dynamic shared memory of the neighbourhood kernel:
// ngacc [256][27] u64, gldm [256][27] u32, hlev [256] u32, ngn [256] u32
constexpr int kNeighSmem = 256 * 27 * 8 + 256 * 27 * 4 + 256 * 4 + 256 * 4;

__device__ __forceinline__ bool sc_failed(const FrScalarArgs& a) {
  return *(const volatile int32_t*)&a.state->status != 0;
}

__device__ __forceinline__ void sc_zyx(const FrScalarArgs& a, int lin, int& z, int& y, int& x) {
  x = lin % a.nx;
  const int t = lin / a.nx;
  y = t % a.ny;
  z = t / a.ny;
}

// Gray level at (z, y, x); 0 outside the volume or the VOI.
__device__ __forceinline__ int sc_level(const FrScalarArgs& a, int z, int y, int x) {
  if ((unsigned)z >= (unsigned)a.nz || (unsigned)y >= (unsigned)a.ny ||
      (unsigned)x >= (unsigned)a.nx)
    return 0;
  return (int)(a.packed[((size_t)z * a.ny + y) * a.px + x] & 0xFFu);
}

// Sum over the block of K doubles (fixed order: deterministic).  sh holds
// K * 32 doubles; every thread gets the totals.
template <int K>
__device__ void block_sum(double (&v)[K], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0) sh[k * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k * 32];
  __syncthreads();
}

template <int K>
__device__ void block_sum_u64(unsigned long long (&v)[K], unsigned long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      unsigned long long x = lane < nw ? sh[k * 32 + lane] : 0ull;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
      if (lane == 0) sh[k * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k * 32];
  __syncthreads();
}

// Fixed-point terms for sums whose order of addition varies between runs
// (the zone table's slot order depends on thread timing): x >= 0 times 2^fb,
// truncated to an unsigned 128-bit integer.  Integer sums do not depend on
// the order of addition, so the total is the same on every run.  The caller
// keeps x < 2^(127 - fb).
__device__ __forceinline__ unsigned __int128 sc_fixed(double x, int fb) {
  if (!(x > 0.0)) return 0;
  int e;
  const double m = frexp(x, &e);  // x = m 2^e, 0.5 <= m < 1
  const unsigned long long mi = (unsigned long long)ldexp(m, 53);  // exact
  const int sh = e - 53 + fb;
  if (sh >= 0) return (unsigned __int128)mi << sh;
  if (sh <= -64) return 0;
  return (unsigned __int128)(mi >> (-sh));
}
__device__ __forceinline__ double sc_unfixed(unsigned __int128 v, int fb) {
  const double hi = (double)(unsigned long long)(v >> 64), lo = (double)(unsigned long long)v;
  return ldexp(hi, 64 - fb) + ldexp(lo, -fb);
}

// Block sum of K unsigned 128-bit integers (exact); sh holds K * 32 values.
template <int K>
__device__ void block_sum_u128(unsigned __int128 (&v)[K], unsigned __int128* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  auto shfl = [](unsigned __int128 x, int o) {
    const unsigned long long lo = __shfl_xor_sync(kFull, (unsigned long long)x, o);
    const unsigned long long hi = __shfl_xor_sync(kFull, (unsigned long long)(x >> 64), o);
    return ((unsigned __int128)hi << 64) | lo;
  };
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[k] += shfl(v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      unsigned __int128 x = lane < nw ? sh[k * 32 + lane] : (unsigned __int128)0;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += shfl(x, o);
      if (lane == 0) sh[k * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[k * 32];
  __syncthreads();
}

__device__ __forceinline__ double sc_ent(double p) { return p > 0.0 ? -p * log2(p) : 0.0; }
__device__ __forceinline__ double sc_div(double a, double b) {
  return b == 0.0 ? __longlong_as_double(0x7ff8000000000000ll) : a / b;
}

// ---------------------------------------------------------------- counting

__global__ void sc_init_kernel(const __grid_constant__ FrScalarArgs a) {
  if (sc_failed(a)) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n_voi;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int lin = a.voi[k];
    a.parent[lin] = lin;
  }
}

// Per VOI voxel: raw / level histograms, GLDM dependence (equal 26-neighbours),
// NGTDM n_i and |i k - sum|, and the zone unions with the 13 forward
// neighbours of equal level.
__global__ void __launch_bounds__(kScThreads) sc_neigh_kernel(const __grid_constant__ FrScalarArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned long long* s_acc = (unsigned long long*)sm;  // [256][27]
  uint32_t* s_gldm = (uint32_t*)(s_acc + 256 * 27);    // [256][27]
  uint32_t* s_hlev = s_gldm + 256 * 27;                 // [256]
  uint32_t* s_ngn = s_hlev + 256;                       // [256]
  for (int i = threadIdx.x; i < 256 * 27; i += blockDim.x) {
    s_acc[i] = 0ull;
    s_gldm[i] = 0u;
  }
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_hlev[i] = s_ngn[i] = 0u;
  __syncthreads();
  if (!sc_failed(a)) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n_voi;
         k += (int64_t)gridDim.x * blockDim.x) {
      const int lin = a.voi[k];
      int z, y, x;
      sc_zyx(a, lin, z, y, x);
      const uint32_t w = a.packed[((size_t)z * a.ny + y) * a.px + x];
      const int g = (int)(w & 0xFFu);
      const int raw = (int)(w >> 8) - 32768;
      atomicAdd(&a.hraw[raw + 32768], 1u);
      atomicAdd(&s_hlev[g], 1u);
      int cnt = 0, sum = 0, eq = 0;
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dz && !dy && !dx) continue;
            const int b = sc_level(a, z + dz, y + dy, x + dx);
            if (!b) continue;
            ++cnt;
            sum += b;
            if (b != g) continue;
            ++eq;
            if (dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0))))
              uf_unite(a.parent, lin, ((z + dz) * a.ny + (y + dy)) * a.nx + (x + dx));
          }
      atomicAdd(&s_gldm[g * 27 + eq], 1u);
      if (cnt) {
        atomicAdd(&s_ngn[g], 1u);
        const int dev = g * cnt - sum;
        atomicAdd(&s_acc[g * 27 + cnt], (unsigned long long)(dev < 0 ? -dev : dev));
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256 * 27; i += blockDim.x) {
    if (s_acc[i]) atomicAdd(&a.ngacc[i], s_acc[i]);
    if (s_gldm[i]) atomicAdd(&a.gldm[i], s_gldm[i]);
  }
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    if (s_hlev[i]) atomicAdd(&a.hlev[i], s_hlev[i]);
    if (s_ngn[i]) atomicAdd(&a.ngn[i], s_ngn[i]);
  }
}

// Co-occurrence pairs (u, u + delta d) of direction blockIdx.y, as packed
// upper-triangle counts over levels (a shared-memory copy per block).
__global__ void __launch_bounds__(kScThreads) sc_glcm_kernel(const __grid_constant__ FrScalarArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* s = (uint32_t*)sm;
  const int ngc = a.ngc, np = ngc * (ngc + 1) / 2, d = blockIdx.y;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s[i] = 0u;
  __syncthreads();
  if (!sc_failed(a)) {
    const int oz = c_dirs[d][0] * a.delta, oy = c_dirs[d][1] * a.delta, ox = c_dirs[d][2] * a.delta;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n_voi;
         k += (int64_t)gridDim.x * blockDim.x) {
      int z, y, x;
      sc_zyx(a, a.voi[k], z, y, x);
      const int g = sc_level(a, z, y, x);
      const int b = sc_level(a, z + oz, y + oy, x + ox);
      if (!b) continue;
      atomicAdd(&s[pk(ngc, min(g, b) - 1, max(g, b) - 1)], 1u);
    }
  }
  __syncthreads();
  uint32_t* dst = a.glcm + (size_t)d * np;
  for (int i = threadIdx.x; i < np; i += blockDim.x)
    if (s[i]) atomicAdd(&dst[i], s[i]);
}

// Runs of direction blockIdx.y: a voxel whose predecessor (u - d) is not of
// its level starts a run, measured by walking forward.
__global__ void __launch_bounds__(kScThreads) sc_glrlm_kernel(const __grid_constant__ FrScalarArgs a) {
  if (sc_failed(a)) return;
  const int d = blockIdx.y;
  const int dz = c_dirs[d][0], dy = c_dirs[d][1], dx = c_dirs[d][2];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n_voi;
       k += (int64_t)gridDim.x * blockDim.x) {
    int z, y, x;
    sc_zyx(a, a.voi[k], z, y, x);
    const int g = sc_level(a, z, y, x);
    if (sc_level(a, z - dz, y - dy, x - dx) == g) continue;
    int len = 1, zz = z + dz, yy = y + dy, xx = x + dx;
    while (sc_level(a, zz, yy, xx) == g) {
      ++len;
      zz += dz;
      yy += dy;
      xx += dx;
    }
    atomicAdd(&a.glrlm[((size_t)d * a.ngc + (g - 1)) * a.lmax + (len - 1)], 1u);
  }
}

// Zone size at each root (the unions are complete).
__global__ void sc_flatten_kernel(const __grid_constant__ FrScalarArgs a) {
  if (sc_failed(a)) return;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n_voi;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int r = uf_find((volatile int*)a.parent, a.voi[k]);
    atomicAdd(&a.zsize[r], 1);
  }
}

// 64-bit mix (MurmurHash3's finaliser) for the zone-key table.
__device__ __forceinline__ unsigned long long sc_mix(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// One entry per zone (at its root): zones per level, per size, and per
// (level, size) in the hash table (linear probing; at least half empty).
__global__ void sc_zone_kernel(const __grid_constant__ FrScalarArgs a) {
  if (sc_failed(a)) return;
  const unsigned long long mask = (unsigned long long)a.hcap - 1ull;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < a.n_voi;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int lin = a.voi[k];
    if (a.parent[lin] != lin) continue;
    int z, y, x;
    sc_zyx(a, lin, z, y, x);
    const int g = sc_level(a, z, y, x);
    const int size = a.zsize[lin];
    atomicAdd(&a.zrow[g], 1u);
    atomicAdd(&a.zcol[size], 1u);
    const unsigned long long key = ((unsigned long long)g << 32) | (unsigned)size;
    unsigned long long slot = sc_mix(key) & mask;
    for (int64_t probe = 0; probe < a.hcap; ++probe) {
      const unsigned long long prev = atomicCAS(&a.hkey[slot], kEmptyKey, key);
      if (prev == kEmptyKey || prev == key) {
        atomicAdd(&a.hcnt[slot], 1u);
        break;
      }
      slot = (slot + 1ull) & mask;
    }
  }
}

// ---------------------------------------------------------------- features

// (1 + d) ln(1 + d) - d >= 0 for d >= -1 (the value at -1 is 1).
__device__ __forceinline__ double sc_bregman(double d) {
  if (d <= -1.0) return 1.0;
  if (fabs(d) < 1e-3) return d * d * (0.5 + d * (-1.0 / 6.0 + d * (1.0 / 12.0 + d * (-1.0 / 20.0))));
  return (1.0 + d) * log1p(d) - d;
}

// GLCM features of direction blockIdx.x (or of the merged matrix), written to
// dirf[blockIdx.x][0..23] (and the IBSI sum variance and dissimilarity at
// [40..41]).  Counts C(i, j): n for i != j, 2n on the diagonal.
__global__ void __launch_bounds__(kScThreads) sc_glcm_feat_kernel(const __grid_constant__ FrScalarArgs a) {
  __shared__ unsigned long long s_marg[256];
  __shared__ unsigned long long s_sbin[512];
  __shared__ unsigned long long s_dbin[256];
  __shared__ double s_red[16 * 32];
  __shared__ int s_present;
  const int d = blockIdx.x, tid = threadIdx.x;
  double* f = a.dirf + d * kScalarDirF;
  const double kNaN = __longlong_as_double(0x7ff8000000000000ll);
  if (sc_failed(a)) {
    if (tid < 24) f[tid] = kNaN;
    if (tid < 2) f[40 + tid] = kNaN;
    return;
  }
  const bool merged = a.agg == 1;
  const int ng = a.state->ng, ngc = a.ngc, np = ngc * (ngc + 1) / 2;
  auto cnt = [&](int i, int j) -> unsigned long long {  // pair count, 0-based levels
    const size_t t = (size_t)pk(ngc, min(i, j), max(i, j));
    if (!merged) return a.glcm[(size_t)d * np + t];
    unsigned long long s = 0;
    for (int q = 0; q < kNumDirs; ++q) s += a.glcm[(size_t)q * np + t];
    return s;
  };
  for (int i = tid; i < 512; i += blockDim.x) s_sbin[i] = 0ull;
  for (int i = tid; i < 256; i += blockDim.x) s_dbin[i] = 0ull;
  if (tid == 0) s_present = 0;
  __syncthreads();
  for (int i = tid; i < 256; i += blockDim.x) {
    unsigned long long c = 0;
    if (i < ng)
      for (int j = 0; j < ng; ++j) c += (i == j ? 2ull : 1ull) * cnt(i, j);
    s_marg[i] = c;
    if (c) atomicAdd(&s_present, 1);
  }
  __syncthreads();
  unsigned long long T = 0;
  for (int i = 0; i < ng; ++i) T += s_marg[i];
  if (T == 0) {
    if (tid < 24) f[tid] = kNaN;
    if (tid < 2) f[40 + tid] = kNaN;
    return;
  }
  const double dT = (double)T;
  double mu = 0.0, hx = 0.0;
  for (int i = 0; i < ng; ++i) {
    const double p = (double)s_marg[i] / dT;
    mu += (i + 1) * p;
    hx += sc_ent(p);
  }
  double sig2 = 0.0;
  for (int i = 0; i < ng; ++i) sig2 += ((i + 1) - mu) * ((i + 1) - mu) * ((double)s_marg[i] / dT);
  // entries
  double v[16];
  for (int k = 0; k < 16; ++k) v[k] = 0.0;
  double maxp = 0.0;
  const double ngd = (double)ng;
  for (int t = tid; t < ng * ng; t += blockDim.x) {
    const int i = t / ng, j = t - i * ng;
    const unsigned long long mi = s_marg[i], mj = s_marg[j];
    const unsigned long long C = (i == j ? 2ull : 1ull) * cnt(i, j);
    if (!mi || !mj) continue;
    // mutual information, nats: sum of q g(p / q - 1) >= 0 over all present pairs
    const long long num = (long long)C * (long long)T - (long long)(mi * mj);
    const double q = ((double)mi / dT) * ((double)mj / dT);
    v[15] += q * sc_bregman((double)num / ((double)mi * (double)mj));
    if (!C) continue;
    const double p = (double)C / dT;
    const double I = i + 1, J = j + 1, tt = I + J - 2.0 * mu, dd = fabs(I - J);
    v[0] += I * J * p;                   // autocorrelation
    v[1] += tt * tt * tt * tt * p;       // cluster prominence
    v[2] += tt * tt * tt * p;            // cluster shade
    v[3] += tt * tt * p;                 // cluster tendency
    v[4] += dd * dd * p;                 // contrast
    v[5] += p * p;                       // joint energy
    v[6] += sc_ent(p);                   // joint entropy
    v[7] += p / (1.0 + dd * dd);         // Idm
    v[8] += p / (1.0 + dd * dd / (ngd * ngd));
    v[9] += p / (1.0 + dd);              // Id
    v[10] += p / (1.0 + dd / ngd);       // Idn
    if (i != j) v[11] += p / (dd * dd);  // inverse variance
    v[12] += (I - mu) * (I - mu) * p;    // sum of squares
    maxp = fmax(maxp, p);
    atomicAdd(&s_sbin[i + j + 2], C);
    atomicAdd(&s_dbin[i > j ? i - j : j - i], C);
  }
  block_sum<16>(v, s_red);
  // maximum probability
  {
    double m = maxp;
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = m;
    __syncthreads();
    if (tid == 0) {
      double mm = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, s_red[w]);
      s_red[0] = mm;
    }
    __syncthreads();
    maxp = s_red[0];
    __syncthreads();
  }
  // MCC: spectral radius of S - u u^T over the levels (absent levels: zero rows)
  float* S = a.mcc_s + (size_t)d * ngc * ngc;
  for (int t = tid; t < ng * ng; t += blockDim.x) {
    const int i = t / ng, j = t - i * ng;
    const unsigned long long mi = s_marg[i], mj = s_marg[j];
    float val = 0.f;
    if (mi && mj) {
      const unsigned long long C = (i == j ? 2ull : 1ull) * cnt(i, j);
      const long long num = (long long)C * (long long)T - (long long)(mi * mj);
      val = (float)((double)num / (dT * sqrt((double)mi * (double)mj)));
    }
    S[(size_t)i * ngc + j] = val;
  }
  __syncthreads();
  float mcc = 0.f;
  if (tid < 32 && s_present >= 2) {
    float* vv = a.mcc_v + (size_t)d * 4 * ngc;
    mcc = spectral_radius(S, ng, ngc, vv, vv + ngc, vv + 2 * ngc, vv + 3 * ngc);
  }
  if (tid == 0) {
    double da = 0.0, de = 0.0, sa = 0.0, se = 0.0;
    for (int k = 0; k < ng; ++k) {
      const double p = (double)s_dbin[k] / dT;
      da += k * p;
      de += sc_ent(p);
    }
    double dv = 0.0;
    for (int k = 0; k < ng; ++k) dv += (k - da) * (k - da) * ((double)s_dbin[k] / dT);
    for (int k = 2; k <= 2 * ng; ++k) {
      const double p = (double)s_sbin[k] / dT;
      sa += k * p;
      se += sc_ent(p);
    }
    double sv = 0.0;
    for (int k = 2; k <= 2 * ng; ++k) sv += (k - sa) * (k - sa) * ((double)s_sbin[k] / dT);
    f[40] = sv;
    f[41] = da;
    const double mi_bits = v[15] * 1.4426950408889634;
    f[0] = v[0];
    f[1] = mu;
    f[2] = v[1];
    f[3] = v[2];
    f[4] = v[3];
    f[5] = v[4];
    f[6] = sc_div(v[0] - mu * mu, sig2);
    f[7] = da;
    f[8] = de;
    f[9] = dv;
    f[10] = v[5];
    f[11] = v[6];
    f[12] = sc_div(-mi_bits, hx);
    f[13] = sqrt(fmax(0.0, -expm1(-2.0 * mi_bits)));
    f[14] = v[7];
    f[15] = v[8];
    f[16] = v[9];
    f[17] = v[10];
    f[18] = v[11];
    f[19] = maxp;
    f[20] = sa;
    f[21] = se;
    f[22] = v[12];
    f[23] = s_present >= 2 ? (double)mcc : kNaN;
  }
}

// GLRLM features of direction blockIdx.x (or of the merged matrix), written to
// dirf[blockIdx.x][24..39].
__global__ void __launch_bounds__(kScThreads) sc_glrlm_feat_kernel(const __grid_constant__ FrScalarArgs a) {
  __shared__ double s_red[13 * 32];
  __shared__ unsigned long long s_ured[3 * 32];
  const int d = blockIdx.x, tid = threadIdx.x;
  double* f = a.dirf + d * kScalarDirF + 24;
  const double kNaN = __longlong_as_double(0x7ff8000000000000ll);
  if (sc_failed(a)) {
    if (tid < 16) f[tid] = kNaN;
    return;
  }
  const bool merged = a.agg == 1;
  const int ng = a.state->ng, L = a.lmax;
  auto R = [&](int i, int l) -> unsigned long long {
    if (!merged) return a.glrlm[((size_t)d * a.ngc + i) * L + l];
    unsigned long long s = 0;
    for (int q = 0; q < kNumDirs; ++q) s += a.glrlm[((size_t)q * a.ngc + i) * L + l];
    return s;
  };
  // totals, row and column sums of squares
  unsigned long long u[3] = {0ull, 0ull, 0ull};  // N, sum_i rows^2, sum_l cols^2
  for (int i = tid; i < ng; i += blockDim.x) {
    unsigned long long r = 0;
    for (int l = 0; l < L; ++l) r += R(i, l);
    u[0] += r;
    u[1] += r * r;
  }
  for (int l = tid; l < L; l += blockDim.x) {
    unsigned long long c = 0;
    for (int i = 0; i < ng; ++i) c += R(i, l);
    u[2] += c * c;
  }
  block_sum_u64<3>(u, s_ured);
  if (u[0] == 0) {
    if (tid < 16) f[tid] = kNaN;
    return;
  }
  const double N = (double)u[0];
  double m[2] = {0.0, 0.0};
  for (int t = tid; t < ng * L; t += blockDim.x) {
    const int i = t / L, l = t - i * L;
    const unsigned long long c = R(i, l);
    if (!c) continue;
    m[0] += (i + 1) * (double)c;
    m[1] += (l + 1) * (double)c;
  }
  block_sum<2>(m, s_red);
  const double mui = m[0] / N, muj = m[1] / N;
  double v[11];
  for (int k = 0; k < 11; ++k) v[k] = 0.0;
  for (int t = tid; t < ng * L; t += blockDim.x) {
    const int i = t / L, l = t - i * L;
    const unsigned long long c = R(i, l);
    if (!c) continue;
    const double p = (double)c / N, I = i + 1, J = l + 1;
    v[0] += p / (J * J);
    v[1] += p * J * J;
    v[2] += (I - mui) * (I - mui) * p;
    v[3] += (J - muj) * (J - muj) * p;
    v[4] += sc_ent(p);
    v[5] += p / (I * I);
    v[6] += p * I * I;
    v[7] += p / (I * I * J * J);
    v[8] += p * I * I / (J * J);
    v[9] += p * J * J / (I * I);
    v[10] += p * I * I * J * J;
  }
  block_sum<11>(v, s_red);
  if (tid == 0) {
    const double nv = (double)a.n_voi * (merged ? kNumDirs : 1);
    f[0] = v[0];
    f[1] = v[1];
    f[2] = (double)u[1] / N;
    f[3] = (double)u[1] / (N * N);
    f[4] = (double)u[2] / N;
    f[5] = (double)u[2] / (N * N);
    f[6] = N / nv;
    f[7] = v[2];
    f[8] = v[3];
    f[9] = v[4];
    f[10] = v[5];
    f[11] = v[6];
    f[12] = v[7];
    f[13] = v[8];
    f[14] = v[9];
    f[15] = v[10];
  }
}

// First order (block 0), GLSZM (block 1), GLDM and NGTDM (block 2), written
// to out[0..17], out[58..92] and their extras out[93..95], out[98..100].
__global__ void __launch_bounds__(kMiscThreads) sc_misc_feat_kernel(const __grid_constant__ FrScalarArgs a) {
  __shared__ double s_red[12 * 32];
  __shared__ unsigned long long s_ured[4 * 32];
  __shared__ unsigned __int128 s_qred[11 * 32];
  __shared__ unsigned long long s_base[kMiscThreads];
  __shared__ int s_val[10];
  __shared__ int s_mm[2];
  __shared__ double s_si[256];
  const int tid = threadIdx.x;
  const double kNaN = __longlong_as_double(0x7ff8000000000000ll);
  double* out = a.out;
  if (sc_failed(a)) {
    if (blockIdx.x == 0 && tid < 18) out[tid] = kNaN;
    if (blockIdx.x == 0 && tid < 3) out[kFirstExtra + tid] = kNaN;
    if (blockIdx.x == 0 && tid == 0) out[kScalarStd] = kNaN;
    if (blockIdx.x == 1 && tid < 16) out[58 + tid] = kNaN;
    if (blockIdx.x == 2 && tid < 19) out[74 + tid] = kNaN;
    if (blockIdx.x == 2 && tid < 3) out[kGldmExtra + tid] = kNaN;
    return;
  }
  const int ng = a.state->ng;
  if (blockIdx.x == 0) {
    // ---- first order from the raw histogram: each thread 64 bins
    constexpr int kPer = 65536 / kMiscThreads;
    const int b0 = tid * kPer;
    unsigned long long u[3] = {0ull, 0ull, 0ull};  // N, sum x (offset), sum x^2
    long long s1 = 0;
    int lo = INT_MAX, hi = INT_MIN;
    for (int b = b0; b < b0 + kPer; ++b) {
      const unsigned c = a.hraw[b];
      if (!c) continue;
      const long long xv = b - 32768;
      u[0] += c;
      s1 += (long long)c * xv;
      u[2] += (unsigned long long)c * (unsigned long long)(xv * xv);
      lo = min(lo, (int)xv);
      hi = max(hi, (int)xv);
    }
    s_base[tid] = u[0];
    u[1] = (unsigned long long)s1;  // two's complement sums add exactly
    if (tid < 2) s_mm[tid] = tid == 0 ? INT_MAX : INT_MIN;
    __syncthreads();
    atomicMin(&s_mm[0], lo);
    atomicMax(&s_mm[1], hi);
    block_sum_u64<3>(u, s_ured);  // contains __syncthreads
    const unsigned long long n = u[0];
    const long long S1 = (long long)u[1];
    const unsigned long long S2 = u[2];
    // exclusive prefix of the per-thread counts (one thread; 1024 values)
    if (tid == 0) {
      unsigned long long run = 0;
      for (int t = 0; t < kMiscThreads; ++t) {
        const unsigned long long c = s_base[t];
        s_base[t] = run;
        run += c;
      }
    }
    __syncthreads();
    // order statistics at the ranks of P10, P25, P50, P75, P90 (k and k + 1)
    const int qs[5] = {10, 25, 50, 75, 90};
    {
      const unsigned long long base = s_base[tid];
      unsigned long long run = base;
      int r = 0;
      for (int b = b0; b < b0 + kPer; ++b) {
        const unsigned c = a.hraw[b];
        if (!c) continue;
        for (r = 0; r < 10; ++r) {
          const unsigned long long num = (n - 1) * (unsigned long long)qs[r >> 1];
          unsigned long long k = num / 100 + (r & 1);
          if (k > n - 1) k = n - 1;
          if (k >= run && k < run + c) s_val[r] = b - 32768;
        }
        run += c;
      }
    }
    __syncthreads();
    const double N = (double)n, mean = (double)S1 / N;
    auto pct = [&](int qi) -> double {
      const unsigned long long num = (n - 1) * (unsigned long long)qs[qi];
      const long long rem = (long long)(num % 100);
      const int xk = s_val[2 * qi], xk1 = s_val[2 * qi + 1];
      if (rem == 0) return (double)xk;
      return xk + (rem / 100.0) * (double)(xk1 - xk);
    };
    // 100 * P_q exactly, for the robust subset P10 <= x <= P90
    auto pct100 = [&](int qi) -> long long {
      const unsigned long long num = (n - 1) * (unsigned long long)qs[qi];
      const long long rem = (long long)(num % 100);
      const long long xk = s_val[2 * qi], xk1 = s_val[2 * qi + 1];
      return 100 * xk + (rem ? rem * (xk1 - xk) : 0);
    };
    const long long r10 = pct100(0), r90 = pct100(4);
    const double med = pct(2);
    double m[7] = {0, 0, 0, 0, 0, 0, 0};  // m2 m3 m4 mad, robust count, robust sum, |x - median|
    for (int b = b0; b < b0 + kPer; ++b) {
      const unsigned c = a.hraw[b];
      if (!c) continue;
      const double xv = b - 32768, dv = xv - mean, dc = (double)c;
      m[0] += dc * dv * dv;
      m[1] += dc * dv * dv * dv;
      m[2] += dc * dv * dv * dv * dv;
      m[3] += dc * fabs(dv);
      m[6] += dc * fabs(xv - med);
      const long long x100 = 100ll * (b - 32768);
      if (x100 >= r10 && x100 <= r90) {
        m[4] += dc;
        m[5] += dc * xv;
      }
    }
    block_sum<7>(m, s_red);
    const double rmean = m[5] / m[4];
    double rm[1] = {0.0};
    for (int b = b0; b < b0 + kPer; ++b) {
      const unsigned c = a.hraw[b];
      if (!c) continue;
      const long long x100 = 100ll * (b - 32768);
      if (x100 >= r10 && x100 <= r90) rm[0] += (double)c * fabs((b - 32768) - rmean);
    }
    block_sum<1>(rm, s_red);
    // discretised entropy and uniformity
    double e[2] = {0.0, 0.0};
    for (int g = tid + 1; g <= ng; g += blockDim.x) {
      const double p = (double)a.hlev[g] / N;
      e[0] += sc_ent(p);
      e[1] += p * p;
    }
    block_sum<2>(e, s_red);
    if (tid == 0) {
      const double m2 = m[0] / N, m3 = m[1] / N, m4 = m[2] / N;
      out[0] = (double)S2;
      out[1] = a.voxel_volume * (double)S2;
      out[2] = e[0];
      out[3] = (double)s_mm[0];
      out[4] = pct(0);
      out[5] = pct(4);
      out[6] = (double)s_mm[1];
      out[7] = mean;
      out[8] = pct(2);
      out[9] = pct(3) - pct(1);
      out[10] = (double)s_mm[1] - (double)s_mm[0];
      out[11] = m[3] / N;
      out[12] = rm[0] / m[4];
      out[13] = sqrt((double)S2 / N);
      out[14] = m2 == 0.0 ? kNaN : m3 / pow(m2, 1.5);
      out[15] = m2 == 0.0 ? kNaN : m4 / (m2 * m2) - (a.kurt_excess ? 3.0 : 0.0);
      out[16] = m2;
      out[17] = e[1];
      // IBSI extras: median absolute deviation, coefficient of variation,
      // quartile coefficient of dispersion
      const double p25 = pct(1), p75 = pct(3);
      out[kFirstExtra] = m[6] / N;
      out[kFirstExtra + 1] = sc_div(sqrt(m2), mean);
      out[kFirstExtra + 2] = sc_div(p75 - p25, p75 + p25);
      // standard deviation (population), the scalar-only statistic
      out[kScalarStd] = sqrt(m2);
    }
  } else if (blockIdx.x == 1) {
    // ---- GLSZM from zones per level, per size and per (level, size)
    unsigned long long u[3] = {0ull, 0ull, 0ull};  // N zones, sum rows^2, sum cols^2
    for (int g = tid + 1; g <= ng; g += blockDim.x) {
      const unsigned long long r = a.zrow[g];
      u[0] += r;
      u[1] += r * r;
    }
    double m[2] = {0.0, 0.0};
    for (int64_t j = tid + 1; j <= a.n_voi; j += blockDim.x) {
      const unsigned long long c = a.zcol[j];
      u[2] += c * c;
      m[1] += (double)j * (double)c;
    }
    for (int g = tid + 1; g <= ng; g += blockDim.x) m[0] += (double)g * (double)a.zrow[g];
    block_sum_u64<3>(u, s_ured);
    block_sum<2>(m, s_red);
    const double N = (double)u[0];
    const double mui = m[0] / N, muj = m[1] / N;
    // every (level, size) cell's terms, summed in fixed point so that the
    // slot order of the zone table does not change the result.  Bits after
    // the point per sum, from its bound (I <= 255, J < 2^31, sum p = 1):
    // <= 1 -> 120; <= 255^2 -> 110; <= 2^62 -> 64; <= 2^78 -> 48.
    constexpr int kFb[11] = {120, 64, 110, 64, 120, 120, 110, 120, 110, 64, 48};
    unsigned __int128 q[11];
    for (int k = 0; k < 11; ++k) q[k] = 0;
    for (int64_t t = tid; t < a.hcap; t += blockDim.x) {
      const unsigned long long key = a.hkey[t];
      if (key == kEmptyKey) continue;
      const double I = (double)(key >> 32), J = (double)(key & 0xffffffffull);
      const double p = (double)a.hcnt[t] / N;
      const double tv[11] = {p / (J * J),          p * J * J,          (I - mui) * (I - mui) * p,
                             (J - muj) * (J - muj) * p, sc_ent(p),     p / (I * I),
                             p * I * I,            p / (I * I * J * J), p * I * I / (J * J),
                             p * J * J / (I * I),  p * I * I * J * J};
#pragma unroll
      for (int k = 0; k < 11; ++k) q[k] += sc_fixed(tv[k], kFb[k]);
    }
    block_sum_u128<11>(q, s_qred);
    double v[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) v[k] = sc_unfixed(q[k], kFb[k]);
    if (tid == 0) {
      double* f = out + 58;
      if (u[0] == 0) {
        for (int k = 0; k < 16; ++k) f[k] = kNaN;
      } else {
        f[0] = v[0];
        f[1] = v[1];
        f[2] = (double)u[1] / N;
        f[3] = (double)u[1] / (N * N);
        f[4] = (double)u[2] / N;
        f[5] = (double)u[2] / (N * N);
        f[6] = N / (double)a.n_voi;
        f[7] = v[2];
        f[8] = v[3];
        f[9] = v[4];
        f[10] = v[5];
        f[11] = v[6];
        f[12] = v[7];
        f[13] = v[8];
        f[14] = v[9];
        f[15] = v[10];
      }
    }
  } else {
    // ---- GLDM from [level][equal neighbours] counts
    // N, sum rows^2, sum cols^2, sum of squared cells
    unsigned long long u[4] = {0ull, 0ull, 0ull, 0ull};
    for (int g = tid + 1; g <= ng; g += blockDim.x) {
      unsigned long long r = 0;
      for (int j = 0; j < 27; ++j) {
        const unsigned long long c = a.gldm[g * 27 + j];
        r += c;
        u[3] += c * c;
      }
      u[0] += r;
      u[1] += r * r;
    }
    if (tid < 27) {
      unsigned long long c = 0;
      for (int g = 1; g <= ng; ++g) c += a.gldm[g * 27 + tid];
      u[2] += c * c;
    }
    block_sum_u64<4>(u, s_ured);
    const double N = (double)u[0];
    double m[2] = {0.0, 0.0};
    for (int t = tid; t < ng * 27; t += blockDim.x) {
      const int g = t / 27 + 1, j = t % 27;
      const double c = (double)a.gldm[g * 27 + j];
      m[0] += g * c;
      m[1] += (j + 1) * c;
    }
    block_sum<2>(m, s_red);
    const double mui = m[0] / N, muj = m[1] / N;
    double v[11];
    for (int k = 0; k < 11; ++k) v[k] = 0.0;
    for (int t = tid; t < ng * 27; t += blockDim.x) {
      const int g = t / 27 + 1, j = t % 27;
      const unsigned c = a.gldm[g * 27 + j];
      if (!c) continue;
      const double p = (double)c / N, I = g, J = j + 1;
      v[0] += p / (J * J);
      v[1] += p * J * J;
      v[2] += (I - mui) * (I - mui) * p;
      v[3] += (J - muj) * (J - muj) * p;
      v[4] += sc_ent(p);
      v[5] += p / (I * I);
      v[6] += p * I * I;
      v[7] += p / (I * I * J * J);
      v[8] += p * I * I / (J * J);
      v[9] += p * J * J / (I * I);
      v[10] += p * I * I * J * J;
    }
    block_sum<11>(v, s_red);
    // ---- NGTDM: n_i, s_i = sum_k acc[i][k] / k
    double w[4] = {0, 0, 0, 0};  // Nvp, sum n_i s_i, sum s_i, levels present
    for (int g = tid; g < 256; g += blockDim.x) {
      double si = 0.0;
      if (g >= 1 && g <= ng)
        for (int k = 1; k <= 26; ++k) si += (double)a.ngacc[g * 27 + k] / (double)k;
      s_si[g] = si;
    }
    __syncthreads();
    for (int g = tid + 1; g <= ng; g += blockDim.x) {
      const double ni = (double)a.ngn[g], si = s_si[g];
      w[0] += ni;
      w[1] += ni * si;
      w[2] += si;
      w[3] += ni > 0.0 ? 1.0 : 0.0;
    }
    block_sum<4>(w, s_red);
    const double Nvp = w[0], sum_ps = w[1] / Nvp, sum_s = w[2], ngp = w[3];
    double x[4] = {0.0, 0.0, 0.0, 0.0};  // c1, busy den, complexity, strength
    for (int t = tid; t < ng * ng; t += blockDim.x) {
      const int i = t / ng + 1, j = t % ng + 1;
      const double ni = (double)a.ngn[i], nj = (double)a.ngn[j];
      if (ni == 0.0 || nj == 0.0) continue;
      const double si = s_si[i], sj = s_si[j];
      const double pi = ni / Nvp, pj = nj / Nvp, dd = (double)(i - j);
      x[0] += pi * pj * dd * dd;
      x[1] += fabs((double)i * ni - (double)j * nj) / Nvp;
      x[2] += fabs(dd) * (pi * si + pj * sj) / (pi + pj);
      x[3] += (pi + pj) * dd * dd;
    }
    block_sum<4>(x, s_red);
    if (tid == 0) {
      double* f = out + 74;
      if (u[0] == 0) {
        for (int k = 0; k < 14; ++k) f[k] = kNaN;
      } else {
        f[0] = v[0];
        f[1] = v[1];
        f[2] = (double)u[1] / N;
        f[3] = (double)u[2] / N;
        f[4] = (double)u[2] / (N * N);
        f[5] = v[2];
        f[6] = v[3];
        f[7] = v[4];
        f[8] = v[5];
        f[9] = v[6];
        f[10] = v[7];
        f[11] = v[8];
        f[12] = v[9];
        f[13] = v[10];
      }
      // IBSI extras: normalised gray level non-uniformity, dependence count
      // percentage, dependence count energy
      double* e = out + kGldmExtra;
      if (u[0] == 0) {
        for (int k = 0; k < 3; ++k) e[k] = kNaN;
      } else {
        e[0] = (double)u[1] / (N * N);
        e[1] = N / (double)a.n_voi;
        e[2] = (double)u[3] / (N * N);
      }
      double* h = out + 88;
      if (Nvp == 0.0) {
        for (int k = 0; k < 5; ++k) h[k] = kNaN;
      } else {
        h[0] = sc_div(1.0, sum_ps);
        h[1] = ngp == 1.0 ? 0.0 : (x[0] / (ngp * (ngp - 1.0))) * (sum_s / Nvp);
        h[2] = sc_div(sum_ps, x[1]);
        h[3] = x[2] / Nvp;
        h[4] = sc_div(x[3], sum_s);
      }
    }
  }
}

// Direction averages (NaN skipped), then the selected features in id order.
__global__ void sc_final_kernel(const __grid_constant__ FrScalarArgs a, double* user_out,
                                const int16_t* __restrict__ row_of_dev) {
  const double kNaN = __longlong_as_double(0x7ff8000000000000ll);
  const int ndir = a.agg == 1 ? 1 : kNumDirs;
  const bool bad = sc_failed(a);
  for (int k = threadIdx.x; k < kScalarDirF; k += blockDim.x) {
    double s = 0.0;
    int c = 0;
    for (int d = 0; d < ndir; ++d) {
      const double v = a.dirf[d * kScalarDirF + k];
      if (isnan(v)) continue;
      s += v;
      ++c;
    }
    a.out[k < 24 ? 18 + k : k < 40 ? 42 + (k - 24) : kGlcmExtra + (k - 40)] = c ? s / c : kNaN;
  }
  __syncthreads();
  for (int f = threadIdx.x; f < kNumScalarFeatures; f += blockDim.x) {
    const int row = row_of_dev[f];
    if (row >= 0) user_out[row] = bad ? kNaN : a.out[f];
  }
}

// ---------------------------------------------------------------- host side

static int sc_grid(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

cudaError_t fr_scalar_configure(int ngc) {
  cudaError_t e = cudaFuncSetAttribute(sc_neigh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kNeighSmem);
  if (e != cudaSuccess) return e;
  const int np = ngc * (ngc + 1) / 2;
  return cudaFuncSetAttribute(sc_glcm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              np * 4);
}

// Every kernel of one scalar extraction, after discretisation and the
// zeroing of the count buffers.  8 launches + 2 per-direction grids.
cudaError_t fr_scalar_launch(const FrScalarArgs& a, double* user_out, const int16_t* row_of_dev,
                             int sms, cudaStream_t s) {
  const int grid = sc_grid(a.n_voi, kScThreads, 8 * sms);
  sc_init_kernel<<<grid, kScThreads, 0, s>>>(a);
  sc_neigh_kernel<<<grid, kScThreads, kNeighSmem, s>>>(a);
  const int gx = sc_grid(a.n_voi, kScThreads * 16, (2 * sms + kNumDirs - 1) / kNumDirs);
  const int np = a.ngc * (a.ngc + 1) / 2;
  sc_glcm_kernel<<<dim3(gx, kNumDirs), kScThreads, np * 4, s>>>(a);
  sc_glrlm_kernel<<<dim3(sc_grid(a.n_voi, kScThreads, (8 * sms) / kNumDirs + 1), kNumDirs),
                    kScThreads, 0, s>>>(a);
  sc_flatten_kernel<<<grid, kScThreads, 0, s>>>(a);
  sc_zone_kernel<<<grid, kScThreads, 0, s>>>(a);
  const int ndir = a.agg == 1 ? 1 : kNumDirs;
  sc_glcm_feat_kernel<<<ndir, kScThreads, 0, s>>>(a);
  sc_glrlm_feat_kernel<<<ndir, kScThreads, 0, s>>>(a);
  sc_misc_feat_kernel<<<3, kMiscThreads, 0, s>>>(a);
  sc_final_kernel<<<1, 128, 0, s>>>(a, user_out, row_of_dev);
  return cudaGetLastError();
}

}  // namespace fr
