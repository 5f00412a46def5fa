// fr_voxel.cuh -- one warp maps one voxel: window gather, first-order
// statistics, and the GLCM / GLRLM / GLSZM / GLDM / NGTDM matrices and
// features of the sub-VOI V(v) = window(v) n VOI.
//
// Definitions (paper: spatial mapping evaluates each feature on the
// neighbourhood of every VOI voxel; Table 2 lists the 93 features; the
// backends follow the IBSI definitions):
//   - window: cube of side s = 2r+1 around v (Chebyshev radius r), clipped
//     to the image; positions outside the VOI carry level 0.
//   - GLCM: 13 directions d, symmetric counts of pairs (u, u + delta*d),
//     features per direction, mean over directions with pairs.
//   - GLRLM: maximal equal-level runs inside V(v) along each direction,
//     features per direction, mean over directions.
//   - GLSZM: 26-connected equal-level zones inside V(v).
//   - GLDM: alpha = 0, distance 1; dependence j = 1 + equal neighbours.
//   - NGTDM: 26-neighbourhood inside V(v), voxels without a neighbour skipped.
//
// Numerics: every matrix count is an exact integer; every numerator that
// can cancel (variances, correlation, cluster shade, skewness, kurtosis) is
// an exact 32-, 64- or 128-bit integer; sums of nonnegative terms
// (emphases, entropies as (c/N) log2(N/c)) accumulate in fp32; the final
// ratios round once in fp32.
//
// Latency: a warp works on one voxel at a time, so the code avoids long
// dependent chains -- integer sums use the single-instruction warp
// reduction, float sums are reduced together, equal matrix keys are merged
// with __match_any_sync before their shared-memory atomic, every
// per-direction feature is finished by its own lane with one division, and
// the 13 GLCM MCC eigenproblems of a voxel are solved concurrently, one lane
// per direction.
#pragma once

#include <cstdint>
#include <type_traits>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

// (dz, dy, dx) of the 13 directions: the vectors of {-1,0,1}^3 that are
// lexicographically greater than (0,0,0), in increasing order.
#define FR_DIRECTIONS                                                   \
  {{0, 0, 1},  {0, 1, -1}, {0, 1, 0},  {0, 1, 1},  {1, -1, -1},          \
   {1, -1, 0}, {1, -1, 1}, {1, 0, -1}, {1, 0, 0},  {1, 0, 1},            \
   {1, 1, -1}, {1, 1, 0},  {1, 1, 1}}
__constant__ signed char c_dirs[13][3] = FR_DIRECTIONS;
constexpr signed char kDirs[13][3] = FR_DIRECTIONS;

// The same table as 6-bit codes (each component + 1 in two bits), so that
// lanes working on different directions decode theirs from registers.
constexpr unsigned long long dir_codes(int lo, int hi) {
  unsigned long long c = 0;
  for (int d = hi - 1; d >= lo; --d)
    c = (c << 6) | (unsigned long long)((kDirs[d][0] + 1) | ((kDirs[d][1] + 1) << 2) |
                                        ((kDirs[d][2] + 1) << 4));
  return c;
}
constexpr unsigned long long kDirCodesLo = dir_codes(0, 10), kDirCodesHi = dir_codes(10, 13);

__device__ __forceinline__ void dir_of(int di, int& dz, int& dy, int& dx) {
  const unsigned c =
      (unsigned)((di < 10 ? kDirCodesLo >> (6 * di) : kDirCodesHi >> (6 * (di - 10))) & 63ull);
  dz = (int)(c & 3u) - 1;
  dy = (int)((c >> 2) & 3u) - 1;
  dx = (int)((c >> 4) & 3u) - 1;
}

// L / w for w = 0..26 with L = lcm(1..26): s_i * L is then an exact
// integer sum of |i*w - S| * (L / w).
struct LdivTable {
  long long v[27];
};
constexpr long long ct_gcd(long long a, long long b) {
  return b == 0 ? a : ct_gcd(b, a % b);
}
constexpr long long ct_lcm_upto(int n) {
  long long l = 1;
  for (int k = 2; k <= n; ++k) l = l / ct_gcd(l, k) * k;
  return l;
}
constexpr long long kLcm26 = ct_lcm_upto(26);
constexpr LdivTable make_ldiv() {
  LdivTable t{};
  t.v[0] = 0;
  for (int w = 1; w <= 26; ++w) t.v[w] = kLcm26 / w;
  return t;
}
__constant__ LdivTable c_ldiv = make_ldiv();

constexpr float kNaNf = __builtin_nanf("");

// Per-voxel window geometry and level summary (warp-uniform).
struct Win {
  int r, s, s2, W;
  Magic ms, ms2;
  int nv;    // voxels in V(v)
  int m;     // distinct levels present
  int lev0;  // smallest present level
  int R;     // largest - smallest present level
  int ng;    // levels of the discretisation
  long long u2;  // sum of squared level counts
};

// Per-warp pointers.
struct Arena {
  uint32_t* kb;
  uint8_t* lvl;
  uint8_t* lut;
  uint8_t* lev;
  uint16_t* st;  // run starts of the sorted keys
  float* fv;
  float* facc;
  float* fcomp;  // rounding error of each facc sum (compensated summation)
  int* nacc;
  float* tmp;
  char* big;  // the selected big region
  int mc, bc;
  BigLayout L;
};

__device__ __forceinline__ void pos_to_zyx(const Win& w, int p, int& z, int& y,
                                           int& x) {
  z = (int)w.ms2.div((unsigned)p);
  int rem = p - z * w.s2;
  y = (int)w.ms.div((unsigned)rem);
  x = rem - y * w.s;
}

__device__ __forceinline__ bool in_cube(const Win& w, int z, int y, int x) {
  return (unsigned)z < (unsigned)w.s && (unsigned)y < (unsigned)w.s &&
         (unsigned)x < (unsigned)w.s;
}

// ------------------------------------------------------------------ reductions
// K float sums reduced together (independent butterflies interleave).
template <int K>
__device__ __forceinline__ void warp_sum_f32x(float (&v)[K]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(kFull, v[k], o);
  }
}

__device__ __forceinline__ unsigned redux_u32(unsigned v) {
  return __reduce_add_sync(kFull, v);
}

// Exact warp sum of nonnegative 64-bit values whose total is below 2^64:
// four single-instruction reductions of 16-bit limbs.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  const unsigned l0 = __reduce_add_sync(kFull, (unsigned)(v & 0xffffu));
  const unsigned l1 = __reduce_add_sync(kFull, (unsigned)((v >> 16) & 0xffffu));
  const unsigned l2 = __reduce_add_sync(kFull, (unsigned)((v >> 32) & 0xffffu));
  const unsigned l3 = __reduce_add_sync(kFull, (unsigned)(v >> 48));
  return (unsigned long long)l0 + ((unsigned long long)l1 << 16) +
         ((unsigned long long)l2 << 32) + ((unsigned long long)l3 << 48);
}

// 64-bit integers to float from two 32-bit conversions (these stay off the
// FP64 pipe, which 64-bit conversions use; at most one extra rounding)
__device__ __forceinline__ float u64_to_f32(unsigned long long x) {
  return fmaf((float)(unsigned)(x >> 32), 4294967296.f, (float)(unsigned)x);
}
__device__ __forceinline__ float s64_to_f32(long long x) {  // |x| < 2^63
  return x < 0 ? -u64_to_f32((unsigned long long)(-x)) : u64_to_f32((unsigned long long)x);
}

__device__ __forceinline__ float i128_to_f32(__int128 v) {
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const float f = fmaf(u64_to_f32((unsigned long long)(u >> 64)), 18446744073709551616.0f,
                       u64_to_f32((unsigned long long)u));
  return neg ? -f : f;
}

// One quotient per lane; a zero denominator gives NaN.
__device__ __forceinline__ float lane_quot(float num, float den) {
  return den == 0.f ? kNaNf : __fdividef(num, den);
}

// ------------------------------------------------------------------ float pairs
// A float pair hi + lo carries about 48 significant bits in fp32 arithmetic
// (GB300's FP64 issues at a small fraction of its fp32 rate).
// f integer-valued (any float of magnitude >= 2^24 is) -> int128, exactly.
__device__ __forceinline__ __int128 f32_to_i128(float f) {
  const unsigned u = __float_as_uint(f);
  const int be = (int)((u >> 23) & 0xFFu);
  if (be == 0) return 0;
  const unsigned mant = (u & 0x7FFFFFu) | 0x800000u;
  const int e = be - 150;  // f = mant * 2^e
  const __int128 v = e >= 0 ? ((__int128)mant << e) : (__int128)(mant >> (-e));
  return (u >> 31) ? -v : v;
}
// x = hi + lo: hi the nearest float, lo the float nearest the exact rest
__device__ __forceinline__ float2 i128_to_ff(__int128 x) {
  const float hi = i128_to_f32(x);
  return make_float2(hi, i128_to_f32(x - f32_to_i128(hi)));
}
// x / t^4 for an integer 1 <= t < 4096: t^4 = dh + dl exactly; q = RN(x.hi /
// dh) leaves the exact residual x.hi - q dh (one FMA), so the pair's quotient
// is q + (residual + x.lo - q dl) / dh
__device__ __forceinline__ float2 ff_div_t4(float2 x, int t) {
  const float t2 = (float)(t * t);
  const float dh = __fmul_rn(t2, t2), dl = fmaf(t2, t2, -dh);
  const float q = __fdiv_rn(x.x, dh);
  const float r = fmaf(-q, dh, x.x);
  const float e = fmaf(-q, dl, __fadd_rn(r, x.y));
  return make_float2(q, __fdividef(e, dh));
}
// (a.hi + a.lo) + (b.hi + b.lo) with the rounding error of the high parts
// kept exactly (TwoSum, additions only); commutative bit for bit
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x), v = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v)),
                            __fadd_rn(a.y, b.y));
  const float hi = __fadd_rn(s, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// ------------------------------------------------------------------ sorting
// Compare-exchange of keys i and i ^ j held in one lane's registers.
__device__ __forceinline__ void cx_reg(uint32_t& lo_slot, uint32_t& hi_slot, bool up) {
  const uint32_t mn = min(lo_slot, hi_slot), mx = max(lo_slot, hi_slot);
  lo_slot = up ? mn : mx;
  hi_slot = up ? mx : mn;
}

// Ascending sort of n keys in a[0..n), padded to P = next power of two with
// 0xffffffff.  Warp-synchronous bitonic network: in registers for P <= 128
// (key 32 r + lane in register r of the lane; partners at distance < 32 by
// shuffle, at 32 and 64 within the lane), in shared memory beyond.
static __device__ void warp_sort(uint32_t* a, int n) {
  const int lane = lane_id();
  int P = 1;
  while (P < n) P <<= 1;
  if (P > 32 && P <= 128) {
    uint32_t x[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = 32 * r + lane;
      x[r] = i < n ? a[i] : 0xffffffffu;
    }
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        if (j == 64) {
          cx_reg(x[0], x[2], ((lane) & k) == 0);
          cx_reg(x[1], x[3], ((32 + lane) & k) == 0);
        } else if (j == 32) {
          cx_reg(x[0], x[1], ((lane) & k) == 0);
          cx_reg(x[2], x[3], ((64 + lane) & k) == 0);
        } else {
          const bool lower = (lane & j) == 0;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const uint32_t y = __shfl_xor_sync(kFull, x[r], j);
            const bool up = ((32 * r + lane) & k) == 0;
            const uint32_t mn = min(x[r], y), mx = max(x[r], y);
            x[r] = (lower == up) ? mn : mx;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = 32 * r + lane;
      if (i < P) a[i] = x[r];
    }
    __syncwarp();
    return;
  }
  if (P <= 32) {
    uint32_t x = lane < n ? a[lane] : 0xffffffffu;
    for (int k = 2; k <= 32; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        uint32_t y = __shfl_xor_sync(kFull, x, j);
        bool up = (lane & k) == 0;
        bool lower = (lane & j) == 0;
        uint32_t mn = x < y ? x : y, mx = x < y ? y : x;
        x = (lower == up) ? mn : mx;
      }
    }
    if (lane < P) a[lane] = x;
    __syncwarp();
    return;
  }
  for (int i = n + lane; i < P; i += 32) a[i] = 0xffffffffu;
  __syncwarp();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < (P >> 1); i += 32) {
        int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
        int hi = lo + j;
        bool up = (lo & k) == 0;
        uint32_t x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
      __syncwarp();
    }
  }
}

// Ascending sort of the n window keys ((x + 32768) << 8 | level) in a[0..n)
// by the intensity x alone: the level is a nondecreasing function of x, so
// keys of equal x are equal words and this is the order of the whole words.
// For 128 < n <= 32 kRadixRounds: least-significant-digit radix sort of
// x - min(x) in 5-bit digits (one bucket per lane), as many passes as the
// window's intensity range has bits (none when every x is equal).  Keys stay
// in registers between passes; each pass counts digits (match_any leaders
// add to hist), scans the 32 counts, and scatters round by round in order,
// so every pass is stable.  hist: 32 ints of warp scratch.  Other n: the
// bitonic network of warp_sort (in registers up to 128 keys, where it was
// measured faster than these passes).  The mapping kernel sorts windows by
// counting (warp_csort) and comes here only for spans too wide for its bins.
constexpr int kRadixRounds = 16;
static __device__ void warp_sort_x(uint32_t* a, int n, int* hist) {
  if (n <= 128 || n > 32 * kRadixRounds) return warp_sort(a, n);
  const int lane = lane_id();
  const int rounds = (n + 31) >> 5;
  uint32_t k[kRadixRounds];
  unsigned lo = 0xffffffffu, hi = 0u;
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    const int i = 32 * r + lane;
    k[r] = 0u;
    if (r < rounds && i < n) {
      k[r] = a[i];
      lo = min(lo, k[r] >> 8);
      hi = max(hi, k[r] >> 8);
    }
  }
  lo = __reduce_min_sync(kFull, lo);
  hi = __reduce_max_sync(kFull, hi);
  if (hi == lo) return;
  const int bits = 32 - __clz(hi - lo);
  const unsigned last = __ballot_sync(kFull, 32 * (rounds - 1) + lane < n);
  for (int sh = 0; sh < bits; sh += 5) {
    hist[lane] = 0;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
      if (r < rounds) {
        const unsigned act = (r == rounds - 1) ? last : kFull;
        if ((act >> lane) & 1u) {
          const unsigned d = (((k[r] >> 8) - lo) >> sh) & 31u;
          const unsigned peers = __match_any_sync(act, d);
          if ((peers & lanemask_lt()) == 0) atomicAdd(&hist[d], __popc(peers));
        }
      }
    }
    __syncwarp();
    {  // exclusive scan of the digit counts
      const int c = hist[lane];
      int inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
      }
      __syncwarp();
      hist[lane] = inc - c;
      __syncwarp();
    }
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
      if (r < rounds) {
        const unsigned act = (r == rounds - 1) ? last : kFull;
        const bool v = (act >> lane) & 1u;
        unsigned d = 0u, peers = 0u;
        if (v) {
          d = (((k[r] >> 8) - lo) >> sh) & 31u;
          peers = __match_any_sync(act, d);
          a[hist[d] + __popc(peers & lanemask_lt())] = k[r];
        }
        __syncwarp();
        if (v && (peers & lanemask_lt()) == 0) hist[d] += __popc(peers);
        __syncwarp();
      }
    }
    if (sh + 5 < bits) {
#pragma unroll
      for (int r = 0; r < kRadixRounds; ++r) {
        const int i = 32 * r + lane;
        if (r < rounds && i < n) k[r] = a[i];
      }
      __syncwarp();
    }
  }
}

// Ascending sort of the n window keys ((x + 32768) << 8 | level) in a[0..n)
// by counting, for n <= 32 kRadixRounds and an intensity span
// x_max - x_min + 1 of at most 2 nwords: one 16-bit count per intensity, two
// to a word of `bins` (nwords words of shared scratch; the words the span
// covers are zeroed first and left zero).  Counts by shared atomics, an
// exclusive scan of the span (a run of words per lane, then across lanes),
// and each key placed at the position its atomic increment returns.  Keys of equal x are equal
// words, so the order in which equal keys land does not matter: the result
// is the one sorted array.  Unlike the radix passes, no round waits for the
// one before it.  Returns false, with a and bins untouched, when the span is
// larger.
constexpr int kCsortMinKeys = 0;  // windows of more keys are sorted by counting
static __device__ bool warp_csort(uint32_t* a, int n, uint32_t* bins, int nwords) {
  const int lane = lane_id();
  const int rounds = (n + 31) >> 5;
  uint32_t k[kRadixRounds];
  unsigned lo = 0xffffffffu, hi = 0u;
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    const int i = 32 * r + lane;
    k[r] = 0u;
    if (r < rounds && i < n) {
      k[r] = a[i];
      lo = min(lo, k[r] >> 8);
      hi = max(hi, k[r] >> 8);
    }
  }
  lo = __reduce_min_sync(kFull, lo);
  hi = __reduce_max_sync(kFull, hi);
  if (hi - lo >= 2u * (unsigned)nwords) return false;
  const int nw = (int)((hi - lo) >> 1) + 1;  // words the span covers
  for (int q = lane; q < nw; q += 32) bins[q] = 0u;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    const int i = 32 * r + lane;
    if (r < rounds && i < n) {
      const unsigned v = (k[r] >> 8) - lo;
      atomicAdd(&bins[v >> 1], 1u << ((v & 1u) << 4));
    }
  }
  __syncwarp();
  {  // exclusive scan: lane takes words [q0, q1)
    const int per = (nw + 31) >> 5;
    const int q0 = min(lane * per, nw), q1 = min(q0 + per, nw);
    unsigned tot = 0u;
    for (int q = q0; q < q1; ++q) {
      const unsigned x = bins[q];
      tot += (x & 0xffffu) + (x >> 16);
    }
    unsigned inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    unsigned run = inc - tot;
    for (int q = q0; q < q1; ++q) {
      const unsigned x = bins[q];
      const unsigned c0 = x & 0xffffu;
      bins[q] = run | ((run + c0) << 16);
      run += c0 + (x >> 16);
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < kRadixRounds; ++r) {
    const int i = 32 * r + lane;
    if (r < rounds && i < n) {
      const unsigned v = (k[r] >> 8) - lo, sh = (v & 1u) << 4;
      const unsigned old = atomicAdd(&bins[v >> 1], 1u << sh);
      a[(old >> sh) & 0xffffu] = k[r];
    }
  }
  __syncwarp();
  for (int q = lane; q < nw; q += 32) bins[q] = 0u;
  __syncwarp();
  return true;
}

// first index in a[lo..hi) with a[i] >= key (a sorted)
__device__ __forceinline__ int lower_bound_u32(const uint32_t* a, int lo, int hi,
                                               uint32_t key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// (c/n) * log2(n/c) for 0 < c <= n; exactly 0 when c == n (a single cell
// has zero entropy, and a zero HX is what makes Imc1 undefined)
__device__ __forceinline__ float ent_term(int c, int n) {
  if (c == n) return 0.f;
  const float fc = (float)c, fn = (float)n;
  return __fdividef(fc, fn) * __log2f(__fdividef(fn, fc));
}

// ------------------------------------------------------------------ gather
// Copy the window of the voxel at tile offset (cx, cy, cz) (window corner)
// from the staged halo tile: kb[0..nv) receives the packed words of V(v)
// (compacted), lvl[p] the gray level (0 outside V(v)).
static __device__ int gather_window(const Win& w, const Arena& A, const uint32_t* tile,
                             int TX, int TY, int cx, int cy, int cz) {
  const int lane = lane_id();
  int nv = 0;
  for (int base = 0; base < w.W; base += 32) {
    int p = base + lane;
    uint32_t word = 0;
    if (p < w.W) {
      int z, y, x;
      pos_to_zyx(w, p, z, y, x);
      word = tile[((cz + z) * TY + (cy + y)) * TX + (cx + x)];
      A.lvl[p] = (uint8_t)(word & 0xffu);
    }
    unsigned b = __ballot_sync(kFull, word != 0u);
    if (word != 0u) A.kb[nv + __popc(b & lanemask_lt())] = word;
    nv += __popc(b);
  }
  __syncwarp();
  return nv;
}

// ------------------------------------------------------------------ first order
// Sorted keys -> the 18 first-order features, the present-level table
// (lev, lut), m, lev0, R and the level-count square sum.
static __device__ void first_order(Win& w, const Arena& A, const FrJob& job,
                            int32_t* dbg_hist) {
  const int lane = lane_id();
  const int N = w.nv;
  const uint32_t* kb = A.kb;
  auto xs = [&](int i) { return (int)(kb[i] >> 8) - 32768; };
  // pass 1: sums and level-run starts
  int s1 = 0;
  unsigned long long s2 = 0;
  int base = 0;
  for (int c = 0; c < N; c += 32) {
    int i = c + lane;
    bool start = false;
    int g = 0;
    if (i < N) {
      const uint32_t k = kb[i];
      const int x = (int)(k >> 8) - 32768;
      s1 += x;
      s2 += (unsigned long long)((long long)x * x);
      g = (int)(k & 0xffu);
      start = (i == 0) || ((kb[i - 1] & 0xffu) != (unsigned)g);
    }
    unsigned b = __ballot_sync(kFull, start);
    if (start) {
      int q = base + __popc(b & lanemask_lt());
      A.lev[q] = (uint8_t)g;
      A.lut[g] = (uint8_t)q;
      A.st[q] = (uint16_t)i;
    }
    base += __popc(b);
  }
  const int m = base;
  if (lane == 0) A.st[m] = (uint16_t)N;
  s1 = (int)redux_u32((unsigned)s1);
  s2 = warp_sum_u64(s2);
  __syncwarp();
  // level counts: entropy, uniformity
  float ent = 0.f;
  unsigned u2 = 0;
  for (int q = lane; q < m; q += 32) {
    int c = (int)A.st[q + 1] - (int)A.st[q];
    ent += ent_term(c, N);
    u2 += (unsigned)(c * c);
    if (dbg_hist) dbg_hist[A.lev[q] - 1] = c;
  }
  u2 = redux_u32(u2);
  // exact percentiles: (N-1)*q = 100*k + rem, P_q = (100 x_k + rem (x_k+1 - x_k)) / 100
  long long num[5];
  const int qs[5] = {10, 25, 50, 75, 90};
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    int hq = (N - 1) * qs[t];
    int k = hq / 100, rem = hq % 100;
    long long xk = xs(k);
    num[t] = 100 * xk + (rem ? (long long)rem * (xs(k + 1) - xk) : 0);
  }
  // pass 2: central moments from d = N x - S1 (exact), robust-range counts
  __int128 d2 = 0, d3 = 0, d4 = 0;
  unsigned long long dabs = 0, medabs = 0;  // medabs: sum |100 x - 100 P50|
  unsigned below10 = 0, upto90 = 0;
  for (int i = lane; i < N; i += 32) {
    const long long x = xs(i);
    const long long d = (long long)N * x - s1;
    const long long dd = d * d;
    d2 += (__int128)dd;
    d3 += (__int128)dd * d;
    d4 += (__int128)dd * dd;
    dabs += (unsigned long long)(d < 0 ? -d : d);
    const long long dm = 100 * x - num[2];
    medabs += (unsigned long long)(dm < 0 ? -dm : dm);
    below10 += (100 * x < num[0]);
    upto90 += (100 * x <= num[4]);
  }
  d2 = warp_sum_i128(d2);
  d3 = warp_sum_i128(d3);
  d4 = warp_sum_i128(d4);
  dabs = warp_sum_u64(dabs);
  medabs = warp_sum_u64(medabs);
  below10 = redux_u32(below10);
  upto90 = redux_u32(upto90);
  // pass 3: robust subset [below10, upto90)
  const int rn = (int)upto90 - (int)below10;
  int rs = 0;
  for (int i = (int)below10 + lane; i < (int)upto90; i += 32) rs += xs(i);
  rs = (int)redux_u32((unsigned)rs);
  unsigned long long rabs = 0;
  for (int i = (int)below10 + lane; i < (int)upto90; i += 32) {
    long long d = (long long)rn * xs(i) - rs;
    rabs += (unsigned long long)(d < 0 ? -d : d);
  }
  rabs = warp_sum_u64(rabs);
  {
    float e1[1] = {ent};
    warp_sum_f32x<1>(e1);
    ent = e1[0];
  }
  if (lane == 0) {
    const float fn = (float)N;
    const float m2 = i128_to_f32(d2);  // = N^3 * variance
    float* f = A.fv;
    f[0] = (float)s2;
    f[1] = (float)job.voxel_volume * (float)s2;
    f[2] = ent;
    f[3] = (float)xs(0);
    f[4] = (float)num[0] * 0.01f;
    f[5] = (float)num[4] * 0.01f;
    f[6] = (float)xs(N - 1);
    f[7] = __fdividef((float)s1, fn);
    f[8] = (float)num[2] * 0.01f;
    f[9] = (float)(num[3] - num[1]) * 0.01f;
    f[10] = (float)(xs(N - 1) - xs(0));
    f[11] = __fdividef((float)dabs, fn * fn);
    f[12] = rn > 0 ? __fdividef((float)rabs, (float)rn * (float)rn) : kNaNf;
    f[13] = sqrtf(__fdividef((float)s2, fn));
    if (m2 == 0.f) {
      f[14] = kNaNf;
      f[15] = kNaNf;
    } else {
      f[14] = __fdividef(i128_to_f32(d3) * sqrtf(fn), m2 * sqrtf(m2));
      // m4 / m2^2 = N d4 / d2^2, and "minus 3" cancels when the kurtosis is
      // near 3: the excess is taken from the exact numerator N d4 - 3 d2^2
      // (int128: d2 < 2^56 keeps d2^2 < 2^112 and N d4 <= N d2^2 < 2^124),
      // else from the same quotient in FP64
      const float fd2 = i128_to_f32(d2);
      float kex;
      if ((d2 >> 56) == 0 && N <= 4096) {
        const __int128 knum = (__int128)N * d4 - 3 * d2 * d2;
        kex = __fdividef(i128_to_f32(knum), fd2 * fd2);
      } else {
        const double q2 = i128_to_f64(d2);
        kex = (float)((double)N * i128_to_f64(d4) / (q2 * q2) - 3.0);
      }
      f[15] = job.kurt_excess ? kex : __fdividef(fn * __fdividef(i128_to_f32(d4), m2), m2);
    }
    f[16] = __fdividef(m2, fn * fn * fn);
    f[17] = __fdividef((float)u2, fn * fn);
    // IBSI extras: median absolute deviation, coefficient of variation
    // sqrt(variance) / mean, quartile coefficient of dispersion (exact
    // numerator and denominator 100 (P75 -+ P25))
    f[kFirstExtra] = __fdividef((float)medabs, 100.f * fn);
    f[kFirstExtra + 1] = lane_quot(sqrtf(__fdividef(m2, fn)), (float)s1);
    f[kFirstExtra + 2] = lane_quot((float)(num[3] - num[1]), (float)(num[3] + num[1]));
  }
  w.m = m;
  w.lev0 = A.lev[0];
  w.R = (int)A.lev[m - 1] - (int)A.lev[0];
  w.u2 = u2;
  __syncwarp();
}

// lvl[p]: level -> compact index + 1 (0 stays 0)
static __device__ void compact_levels(const Win& w, const Arena& A) {
  for (int p = lane_id(); p < w.W; p += 32) {
    int g = A.lvl[p];
    if (g) A.lvl[p] = (uint8_t)(A.lut[g] + 1);
  }
  __syncwarp();
}

// Per-direction accumulation: lane f < nf adds finite v into facc[f].  The
// sum is compensated (Knuth's TwoSum keeps each addition's rounding error in
// fcomp): per-direction values of either sign can cancel to a mean far below
// them (ClusterShade), where a plain fp32 sum loses the digits.
__device__ __forceinline__ void acc_reset(const Arena& A) {
  const int lane = lane_id();
  A.facc[lane] = 0.f;
  A.fcomp[lane] = 0.f;
  A.nacc[lane] = 0;
  __syncwarp();
}
__device__ __forceinline__ void acc_lane(const Arena& A, int nf, float v) {
  const int lane = lane_id();
  if (lane < nf && !isnan(v)) {
    const float a = A.facc[lane], s = a + v, bv = s - a;
    A.fcomp[lane] += (a - (s - bv)) + (v - bv);
    A.facc[lane] = s;
    A.nacc[lane] += 1;
  }
}
// Compensated (TwoSum) accumulation of one value into (s, c).
__device__ __forceinline__ void two_sum_add(float& s, float& c, float v) {
  const float t = s + v, bv = t - s;
  c += (s - (t - bv)) + (v - bv);
  s = t;
}

__device__ __forceinline__ void acc_store(const Arena& A, int nf, int f0) {
  __syncwarp();
  const int lane = lane_id();
  if (lane < nf)
    A.fv[f0 + lane] = A.nacc[lane] ? __fdividef(A.facc[lane] + A.fcomp[lane], (float)A.nacc[lane])
                                   : kNaNf;
  __syncwarp();
}

// ------------------------------------------------------------------ MCC
__device__ __forceinline__ float warp_max_pos_f32(float v) {
  // v >= 0: the ordering of nonnegative floats matches their bit patterns
  return __int_as_float(__reduce_max_sync(kFull, __float_as_int(v)));
}

__device__ __forceinline__ int sturm_below(const float* dd, const float* ee, int n,
                                           float t) {
  int c = 0;
  float q = dd[0] - t;
  if (q < 0.f) ++c;
  for (int i = 1; i < n; ++i) {
    if (fabsf(q) < 1e-30f) q = -1e-30f;
    q = dd[i] - t - __fdividef(ee[i - 1] * ee[i - 1], q);
    if (q < 0.f) ++c;
  }
  return c;
}

// Largest |eigenvalue| of the symmetric n x n matrix A (stride mc, fp32):
// Householder tridiagonalisation (warp-cooperative, A overwritten), then
// Sturm-sequence multisection over 32 shifts per round.  Used for
// directions with more than kCapL present levels.
static __device__ float spectral_radius(float* A, int n, int mc, float* vv, float* ww,
                                 float* dd, float* ee) {
  const int lane = lane_id();
  for (int k = 0; k + 2 < n; ++k) {
    float tail = 0.f;
    for (int i = k + 2 + lane; i < n; i += 32) {
      float x = A[i * mc + k];
      tail += x * x;
    }
    {
      float t1[1] = {tail};
      warp_sum_f32x<1>(t1);
      tail = t1[0];
    }
    const float x1 = A[(k + 1) * mc + k];
    if (tail == 0.f) {
      if (lane == 0) {
        dd[k] = A[k * mc + k];
        ee[k] = x1;
      }
      continue;
    }
    const float alpha = -copysignf(sqrtf(tail + x1 * x1), x1);
    const float inv = rsqrtf(2.f * (alpha * alpha - alpha * x1));
    for (int i = k + 1 + lane; i < n; i += 32)
      vv[i] = (i == k + 1 ? x1 - alpha : A[i * mc + k]) * inv;
    __syncwarp();
    float kp = 0.f;
    for (int i = k + 1 + lane; i < n; i += 32) {
      float acc = 0.f;
      for (int j = k + 1; j < n; ++j) acc += A[i * mc + j] * vv[j];
      ww[i] = acc;
      kp += vv[i] * acc;
    }
    {
      float t1[1] = {kp};
      warp_sum_f32x<1>(t1);
      kp = t1[0];
    }
    for (int i = k + 1 + lane; i < n; i += 32) ww[i] -= kp * vv[i];
    __syncwarp();
    for (int i = k + 1 + lane; i < n; i += 32) {
      const float vi = vv[i], wi = ww[i];
      for (int j = k + 1; j < n; ++j) A[i * mc + j] -= 2.f * (vi * ww[j] + wi * vv[j]);
    }
    if (lane == 0) {
      dd[k] = A[k * mc + k];
      ee[k] = alpha;
    }
    __syncwarp();
  }
  __syncwarp();
  if (lane == 0) {
    if (n >= 2) {
      dd[n - 2] = A[(n - 2) * mc + (n - 2)];
      ee[n - 2] = A[(n - 1) * mc + (n - 2)];
    }
    dd[n - 1] = A[(n - 1) * mc + (n - 1)];
  }
  __syncwarp();
  float bnd = 0.f;
  for (int i = lane; i < n; i += 32) {
    float r = fabsf(dd[i]);
    if (i > 0) r += fabsf(ee[i - 1]);
    if (i < n - 1) r += fabsf(ee[i]);
    bnd = fmaxf(bnd, r);
  }
  bnd = warp_max_pos_f32(bnd);
  float lo = 0.f, hi = bnd * 1.0001f + 1e-20f;
  for (int round = 0; round < 6; ++round) {
    const float step = (hi - lo) * (1.f / 33.f);
    const float sig = lo + step * (float)(lane + 1);
    const int cnt = (n - sturm_below(dd, ee, n, sig)) + sturm_below(dd, ee, n, -sig);
    const unsigned msk = __ballot_sync(kFull, cnt > 0);
    if (msk == 0u) {
      hi = lo + step;
    } else {
      const int L = 31 - __clz(msk);
      const float nlo = lo + step * (float)(L + 1);
      const float nhi = (L == 31) ? hi : lo + step * (float)(L + 2);
      lo = nlo;
      hi = nhi;
    }
  }
  return 0.5f * (lo + hi);
}

// Index of (i, j), i <= j, in the packed upper triangle of an n x n matrix
// (row i holds columns i..n-1).
__host__ __device__ constexpr int pk(int n, int i, int j) {
  return i * n - ((i * (i - 1)) >> 1) + (j - i);
}

// Sturm count of the symmetric tridiagonal (d, e2 = squared off-diagonal)
// times sg (+1 or -1) at the shift t: the number of its eigenvalues below t.
template <int N>
__device__ __forceinline__ int sturm_count(const float (&d)[N], const float (&e2)[N], float sg,
                                           float t) {
  float q = sg * d[0] - t;
  int c = q < 0.f;
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const float qk = fabsf(q) < 1e-30f ? -1e-30f : q;
    q = sg * d[i] - t - __fdividef(e2[i - 1], qk);
    c += q < 0.f;
  }
  return c;
}

// The same count from the leading principal minors of the first n rows
// (rows beyond n are zero padding and left out):
// p_k = det(sg T_k - t I) = (sg d_k - t) p_{k-1} - e2_{k-1} p_{k-2}, p_0 = 1,
// and each sign change between p_{k-1} and p_k is one eigenvalue below t.
// Two dependent operations per row instead of a reciprocal.  The caller
// scales T (and t) to spectral radius <= 1, which keeps every minor of at
// most 12 rows within float range; a minor that is exactly zero takes the
// sign opposite to the one before it (a bias of 1e-37, below the rounding of
// any other value), as the ratio form's guard does.
template <int N>
__device__ __forceinline__ int sturm_minors(const float (&d)[N], const float (&e2)[N], float sg,
                                            float t, int n) {
  float p0 = 1.f;
  float p1 = fmaf(sg, d[0], -t) - 1e-37f;
  int c = (int)(__float_as_uint(p1) >> 31);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    if (i < n) {
      const float q = fmaf(fmaf(sg, d[i], -t), p1, -e2[i - 1] * p0) - copysignf(1e-37f, p1);
      c += (int)((__float_as_uint(q) ^ __float_as_uint(p1)) >> 31);
      p0 = p1;
      p1 = q;
    }
  }
  return c;
}

// Rounds of the paired MCC solve: both-ends bisection (one bit per round),
// then trisection of the deciding end (log2 3 bits per round); about 22 bits
// in all.
constexpr int kMccRounds1 = 22;
constexpr int kMccRounds2 = 14;

// Largest |eigenvalue| of the symmetric n x n matrix (n <= N <= 32, packed
// upper triangle, pk(n, i, j)) at src, by one warp with the matrix in
// registers: lane i holds row i (zero beyond n; zero rows and columns only
// add the eigenvalue 0, which every deflated S - u u^T already has).  Householder
// tridiagonalisation with the step loop unrolled, so every row element is a
// register: per step the column's tail norm is one warp sum, p = A v takes
// v_j from lane j by shuffle, and the rank-2 update A -= 2 (v w^T + w v^T)
// takes w_j the same way; rows above the step are never read again, so they
// are left as they are.  Then Sturm-count multisection of [0, B] (B the
// Gershgorin bound) over 32 shifts per round, one per lane, counting the
// eigenvalues of either sign beyond the shift by the signs of the leading
// minors of the n x n block of T / B.  Every lane returns the same value
// (warp sums by xor butterflies give every lane identical totals).
template <int N>
__device__ float pool_rho_regs(const float* __restrict__ src, int n) {
  static_assert(N <= 32, "one row per lane");
  const int lane = lane_id();
  float a[N];
  // packed index of (min(lane, j), max(lane, j)), stepped along the row
  int idx = lane;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    a[j] = (lane < n && j < n) ? src[idx] : 0.f;
    idx += j < lane ? max(n - j - 1, 0) : 1;  // >= 0 on lanes beyond the matrix too
  }
  float dk = 0.f, ek = 0.f;  // lane k ends with d_k and e_k (the (k, k+1) entry)
#pragma unroll
  for (int k = 0; k + 2 < N; ++k) {
    const float x = lane > k ? a[k] : 0.f;
    const float x1 = __shfl_sync(kFull, a[k], k + 1);
    float t1[1] = {lane > k + 1 ? x * x : 0.f};
    warp_sum_f32x<1>(t1);
    const float tail = t1[0];
    if (lane == k) dk = a[k];
    if (tail == 0.f) {  // the column is already reduced (the same on every lane)
      if (lane == k) ek = x1;
      continue;
    }
    const float alpha = -copysignf(sqrtf(tail + x1 * x1), x1);
    const float inv = rsqrtf(2.f * (alpha * alpha - alpha * x1));
    const float v = lane > k ? (lane == k + 1 ? x1 - alpha : x) * inv : 0.f;
    float vb[N];
    float p = 0.f;
#pragma unroll
    for (int j = k + 1; j < N; ++j) {
      vb[j] = __shfl_sync(kFull, v, j);
      p = fmaf(a[j], vb[j], p);
    }
    float kp[1] = {v * p};
    warp_sum_f32x<1>(kp);
    const float w = p - kp[0] * v;
#pragma unroll
    for (int j = k + 1; j < N; ++j) {
      const float wj = __shfl_sync(kFull, w, j);
      a[j] -= 2.f * (v * wj + w * vb[j]);
    }
    if (lane == k) ek = alpha;
  }
  if (lane == N - 2) {
    dk = a[N - 2];
    ek = a[N - 1];
  }
  if (lane == N - 1) dk = a[N - 1];
  // the tridiagonal (d, e^2) in every lane
  float d[N], e2[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d[i] = __shfl_sync(kFull, dk, i);
    const float e = __shfl_sync(kFull, ek, i);
    e2[i] = e * e;
  }
  float bnd = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float r = fabsf(d[i]);
    if (i > 0) r += sqrtf(e2[i - 1]);
    if (i < N - 1) r += sqrtf(e2[i]);
    bnd = fmaxf(bnd, r);
  }
  float lo = 0.f, hi = bnd * 1.0001f + 1e-20f;
  // the counts run on T / hi (shifts sig / hi): spectral radius <= 1
  const float sc = __fdividef(1.f, hi);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d[i] *= sc;
    e2[i] = (e2[i] * sc) * sc;
  }
  for (int round = 0; round < 6; ++round) {
    const float step = (hi - lo) * (1.f / 33.f);
    const float sig = lo + step * (float)(lane + 1);
    // eigenvalues above sig plus eigenvalues below -sig (rows beyond n are
    // zero padding: their eigenvalues 0 lie between)
    const int cnt = (n - sturm_minors<N>(d, e2, 1.f, sig * sc, n)) +
                    sturm_minors<N>(d, e2, 1.f, -sig * sc, n);
    const unsigned msk = __ballot_sync(kFull, cnt > 0);
    if (msk == 0u) {
      hi = lo + step;
    } else {
      const int L = 31 - __clz(msk);
      const float nlo = lo + step * (float)(L + 1);
      const float nhi = (L == 31) ? hi : lo + step * (float)(L + 2);
      lo = nlo;
      hi = nhi;
    }
  }
  return 0.5f * (lo + hi);
}

// Largest |eigenvalue| of two symmetric matrices of at most 16 rows at once,
// one per half-warp: lanes 16 h .. 16 h + 15 take the n x n matrix at src
// (packed upper triangle, pk(n, i, j); n = 0: no matrix), lane i of the half
// holding row i.  Householder steps as in pool_rho_regs with every sum over
// the half (xor butterflies of width 16); a column already reduced
// takes a zero reflector instead of a branch, so both halves run the same
// instructions and every shuffle sees the whole warp.  Then Sturm-count
// multisection over 16 shifts per round, one per lane of the half, of
// [max_i |T e_i|, B] (B the smaller of the Gershgorin and Frobenius bounds;
// |T e_i| <= rho), until the bracket is at most max(1e-6, 2e-5 lo) wide.  A
// shift counts the eigenvalues of either sign beyond it until the counts at
// the bracket's lower end show one end of the spectrum alone beyond it; that
// end decides the radius, and later rounds count it alone.  The counts are
// the sign changes of the leading minors of the n x n block of T / B.  Every
// lane of a half returns its matrix's value.
static __device__ __forceinline__ float pool_rho_half16(const float* __restrict__ src, int n) {
  constexpr int N = 16;
  const int lane = lane_id();
  const int r = lane & 15, half = lane >> 4;
  float a[N];
  // packed index of (min(r, j), max(r, j)), stepped along the row
  int idx = r;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    a[j] = (r < n && j < n) ? src[idx] : 0.f;
    idx += j < r ? max(n - j - 1, 0) : 1;  // >= 0 on lanes beyond the matrix too
  }
  float dk = 0.f, ek = 0.f;  // lane k of the half ends with d_k and e_k
#pragma unroll
  for (int k = 0; k + 2 < N; ++k) {
    const float x = r > k ? a[k] : 0.f;
    const float x1 = __shfl_sync(kFull, a[k], k + 1, 16);
    float tail = r > k + 1 ? x * x : 0.f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) tail += __shfl_xor_sync(kFull, tail, o);
    if (r == k) dk = a[k];
    const bool red = tail == 0.f;  // the same on every lane of the half
    const float alpha = red ? x1 : -copysignf(sqrtf(tail + x1 * x1), x1);
    const float inv = red ? 0.f : rsqrtf(2.f * (alpha * alpha - alpha * x1));
    if (r == k) ek = alpha;
    const float v = r > k ? (r == k + 1 ? x1 - alpha : x) * inv : 0.f;
    float vb[N];
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int j = k + 1; j < N; ++j) {
      vb[j] = __shfl_sync(kFull, v, j, 16);
      if ((j - k) & 1)
        p1 = fmaf(a[j], vb[j], p1);
      else
        p0 = fmaf(a[j], vb[j], p0);
    }
    const float p = p0 + p1;
    float kp = v * p;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) kp += __shfl_xor_sync(kFull, kp, o);
    const float w = p - kp * v;
    const float v2 = -2.f * v, w2 = -2.f * w;
#pragma unroll
    for (int j = k + 1; j < N; ++j) {
      const float wj = __shfl_sync(kFull, w, j, 16);
      a[j] = fmaf(v2, wj, fmaf(w2, vb[j], a[j]));
    }
  }
  if (r == N - 2) {
    dk = a[N - 2];
    ek = a[N - 1];
  }
  if (r == N - 1) dk = a[N - 1];
  float d[N], e2[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d[i] = __shfl_sync(kFull, dk, i, 16);
    const float e = __shfl_sync(kFull, ek, i, 16);
    e2[i] = e * e;
  }
  float gb = 0.f, fro = 0.f, cn = 0.f;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float g = fabsf(d[i]), c = d[i] * d[i];
    if (i > 0) {
      g += sqrtf(e2[i - 1]);
      c += e2[i - 1];
    }
    if (i < N - 1) {
      g += sqrtf(e2[i]);
      c += e2[i];
    }
    gb = fmaxf(gb, g);
    cn = fmaxf(cn, c);
    fro = fmaf(d[i], d[i], fmaf(2.f, e2[i], fro));
  }
  float lo = sqrtf(cn) * 0.9999f, hi = fminf(gb, sqrtf(fro)) * 1.0001f + 1e-20f;
  // the counts run on T / hi (shifts sig / hi): spectral radius <= 1
  const float sc = __fdividef(1.f, hi);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d[i] *= sc;
    e2[i] = (e2[i] * sc) * sc;
  }
  int ends = 0;  // 0: both ends; 1: the top end decides; 2: the bottom end
  for (int round = 0; round < 8; ++round) {
    const bool done = hi - lo <= fmaxf(1e-6f, 2e-5f * lo);
    if (__all_sync(kFull, done)) break;
    const float step = (hi - lo) * (1.f / 17.f);
    const float sig = lo + step * (float)(r + 1);
    // eigenvalues above sig (below -sig: of -T above sig) at the end taken,
    // and below -sig while both ends are counted; rows beyond n are zero
    // padding, whose eigenvalues 0 lie between
    const int ca = n - sturm_minors<N>(d, e2, ends == 2 ? -1.f : 1.f, sig * sc, n);
    const int cb = ends == 0 ? sturm_minors<N>(d, e2, 1.f, -sig * sc, n) : 0;
    const unsigned msk = (__ballot_sync(kFull, ca + cb > 0) >> (16 * half)) & 0xFFFFu;
    const int L = msk ? 31 - __clz(msk) : 0;
    const int at = __shfl_sync(kFull, (ca > 0 ? 1 : 0) | (cb > 0 ? 2 : 0), L, 16);
    if (!done) {
      if (msk == 0u) {
        hi = lo + step;
      } else {
        const float nlo = lo + step * (float)(L + 1);
        const float nhi = (L == 15) ? hi : lo + step * (float)(L + 2);
        lo = nlo;
        hi = nhi;
        if (ends == 0 && at != 3) ends = at;
      }
    }
  }
  return 0.5f * (lo + hi);
}

// Largest |eigenvalue| of a symmetric N x N matrix read from a packed upper
// triangle in the kCapL x kCapL layout, by one thread with every value in
// registers.  Rows and columns beyond the matrix hold zeros: they only add
// the eigenvalue 0, which every deflated matrix A = S - u u^T already has
// (A u = 0), so the radius is unchanged and one fixed N serves all smaller
// matrices.  Householder tridiagonalisation (indices are compile-time
// constants, so the loops unroll into independent FMAs), then Sturm
// bisection of the two ends of the spectrum, counted from the leading minors
// of the n x n block (n = the direction's present levels) of T / bound.  Two lanes solve each matrix
// (h = 0, 1; pm = the pair's lane mask) and share every round's result: while
// both ends are open, lane 0 bisects the top end and lane 1 the bottom one;
// then the pair trisects the deciding end, one shift each.  Both lanes end
// with the same bracket and return the same value.
template <int N>
__device__ __forceinline__ float rho_reg(const float* __restrict__ P, int h, unsigned pm, int n) {
  constexpr int NP = N * (N + 1) / 2;
  float a[NP];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) a[pk(N, i, j)] = P[pk(kCapL, i, j)];
  float d[N], e2[N];
#pragma unroll
  for (int k = 0; k + 2 < N; ++k) {
    // reflect x = A(k, k+1..N-1) onto alpha e_1, |alpha| = |x|
    const float x1 = a[pk(N, k, k + 1)];
    float nrm2 = x1 * x1;
#pragma unroll
    for (int i = k + 2; i < N; ++i) nrm2 = fmaf(a[pk(N, k, i)], a[pk(N, k, i)], nrm2);
    const float sq = sqrtf(nrm2);
    // |x - alpha e_1|^2 = 2 (|x|^2 + |x_1| |x|); a zero row keeps H = I
    const float inv = nrm2 > 0.f ? rsqrtf(2.f * fmaf(fabsf(x1), sq, nrm2)) : 0.f;
    d[k] = a[pk(N, k, k)];
    e2[k] = nrm2;
    a[pk(N, k, k + 1)] = (x1 + copysignf(sq, x1)) * inv;  // unit v, in row k
#pragma unroll
    for (int i = k + 2; i < N; ++i) a[pk(N, k, i)] *= inv;
    // w = A v - (v^T A v) v on the trailing block; A <- A - 2 (v w^T + w v^T)
    float w[N];
    float Kv = 0.f;
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int j = k + 1; j < N; ++j)
        acc = fmaf(a[i <= j ? pk(N, i, j) : pk(N, j, i)], a[pk(N, k, j)], acc);
      w[i] = acc;
      Kv = fmaf(a[pk(N, k, i)], acc, Kv);
    }
#pragma unroll
    for (int i = k + 1; i < N; ++i) w[i] = fmaf(-Kv, a[pk(N, k, i)], w[i]);
#pragma unroll
    for (int i = k + 1; i < N; ++i)
#pragma unroll
      for (int j = i; j < N; ++j)
        a[pk(N, i, j)] = fmaf(-2.f * a[pk(N, k, i)], w[j],
                              fmaf(-2.f * w[i], a[pk(N, k, j)], a[pk(N, i, j)]));
  }
  d[N - 2] = a[pk(N, N - 2, N - 2)];
  e2[N - 2] = a[pk(N, N - 2, N - 1)] * a[pk(N, N - 2, N - 1)];
  d[N - 1] = a[pk(N, N - 1, N - 1)];
  e2[N - 1] = 0.f;
  // bound on |lambda|: the smaller of the Gershgorin and Frobenius bounds
  float bnd = 0.f, dmax = d[0], dmin = d[0], fro = 0.f;
  float e[N];
#pragma unroll
  for (int i = 0; i < N; ++i) e[i] = sqrtf(e2[i]);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float r = fabsf(d[i]) + e[i];
    if (i > 0) r += e[i - 1];
    bnd = fmaxf(bnd, r);
    dmax = fmaxf(dmax, d[i]);
    dmin = fminf(dmin, d[i]);
    fro = fmaf(d[i], d[i], fmaf(2.f, e2[i], fro));
  }
  bnd = fminf(bnd, sqrtf(fro)) * 1.0001f + 1e-20f;
  // the counts run on T / bnd (shifts t / bnd): spectral radius <= 1
  const float sc = __fdividef(1.f, bnd);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    d[i] *= sc;
    e2[i] = (e2[i] * sc) * sc;
  }
  // A has the eigenvalue 0, so lambda_max >= 0 >= lambda_min and the radius
  // is max(lambda_max, -lambda_min).  Bracket both ends (lambda_max in
  // [max d_i, bnd], lambda_min in [-bnd, min d_i], by interlacing) until the
  // brackets show which end decides the radius, then refine that end alone.
  float hl = fmaxf(dmax, 0.f), hh = bnd, ll = -bnd, lh = fminf(dmin, 0.f);
  int it = 0;
  for (; it < kMccRounds1; ++it) {
    if (hl >= -ll || -lh >= hh) break;  // one end dominates
    // lane 0: top bracket [hl, hh] of A; lane 1: top bracket [-lh, -ll] of -A
    const float lo = h ? -lh : hl, hi = h ? -ll : hh;
    const float t = 0.5f * (lo + hi);
    // every eigenvalue < t (the n x n block's; t > 0, so the padding's zeros too)
    const bool below = sturm_minors<N>(d, e2, h ? -1.f : 1.f, t * sc, n) == n;
    const float nlo = below ? lo : t, nhi = below ? t : hi;
    const float olo = __shfl_xor_sync(pm, nlo, 16), ohi = __shfl_xor_sync(pm, nhi, 16);
    hl = h ? olo : nlo;
    hh = h ? ohi : nhi;
    lh = -(h ? nlo : olo);
    ll = -(h ? nhi : ohi);
  }
  if (it == kMccRounds1) return fmaxf(fabsf(0.5f * (hl + hh)), fabsf(0.5f * (ll + lh)));
  const bool top = hl >= -ll;
  const float sg = top ? 1.f : -1.f;
  float lo = top ? hl : -lh, hi = top ? hh : -ll;
  for (int r = 0; r < kMccRounds2; ++r) {
    // the bracket is fine enough: half-width <= max(5e-7, 1e-5 lambda)
    if (hi - lo <= fmaxf(1e-6f, 2e-5f * lo)) break;
    const float st = (hi - lo) * (1.f / 3.f);
    const float t1 = lo + st, t2 = lo + 2.f * st;
    const int c = sturm_minors<N>(d, e2, sg, (h ? t2 : t1) * sc, n);
    const int co = __shfl_xor_sync(pm, c, 16);
    const int c1 = h ? co : c, c2 = h ? c : co;
    if (c1 == n) {
      hi = t1;
    } else if (c2 == n) {
      lo = t1;
      hi = t2;
    } else {
      lo = t2;
    }
  }
  return 0.5f * (lo + hi);
}

// ------------------------------------------------------------------ slice bit masks
// For windows of side S <= 7 a set of window positions is S words, word z
// holding slice z with bit y S + x (32-bit words up to S = 5, 64-bit at 7).
// Lane a holds the set of compact level a; shifting a set along a direction
// d moves whole words by dz and bits by dy S + dx.
template <int S>
struct SliceT {
  using W = typename std::conditional<(S * S <= 32), uint32_t, unsigned long long>::type;
  static constexpr int kChunks = (S * S + 31) / 32;
  static __device__ __forceinline__ W full() { return (W)(((unsigned long long)1 << (S * S)) - 1ull); }
  // in-slice positions whose row y + dy (column x + dx) stays inside
  static __device__ __forceinline__ W rows_ok(int dy) {
    constexpr unsigned long long row0 = ((unsigned long long)1 << S) - 1ull;
    constexpr unsigned long long allr = ((unsigned long long)1 << (S * S)) - 1ull;
    return (W)(dy > 0 ? (allr >> S) : dy < 0 ? (allr & ~row0) : allr);
  }
  static __device__ __forceinline__ W cols_ok(int dx) {
    unsigned long long c = 0;
#pragma unroll
    for (int y = 0; y < S; ++y)
      c |= (dx > 0 ? (((unsigned long long)1 << (S - 1)) - 1ull)
                   : dx < 0 ? ((((unsigned long long)1 << S) - 1ull) & ~1ull)
                            : (((unsigned long long)1 << S) - 1ull))
           << (y * S);
    return (W)c;
  }
};

template <typename W>
__device__ __forceinline__ W shift_bits(W x, int k) {  // bit b + k -> b (k may be < 0)
  return k >= 0 ? (W)(x >> k) : (W)(x << (-k));
}

// One direction d = (dz, dy, dx), dz in {0, 1}, as shift parameters.
template <int S>
struct SliceDir {
  using W = typename SliceT<S>::W;
  int dz, k;
  W mf, mb;  // u + d (u - d) inside, in-slice part
  __device__ __forceinline__ SliceDir(int dz_, int dy, int dx) {
    dz = dz_;
    k = dy * S + dx;
    mf = SliceT<S>::rows_ok(dy) & SliceT<S>::cols_ok(dx);
    mb = SliceT<S>::rows_ok(-dy) & SliceT<S>::cols_ok(-dx);
  }
  // o(u) = x(u + d)
  __device__ __forceinline__ void fwd(const W (&x)[S], W (&o)[S]) const {
#pragma unroll
    for (int z = 0; z < S; ++z) {
      const W src = dz ? (z + 1 < S ? x[z + 1 < S ? z + 1 : z] : (W)0) : x[z];
      o[z] = shift_bits<W>(src, k) & mf;
    }
  }
  // o(u) = x(u - d)
  __device__ __forceinline__ void bwd(const W (&x)[S], W (&o)[S]) const {
#pragma unroll
    for (int z = 0; z < S; ++z) {
      const W src = dz ? (z >= 1 ? x[z >= 1 ? z - 1 : z] : (W)0) : x[z];
      o[z] = shift_bits<W>(src, -k) & mb;
    }
  }
};

template <typename W>
__device__ __forceinline__ int popc_w(W x) {
  if (sizeof(W) == 8) return __popcll((unsigned long long)x);
  return __popc((unsigned)x);
}

// This lane's compact-level set (level `lane`; empty past m) and the VOI set,
// by one ballot per slice chunk and level.
template <int S>
__device__ __forceinline__ void slice_masks(const Win& w, const Arena& A,
                                            typename SliceT<S>::W (&L)[S],
                                            typename SliceT<S>::W (&V)[S]) {
  using W = typename SliceT<S>::W;
  const int lane = lane_id();
#pragma unroll
  for (int z = 0; z < S; ++z) {
    W l = 0, v = 0;
#pragma unroll
    for (int c = 0; c < SliceT<S>::kChunks; ++c) {
      const int bit = 32 * c + lane;
      const int lv = bit < S * S ? (int)A.lvl[z * S * S + bit] : 0;
      v |= (W)__ballot_sync(kFull, lv != 0) << (32 * c);
      for (int a = 0; a < w.m; ++a) {
        const unsigned bal = __ballot_sync(kFull, lv == a + 1);
        if (lane == a) l |= (W)bal << (32 * c);
      }
    }
    L[z] = l;
    V[z] = v;
  }
}

// Warp sum of K <= 16 values per lane, scattered: lane L receives the total
// of v[L >> 1] (zero for L >> 1 >= K).  Recursive halving: at offset o a lane
// keeps the half of its partial sums selected by its bit o and sends the
// other half, so 16 sums cost 15 exchanges instead of 80.
template <int K>
__device__ __forceinline__ float warp_rsum_f32(const float (&v)[K]) {
  static_assert(K <= 16, "at most 16 sums");
  const int lane = lane_id();
  float x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = k < K ? v[k] : 0.f;
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? x[i] : x[i + h];
      const float keep = up ? x[i + h] : x[i];
      x[i] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return x[0] + __shfl_xor_sync(kFull, x[0], 1);
}

// Which of the 12 GLCM per-direction sums the feature of lane L reads
// (4 bits per lane; 0 where none): Autocorrelation .. SumEntropy order.
constexpr unsigned long long kGlcmSumLo =  // lanes 0..15
    (11ull << (4 * 2)) | (10ull << (4 * 4)) | (3ull << (4 * 8)) | (1ull << (4 * 11)) |
    (2ull << (4 * 12)) | (2ull << (4 * 13)) | (4ull << (4 * 14)) | (5ull << (4 * 15));
constexpr unsigned long long kGlcmSumHi =  // lanes 16..31
    (6ull << (4 * 0)) | (7ull << (4 * 1)) | (8ull << (4 * 2)) | (9ull << (4 * 5));
__device__ __forceinline__ int glcm_sum_of_lane(int lane) {
  return (int)((lane < 16 ? kGlcmSumLo >> (4 * lane) : kGlcmSumHi >> (4 * (lane - 16))) & 15ull);
}

// Pair t (0 <= t < m (m + 1) / 2) of the packed upper triangle of an m x m
// matrix as its row a and column b >= a: row a starts at a m - a (a - 1) / 2.
__device__ __forceinline__ void pair_of(int t, int m, int& a, int& b) {
  const float q = (float)(2 * m + 1);
  a = (int)((q - sqrtf(q * q - 8.f * (float)t)) * 0.5f);
  a = max(0, min(a, m - 1));
  while (a + 1 < m && (a + 1) * m - (((a + 1) * a) >> 1) <= t) ++a;
  while (a > 0 && a * m - ((a * (a - 1)) >> 1) > t) --a;
  b = a + (t - (a * m - ((a * (a - 1)) >> 1)));
}

// (1 + d) ln(1 + d) - d >= 0 (d > -1) without the cancellation near d = 0:
// for |d| < 1/4 its Taylor series sum_{k>=2} (-d)^k / (k (k - 1)), cut after
// d^13 (the next term is below 1e-9 of the sum); beyond, the hardware log2
// (absolute error ~1e-7 near 1, where the result is > 0.02).
__device__ __forceinline__ float kl_term(float d) {
  if (fabsf(d) < 0.25f) {
    float s = -1.f / 156.f;
    s = fmaf(s, d, 1.f / 132.f);
    s = fmaf(s, d, -1.f / 110.f);
    s = fmaf(s, d, 1.f / 90.f);
    s = fmaf(s, d, -1.f / 72.f);
    s = fmaf(s, d, 1.f / 56.f);
    s = fmaf(s, d, -1.f / 42.f);
    s = fmaf(s, d, 1.f / 30.f);
    s = fmaf(s, d, -1.f / 20.f);
    s = fmaf(s, d, 1.f / 12.f);
    s = fmaf(s, d, -1.f / 6.f);
    s = fmaf(s, d, 0.5f);
    return d * d * s;
  }
  const float x = 1.f + d;
  return fmaf(x * __log2f(x), 0.69314718055994531f, -d);
}

// ------------------------------------------------------------------ GLCM
// The CTA's pool of many-level MCC solves (more than kCapL present levels):
// a warp that meets one writes S - u u^T to its global scratch and lists the
// task; after the GLCM family every warp of the CTA takes tasks from the list
// and writes the radius into the owner's results, so one voxel's many-level
// directions no longer hold the whole CTA at the next barrier.
struct FbPool {
  int* count;        // tasks of up to 16 rows listed this round (from the front)
  int* next;         // next of them to take
  int* count_big;    // tasks of more rows (from the back of the list)
  int* next_big;
  int* tasks;        // owner warp << 16 | direction << 8 | size
  float* scratch;    // this warp's matrices, kNumDirs x kMCap^2
  int warp;
};

// Lists warp-owner direction d's m x m solve: up to 16 rows at the front of
// the list (the pool solves two at a time), more at the back.
__device__ __forceinline__ void pool_list(const FbPool* pool, int d, int m) {
  const int task = (pool->warp << 16) | (d << 8) | m;
  if (m <= 16)
    pool->tasks[atomicAdd(pool->count, 1)] = task;
  else
    pool->tasks[kFbTasks - 1 - atomicAdd(pool->count_big, 1)] = task;
}

// After the 13 directions: the deferred MCC solves (one lane per direction),
// the direction means, and ClusterShade's mean (in float pairs).
static __device__ void glcm_finish(const Arena& A, const FrJob& job) {
  const int lane = lane_id();
  const bool want_mcc = (job.families & kFamMCC) != 0;
  int* mn = (int*)(A.big + A.L.mn);
  float* mres = (float*)(A.big + A.L.mres);
  float* slots = (float*)(A.big + A.L.slots);
  float2* csn = (float2*)(A.big + A.L.csn);
  int* cst = (int*)(A.big + A.L.cst);
  __syncwarp();
  if (want_mcc) {
    // one register-resident size for the warp: the smallest that holds every
    // direction's matrix (zero padding leaves the radius unchanged); lanes d
    // and d + 16 solve direction d together
    const int dl = lane & 15, h = lane >> 4;
    const int nl = (dl < kNumDirs) ? mn[dl] : 0;
    const int nmax = __reduce_max_sync(kFull, nl);
    if (nl >= 2) {
      const float* P = slots + dl * kSlot;
      const unsigned pm = (1u << dl) | (1u << (dl + 16));
      const float r = nmax <= 4   ? rho_reg<4>(P, h, pm, nl)
                      : nmax <= 8 ? rho_reg<8>(P, h, pm, nl)
                                  : rho_reg<kCapL>(P, h, pm, nl);
      if (!h) mres[dl] = r;
    }
    __syncwarp();
    if (lane == 23) {
      float s = 0.f;
      int c = 0;
      for (int d = 0; d < kNumDirs; ++d) {
        const float v = mres[d];
        if (!isnan(v)) {
          s += v;
          ++c;
        }
      }
      A.facc[23] = s;
      A.fcomp[23] = 0.f;
      A.nacc[23] = c;
    }
  }
  acc_store(A, want_mcc ? 24 : 23, 18);
  if (lane == 24 || lane == 25)
    A.fv[kGlcmExtra + lane - 24] =
        A.nacc[lane] ? __fdividef(A.facc[lane] + A.fcomp[lane], (float)A.nacc[lane]) : kNaNf;
  {
    __syncwarp();
    const int t = lane < kNumDirs ? cst[lane] : 0;
    float2 v = make_float2(0.f, 0.f);
    if (t > 0) v = ff_div_t4(csn[lane], t);
    const int n = __popc(__ballot_sync(kFull, t > 0));
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const float2 w = make_float2(__shfl_xor_sync(kFull, v.x, o), __shfl_xor_sync(kFull, v.y, o));
      v = ff_add(v, w);
    }
    if (lane == 3 && n) {
      const float fn = (float)n, q = __fdiv_rn(v.x, fn);
      A.fv[18 + 3] = q + __fdividef(__fadd_rn(fmaf(-q, fn, v.x), v.y), fn);
    }
    if (lane < kNumDirs) cst[lane] = 0;  // leave the big region zero
    __syncwarp();
  }
}

// S > 0: windows of side S with at most 32 levels, distance 1, per-direction
// aggregation: pair counts from level bit masks (lane a holds level a's set;
// a pair lane counts |L_a & fwd(L_b)| + |L_b & fwd(L_a)|), so there is no
// shared-memory count matrix.  S == 0: any window; pairs counted into a
// shared-memory matrix of compact levels.
template <int S>
static __device__ void glcm_family_impl(const Win& w, const Arena& A, const FrJob& job,
                                        int32_t* dbg_glcm, const FbPool* pool) {
  const int lane = lane_id();
  const int m = w.m, mc = A.mc;
  int* cnt = (int*)(A.big + A.L.cnt);
  int* marg = (int*)(A.big + A.L.marg);
  int* prank = (int*)(A.big + A.L.prank);  // rank of a present level
  int* sbin = (int*)(A.big + A.L.sbin);
  int* dbin = (int*)(A.big + A.L.dbin);
  float* vv = (float*)(A.big + A.L.vec);
  float* ww = vv + mc;
  float* dd = ww + mc;
  float* ee = dd + mc;
  int* mn = (int*)(A.big + A.L.mn);
  float* mres = (float*)(A.big + A.L.mres);
  float* slots = (float*)(A.big + A.L.slots);
  const bool want_mcc = (job.families & kFamMCC) != 0;
  const float ngf = (float)w.ng;
  Magic mm;
  mm.init((unsigned)m);
  const int mm2 = m * m;
  // merged aggregation: the 13 directions' pairs go into one matrix, whose
  // features (and MCC, in slot 0) are taken once
  const bool merged = job.agg == 1;
  if (merged && want_mcc && lane < kNumDirs) {
    mn[lane] = 0;
    mres[lane] = kNaNf;
  }
  acc_reset(A);
  // ClusterShade: per-direction values of either sign (hundreds, for
  // near-symmetric windows) can average to ~1e-2, below what fp32 keeps
  // after rounding each; their exact numerators (as float pairs, about 48
  // bits) and totals are kept per direction and averaged in float pairs
  // after the loop
  float2* csn = (float2*)(A.big + A.L.csn);
  int* cst = (int*)(A.big + A.L.cst);
  if (lane < kNumDirs) cst[lane] = 0;
  constexpr int SS = S > 0 ? S : 1;
  using W = typename SliceT<SS>::W;
  W Lm[SS], Vm[SS];
  if constexpr (S > 0) slice_masks<S>(w, A, Lm, Vm);
  const int npairs = m * (m + 1) / 2;
  // this lane's level pair in the first two rounds of the pair loop (the
  // same for every direction), 5 bits per level: a0 b0 a1 b1
  unsigned pairs01 = 0;
  if constexpr (S > 0) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int t = 32 * r + lane;
      int a = 0, b = 0;
      if (t < npairs) pair_of(t, m, a, b);
      pairs01 |= (unsigned)(a | (b << 5)) << (10 * r);
    }
  }
  int np = 0;
  for (int di = 0; di < kNumDirs; ++di) {
    const int ddz = c_dirs[di][0] * job.delta, ddy = c_dirs[di][1] * job.delta,
              ddx = c_dirs[di][2] * job.delta;
    const int off = ddz * w.s2 + ddy * w.s + ddx;
    // pairs -> upper-triangle counts over compact indices (equal keys merged)
    if (!merged) np = 0;
    W fL[SS];        // mask path: this lane's level set moved back along d
    unsigned cmask = 0;  // mask path: this lane's marginal count
    if constexpr (S > 0) {
      const SliceDir<S> D(c_dirs[di][0], c_dirs[di][1], c_dirs[di][2]);
      W fV[S], bV[S];
      D.fwd(Lm, fL);
      D.fwd(Vm, fV);
      D.bwd(Vm, bV);
      unsigned npz = 0;
#pragma unroll
      for (int z = 0; z < S; ++z) {
        cmask += (unsigned)(popc_w<W>(Lm[z] & fV[z]) + popc_w<W>(Lm[z] & bV[z]));
        npz += (unsigned)popc_w<W>(Vm[z] & fV[z]);
      }
      np = (int)npz;
    }
    for (int base = 0; S == 0 && base < w.W; base += 32) {
      const int p = base + lane;
      int key = -1;
      if (p < w.W) {
        const int a = A.lvl[p];
        if (a) {
          int z, y, x;
          pos_to_zyx(w, p, z, y, x);
          if (in_cube(w, z + ddz, y + ddy, x + ddx)) {
            const int b = A.lvl[p + off];
            if (b) key = (min(a, b) - 1) * mc + (max(a, b) - 1);
          }
        }
      }
      const unsigned act = __ballot_sync(kFull, key >= 0);
      if (key >= 0) {
        const unsigned grp = __match_any_sync(act, key);
        if ((grp & lanemask_lt()) == 0) atomicAdd(&cnt[key], __popc(grp));
      }
      np += __popc(act);
    }
    __syncwarp();
    if (merged && di < kNumDirs - 1) continue;
    const int ds = merged ? 0 : di;  // slot / record of this matrix
    if (np == 0) {
      if (lane == 0) {
        mn[ds] = 0;
        mres[ds] = kNaNf;
      }
      acc_lane(A, 23, kNaNf);
      continue;
    }
    const int T = 2 * np;
    const float fT = (float)T;
    // marginals (lane a sums row a of the symmetric matrix) and present list
    // 64-bit where a merged matrix (13 directions, up to 13 x 3375 pairs)
    // can pass 2^32
    unsigned m1 = 0;
    unsigned long long m2 = 0;
    float hx = 0.f;
    int present = 0;
    int prank_l = 0;  // mask path: rank of this lane's level among present ones
    for (int a0 = 0; a0 < m; a0 += 32) {
      const int a = a0 + lane;
      int c = 0;
      if (a < m) {
        if constexpr (S > 0) {
          c = (int)cmask;
        } else {
          for (int b = 0; b < m; ++b)
            c += b > a ? cnt[a * mc + b] : (b == a ? 2 * cnt[a * mc + a] : cnt[b * mc + a]);
          marg[a] = c;
        }
        if (c) {
          const unsigned i = A.lev[a];
          m1 += i * (unsigned)c;
          m2 += (unsigned long long)(i * i) * (unsigned)c;
          hx += ent_term(c, T);
        }
      }
      const unsigned pb = __ballot_sync(kFull, c > 0);
      if constexpr (S > 0) {
        prank_l = __popc(pb & lanemask_lt());
      } else {
        if (c > 0) prank[a] = present + __popc(pb & lanemask_lt());
      }
      present += __popc(pb);
    }
    m1 = redux_u32(m1);
    m2 = merged ? warp_sum_u64(m2) : redux_u32((unsigned)m2);  // < 2^32 per direction
    // MCC matrix of up to kCapL present levels: written by the entries pass
    // into this direction's slot (zero first: the padding beyond them)
    const bool slot = want_mcc && present >= 2 && present <= kCapL;
    // counts are cleared as the entries pass reads them, unless the
    // many-level MCC solve still needs them
    const bool clear_now = !want_mcc || present <= kCapL;
    // mask path, many levels: the pair lanes write S - u u^T for the
    // warp-cooperative solve into the (zero) count region
    const bool fill_s = S > 0 && want_mcc && present > kCapL;
    const bool pooled = pool != nullptr && want_mcc && present > kCapL;
    // pooled: packed upper triangle over the m compact levels in the warp's
    // global scratch (every pair written); else dense (stride mc) in place
    // of the counts, which are zero where no present pair writes
    float* Sm = pooled ? pool->scratch + (size_t)ds * kFbDir : (float*)cnt;
    const int ms = mc;
    float* P = slots + ds * kSlot;
    const float invT = __fdividef(1.f, fT);
    if (slot)
      for (int t = lane; t < kSlot; t += 32) P[t] = 0.f;
    __syncwarp();
    // entries: linear sums, entropies, mutual information, sum / difference
    // bins, the MCC slot
    unsigned long long a1 = 0, e2 = 0, mi0 = 0;
    unsigned maxc = 0;
    // MI = sum over all level pairs of p ln(p/q) - p + q (q = p_a p_b; the
    // extra terms sum to zero), every term >= 0: q g(p/q) where p > 0, and
    // q where p = 0 (its sum kept exact in mi0 T^2); nats until the end
    float hxy = 0.f, mi = 0.f;
    const float fT2 = fT * fT;
    if constexpr (S > 0) {
      // one lane per level pair (a <= b), 32 pairs a round
      for (int t0 = 0; t0 < npairs; t0 += 32) {
        const int t = t0 + lane;
        const bool valid = t < npairs;
        int a = 0, b = 0;
        if (valid) {
          if (t0 < 64) {
            const unsigned pr = pairs01 >> (10 * (t0 >> 5));
            a = (int)(pr & 31u);
            b = (int)((pr >> 5) & 31u);
          } else {
            pair_of(t, m, a, b);
          }
        }
        int n = 0;
#pragma unroll
        for (int z = 0; z < S; ++z) {
          const W la = __shfl_sync(kFull, Lm[z], a);
          const W fa = __shfl_sync(kFull, fL[z], a);
          const W lb = __shfl_sync(kFull, Lm[z], b);
          const W fb = __shfl_sync(kFull, fL[z], b);
          n += a == b ? popc_w<W>(la & fa) : popc_w<W>(la & fb) + popc_w<W>(lb & fa);
        }
        const int ca = __shfl_sync(kFull, (int)cmask, a), cb = __shfl_sync(kFull, (int)cmask, b);
        const int pa = __shfl_sync(kFull, prank_l, a), pbk = __shfl_sync(kFull, prank_l, b);
        if (!valid) continue;
        if (!ca || !cb) {
          if (fill_s && pooled) Sm[t] = 0.f;  // a level absent along the direction
          continue;
        }
        if (!n) {
          // an empty pair of present levels: its q = p_a p_b enters MI, and
          // S - u u^T is dense there (-u_a u_b)
          const long long cc = (long long)ca * cb;
          mi0 += (a == b ? 1ull : 2ull) * (unsigned long long)cc;
          const float v = (float)(-cc) * rsqrtf((float)ca * (float)cb) * invT;
          if (slot) P[pk(kCapL, pa, pbk)] = v;
          if (fill_s) {
            if (pooled) {
              Sm[t] = v;  // t = pk(m, a, b)
            } else {
              Sm[a * ms + b] = v;
              Sm[b * ms + a] = v;
            }
          }
          continue;
        }
        const unsigned i = A.lev[a], j = A.lev[b];
        const int C = (a == b) ? 2 * n : n;
        const unsigned mult = (a == b) ? 1u : 2u;
        a1 += (unsigned long long)(mult * (unsigned)C) * (i * j);
        e2 += (unsigned long long)(mult * (unsigned)C) * (unsigned)C;
        maxc = max(maxc, (unsigned)C);
        const float fm = (float)mult;
        hxy += fm * ent_term(C, T);
        const long long ct = (long long)C * T, cc = (long long)ca * cb;
        if (ct != cc)  // p = p_x p_y exactly contributes nothing
          mi += fm * __fdividef((float)cc, fT2) * kl_term(__fdividef((float)(ct - cc), (float)cc));
        const float v = (float)(ct - cc) * rsqrtf((float)ca * (float)cb) * invT;
        if (slot) P[pk(kCapL, pa, pbk)] = v;
        if (fill_s) {
          if (pooled) {
            Sm[t] = v;
          } else {
            Sm[a * ms + b] = v;
            Sm[b * ms + a] = v;
          }
        }
        atomicAdd(&sbin[i + j - 2 * w.lev0], 2 * n);
        atomicAdd(&dbin[j - i], 2 * n);
        if (dbg_glcm) {
          int32_t* g = dbg_glcm + (size_t)ds * w.ng * w.ng;
          g[(i - 1) * w.ng + (j - 1)] = C;
          g[(j - 1) * w.ng + (i - 1)] = C;
        }
      }
    }
    for (int t0 = 0; S == 0 && t0 < mm2; t0 += 32) {
      const int t = t0 + lane;
      if (t >= mm2) continue;
      const int a = (int)mm.div((unsigned)t), b = t - a * m;
      if (b < a) continue;
      const int n = cnt[a * mc + b];
      if (!n) {
        const int ca = marg[a], cb = marg[b];
        if (ca && cb) {
          // an empty pair of present levels: its q = p_a p_b enters MI, and
          // S - u u^T is dense there (-u_a u_b)
          const long long cc = (long long)ca * cb;
          mi0 += (a == b ? 1ull : 2ull) * (unsigned long long)cc;
          if (slot)
            P[pk(kCapL, prank[a], prank[b])] =
                (float)(-cc) * rsqrtf((float)ca * (float)cb) * invT;
        }
        continue;
      }
      const unsigned i = A.lev[a], j = A.lev[b];
      const int C = (a == b) ? 2 * n : n;
      const unsigned mult = (a == b) ? 1u : 2u;
      a1 += (unsigned long long)(mult * (unsigned)C) * (i * j);
      e2 += (unsigned long long)(mult * (unsigned)C) * (unsigned)C;
      maxc = max(maxc, (unsigned)C);
      const float fm = (float)mult;
      hxy += fm * ent_term(C, T);
      const int ca = marg[a], cb = marg[b];
      const long long ct = (long long)C * T, cc = (long long)ca * cb;
      if (ct != cc)  // p = p_x p_y exactly contributes nothing
        mi += fm * __fdividef((float)cc, fT2) * kl_term(__fdividef((float)(ct - cc), (float)cc));
      if (clear_now) cnt[a * mc + b] = 0;
      // A(a', b') = (C T - c_a c_b) / (T sqrt(c_a c_b)) over present ranks
      if (slot)
        P[pk(kCapL, prank[a], prank[b])] =
            (float)(ct - cc) * rsqrtf((float)ca * (float)cb) * invT;
      atomicAdd(&sbin[i + j - 2 * w.lev0], 2 * n);
      atomicAdd(&dbin[j - i], 2 * n);
      if (dbg_glcm) {
        int32_t* g = dbg_glcm + (size_t)ds * w.ng * w.ng;
        g[(i - 1) * w.ng + (j - 1)] = C;
        g[(j - 1) * w.ng + (i - 1)] = C;
      }
    }
    if (merged) {
      a1 = warp_sum_u64(a1);
      e2 = warp_sum_u64(e2);
      mi0 = warp_sum_u64(mi0);
    } else {  // one direction: each < 2^32
      a1 = redux_u32((unsigned)a1);
      e2 = redux_u32((unsigned)e2);
      mi0 = redux_u32((unsigned)mi0);
    }
    maxc = __reduce_max_sync(kFull, maxc);
    __syncwarp();
    // MCC: the deflated A = S - u u^T, S = D^-1/2 P D^-1/2 over present levels
    if (want_mcc) {
      const int nd = present;
      if (nd < 2) {
        if (lane == 0) {
          mn[ds] = 0;
          mres[ds] = kNaNf;
        }
      } else if (slot) {
        if (lane == 0) mn[ds] = nd;  // solved after the 13 directions
      } else {
        // many levels: warp-cooperative solve now, on S in place of the counts
        // (the mask path wrote S during its pair rounds)
        for (int t = lane; S == 0 && t < mm2; t += 32) {
          const int a = (int)mm.div((unsigned)t), b = t - a * m;
          if (b < a) continue;
          const int n = cnt[a * mc + b];
          const int ca = marg[a], cb = marg[b];
          float v = 0.f;
          if (ca && cb) {
            const int C = (a == b) ? 2 * n : n;
            const long long num = (long long)C * T - (long long)ca * cb;
            v = __fdividef((float)num * rsqrtf((float)ca * (float)cb), fT);
          }
          if (pooled) {
            Sm[pk(m, a, b)] = v;
          } else {
            Sm[a * ms + b] = v;
            Sm[b * ms + a] = v;
          }
        }
        __syncwarp();
        if (pooled) {
          if (lane == 0) {
            mn[ds] = 0;
            mres[ds] = kNaNf;  // the pool writes the radius
            pool_list(pool, ds, m);
          }
        } else {
          const float rho = spectral_radius(Sm, m, mc, vv, ww, dd, ee);
          if (lane == 0) {
            mn[ds] = 0;
            mres[ds] = rho;
          }
        }
        __syncwarp();
        for (int t = lane; t < mm2; t += 32) {
          const int a = (int)mm.div((unsigned)t);
          cnt[a * mc + (t - a * m)] = 0;
        }
      }
    }
    __syncwarp();
    for (int a = lane; S == 0 && a < m; a += 32) {  // leave the big region zero
      marg[a] = 0;
      prank[a] = 0;
    }
    // difference and sum distributions (bins relative to the smallest level)
    unsigned dk = 0, sk = 0;
    unsigned long long dk2 = 0, sk2 = 0;
    float de = 0.f, idm = 0.f, idmn = 0.f, idd = 0.f, idn = 0.f, iv = 0.f, se = 0.f,
          ce2 = 0.f, ce4 = 0.f;
    __int128 ce3 = 0;
    const int nb = 2 * w.R + 1;
    for (int k = lane; k < nb; k += 32) {
      if (k <= w.R) {
        const int c = dbin[k];
        if (c) {
          dbin[k] = 0;
          const float fk = (float)k, fc = (float)c;
          dk += (unsigned)(k * c);
          dk2 += (unsigned long long)(k * k) * (unsigned)c;
          de += ent_term(c, T);
          idm += __fdividef(fc, 1.f + fk * fk);
          idmn += __fdividef(fc, 1.f + __fdividef(fk * fk, ngf * ngf));
          idd += __fdividef(fc, 1.f + fk);
          idn += __fdividef(fc, 1.f + __fdividef(fk, ngf));
          if (k) iv += __fdividef(fc, fk * fk);
        }
      }
      const int c = sbin[k];
      if (c) {
        sbin[k] = 0;
        const int kk = k + 2 * w.lev0;
        sk += (unsigned)(kk * c);
        sk2 += (unsigned long long)(kk * kk) * (unsigned)c;
        se += ent_term(c, T);
        // T (k - 2 mu): |e| < 2^24 per direction, < 2^26 merged
        const int e = T * kk - 2 * (int)m1;
        const float fe = (float)e, fe2 = fe * fe;
        ce2 += (float)c * fe2;
        ce4 += (float)c * fe2 * fe2;
        ce3 += (__int128)((long long)e * e) * ((long long)c * e);
      }
    }
    dk = redux_u32(dk);
    dk2 = merged ? warp_sum_u64(dk2) : redux_u32((unsigned)dk2);
    sk2 = merged ? warp_sum_u64(sk2) : redux_u32((unsigned)sk2);
    sk = redux_u32(sk);
    ce3 = warp_sum_i128(ce3);
    const float fs[12] = {hx, hxy, mi, de, idm, idmn, idd, idn, iv, se, ce2, ce4};
    // lanes 2k, 2k + 1 hold the total of fs[k]; MI (k = 2) in bits
    float tot = warp_rsum_f32<12>(fs);
    if ((lane >> 1) == 2) tot = (tot + __fdividef((float)mi0, fT2)) * 1.44269504088896341f;
    const float fa = __shfl_sync(kFull, tot, 2 * glcm_sum_of_lane(lane));  // this lane's sum
    const float f0 = __shfl_sync(kFull, tot, 0);                            // HX
    // one lane per feature
    float num = kNaNf, den = 1.f;
    const long long var_num = (long long)T * (long long)m2 - (long long)m1 * m1;  // T^2 sigma^2
    if (lane == 0) { num = (float)a1; den = fT; }
    if (lane == 1) { num = (float)m1; den = fT; }
    if (lane == 2) { num = fa; den = fT * fT * fT * fT * fT; }
    if (lane == 3) {
      num = i128_to_f32(ce3);
      den = fT * fT * fT * fT;
      csn[ds] = i128_to_ff(ce3);
      cst[ds] = T;
    }
    if (lane == 4) { num = fa; den = fT * fT * fT; }
    if (lane == 5) { num = (float)dk2; den = fT; }
    if (lane == 6) { num = (float)((long long)T * (long long)a1 - (long long)m1 * m1); den = (float)var_num; }
    if (lane == 7) { num = (float)dk; den = fT; }
    if (lane == 8) { num = fa; }
    if (lane == 9) { num = (float)((long long)T * (long long)dk2 - (long long)dk * dk); den = fT * fT; }
    if (lane == 10) { num = (float)e2; den = fT * fT; }
    if (lane == 11) { num = fa; }
    if (lane == 12) { num = -fa; den = f0; }
    if (lane == 13) { num = sqrtf(fmaxf(0.f, -expm1f(-2.f * fa))); }
    if (lane >= 14 && lane <= 18) { num = fa; den = fT; }
    if (lane == 19) { num = (float)maxc; den = fT; }
    if (lane == 20) { num = (float)sk; den = fT; }
    if (lane == 21) { num = fa; }
    if (lane == 22) { num = (float)var_num; den = fT * fT; }
    // IBSI extras (lanes 24, 25): sum variance, dissimilarity
    if (lane == 24) { num = (float)((long long)T * (long long)sk2 - (long long)sk * sk); den = fT * fT; }
    if (lane == 25) { num = (float)dk; den = fT; }
    acc_lane(A, 26, lane_quot(num, den));
  }
}

// One warp's share of the CTA pool: take listed tasks until none is left;
// each loads the owner's matrix into the warp's registers (a row per lane),
// solves it there (pool_rho_regs) and stores the radius in the owner's
// results.  Every consumer warp calls this between two CTA barriers (the
// list is complete).
static __device__ void fb_pool_work(const FbPool& P, const FrMapArgs& args, int W,
                                    unsigned char* arenas, int arena_bytes, int arena_off_big,
                                    char* my_big) {
  const int lane = lane_id();
  const BigLayout L = fr_big_layout(kMCap, kBinCap, W);
  const int count = *(volatile int*)P.count, count_big = *(volatile int*)P.count_big;
  (void)my_big;
  const float* fb = args.fb + (size_t)blockIdx.x * args.consumer_warps * args.fb_stride;
  // tasks have more than kCapL levels: two of 13..16 rows at once, one per
  // half-warp, then the larger ones (17..kMCap rows) by the whole warp
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(P.next, 2);
    t = __shfl_sync(kFull, t, 0);
    if (t >= count) break;
    const int task0 = P.tasks[t];
    const int task1 = t + 1 < count ? P.tasks[t + 1] : -1;
    const int task = (lane >> 4) ? task1 : task0;
    const int n = task >= 0 ? (task & 0xFF) : 0;
    const int owner = task >> 16, d = (task >> 8) & 0xFF;
    const float* src = n > 0 ? fb + (size_t)owner * args.fb_stride + (size_t)d * kFbDir : fb;
    const float rho = pool_rho_half16(src, n);
    if ((lane & 15) == 0 && n > 0) {
      float* mres = (float*)(arenas + (size_t)owner * arena_bytes + arena_off_big + L.mres);
      mres[d] = rho;
    }
    __syncwarp();
  }
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(P.next_big, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= count_big) break;
    const int task = P.tasks[kFbTasks - 1 - t];
    const int owner = task >> 16, d = (task >> 8) & 0xFF, n = task & 0xFF;
    const float* src = fb + (size_t)owner * args.fb_stride + (size_t)d * kFbDir;
    const float rho = pool_rho_regs<kMCap>(src, n);
    if (lane == 0) {
      float* mres = (float*)(arenas + (size_t)owner * arena_bytes + arena_off_big + L.mres);
      mres[d] = rho;
    }
    __syncwarp();
  }
}

// pool: many-level MCC solves go to the CTA pool (windows in shared memory);
// null solves them inline.  The caller runs glcm_finish after the pool.
// GLCM of windows of side S in {3, 5, 7} with at most DirLayout<S>::kLv levels
// (distance 1, per-direction aggregation): lane d < 13 takes direction d
// through every step on its own -- pair counts from the level sets, the
// entry sums, its MCC slot, the difference and sum distributions and the 26
// per-direction features -- so no step needs a warp reduction; the direction
// means are then taken per feature in direction order.  Each lane keeps its
// pair counts in a row of a shared table; the distributions are read from it
// in two orders of the level pairs fixed once per voxel (by gray-level
// difference, by gray-level sum; ties by pair index), so that every class of
// equal difference (sum) is contiguous and its count is final at its last
// pair.
// Layout of the path, per window side: up to 16 levels.  Sides 3 and 5 keep
// everything in the shared-memory big region, with byte pair counts (a
// direction of a side-5 window has at most 100 voxel pairs, so a count
// 2n <= 200).  Side 7 needs 16-bit counts, and its count rows fill the big
// region up to the MCC bookkeeping, so its level sets, marginals, pair orders
// and class counts go to the window-key buffer (free once first order is
// done; 512 keys, 2 KB, at side 7).  Count rows have an odd number of words
// and the marginals are level-major, so the 13 lanes touch distinct banks.
template <int S>
struct DirLayout {
  static constexpr int kLv = 16;
  static constexpr int kPairs = kLv * (kLv + 1) / 2;  // 136
  using Cnt = typename std::conditional<(S <= 5), uint8_t, uint16_t>::type;
  static constexpr bool kSplit = S == 7;              // side tables in the key buffer
  static constexpr int kRow = S <= 5 ? 140 : 138;     // counts per row
  static constexpr int kMg = S <= 5 ? 320 : 896;      // marginals [kLv][13]
  static constexpr int kW = S <= 5 ? 764 : 0;         // count rows (big region)
  static constexpr int kRowsEnd = kW + 13 * kRow * (int)sizeof(Cnt);
  static constexpr int kOrd = S <= 5 ? kRowsEnd : kMg + kLv * 13 * 2;
  static constexpr int kOrdLen = (kPairs + 3) & ~3;
  static constexpr int kCnt = kOrd + 4 * kOrdLen;
  static constexpr int kSideEnd = kCnt + 192;
  static constexpr int kBytes = ((kSplit ? kRowsEnd : kSideEnd) + 15) / 16 * 16;  // of big
};

template <int S>
__device__ void glcm_dir_lanes(const Win& w, const Arena& A, const FrJob& job,
                               int32_t* dbg_glcm, const FbPool* pool) {
  using W = typename SliceT<S>::W;
  using Lay = DirLayout<S>;
  using Cnt = typename Lay::Cnt;
  constexpr int kRounds = (Lay::kPairs + 31) / 32;
  static_assert(Lay::kLv * S * sizeof(W) <= Lay::kMg, "level sets");
  static_assert(Lay::kMg + Lay::kLv * 13 * 2 <= (Lay::kSplit ? Lay::kOrd : Lay::kW), "marginals");
  static_assert(13 * 27 * 4 <= Lay::kRowsEnd - Lay::kW, "per-direction features over the rows");
  static_assert(Lay::kBytes <= 3648, "below the MCC bookkeeping");
  static_assert(!Lay::kSplit || Lay::kSideEnd <= 512 * 4, "side tables in the side-7 key buffer");
  static_assert(S > 5 || 2 * S * S * (S - 1) < 256, "byte counts");
  const int lane = lane_id();
  const int m = w.m;
  const int npairs = m * (m + 1) / 2;
  const bool want_mcc = (job.families & kFamMCC) != 0;
  char* const side = Lay::kSplit ? (char*)A.kb : A.big;  // region of the side tables
  W* Lsm = (W*)side;                                    // [m][S] level sets
  uint16_t* mg = (uint16_t*)(side + Lay::kMg);          // [kLv][13] marginals
  Cnt* wt = (Cnt*)(A.big + Lay::kW);                    // [13][kRow] pair counts
  uint8_t* kord = (uint8_t*)(side + Lay::kOrd);         // pair at each difference position
  uint8_t* sord = kord + Lay::kOrdLen;                  // pair at each sum position
  uint8_t* kpos = sord + Lay::kOrdLen;                  // difference | 0x80 at a class end
  uint8_t* spos = kpos + Lay::kOrdLen;                  // sum - 2 lev0 | 0x80 at a class end
  uint8_t* cntk = (uint8_t*)(side + Lay::kCnt);         // [64] by difference
  uint8_t* cnts = cntk + 64;                            // [128] by sum - 2 lev0
  float* fvd = (float*)(A.big + Lay::kW);               // [13][27], after the rows are read
  int* mn = (int*)(A.big + A.L.mn);
  float* mres = (float*)(A.big + A.L.mres);
  float* slots = (float*)(A.big + A.L.slots);
  float2* csn = (float2*)(A.big + A.L.csn);
  int* cst = (int*)(A.big + A.L.cst);
  acc_reset(A);
  for (int q = lane; q < 48; q += 32) ((unsigned*)cntk)[q] = 0u;
  W Lm[S], Vm[S];
  slice_masks<S>(w, A, Lm, Vm);
  if (lane < m)
#pragma unroll
    for (int z = 0; z < S; ++z) Lsm[lane * S + z] = Lm[z];
  if (lane < kNumDirs) cst[lane] = 0;
  __syncwarp();
  // the two orders of the level pairs: counting sort by value (difference
  // k <= 63, sum s - 2 lev0 <= 126), ties by pair index
  int pk_[kRounds], ps_[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int t = 32 * r + lane;
    pk_[r] = ps_[r] = -1;
    if (t < npairs) {
      int a, b;
      pair_of(t, m, a, b);
      pk_[r] = (int)A.lev[b] - (int)A.lev[a];
      ps_[r] = (int)A.lev[a] + (int)A.lev[b] - 2 * w.lev0;
    }
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {  // class sizes: the leader of each group adds
    const bool v = pk_[r] >= 0;
    const unsigned act = __ballot_sync(kFull, v);
    if (v) {
      const unsigned gk = __match_any_sync(act, pk_[r]), gs = __match_any_sync(act, ps_[r]);
      if ((gk & lanemask_lt()) == 0) cntk[pk_[r]] += (uint8_t)__popc(gk);
      if ((gs & lanemask_lt()) == 0) cnts[ps_[r]] += (uint8_t)__popc(gs);
    }
    __syncwarp();
  }
  {  // exclusive prefix sums: class starts (64 differences: 2 per lane;
     // 128 sums: 4 per lane)
    const int k0 = cntk[2 * lane], k1 = cntk[2 * lane + 1];
    const int s0 = cnts[4 * lane], s1 = cnts[4 * lane + 1], s2 = cnts[4 * lane + 2],
              s3 = cnts[4 * lane + 3];
    int ik = k0 + k1, is = s0 + s1 + s2 + s3;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int yk = __shfl_up_sync(kFull, ik, o), ys = __shfl_up_sync(kFull, is, o);
      if (lane >= o) {
        ik += yk;
        is += ys;
      }
    }
    const int ek = ik - (k0 + k1), es = is - (s0 + s1 + s2 + s3);
    __syncwarp();
    cntk[2 * lane] = (uint8_t)ek;
    cntk[2 * lane + 1] = (uint8_t)(ek + k0);
    cnts[4 * lane] = (uint8_t)es;
    cnts[4 * lane + 1] = (uint8_t)(es + s0);
    cnts[4 * lane + 2] = (uint8_t)(es + s0 + s1);
    cnts[4 * lane + 3] = (uint8_t)(es + s0 + s1 + s2);
    __syncwarp();
  }
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {  // positions: class start + rank in pair order
    const bool v = pk_[r] >= 0;
    const unsigned act = __ballot_sync(kFull, v);
    int posk = 0, poss = 0;
    unsigned gk = 0, gs = 0;
    if (v) {
      gk = __match_any_sync(act, pk_[r]);
      gs = __match_any_sync(act, ps_[r]);
      posk = cntk[pk_[r]] + __popc(gk & lanemask_lt());
      poss = cnts[ps_[r]] + __popc(gs & lanemask_lt());
      kord[posk] = (uint8_t)(32 * r + lane);
      kpos[posk] = (uint8_t)pk_[r];
      sord[poss] = (uint8_t)(32 * r + lane);
      spos[poss] = (uint8_t)ps_[r];
    }
    __syncwarp();
    if (v) {
      if ((gk & lanemask_lt()) == 0) cntk[pk_[r]] += (uint8_t)__popc(gk);
      if ((gs & lanemask_lt()) == 0) cnts[ps_[r]] += (uint8_t)__popc(gs);
    }
    __syncwarp();
  }
  {  // mark the last position of every class
    int fk[kRounds], fs[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int p = 32 * r + lane;
      fk[r] = fs[r] = 0;
      if (p < npairs) {
        fk[r] = (p == npairs - 1 || kpos[p + 1] != kpos[p]) ? 0x80 : 0;
        fs[r] = (p == npairs - 1 || spos[p + 1] != spos[p]) ? 0x80 : 0;
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int p = 32 * r + lane;
      if (p < npairs) {
        kpos[p] |= (uint8_t)fk[r];
        spos[p] |= (uint8_t)fs[r];
      }
    }
    __syncwarp();
  }
  // lanes d and d + 16 share direction d: both take the marginals; lane h
  // takes the pair rows a = h, h + 2, ..., their sums meet by one exchange;
  // lane 0 of the pair reads the difference order, lane 1 the sum order
  const int d = lane & 15, h = lane >> 4;
  const unsigned pm = (1u << d) | (1u << (d + 16));
  constexpr unsigned kPairLanes = ((1u << kNumDirs) - 1u) * 0x10001u;
  if (d < kNumDirs) {
    int dz, dy, dx;
    dir_of(d, dz, dy, dx);
    const SliceDir<S> D(dz, dy, dx);
    W fV[S], bV[S];
    D.fwd(Vm, fV);
    D.bwd(Vm, bV);
    unsigned npz = 0;
#pragma unroll
    for (int z = 0; z < S; ++z) npz += (unsigned)popc_w<W>(Vm[z] & fV[z]);
    const int T = 2 * (int)npz;
    float fval[26];
#pragma unroll
    for (int f = 0; f < 26; ++f) fval[f] = kNaNf;
    if (T == 0) {
      if (!h) {
        mn[d] = 0;
        mres[d] = kNaNf;
      }
    } else {
      const float fT = (float)T, fT2 = fT * fT, invT = __fdividef(1.f, fT);
      Cnt* wrow = wt + d * Lay::kRow;
      // marginals c_a = |L_a & fwd(V)| + |L_a & bwd(V)| (both lanes)
      unsigned m1 = 0, m2 = 0, pmask = 0;
      float hx = 0.f;
      for (int a = 0; a < m; ++a) {
        unsigned c = 0;
#pragma unroll
        for (int z = 0; z < S; ++z) {
          const W la = Lsm[a * S + z];
          c += (unsigned)(popc_w<W>(la & fV[z]) + popc_w<W>(la & bV[z]));
        }
        if (!h) mg[a * kNumDirs + d] = (uint16_t)c;
        if (c) {
          const unsigned i = A.lev[a];
          m1 += i * c;
          m2 += i * i * c;
          hx += ent_term((int)c, T);
          pmask |= 1u << a;
        }
      }
      const int present = __popc(pmask);
      // more than kCapL present levels: the dense S - u u^T over the m
      // compact levels goes to this warp's global scratch and the solve to
      // the CTA pool (which writes mres[d]); else the register solve's slot
      const bool many = want_mcc && present > kCapL;
      const bool slot = want_mcc && present >= 2 && !many;
      float* P = slots + d * kSlot;
      // packed upper triangle over the m compact levels (pair index t)
      float* Sm = many ? pool->scratch + (size_t)d * kFbDir : nullptr;
      if (slot)
        for (int t = h; t < kSlot; t += 2) P[t] = 0.f;
      if (!h) {
        mn[d] = slot ? present : 0;
        if (!slot) mres[d] = kNaNf;
        if (many) pool_list(pool, d, m);
      }
      __syncwarp(pm);
      unsigned a1 = 0, e2 = 0, maxc = 0;
      unsigned long long mi0 = 0;
      float hxy = 0.f, mi = 0.f;
      for (int a = h; a < m; a += 2) {
        W la[S], fa[S], ba[S];
#pragma unroll
        for (int z = 0; z < S; ++z) la[z] = Lsm[a * S + z];
        D.fwd(la, fa);
        D.bwd(la, ba);
        const int ca = mg[a * kNumDirs + d];
        const unsigned i = A.lev[a];
        const int pa = __popc(pmask & ((1u << a) - 1u));
        int t = a * m - ((a * (a - 1)) >> 1);  // pair (a, a)
        for (int b = a; b < m; ++b, ++t) {
          int n = 0;
          if (b == a) {
#pragma unroll
            for (int z = 0; z < S; ++z) n += popc_w<W>(la[z] & fa[z]);
          } else {
#pragma unroll
            for (int z = 0; z < S; ++z) {
              const W lb = Lsm[b * S + z];
              n += popc_w<W>(lb & fa[z]) + popc_w<W>(lb & ba[z]);
            }
          }
          wrow[t] = (uint16_t)(2 * n);  // the pair's weight in both distributions
          const int cb = mg[b * kNumDirs + d];
          if (!ca || !cb) {
            if (many) Sm[t] = 0.f;  // a level absent along d
            continue;
          }
          const unsigned mult = (a == b) ? 1u : 2u;
          const int pb = __popc(pmask & ((1u << b) - 1u));
          const long long cc = (long long)ca * cb;
          if (!n) {
            // an empty pair of present levels: q = p_a p_b enters MI, and
            // S - u u^T is dense there (-u_a u_b)
            mi0 += mult * (unsigned long long)cc;
            const float v = (float)(-cc) * rsqrtf((float)ca * (float)cb) * invT;
            if (slot) P[pk(kCapL, pa, pb)] = v;
            if (many) Sm[t] = v;
            continue;
          }
          const unsigned j = A.lev[b];
          const int C = (a == b) ? 2 * n : n;
          a1 += mult * (unsigned)C * (i * j);
          e2 += mult * (unsigned)C * (unsigned)C;
          maxc = max(maxc, (unsigned)C);
          const float fm = (float)mult;
          hxy += fm * ent_term(C, T);
          const long long ct = (long long)C * T;
          if (ct != cc)  // p = p_x p_y exactly contributes nothing
            mi += fm * __fdividef((float)cc, fT2) * kl_term(__fdividef((float)(ct - cc), (float)cc));
          {
            const float v = (float)(ct - cc) * rsqrtf((float)ca * (float)cb) * invT;
            if (slot) P[pk(kCapL, pa, pb)] = v;
            if (many) Sm[t] = v;
          }
          if (dbg_glcm) {
            int32_t* g = dbg_glcm + (size_t)d * w.ng * w.ng;
            g[(i - 1) * w.ng + (j - 1)] = C;
            g[(j - 1) * w.ng + (i - 1)] = C;
          }
        }
      }
      // the two halves' sums (a + b == b + a: both lanes get the same value)
      a1 += __shfl_xor_sync(pm, a1, 16);
      e2 += __shfl_xor_sync(pm, e2, 16);
      maxc = max(maxc, __shfl_xor_sync(pm, maxc, 16));
      mi0 += __shfl_xor_sync(pm, mi0, 16);
      hxy += __shfl_xor_sync(pm, hxy, 16);
      mi += __shfl_xor_sync(pm, mi, 16);
      __syncwarp(pm);  // the row is complete
      if (!h) {
        // difference distribution: pairs in difference order, a class's
        // count is complete at its last pair
        const float ngf = (float)w.ng;
        unsigned dk = 0, dk2 = 0;
        float de = 0.f, idm = 0.f, idmn = 0.f, idd = 0.f, idn = 0.f, iv = 0.f;
        int acc = 0;
        for (int p = 0; p < npairs; ++p) {
          const int v = kpos[p];
          acc += wrow[kord[p]];
          if (!(v & 0x80)) continue;
          const int c = acc;
          acc = 0;
          if (!c) continue;
          const int k = v & 0x7F;
          const float fk = (float)k, fc = (float)c;
          dk += (unsigned)(k * c);
          dk2 += (unsigned)(k * k * c);
          de += ent_term(c, T);
          idm += __fdividef(fc, 1.f + fk * fk);
          idmn += __fdividef(fc, 1.f + __fdividef(fk * fk, ngf * ngf));
          idd += __fdividef(fc, 1.f + fk);
          idn += __fdividef(fc, 1.f + __fdividef(fk, ngf));
          if (k) iv += __fdividef(fc, fk * fk);
        }
        const float MI = (mi + __fdividef(u64_to_f32(mi0), fT2)) * 1.44269504088896341f;  // bits
        const long long var_num = (long long)T * (long long)m2 - (long long)m1 * m1;
        fval[0] = __fdividef((float)a1, fT);
        fval[1] = __fdividef((float)m1, fT);
        fval[5] = __fdividef((float)dk2, fT);
        fval[6] = lane_quot(s64_to_f32((long long)T * (long long)a1 - (long long)m1 * m1),
                            s64_to_f32(var_num));
        fval[7] = __fdividef((float)dk, fT);
        fval[8] = de;
        fval[9] = __fdividef(s64_to_f32((long long)T * (long long)dk2 - (long long)dk * dk), fT2);
        fval[10] = __fdividef((float)e2, fT2);
        fval[11] = hxy;
        fval[12] = lane_quot(-MI, hx);
        fval[13] = sqrtf(fmaxf(0.f, -expm1f(-2.f * MI)));
        fval[14] = __fdividef(idm, fT);
        fval[15] = __fdividef(idmn, fT);
        fval[16] = __fdividef(idd, fT);
        fval[17] = __fdividef(idn, fT);
        fval[18] = __fdividef(iv, fT);
        fval[19] = __fdividef((float)maxc, fT);
        fval[22] = __fdividef(s64_to_f32(var_num), fT2);
        fval[25] = __fdividef((float)dk, fT);
      } else {
        // sum distribution, the same way
        unsigned sk = 0, sk2 = 0;
        float se = 0.f, ce2 = 0.f, ce4 = 0.f;
        __int128 ce3 = 0;
        int acc = 0;
        for (int p = 0; p < npairs; ++p) {
          const int v = spos[p];
          acc += wrow[sord[p]];
          if (!(v & 0x80)) continue;
          const int c = acc;
          acc = 0;
          if (!c) continue;
          const int kk = (v & 0x7F) + 2 * w.lev0;
          sk += (unsigned)(kk * c);
          sk2 += (unsigned)(kk * kk) * (unsigned)c;
          se += ent_term(c, T);
          // T (k - 2 mu): |e| < 2^24 per direction
          const int e = T * kk - 2 * (int)m1;
          const float fe = (float)e, fe2 = fe * fe;
          ce2 += (float)c * fe2;
          ce4 += (float)c * fe2 * fe2;
          ce3 += (__int128)((long long)e * e) * ((long long)c * e);
        }
        fval[2] = __fdividef(ce4, fT * fT * fT * fT * fT);
        fval[3] = __fdividef(i128_to_f32(ce3), fT * fT * fT * fT);
        csn[d] = i128_to_ff(ce3);
        cst[d] = T;
        fval[4] = __fdividef(ce2, fT * fT * fT);
        fval[20] = __fdividef((float)sk, fT);
        fval[21] = se;
        fval[24] = __fdividef(s64_to_f32((long long)T * (long long)sk2 - (long long)sk * sk), fT2);
      }
    }
    // every direction's rows are read: the features may reuse them; each
    // lane of a pair writes its own features (fval[23], MCC, stays NaN)
    __syncwarp(kPairLanes);
    float* row = fvd + d * 27;
    const unsigned mine = h ? 0x0130001Cu : 0x02CFFFE3u;  // bit f: this lane's feature f
#pragma unroll
    for (int f = 0; f < 26; ++f)
      if ((mine >> f) & 1u) row[f] = fval[f];
  }
  __syncwarp();
  // direction means, per feature in direction order (compensated)
  if (lane < 26) {
    float s = 0.f, c = 0.f;
    int n = 0;
    for (int d = 0; d < kNumDirs; ++d) {
      const float v = fvd[d * 27 + lane];
      if (!isnan(v)) {
        two_sum_add(s, c, v);
        ++n;
      }
    }
    A.facc[lane] = s;
    A.fcomp[lane] = c;
    A.nacc[lane] = n;
  }
  __syncwarp();
  // leave the region zero (the count-matrix path and the later families
  // expect it so)
  for (int q = lane; q < Lay::kBytes / 16; q += 32) ((uint4*)A.big)[q] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
}

static __device__ void glcm_family(const Win& w, const Arena& A, const FrJob& job,
                                   int32_t* dbg_glcm, const FbPool* pool) {
  if (A.mc != kMCap) pool = nullptr;
  // the lane-per-direction path: windows in shared memory, distance 1,
  // per-direction aggregation; more than kCapL present levels need the pool
  const bool want_mcc = (job.families & kFamMCC) != 0;
  if (A.mc == kMCap && A.L.mn >= 3648 && job.delta == 1 && job.agg != 1 &&
      (w.m <= kCapL || pool != nullptr || !want_mcc)) {
    if (w.s == 3 && w.m <= DirLayout<3>::kLv) return glcm_dir_lanes<3>(w, A, job, dbg_glcm, pool);
    if (w.s == 5 && w.m <= DirLayout<5>::kLv) return glcm_dir_lanes<5>(w, A, job, dbg_glcm, pool);
    if (w.s == 7 && w.m <= DirLayout<7>::kLv) return glcm_dir_lanes<7>(w, A, job, dbg_glcm, pool);
  }
  if (w.m <= 32 && job.delta == 1 && job.agg != 1) {
    if (w.s == 3) return glcm_family_impl<3>(w, A, job, dbg_glcm, pool);
    if (w.s == 5) return glcm_family_impl<5>(w, A, job, dbg_glcm, pool);
    if (w.s == 7) return glcm_family_impl<7>(w, A, job, dbg_glcm, pool);
  }
  glcm_family_impl<0>(w, A, job, dbg_glcm, pool);
}

// ------------------------------------------------------------------ GLRLM
// GLRLM of windows of side S <= 5 with at most 32 levels: lane a counts the
// runs of level a along each direction from its level set: starts are the
// voxels whose predecessor u - d is not in the set, R_j the voxels that begin
// a chain of j, so runs of length >= j number |starts & R_j|.
template <int S>
__device__ void glrlm_masks(const Win& w, const Arena& A, bool merged, int32_t* dbg_glrlm) {
  using W = typename SliceT<S>::W;
  const int lane = lane_id();
  W L[S], V[S];
  slice_masks<S>(w, A, L, V);
  (void)V;
  const bool ok = lane < w.m;
  const unsigned i = ok ? (unsigned)A.lev[lane] : 1u;
  const float fi2 = (float)(i * i), inv_i2 = __fdividef(1.f, fi2);
  const float nvf = merged ? (float)(kNumDirs * w.nv) : (float)w.nv;
  acc_reset(A);
  unsigned h[S];
#pragma unroll
  for (int j = 0; j < S; ++j) h[j] = 0u;
  for (int di = 0; di < kNumDirs; ++di) {
    const SliceDir<S> D(c_dirs[di][0], c_dirs[di][1], c_dirs[di][2]);
    W st[S], R[S], T[S];
    D.bwd(L, T);
    unsigned c[S + 1];
    c[0] = 0u;
#pragma unroll
    for (int z = 0; z < S; ++z) {
      st[z] = L[z] & ~T[z];
      R[z] = L[z];
      c[0] += (unsigned)popc_w<W>(st[z]);
    }
#pragma unroll
    for (int j = 1; j < S; ++j) {
      D.fwd(R, T);
      c[j] = 0u;
#pragma unroll
      for (int z = 0; z < S; ++z) {
        R[z] = L[z] & T[z];
        c[j] += (unsigned)popc_w<W>(st[z] & R[z]);
      }
    }
    c[S] = 0u;
#pragma unroll
    for (int j = 0; j < S; ++j) h[j] += c[j] - c[j + 1];  // runs of length j + 1
    if (merged && di < kNumDirs - 1) continue;
    const int ds = merged ? 0 : di;
    unsigned row = 0, si = 0, si2 = 0, sj = 0, sj2 = 0;
    float fs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sre lgl srl srh lrl lrh
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const unsigned cnt = h[j];
      const unsigned J = (unsigned)(j + 1);
      const float fc = (float)cnt, fj2 = (float)(J * J), inv_j2 = 1.f / (float)(J * J);
      row += cnt;
      sj += cnt * J;
      sj2 += cnt * J * J;
      fs[0] += fc * inv_j2;
      fs[1] += fc * inv_i2;
      fs[2] += fc * inv_i2 * inv_j2;
      fs[3] += fc * fi2 * inv_j2;
      fs[4] += fc * fj2 * inv_i2;
      fs[5] += fc * fi2 * fj2;
      if (dbg_glrlm && cnt) dbg_glrlm[((size_t)ds * w.ng + (i - 1)) * w.s + j] = (int)cnt;
    }
    si = row * i;
    si2 = row * i * i;
    const unsigned nr = redux_u32(row);
    unsigned rlnu = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const unsigned col = redux_u32(h[j]);
      rlnu += col * col;
    }
    float ent = 0.f;
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (h[j]) ent += ent_term((int)h[j], (int)nr);
    const unsigned glnu = redux_u32(row * row);
    si = redux_u32(si);
    si2 = redux_u32(si2);
    sj = redux_u32(sj);
    sj2 = redux_u32(sj2);
    float fsr[7] = {fs[0], fs[1], fs[2], fs[3], fs[4], fs[5], ent};
    warp_sum_f32x<7>(fsr);
    const float N = (float)nr;
    float num = kNaNf, den = N;
    if (lane == 0) { num = fsr[0]; }
    if (lane == 1) { num = (float)sj2; }
    if (lane == 2) { num = (float)glnu; }
    if (lane == 3) { num = (float)glnu; den = N * N; }
    if (lane == 4) { num = (float)rlnu; }
    if (lane == 5) { num = (float)rlnu; den = N * N; }
    if (lane == 6) { num = N; den = nvf; }
    if (lane == 7) { num = (float)((long long)nr * si2 - (long long)si * si); den = N * N; }
    if (lane == 8) { num = (float)((long long)nr * sj2 - (long long)sj * sj); den = N * N; }
    if (lane == 9) { num = fsr[6]; den = 1.f; }
    if (lane == 10) { num = fsr[1]; }
    if (lane == 11) { num = (float)si2; }
    if (lane == 12) { num = fsr[2]; }
    if (lane == 13) { num = fsr[3]; }
    if (lane == 14) { num = fsr[4]; }
    if (lane == 15) { num = fsr[5]; }
    acc_lane(A, 16, lane_quot(num, den));
#pragma unroll
    for (int j = 0; j < S; ++j) h[j] = 0u;
  }
  acc_store(A, 16, 42);
}

// GLRLM feature f (0..15) of one direction from its run totals; NaN where
// the denominator is 0.  Every lane evaluates the chain for its own f.
__device__ __forceinline__ float glrlm_feature(int f, const float (&fsr)[7], unsigned nr,
                                               unsigned sj2, unsigned glnu, unsigned rlnu,
                                               unsigned si, unsigned si2, unsigned sj, float nvf) {
  const float N = (float)nr;
  float num = kNaNf, den = N;
  if (f == 0) { num = fsr[0]; }
  if (f == 1) { num = (float)sj2; }
  if (f == 2) { num = (float)glnu; }
  if (f == 3) { num = (float)glnu; den = N * N; }
  if (f == 4) { num = (float)rlnu; }
  if (f == 5) { num = (float)rlnu; den = N * N; }
  if (f == 6) { num = N; den = nvf; }
  if (f == 7) { num = (float)((long long)nr * si2 - (long long)si * si); den = N * N; }
  if (f == 8) { num = (float)((long long)nr * sj2 - (long long)sj * sj); den = N * N; }
  if (f == 9) { num = fsr[6]; den = 1.f; }
  if (f == 10) { num = fsr[1]; }
  if (f == 11) { num = (float)si2; }
  if (f == 12) { num = fsr[2]; }
  if (f == 13) { num = fsr[3]; }
  if (f == 14) { num = fsr[4]; }
  if (f == 15) { num = fsr[5]; }
  return lane_quot(num, den);
}

// GLRLM (per-direction aggregation) of windows of side S <= 5 with at most
// 16 levels: the warp splits into segments of Wd = 8 or 16 lanes, one
// direction per segment and one level per lane, so a pass covers 32 / Wd
// directions (4 or 2) instead of one.  Run counts as in glrlm_masks; the
// per-direction totals are segment reductions; each lane finishes 16 / Wd of
// the direction's features and keeps their direction sums (compensated) in
// registers; the segments' sums are merged at the end.
template <int S>
__device__ void glrlm_masks_packed(const Win& w, const Arena& A, int32_t* dbg_glrlm) {
  using W = typename SliceT<S>::W;
  const int lane = lane_id();
  W L0[S], V[S];
  slice_masks<S>(w, A, L0, V);
  (void)V;
  const int m = w.m;
  const int Wd = m <= 8 ? 8 : 16;
  const int G = 32 / Wd;
  const int sl = lane & (Wd - 1), g = lane / Wd;
  const unsigned segmask = ((1u << Wd) - 1u) << (g * Wd);
  const bool ok = sl < m;
  W L[S];
#pragma unroll
  for (int z = 0; z < S; ++z) {
    const W v = __shfl_sync(kFull, L0[z], sl);
    L[z] = ok ? v : (W)0;
  }
  const unsigned i = ok ? (unsigned)A.lev[sl] : 1u;
  const float fi2 = (float)(i * i), inv_i2 = __fdividef(1.f, fi2);
  const float nvf = (float)w.nv;
  float as[2] = {0.f, 0.f}, ac[2] = {0.f, 0.f};
  int an[2] = {0, 0};
  for (int d0 = 0; d0 < kNumDirs; d0 += G) {
    const int di = d0 + g;
    const bool dok = di < kNumDirs;
    int dz, dy, dx;
    dir_of(dok ? di : 0, dz, dy, dx);
    const SliceDir<S> D(dz, dy, dx);
    W st[S], R[S], T[S];
    D.bwd(L, T);
    unsigned c[S + 1];
    c[0] = 0u;
#pragma unroll
    for (int z = 0; z < S; ++z) {
      st[z] = L[z] & ~T[z];
      R[z] = L[z];
      c[0] += (unsigned)popc_w<W>(st[z]);
    }
#pragma unroll
    for (int j = 1; j < S; ++j) {
      D.fwd(R, T);
      c[j] = 0u;
#pragma unroll
      for (int z = 0; z < S; ++z) {
        R[z] = L[z] & T[z];
        c[j] += (unsigned)popc_w<W>(st[z] & R[z]);
      }
    }
    c[S] = 0u;
    unsigned h[S];
    unsigned row = 0, sj = 0, sj2 = 0;
    float fs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sre lgl srl srh lrl lrh
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const unsigned cnt = c[j] - c[j + 1];  // runs of length j + 1
      h[j] = cnt;
      const unsigned J = (unsigned)(j + 1);
      const float fc = (float)cnt, fj2 = (float)(J * J), inv_j2 = 1.f / (float)(J * J);
      row += cnt;
      sj += cnt * J;
      sj2 += cnt * J * J;
      fs[0] += fc * inv_j2;
      fs[1] += fc * inv_i2;
      fs[2] += fc * inv_i2 * inv_j2;
      fs[3] += fc * fi2 * inv_j2;
      fs[4] += fc * fj2 * inv_i2;
      fs[5] += fc * fi2 * fj2;
      if (dbg_glrlm && cnt && dok)
        dbg_glrlm[((size_t)di * w.ng + (i - 1)) * w.s + j] = (int)cnt;
    }
    const unsigned nr = __reduce_add_sync(segmask, row);
    unsigned rlnu = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const unsigned col = __reduce_add_sync(segmask, h[j]);
      rlnu += col * col;
    }
    float ent = 0.f;
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (h[j]) ent += ent_term((int)h[j], (int)nr);
    const unsigned glnu = __reduce_add_sync(segmask, row * row);
    const unsigned si = __reduce_add_sync(segmask, row * i);
    const unsigned si2 = __reduce_add_sync(segmask, row * i * i);
    const unsigned sjt = __reduce_add_sync(segmask, sj);
    const unsigned sj2t = __reduce_add_sync(segmask, sj2);
    float fsr[7] = {fs[0], fs[1], fs[2], fs[3], fs[4], fs[5], ent};
    for (int o = Wd >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 7; ++k) fsr[k] += __shfl_xor_sync(kFull, fsr[k], o);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int f = sl + k * Wd;
      if (f < 16) {
        const float v = glrlm_feature(f, fsr, nr, sj2t, glnu, rlnu, si, si2, sjt, nvf);
        if (dok && !isnan(v)) {
          two_sum_add(as[k], ac[k], v);
          ++an[k];
        }
      }
    }
  }
  // merge the segments' direction sums
  for (int o = Wd; o < 32; o <<= 1)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float so = __shfl_xor_sync(kFull, as[k], o), co = __shfl_xor_sync(kFull, ac[k], o);
      const int no = __shfl_xor_sync(kFull, an[k], o);
      two_sum_add(as[k], ac[k], so);
      ac[k] += co;
      an[k] += no;
    }
  if (g == 0)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int f = sl + k * Wd;
      if (f < 16) A.fv[42 + f] = an[k] ? __fdividef(as[k] + ac[k], (float)an[k]) : kNaNf;
    }
  __syncwarp();
}

// GLRLM of windows of side S <= 5 with at most 16 levels (per-direction
// aggregation): lanes d and d + 16 take direction d.  The set E_d of VOI
// voxels whose successor u + d has the same level is built once per direction
// (the union over levels of L_a & fwd(L_a)); run starts are V minus bwd(E_d),
// and R_j = E_d & fwd(R_{j-1}) marks the voxels that begin a chain of j + 1
// equal levels, for every level at once.  Each lane of the pair then counts
// the runs of its levels (a = h, h + 2, ...) as |L_a & starts & R_j|, keeps
// their per-cell terms, and the pair's sums meet by one exchange each; the
// direction means follow per feature in direction order.
constexpr int kRunLevels = 16;
// byte offsets in the shared-memory big region (everything below byte 2512 is
// cleared on exit; the run-count cells from byte 3264 lie in bytes that no
// family needs zero: GLCM's solver scratch and MCC slots, written before use)
constexpr int kRunR = 320, kRunS0 = 1360, kRunF = 1620, kRunClear = 2512, kRunCells = 3264;

template <int S>
__device__ void glrlm_dir_lanes(const Win& w, const Arena& A, int32_t* dbg_glrlm) {
  using W = typename SliceT<S>::W;
  static_assert(sizeof(W) == 4 && kRunLevels * S * 4 <= kRunR, "level sets");
  static_assert(kRunR + 13 * (S - 1) * S * 4 <= kRunS0 && kRunS0 + 13 * S * 4 <= kRunF, "sets");
  static_assert(kRunF + 13 * 17 * 4 <= kRunClear, "feature rows");
  static_assert(kRunCells + 32 * 8 * S * 2 <= 8000, "run-count cells");
  const int lane = lane_id();
  const int m = w.m;
  W* Lsm = (W*)A.big;                              // [m][S]
  W* Rsm = (W*)(A.big + kRunR);                    // [13][S - 1][S]: R_1 .. R_{S-1}
  W* S0sm = (W*)(A.big + kRunS0);                  // [13][S] run starts
  float* fvd = (float*)(A.big + kRunF);            // [13][17] features
  uint16_t* cells = (uint16_t*)(A.big + kRunCells);  // [32 lanes][8][S] run counts
  W Lm[S], Vm[S];
  slice_masks<S>(w, A, Lm, Vm);
  if (lane < m)
#pragma unroll
    for (int z = 0; z < S; ++z) Lsm[lane * S + z] = Lm[z];
  __syncwarp();
  const int d = lane & 15, h = lane >> 4;
  const unsigned pm = (1u << d) | (1u << (d + 16));
  if (d < kNumDirs) {
    int dz, dy, dx;
    dir_of(d, dz, dy, dx);
    const SliceDir<S> D(dz, dy, dx);
    // E_d over this lane's levels, then the pair's union
    W E[S];
#pragma unroll
    for (int z = 0; z < S; ++z) E[z] = 0;
    for (int a = h; a < m; a += 2) {
      W la[S], fa[S];
#pragma unroll
      for (int z = 0; z < S; ++z) la[z] = Lsm[a * S + z];
      D.fwd(la, fa);
#pragma unroll
      for (int z = 0; z < S; ++z) E[z] |= la[z] & fa[z];
    }
#pragma unroll
    for (int z = 0; z < S; ++z) E[z] |= __shfl_xor_sync(pm, E[z], 16);
    W* Rd = Rsm + d * (S - 1) * S;
    W* S0 = S0sm + d * S;
    if (!h) {
      W T[S], R[S];
      D.bwd(E, T);
#pragma unroll
      for (int z = 0; z < S; ++z) {
        S0[z] = Vm[z] & ~T[z];
        R[z] = E[z];
      }
#pragma unroll
      for (int j = 1; j < S; ++j) {
#pragma unroll
        for (int z = 0; z < S; ++z) Rd[(j - 1) * S + z] = R[z];
        if (j + 1 < S) {
          D.fwd(R, T);
#pragma unroll
          for (int z = 0; z < S; ++z) R[z] = E[z] & T[z];
        }
      }
    }
    __syncwarp(pm);
    // runs of this lane's levels: c_j = |L_a & starts & R_j|, runs of length
    // exactly j + 1 = c_j - c_{j+1}
    uint16_t* mycells = cells + lane * 8 * S;
    unsigned nr = 0, sj = 0, sj2 = 0, glnu = 0, si = 0, si2 = 0;
    unsigned col[S];
#pragma unroll
    for (int j = 0; j < S; ++j) col[j] = 0;
    float fs[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sre lgl srl srh lrl lrh
    int q = 0;
    for (int a = h; a < m; a += 2, ++q) {
      W base[S];
      unsigned c[S + 1];
      c[0] = 0;
#pragma unroll
      for (int z = 0; z < S; ++z) {
        base[z] = Lsm[a * S + z] & S0[z];
        c[0] += (unsigned)popc_w<W>(base[z]);
      }
#pragma unroll
      for (int j = 1; j < S; ++j) {
        c[j] = 0;
#pragma unroll
        for (int z = 0; z < S; ++z) c[j] += (unsigned)popc_w<W>(base[z] & Rd[(j - 1) * S + z]);
      }
      c[S] = 0;
      const unsigned i = A.lev[a];
      const float fi2 = (float)(i * i), inv_i2 = __fdividef(1.f, fi2);
      unsigned row = 0;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const unsigned cnt = c[j] - c[j + 1];
        mycells[q * S + j] = (uint16_t)cnt;
        const unsigned J = (unsigned)(j + 1);
        const float fc = (float)cnt, fj2 = (float)(J * J), inv_j2 = 1.f / (float)(J * J);
        row += cnt;
        col[j] += cnt;
        sj += cnt * J;
        sj2 += cnt * J * J;
        fs[0] += fc * inv_j2;
        fs[1] += fc * inv_i2;
        fs[2] += fc * inv_i2 * inv_j2;
        fs[3] += fc * fi2 * inv_j2;
        fs[4] += fc * fj2 * inv_i2;
        fs[5] += fc * fi2 * fj2;
        if (dbg_glrlm && cnt) dbg_glrlm[((size_t)d * w.ng + (i - 1)) * w.s + j] = (int)cnt;
      }
      nr += row;
      glnu += row * row;
      si += row * i;
      si2 += row * i * i;
    }
    // the pair's totals (integer sums, and a + b == b + a for the floats)
    nr += __shfl_xor_sync(pm, nr, 16);
    sj += __shfl_xor_sync(pm, sj, 16);
    sj2 += __shfl_xor_sync(pm, sj2, 16);
    glnu += __shfl_xor_sync(pm, glnu, 16);
    si += __shfl_xor_sync(pm, si, 16);
    si2 += __shfl_xor_sync(pm, si2, 16);
    unsigned rlnu = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      const unsigned cj = col[j] + __shfl_xor_sync(pm, col[j], 16);
      rlnu += cj * cj;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) fs[k] += __shfl_xor_sync(pm, fs[k], 16);
    float ent = 0.f;
    for (int qq = 0; qq < q; ++qq)
#pragma unroll
      for (int j = 0; j < S; ++j) {
        const int cnt = mycells[qq * S + j];
        if (cnt) ent += ent_term(cnt, (int)nr);
      }
    ent += __shfl_xor_sync(pm, ent, 16);
    const float fsr[7] = {fs[0], fs[1], fs[2], fs[3], fs[4], fs[5], ent};
    const float nvf = (float)w.nv;
    float* row = fvd + d * 17;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int f = 8 * h + k;
      row[f] = glrlm_feature(f, fsr, nr, sj2, glnu, rlnu, si, si2, sj, nvf);
    }
  }
  __syncwarp();
  // direction means, per feature in direction order (compensated)
  if (lane < 16) {
    float s = 0.f, c = 0.f;
    int n = 0;
    for (int dd = 0; dd < kNumDirs; ++dd) {
      const float v = fvd[dd * 17 + lane];
      if (!isnan(v)) {
        two_sum_add(s, c, v);
        ++n;
      }
    }
    A.fv[42 + lane] = n ? __fdividef(s + c, (float)n) : kNaNf;
  }
  __syncwarp();
  for (int t = lane; t < kRunClear / 16; t += 32) ((uint4*)A.big)[t] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
}

// GLRLM of windows of side 7 with at most kMCap levels (per-direction
// aggregation), every count in registers: lanes d and d + 16 take direction
// d.  As in glrlm_dir_lanes, E_d (voxels whose successor u + d has the same
// level) is the pair's union over levels, the run starts are V minus
// bwd(E_d), and R_1 = E_d, R_{j+1} = E_d & fwd(R_j) mark the voxels that
// begin a chain of j + 1 equal levels.  The chain is walked once, j outer:
// at step j each lane counts c_j(a) = |L_a & starts & R_j| for its levels
// (a = h, h + 2, ...) and finishes the cells of length j, c_{j-1}(a) - c_j(a),
// keeping only the previous count per level.  The cell sums factor by
// length: the length weights (1/j^2, j^2) multiply per-length totals over
// levels (count, count/i^2, count i^2), so a cell costs one subtraction,
// one FMA, one integer multiply-add and its entropy term.  No run count is
// stored; the region keeps only the level sets and per-level constants.
constexpr int kRun7L = 0, kRun7Inv = 1536, kRun7I2 = 1664, kRun7F = 1792, kRun7Clear = 2688;

template <int S>
__device__ void glrlm_dir_regs(const Win& w, const Arena& A, int32_t* dbg_glrlm) {
  using W = typename SliceT<S>::W;
  constexpr int kQ = (kMCap + 1) / 2;  // levels per lane
  static_assert(kMCap * S * (int)sizeof(W) <= kRun7Inv - kRun7L, "level sets");
  static_assert(kRun7Inv + kMCap * 4 <= kRun7I2 && kRun7I2 + kMCap * 4 <= kRun7F, "tables");
  static_assert(kRun7F + 13 * 17 * 4 <= kRun7Clear, "feature rows");
  const int lane = lane_id();
  const int m = w.m;
  W* Lsm = (W*)(A.big + kRun7L);          // [m][S]
  float* inv_i2 = (float*)(A.big + kRun7Inv);  // [m] 1 / i^2
  unsigned* i2t = (unsigned*)(A.big + kRun7I2);  // [m] i^2
  float* fvd = (float*)(A.big + kRun7F);       // [13][17] features
  W Lm[S], Vm[S];
  slice_masks<S>(w, A, Lm, Vm);
  if (lane < m) {
#pragma unroll
    for (int z = 0; z < S; ++z) Lsm[lane * S + z] = Lm[z];
    const unsigned i = A.lev[lane];
    i2t[lane] = i * i;
    inv_i2[lane] = __fdividef(1.f, (float)(i * i));
  }
  __syncwarp();
  const int d = lane & 15, h = lane >> 4;
  const unsigned pm = (1u << d) | (1u << (d + 16));
  if (d < kNumDirs) {
    int dz, dy, dx;
    dir_of(d, dz, dy, dx);
    const SliceDir<S> D(dz, dy, dx);
    W E[S];
#pragma unroll
    for (int z = 0; z < S; ++z) E[z] = 0;
    for (int a = h; a < m; a += 2) {
      W la[S], fa[S];
#pragma unroll
      for (int z = 0; z < S; ++z) la[z] = Lsm[a * S + z];
      D.fwd(la, fa);
#pragma unroll
      for (int z = 0; z < S; ++z) E[z] |= la[z] & fa[z];
    }
#pragma unroll
    for (int z = 0; z < S; ++z) E[z] |= __shfl_xor_sync(pm, E[z], 16);
    W st[S], R[S];
    {
      W T[S];
      D.bwd(E, T);
#pragma unroll
      for (int z = 0; z < S; ++z) {
        st[z] = Vm[z] & ~T[z];
        R[z] = E[z];
      }
    }
    // every run has exactly one start: the direction's run total
    unsigned nr = 0;
#pragma unroll
    for (int z = 0; z < S; ++z) nr += (unsigned)popc_w<W>(st[z]);
    unsigned prev[kQ];
    unsigned live = 0;  // bit q: level h + 2 q has runs longer than the current j
    unsigned glnu = 0, si = 0, si2 = 0, sj = 0, sj2 = 0, rlnu = 0;
    float f_inv_i2 = 0.f, f_j = 0.f, f_j_inv_i2 = 0.f, f_j_i2 = 0.f, f_jj_inv_i2 = 0.f,
          f_jj_i2 = 0.f, ent = 0.f;
    // j = 0: runs starting at each level (the rows)
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const int a = h + 2 * q;
      unsigned c = 0;
      if (a < m) {
#pragma unroll
        for (int z = 0; z < S; ++z) c += (unsigned)popc_w<W>(Lsm[a * S + z] & st[z]);
        glnu += c * c;
        const unsigned ii = i2t[a];
        si2 += c * ii;
        si += c * (unsigned)A.lev[a];
        f_inv_i2 += (float)c * inv_i2[a];
      }
      prev[q] = c;
      if (c) live |= 1u << q;
    }
#pragma unroll
    for (int j = 1; j <= S; ++j) {
      // X = starts that begin a chain of j + 1 (empty past the window side)
      W X[S];
      if (j < S) {
#pragma unroll
        for (int z = 0; z < S; ++z) X[z] = st[z] & R[z];
      }
      // cells of length j: prev - c_j
      unsigned col = 0, ui2 = 0;
      float tinv = 0.f;
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int a = h + 2 * q;
        // a level without runs longer than j - 1 has none longer than j:
        // its counts stay zero and it is left out (a < m where live)
        if ((live >> q) & 1u) {
          unsigned c = 0;
          if (j < S) {
#pragma unroll
            for (int z = 0; z < S; ++z) c += (unsigned)popc_w<W>(Lsm[a * S + z] & X[z]);
          }
          const unsigned cnt = prev[q] - c;
          prev[q] = c;
          if (!c) live &= ~(1u << q);
          if (cnt) {
            col += cnt;
            ui2 += cnt * i2t[a];
            tinv += (float)cnt * inv_i2[a];
            ent += ent_term((int)cnt, (int)nr);
            if (dbg_glrlm)
              dbg_glrlm[((size_t)d * w.ng + (A.lev[a] - 1)) * w.s + (j - 1)] = (int)cnt;
          }
        }
      }
      const float fj2 = (float)(j * j), inv_j2 = 1.f / (float)(j * j);
      const unsigned colt = col + __shfl_xor_sync(pm, col, 16);
      rlnu += colt * colt;
      sj += col * (unsigned)j;
      sj2 += col * (unsigned)(j * j);
      f_j += (float)col * inv_j2;
      f_j_inv_i2 += tinv * inv_j2;
      f_j_i2 += (float)ui2 * inv_j2;
      f_jj_inv_i2 += tinv * fj2;
      f_jj_i2 += (float)ui2 * fj2;
      if (j + 1 < S) {
        W T[S];
        D.fwd(R, T);
#pragma unroll
        for (int z = 0; z < S; ++z) R[z] = E[z] & T[z];
      }
    }
    // the pair's totals (rlnu is already the pair's)
    glnu += __shfl_xor_sync(pm, glnu, 16);
    si += __shfl_xor_sync(pm, si, 16);
    si2 += __shfl_xor_sync(pm, si2, 16);
    sj += __shfl_xor_sync(pm, sj, 16);
    sj2 += __shfl_xor_sync(pm, sj2, 16);
    float fs[7] = {f_j, f_inv_i2, f_j_inv_i2, f_j_i2, f_jj_inv_i2, f_jj_i2, ent};
#pragma unroll
    for (int k = 0; k < 7; ++k) fs[k] += __shfl_xor_sync(pm, fs[k], 16);
    const float nvf = (float)w.nv;
    float* row = fvd + d * 17;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int f = 8 * h + k;
      row[f] = glrlm_feature(f, fs, nr, sj2, glnu, rlnu, si, si2, sj, nvf);
    }
  }
  __syncwarp();
  if (lane < 16) {
    float s = 0.f, c = 0.f;
    int n = 0;
    for (int dd = 0; dd < kNumDirs; ++dd) {
      const float v = fvd[dd * 17 + lane];
      if (!isnan(v)) {
        two_sum_add(s, c, v);
        ++n;
      }
    }
    A.fv[42 + lane] = n ? __fdividef(s + c, (float)n) : kNaNf;
  }
  __syncwarp();
  for (int t = lane; t < kRun7Clear / 16; t += 32) ((uint4*)A.big)[t] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
}

// merged: the 13 directions' runs go into one matrix, whose features are
// taken once (RunPercentage over 13 N_v: each voxel lies on one run per
// direction).
static __device__ void glrlm_family(const Win& w, const Arena& A, bool merged, int32_t* dbg_glrlm) {
  if (!merged && w.m <= kRunLevels && A.mc == kMCap) {
    if (w.s == 3) return glrlm_dir_lanes<3>(w, A, dbg_glrlm);
    if (w.s == 5) return glrlm_dir_lanes<5>(w, A, dbg_glrlm);
  }
  if (!merged && A.mc == kMCap && w.s == 7) return glrlm_dir_regs<7>(w, A, dbg_glrlm);
  if (!merged && w.m <= 16) {
    if (w.s == 3) return glrlm_masks_packed<3>(w, A, dbg_glrlm);
    if (w.s == 5) return glrlm_masks_packed<5>(w, A, dbg_glrlm);
  }
  if (w.m <= 32) {
    if (w.s == 3) return glrlm_masks<3>(w, A, merged, dbg_glrlm);
    if (w.s == 5) return glrlm_masks<5>(w, A, merged, dbg_glrlm);
  }
  const int lane = lane_id();
  const int m = w.m;
  int* hist = (int*)(A.big + A.L.rhist);  // [mc][16]
  int* lnc = (int*)(A.big + A.L.rlen);    // column sums when m > 32
  acc_reset(A);
  const float nvf = merged ? (float)(kNumDirs * w.nv) : (float)w.nv;
  int nr = 0;
  for (int di = 0; di < kNumDirs; ++di) {
    const int dz = c_dirs[di][0], dy = c_dirs[di][1], dx = c_dirs[di][2];
    const int off = dz * w.s2 + dy * w.s + dx;
    if (!merged) nr = 0;
    for (int base = 0; base < w.W; base += 32) {
      const int p = base + lane;
      int key = -1;
      if (p < w.W) {
        const int a = A.lvl[p];
        if (a) {
          int z, y, x;
          pos_to_zyx(w, p, z, y, x);
          if (!(in_cube(w, z - dz, y - dy, x - dx) && A.lvl[p - off] == a)) {
            int len = 1, q = p + off, zz = z + dz, yy = y + dy, xx = x + dx;
            while (in_cube(w, zz, yy, xx) && A.lvl[q] == a) {
              ++len;
              q += off;
              zz += dz;
              yy += dy;
              xx += dx;
            }
            key = (a - 1) * 16 + (len - 1);
          }
        }
      }
      const unsigned act = __ballot_sync(kFull, key >= 0);
      if (key >= 0) {
        const unsigned grp = __match_any_sync(act, key);
        if ((grp & lanemask_lt()) == 0) atomicAdd(&hist[key], __popc(grp));
      }
      nr += __popc(act);
    }
    __syncwarp();
    if (merged && di < kNumDirs - 1) continue;
    const int ds = merged ? 0 : di;  // record of this matrix
    // row walk: lane a owns gray level a; columns are run lengths
    unsigned si = 0, si2 = 0, sj = 0, sj2 = 0, glnu = 0, rlnu = 0;
    float fs[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sre lgl srl srh lrl lrh ent
    for (int a0 = 0; a0 < m; a0 += 32) {
      const int a = a0 + lane;
      const bool ok = a < m;
      const unsigned i = ok ? A.lev[a] : 1u;
      const float fi2 = (float)(i * i), inv_i2 = __fdividef(1.f, fi2);
      unsigned row = 0;
      for (int jl = 0; jl < w.s; ++jl) {
        const int c = ok ? hist[a * 16 + jl] : 0;
        const unsigned col = redux_u32((unsigned)c);
        if (m <= 32)
          rlnu += col * col;
        else if (lane == 0)
          lnc[jl] += (int)col;
        if (c) {
          hist[a * 16 + jl] = 0;
          const unsigned J = (unsigned)(jl + 1);
          const float fc = (float)c, fj2 = (float)(J * J), inv_j2 = __fdividef(1.f, fj2);
          row += (unsigned)c;
          si += (unsigned)c * i;
          si2 += (unsigned)c * i * i;
          sj += (unsigned)c * J;
          sj2 += (unsigned)c * J * J;
          fs[0] += fc * inv_j2;
          fs[1] += fc * inv_i2;
          fs[2] += fc * inv_i2 * inv_j2;
          fs[3] += fc * fi2 * inv_j2;
          fs[4] += fc * fj2 * inv_i2;
          fs[5] += fc * fi2 * fj2;
          fs[6] += ent_term(c, nr);
          if (dbg_glrlm) dbg_glrlm[((size_t)ds * w.ng + (i - 1)) * w.s + jl] = c;
        }
      }
      glnu += row * row;
    }
    if (m > 32) {
      __syncwarp();
      if (lane < 16) {
        const unsigned c = (unsigned)lnc[lane];
        lnc[lane] = 0;
        rlnu = c * c;
      }
      rlnu = redux_u32(rlnu);
    }
    si = redux_u32(si);
    si2 = redux_u32(si2);
    sj = redux_u32(sj);
    sj2 = redux_u32(sj2);
    glnu = redux_u32(glnu);
    warp_sum_f32x<7>(fs);
    const float N = (float)nr;
    float num = kNaNf, den = N;
    if (lane == 0) { num = fs[0]; }
    if (lane == 1) { num = (float)sj2; }
    if (lane == 2) { num = (float)glnu; }
    if (lane == 3) { num = (float)glnu; den = N * N; }
    if (lane == 4) { num = (float)rlnu; }
    if (lane == 5) { num = (float)rlnu; den = N * N; }
    if (lane == 6) { num = N; den = nvf; }
    if (lane == 7) { num = (float)((long long)nr * si2 - (long long)si * si); den = N * N; }
    if (lane == 8) { num = (float)((long long)nr * sj2 - (long long)sj * sj); den = N * N; }
    if (lane == 9) { num = fs[6]; den = 1.f; }
    if (lane == 10) { num = fs[1]; }
    if (lane == 11) { num = (float)si2; }
    if (lane == 12) { num = fs[2]; }
    if (lane == 13) { num = fs[3]; }
    if (lane == 14) { num = fs[4]; }
    if (lane == 15) { num = fs[5]; }
    acc_lane(A, 16, lane_quot(num, den));
  }
  acc_store(A, 16, 42);
}

// ------------------------------------------------------------------ GLSZM
__device__ __forceinline__ int uf_find(volatile int* parent, int x) {
  int cur = parent[x];
  if (cur != x) {
    int prev = x, next;
    while (cur > (next = parent[cur])) {
      parent[prev] = next;  // path halving; only ever points to an ancestor
      prev = cur;
      cur = next;
    }
  }
  return cur;
}

__device__ __forceinline__ void uf_unite(int* parent, int a, int b) {
  volatile int* vp = parent;
  while (true) {
    a = uf_find(vp, a);
    b = uf_find(vp, b);
    if (a == b) return;
    if (a < b) {
      int t = a;
      a = b;
      b = t;
    }
    // hook root a under the smaller root b if a is still a root
    if (atomicCAS(&parent[a], a, b) == a) return;
  }
}

// Per-lane partial sums over zones (level value i, size j): sum i, i^2,
// j^2, and 1/j^2, 1/i^2, 1/(i^2 j^2), i^2/j^2, j^2/i^2, i^2 j^2.
struct ZoneAcc {
  unsigned si = 0, si2 = 0, sj2 = 0;
  float fs[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sae lgl sal sah lal lah ze

  __device__ __forceinline__ void add(unsigned i, unsigned j) {
    si += i;
    si2 += i * i;
    sj2 += j * j;
    const float fi2 = (float)(i * i), fj2 = (float)(j * j);
    const float inv_i2 = __fdividef(1.f, fi2), inv_j2 = __fdividef(1.f, fj2);
    fs[0] += inv_j2;
    fs[1] += inv_i2;
    fs[2] += inv_i2 * inv_j2;
    fs[3] += fi2 * inv_j2;
    fs[4] += fj2 * inv_i2;
    fs[5] += fi2 * fj2;
  }
};

// Bit masks over a cube of side S (bit p = (z S + y) S + x) for the
// 26-neighbour dilation: kind 0: x != 0, 1: x != S-1, 2: y != 0, 3: y != S-1,
// 4: inside the cube.
template <int S>
__host__ __device__ constexpr uint32_t cube_mask(int word, int kind) {
  uint32_t m = 0;
  for (int b = 0; b < 32; ++b) {
    const int p = 32 * word + b;
    if (p >= S * S * S) continue;
    const int x = p % S, y = (p / S) % S;
    const bool ok = kind == 0 ? x != 0 : kind == 1 ? x != S - 1 : kind == 2 ? y != 0
                  : kind == 3 ? y != S - 1 : true;
    if (ok) m |= 1u << b;
  }
  return m;
}

// Word i of the NW-word bit set f shifted towards higher (K > 0) or lower
// (K < 0) bit indices by |K| bits.
template <int NW, int K>
__device__ __forceinline__ uint32_t shifted(const uint32_t (&f)[NW], int i) {
  constexpr int A = K > 0 ? K : -K, Q = A / 32, R = A % 32;
  if (K > 0) {
    const uint32_t hi = i - Q >= 0 ? f[i - Q] : 0u;
    const uint32_t lo = i - Q - 1 >= 0 ? f[i - Q - 1] : 0u;
    return R ? __funnelshift_l(lo, hi, R) : hi;
  } else {
    const uint32_t lo = i + Q < NW ? f[i + Q] : 0u;
    const uint32_t hi = i + Q + 1 < NW ? f[i + Q + 1] : 0u;
    return R ? __funnelshift_r(lo, hi, R) : lo;
  }
}

// o = (f dilated by the 26-neighbourhood, inside the cube) & lim, done as
// three separable 3-tap dilations (x, then y, then z).
template <int S, int NW>
__device__ __forceinline__ void dilate26(const uint32_t (&f)[NW], const uint32_t (&lim)[NW],
                                         uint32_t (&o)[NW]) {
  uint32_t a[NW], b[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i)
    a[i] = f[i] | (shifted<NW, 1>(f, i) & cube_mask<S>(i, 0)) |
           (shifted<NW, -1>(f, i) & cube_mask<S>(i, 1));
#pragma unroll
  for (int i = 0; i < NW; ++i)
    b[i] = a[i] | (shifted<NW, S>(a, i) & cube_mask<S>(i, 2)) |
           (shifted<NW, -S>(a, i) & cube_mask<S>(i, 3));
#pragma unroll
  for (int i = 0; i < NW; ++i)
    o[i] = (b[i] | (shifted<NW, S * S>(b, i) & cube_mask<S>(i, 4)) | shifted<NW, -S * S>(b, i)) &
           lim[i];
}

// Zones of V(v) for a window of side S: lane a owns compact level a (and
// a + 32, ...): its level set as a bit mask (one ballot per 32 positions),
// then repeatedly flood-fills from the lowest remaining voxel by 26-neighbour
// dilations until the set stops growing; each fill is one zone.  Appends
// zone keys (size << 8 | level) to A.kb and returns the zone count.
template <int S>
__device__ int glszm_zones_bits(const Win& w, const Arena& A, int* counter, ZoneAcc& z,
                                unsigned& glnu, int32_t* dbg_glszm) {
  constexpr int NW = (S * S * S + 31) / 32;
  const int lane = lane_id();
  if (lane == 0) *counter = 0;
  __syncwarp();
  for (int a0 = 0; a0 < w.m; a0 += 32) {
    const int a = a0 + lane;
    uint32_t L[NW];
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const int p = 32 * k + lane;
      const int lv = p < S * S * S ? (int)A.lvl[p] - 1 - a0 : -1;  // compact level - a0
      uint32_t word = 0u;
      const int top = min(32, w.m - a0);
      for (int c = 0; c < top; ++c) {
        const uint32_t bal = __ballot_sync(kFull, lv == c);
        if (lane == c) word = bal;
      }
      L[k] = a < w.m ? word : 0u;
    }
    unsigned cnt = 0;
    const unsigned i = a < w.m ? (unsigned)A.lev[a] : 0u;
    while (true) {
      bool any = false;
#pragma unroll
      for (int k = 0; k < NW; ++k) any |= L[k] != 0u;
      if (!any) break;
      uint32_t F[NW];
      bool found = false;
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        F[k] = (!found && L[k]) ? (L[k] & (0u - L[k])) : 0u;
        found |= L[k] != 0u;
      }
      while (true) {
        uint32_t G[NW];
        dilate26<S, NW>(F, L, G);
        bool grew = false;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
          grew |= G[k] != F[k];
          F[k] = G[k];
        }
        if (!grew) break;
      }
      unsigned size = 0;
#pragma unroll
      for (int k = 0; k < NW; ++k) {
        size += __popc(F[k]);
        L[k] &= ~F[k];
      }
      const int slot = atomicAdd(counter, 1);
      A.kb[slot] = (size << 8) | (unsigned)a;
      z.add(i, size);
      ++cnt;
      if (dbg_glszm) atomicAdd(&dbg_glszm[(size_t)(i - 1) * w.W + (size - 1)], 1);
    }
    glnu += cnt * cnt;
  }
  __syncwarp();
  const int nz = *counter;
  __syncwarp();
  return nz;
}

// Zones by a lock-free union-find over the window (any window size).
static __device__ int glszm_zones_uf(const Win& w, const Arena& A, ZoneAcc& z, unsigned& glnu,
                              int32_t* dbg_glszm) {
  const int lane = lane_id();
  const int m = w.m;
  int* parent = (int*)(A.big + A.L.parent);
  int* zsz = (int*)(A.big + A.L.zsz);
  int* zlv = (int*)(A.big + A.L.zlv);
  for (int p = lane; p < w.W; p += 32) {
    parent[p] = p;
    zsz[p] = 0;
  }
  for (int a = lane; a < m; a += 32) zlv[a] = 0;
  __syncwarp();
  for (int p = lane; p < w.W; p += 32) {
    const int a = A.lvl[p];
    if (!a) continue;
    int zz, y, x;
    pos_to_zyx(w, p, zz, y, x);
    for (int di = 0; di < kNumDirs; ++di) {
      const int dz = c_dirs[di][0], dy = c_dirs[di][1], dx = c_dirs[di][2];
      if (!in_cube(w, zz + dz, y + dy, x + dx)) continue;
      const int q = p + dz * w.s2 + dy * w.s + dx;
      if (A.lvl[q] == a) uf_unite(parent, p, q);
    }
  }
  __syncwarp();
  for (int p = lane; p < w.W; p += 32) {
    if (!A.lvl[p]) continue;
    atomicAdd(&zsz[uf_find((volatile int*)parent, p)], 1);
  }
  __syncwarp();
  // zones: roots of V(v) components -> keys (size << 8 | compact level)
  int nz = 0;
  for (int base = 0; base < w.W; base += 32) {
    const int p = base + lane;
    bool root = false;
    int a = 0, size = 0;
    if (p < w.W) {
      a = A.lvl[p];
      root = a && parent[p] == p;
      if (root) size = zsz[p];
    }
    const unsigned b = __ballot_sync(kFull, root);
    if (root) {
      A.kb[nz + __popc(b & lanemask_lt())] = ((uint32_t)size << 8) | (uint32_t)(a - 1);
      const unsigned i = A.lev[a - 1];
      z.add(i, (unsigned)size);
      atomicAdd(&zlv[a - 1], 1);
      if (dbg_glszm) atomicAdd(&dbg_glszm[(size_t)(i - 1) * w.W + (size - 1)], 1);
    }
    nz += __popc(b);
  }
  __syncwarp();
  for (int a = lane; a < m; a += 32) {
    const unsigned c = (unsigned)zlv[a];
    zlv[a] = 0;
    glnu += c * c;
  }
  // the big region is shared by the families, which count into it from zero
  for (int p = lane; p < w.W; p += 32) {
    parent[p] = 0;
    zsz[p] = 0;
  }
  return nz;
}

static __device__ void glszm_family(const Win& w, const Arena& A, int32_t* dbg_glszm) {
  const int lane = lane_id();
  ZoneAcc z;
  unsigned glnu = 0;
  int* counter = (int*)(A.big + A.L.zlv);
  int nz;
  if (w.s == 3)
    nz = glszm_zones_bits<3>(w, A, counter, z, glnu, dbg_glszm);
  else if (w.s == 5)
    nz = glszm_zones_bits<5>(w, A, counter, z, glnu, dbg_glszm);
  else if (w.s == 7)
    nz = glszm_zones_bits<7>(w, A, counter, z, glnu, dbg_glszm);
  else
    nz = glszm_zones_uf(w, A, z, glnu, dbg_glszm);
  if (lane == 0) *counter = 0;
  unsigned si = z.si, si2 = z.si2, sj2 = z.sj2;
  float (&fs)[7] = z.fs;
  __syncwarp();
  warp_sort(A.kb, nz);
  unsigned sznu = 0;
  for (int i = lane; i < nz; i += 32) {
    const uint32_t key = A.kb[i];
    if (i == 0 || A.kb[i - 1] != key) {
      const int c = lower_bound_u32(A.kb, i, nz, key + 1) - i;
      fs[6] += ent_term(c, nz);
    }
    if (i == 0 || (A.kb[i - 1] >> 8) != (key >> 8)) {
      const unsigned c = (unsigned)(lower_bound_u32(A.kb, i, nz, ((key >> 8) + 1) << 8) - i);
      sznu += c * c;
    }
  }
  si = redux_u32(si);
  si2 = redux_u32(si2);
  sj2 = redux_u32(sj2);
  sznu = redux_u32(sznu);
  glnu = redux_u32(glnu);
  warp_sum_f32x<7>(fs);
  const float N = (float)nz;
  const unsigned sj = (unsigned)w.nv;  // zone sizes add up to N_v
  float num = kNaNf, den = N;
  if (lane == 0) { num = fs[0]; }
  if (lane == 1) { num = (float)sj2; }
  if (lane == 2) { num = (float)glnu; }
  if (lane == 3) { num = (float)glnu; den = N * N; }
  if (lane == 4) { num = (float)sznu; }
  if (lane == 5) { num = (float)sznu; den = N * N; }
  if (lane == 6) { num = N; den = (float)w.nv; }
  if (lane == 7) { num = (float)((long long)nz * si2 - (long long)si * si); den = N * N; }
  if (lane == 8) { num = (float)((long long)nz * sj2 - (long long)sj * sj); den = N * N; }
  if (lane == 9) { num = fs[6]; den = 1.f; }
  if (lane == 10) { num = fs[1]; }
  if (lane == 11) { num = (float)si2; }
  if (lane == 12) { num = fs[2]; }
  if (lane == 13) { num = fs[3]; }
  if (lane == 14) { num = fs[4]; }
  if (lane == 15) { num = fs[5]; }
  if (lane < 16) A.fv[58 + lane] = lane_quot(num, den);
  __syncwarp();
}

// ------------------------------------------------------------------ GLDM + NGTDM
// Neighbour pass of windows of side S <= 7 on a padded copy: cell
// ((z+1) P + y+1) P + x+1 (P = S + 2) holds the compact level a | gray level
// << 8 of each VOI voxel, 0 elsewhere (the border too), so the 26 neighbour
// reads are unconditional with compile-time offsets.  GLDM counts go to
// gh[a][k]; NGTDM per (level, neighbour count w) to ngacc as one 32-bit word,
// count << 22 | sum of |i w - S| (per cell: count <= 343, sum < 2^22), which
// the caller turns into n_i and s_i L (clearing them).  The padded copy and
// ngacc share bytes with regions the GLCM family leaves non-zero (its MCC
// slots), so both are cleared here first; the copy is cleared again on exit.
template <int S>
__device__ void gldm_ngtdm_pass_padded(const Win& w, const Arena& A, bool do_gldm,
                                       bool do_ngtdm) {
  constexpr int P = S + 2, P2 = P * P, S3 = S * S * S;
  const int lane = lane_id();
  uint16_t* pad = (uint16_t*)(A.big + A.L.pad);
  int* gh = (int*)(A.big + A.L.ghist);
  unsigned* ngacc = (unsigned*)(A.big + A.L.ngacc);
  for (int t = lane; t < (P * P2 + 1) / 2; t += 32) ((unsigned*)pad)[t] = 0u;
  if (do_ngtdm)
    for (int t = lane; t < w.m * 27; t += 32) ngacc[t] = 0u;
  __syncwarp();
  for (int p = lane; p < S3; p += 32) {
    const int a = A.lvl[p];
    if (a) {
      const int z = p / (S * S), y = (p / S) % S, x = p % S;
      pad[((z + 1) * P + y + 1) * P + x + 1] = (uint16_t)(a | ((int)A.lev[a - 1] << 8));
    }
  }
  __syncwarp();
  for (int base = 0; base < S3; base += 32) {
    const int p = base + lane;
    int key = -1;
    if (p < S3) {
      const int z = p / (S * S), y = (p / S) % S, x = p % S;
      const uint16_t* c = pad + ((z + 1) * P + y + 1) * P + x + 1;
      const unsigned v = *c;
      const int a = (int)(v & 0xFFu);
      if (a) {
        int keq = 0, nw = 0, ssum = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dz && !dy && !dx) continue;
              const unsigned u = c[dz * P2 + dy * P + dx];
              const int b = (int)(u & 0xFFu);
              nw += b != 0;
              ssum += (int)(u >> 8);
              keq += b == a;
            }
        key = (a - 1) * 28 + keq;
        if (do_ngtdm && nw > 0) {
          const int dlt = abs((int)(v >> 8) * nw - ssum);
          atomicAdd(&ngacc[(a - 1) * 27 + nw], (unsigned)dlt + (1u << 22));
        }
      }
    }
    if (do_gldm) {
      const unsigned act = __ballot_sync(kFull, key >= 0);
      if (key >= 0) {
        const unsigned grp = __match_any_sync(act, key);
        if ((grp & lanemask_lt()) == 0) atomicAdd(&gh[key], __popc(grp));
      }
    }
  }
  __syncwarp();
  for (int p = lane; p < S3; p += 32)  // leave the padded copy zero
    if (A.lvl[p]) {
      const int z = p / (S * S), y = (p / S) % S, x = p % S;
      pad[((z + 1) * P + y + 1) * P + x + 1] = 0;
    }
}

static __device__ void gldm_ngtdm_family(const Win& w, const Arena& A, const FrJob& job,
                                  int32_t* dbg_gldm, int32_t* dbg_ngn,
                                  long long* dbg_ngs) {
  const int lane = lane_id();
  const int m = w.m;
  const bool do_gldm = (job.families & kFamGLDM) != 0;
  const bool do_ngtdm = (job.families & kFamNGTDM) != 0;
  int* gh = (int*)(A.big + A.L.ghist);  // [mc][28]
  int* ngn = (int*)(A.big + A.L.ngn);
  unsigned long long* ngs = (unsigned long long*)(A.big + A.L.ngs);
  if (w.s == 3 || w.s == 5 || w.s == 7) {
    if (w.s == 3) gldm_ngtdm_pass_padded<3>(w, A, do_gldm, do_ngtdm);
    if (w.s == 5) gldm_ngtdm_pass_padded<5>(w, A, do_gldm, do_ngtdm);
    if (w.s == 7) gldm_ngtdm_pass_padded<7>(w, A, do_gldm, do_ngtdm);
    if (do_ngtdm) {
      // n_i and s_i L from the (level, neighbour count) words
      unsigned* ngacc = (unsigned*)(A.big + A.L.ngacc);
      for (int a = lane; a < m; a += 32) {
        unsigned n = 0;
        unsigned long long sl = 0;
        for (int k = 1; k <= 26; ++k) {
          const unsigned c = ngacc[a * 27 + k];
          if (!c) continue;
          ngacc[a * 27 + k] = 0;
          n += c >> 22;
          sl += (unsigned long long)(c & 0x3FFFFFu) * (unsigned long long)c_ldiv.v[k];
        }
        ngn[a] = (int)n;
        ngs[a] = sl;
      }
    }
  }
  for (int base = 0; w.s != 3 && w.s != 5 && w.s != 7 && base < w.W; base += 32) {
    const int p = base + lane;
    int key = -1;
    if (p < w.W) {
      const int a = A.lvl[p];
      if (a) {
        int z, y, x;
        pos_to_zyx(w, p, z, y, x);
        int keq = 0, nw = 0, ssum = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (!dz && !dy && !dx) continue;
              if (!in_cube(w, z + dz, y + dy, x + dx)) continue;
              const int b = A.lvl[p + dz * w.s2 + dy * w.s + dx];
              if (!b) continue;
              ++nw;
              ssum += A.lev[b - 1];
              keq += (b == a);
            }
        key = (a - 1) * 28 + keq;
        if (do_ngtdm && nw > 0) {
          const long long i = A.lev[a - 1];
          long long dlt = i * nw - ssum;
          if (dlt < 0) dlt = -dlt;
          atomicAdd(&ngn[a - 1], 1);
          atomicAdd(&ngs[a - 1], (unsigned long long)(dlt * c_ldiv.v[nw]));
        }
      }
    }
    if (do_gldm) {
      const unsigned act = __ballot_sync(kFull, key >= 0);
      if (key >= 0) {
        const unsigned grp = __match_any_sync(act, key);
        if ((grp & lanemask_lt()) == 0) atomicAdd(&gh[key], __popc(grp));
      }
    }
  }
  __syncwarp();
  const int N = w.nv;
  if (do_gldm) {
    unsigned si = 0, si2 = 0, sj = 0, sj2 = 0, dnu = 0, dce = 0;  // dce: sum c^2
    float fs[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sde lgl sdl sdh ldl ldh de
    // column sums (dependence counts over all levels) first, then one lane
    // per (level, dependence count) cell
    if (lane < 27) {
      unsigned col = 0;
      for (int a = 0; a < m; ++a) col += (unsigned)gh[a * 28 + lane];
      dnu = col * col;
    }
    dnu = redux_u32(dnu);
    __syncwarp();
    for (int t = lane; t < m * 27; t += 32) {
      const int a = t / 27, k = t - 27 * a;
      const int c = gh[a * 28 + k];
      if (!c) continue;
      gh[a * 28 + k] = 0;
      const unsigned i = A.lev[a];
      const float fi2 = (float)(i * i), inv_i2 = __fdividef(1.f, fi2);
      const unsigned J = (unsigned)(k + 1);
      const float fc = (float)c, fj2 = (float)(J * J), inv_j2 = __fdividef(1.f, fj2);
      si += (unsigned)c * i;
      si2 += (unsigned)c * i * i;
      sj += (unsigned)c * J;
      sj2 += (unsigned)c * J * J;
      fs[0] += fc * inv_j2;
      fs[1] += fc * inv_i2;
      fs[2] += fc * inv_i2 * inv_j2;
      fs[3] += fc * fi2 * inv_j2;
      fs[4] += fc * fj2 * inv_i2;
      fs[5] += fc * fi2 * fj2;
      fs[6] += ent_term(c, N);
      dce += (unsigned)(c * c);
      if (dbg_gldm) dbg_gldm[(i - 1) * 27 + k] = c;
    }
    si = redux_u32(si);
    si2 = redux_u32(si2);
    sj = redux_u32(sj);
    sj2 = redux_u32(sj2);
    dce = redux_u32(dce);
    warp_sum_f32x<7>(fs);
    const float fN = (float)N;
    float num = kNaNf, den = fN;
    if (lane == 0) { num = fs[0]; }
    if (lane == 1) { num = (float)sj2; }
    if (lane == 2) { num = (float)w.u2; }
    if (lane == 3) { num = (float)dnu; }
    if (lane == 4) { num = (float)dnu; den = fN * fN; }
    if (lane == 5) { num = (float)((long long)N * si2 - (long long)si * si); den = fN * fN; }
    if (lane == 6) { num = (float)((long long)N * sj2 - (long long)sj * sj); den = fN * fN; }
    if (lane == 7) { num = fs[6]; den = 1.f; }
    if (lane == 8) { num = fs[1]; }
    if (lane == 9) { num = (float)si2; }
    if (lane == 10) { num = fs[2]; }
    if (lane == 11) { num = fs[3]; }
    if (lane == 12) { num = fs[4]; }
    if (lane == 13) { num = fs[5]; }
    // IBSI extras: grey level non-uniformity normalised, dependence count
    // percentage N / N_v, dependence count energy sum p^2
    if (lane == 14) { num = (float)w.u2; den = fN * fN; }
    if (lane == 15) { num = fN; den = (float)w.nv; }
    if (lane == 16) { num = (float)dce; den = fN * fN; }
    if (lane < 14) A.fv[74 + lane] = lane_quot(num, den);
    if (lane >= 14 && lane < 17) A.fv[kGldmExtra + lane - 14] = lane_quot(num, den);
  }
  __syncwarp();
  if (do_ngtdm) {
    // per-level sums over present levels, then the pairwise sums
    const float invL = (float)(1.0 / (double)kLcm26);
    unsigned nvp = 0, ngp = 0;
    unsigned long long sls = 0;
    float nsf = 0.f;
    for (int a = lane; a < m; a += 32) {
      const int n = ngn[a];
      if (!n) continue;
      const unsigned long long sl = ngs[a];
      nvp += (unsigned)n;
      sls += sl;
      nsf += (float)n * ((float)sl * invL);
      ++ngp;
      if (dbg_ngn) {
        dbg_ngn[A.lev[a] - 1] = n;
        dbg_ngs[A.lev[a] - 1] = (long long)sl;
      }
    }
    nvp = redux_u32(nvp);
    ngp = redux_u32(ngp);
    sls = warp_sum_u64(sls);
    unsigned long long c1 = 0, bden = 0, str = 0;
    float cpl = 0.f;
    for (int a = lane; a < m; a += 32) {
      const long long na = ngn[a];
      if (!na) continue;
      const long long ia = A.lev[a];
      const float sa = (float)ngs[a] * invL;
      for (int b = 0; b < m; ++b) {
        const long long nb = ngn[b];
        if (!nb) continue;
        const long long ib = A.lev[b];
        const long long d = ia - ib;
        c1 += (unsigned long long)(na * nb * d * d);
        const long long bd = ia * na - ib * nb;
        bden += (unsigned long long)(bd < 0 ? -bd : bd);
        str += (unsigned long long)((na + nb) * d * d);
        const float sb = (float)ngs[b] * invL;
        cpl += __fdividef((float)(d < 0 ? -d : d) * ((float)na * sa + (float)nb * sb),
                          (float)(na + nb));
      }
    }
    c1 = warp_sum_u64(c1);
    bden = warp_sum_u64(bden);
    str = warp_sum_u64(str);
    float fs[2] = {nsf, cpl};
    warp_sum_f32x<2>(fs);
    __syncwarp();
    for (int a = lane; a < m; a += 32) {
      ngn[a] = 0;
      ngs[a] = 0ull;
    }
    const float fv = (float)nvp, slsf = (float)sls * invL;
    float num = kNaNf, den = 1.f;
    if (nvp) {
      if (lane == 0) { num = fv; den = fs[0]; }
      if (lane == 1) { if (ngp == 1) {
            num = 0.f;
          } else {
            num = (float)c1 * slsf;
            den = fv * fv * (float)ngp * (float)(ngp - 1) * fv;
          } }
      if (lane == 2) { num = fs[0]; den = (float)bden; }
      if (lane == 3) { num = fs[1]; den = fv; }
      if (lane == 4) { num = (float)str; den = fv * slsf; }
    }
    if (lane < 5) A.fv[88 + lane] = (nvp == 0) ? kNaNf : lane_quot(num, den);
  }
  __syncwarp();
}

}  // namespace fr
