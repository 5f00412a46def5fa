// fr_device.cuh -- warp primitives, exact-integer helpers and the mbarrier /
// TMA wrappers (inline PTX for sm_103a) used by the mapping kernel.
#pragma once

#include <cstdint>

#include <cuda.h>

namespace fr {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ int warp_sum_i32(int v) {
  return __reduce_add_sync(kFull, v);
}
__device__ __forceinline__ unsigned warp_sum_u32(unsigned v) {
  return __reduce_add_sync(kFull, v);
}
__device__ __forceinline__ int warp_max_i32(int v) {
  return __reduce_max_sync(kFull, v);
}
__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ __int128 warp_sum_i128(__int128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long lo = (unsigned long long)v;
    long long hi = (long long)(v >> 64);
    unsigned long long olo = __shfl_xor_sync(kFull, lo, o);
    long long ohi = __shfl_xor_sync(kFull, hi, o);
    v += ((__int128)ohi << 64) | (__int128)olo;
  }
  return v;
}

// Exact int128 -> double (one rounding of the 128-bit value's hi part is at
// most 2^-53 relative; the lo part adds exactly below it).
__device__ __forceinline__ double i128_to_f64(__int128 v) {
  bool neg = v < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  unsigned long long hi = (unsigned long long)(u >> 64);
  unsigned long long lo = (unsigned long long)u;
  double d = (double)hi * 18446744073709551616.0 + (double)lo;
  return neg ? -d : d;
}

// Floor division by a small positive d (p < 2^16, d < 2^12) by multiply-high.
struct Magic {
  unsigned m;
  __device__ __forceinline__ void init(unsigned d) { m = 0xffffffffu / d + 1u; }
  __device__ __forceinline__ unsigned div(unsigned p) const {
    return __umulhi(p, m);
  }
};

// ---------------------------------------------------------------- time
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar,
                                                      unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most
// timeout_ns; also gives up when *abort becomes nonzero.  Returns false when
// the wait ended without the phase completing.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long timeout_ns,
                                                  const volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((++spins & 63u) == 0) {
      if (*abort) return false;
      if ((long long)(global_ns() - t0) > timeout_ns) return false;
      __nanosleep(256);
    }
  }
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tmap_prefetch(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(m) : "memory");
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m)
               : "memory");
}

// 3-D tiled bulk tensor load global -> shared, completing on an mbarrier.
// x must be a multiple of 4 (16 bytes of uint32); y and z are unconstrained
// (out-of-range elements are filled with zero).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* m,
                                            int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_"
      "tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace fr
