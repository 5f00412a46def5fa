// fr_map_kernel.cu -- the persistent mapping kernel.
//
// One CTA = NW warps, resident for the whole launch; each warp maps whole
// voxels (fr_voxel.cuh).  Work items (up to N voxels of one brick of one VOI)
// come from a device queue; each item's brick halo -- a 3-D box of the packed
// level/intensity volume -- is staged into shared memory by one TMA tiled
// load completing on an mbarrier.  Thread 0 is the feeder: it claims the next
// item and starts its load into a buffer as soon as every warp has gathered
// its window from that buffer, so the copy overlaps the texture work of the
// current item (`stages` buffers let it run further ahead).  No warp is set
// aside for the copies.  Every wait is bounded in time; a wait that runs out
// records FR_ERR_TIMEOUT and the CTA leaves after its own copies have landed.
#include <cstdint>

#include "fr_device.cuh"
#include "fr_internal.h"
#include "fr_voxel.cuh"

namespace fr {

constexpr int kStatusTimeout = 6;      // FR_ERR_TIMEOUT
constexpr int kStatusUnsupported = 7;  // FR_ERR_UNSUPPORTED

// Shared-memory layout of a CTA (host and device agree through this).
struct CtaLayout {
  int32_t tiles, bars, slots, fb, arenas, bytes;
};

__host__ __device__ inline CtaLayout fr_cta_layout(int stages, int tile_bytes,
                                                   int nw, int arena_bytes) {
  CtaLayout c;
  c.tiles = 0;
  c.bars = stages * tile_bytes;
  c.slots = c.bars + 2 * stages * 8;
  c.fb = c.slots + stages * 4;  // pool: count, next, count_big, next_big, kFbTasks tasks
  c.arenas = fr_align(c.fb + (4 + kFbTasks) * 4, 128);
  c.bytes = c.arenas + nw * arena_bytes;
  return c;
}

// Consumer warps of a CTA map their voxels of an item family by family, in
// step: a named barrier (id 1, consumer threads only) after each family keeps
// the warps in the same code region, so they share the instruction cache.
__device__ __forceinline__ void consumer_bar(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// OR of a per-thread flag over the consumer threads (a barrier as well).
__device__ __forceinline__ bool consumer_any(bool flag, int nthreads) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\t"
      "selp.s32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((unsigned)flag), "r"(nthreads)
      : "memory");
  return r != 0;
}

// The feeder's state (meaningful in thread 0 only): which buffers hold a
// copy that has not been waited for, and with which barrier parity.
struct Feeder {
  unsigned char* tiles;
  uint64_t* full;
  volatile int* slot;
  int tile_bytes;
  const CUtensorMap* last;
  bool pending[kMaxStages];
  unsigned ppar[kMaxStages];
};

// Thread 0: claim the next item (skipping VOIs whose preparation failed) and
// start its halo copy into buffer `stage`, whose barrier phase `parity` it
// completes; past the end of the queue the buffer gets the sentinel -1 and
// the phase completes without a copy.
__device__ __noinline__ void feed(const FrMapArgs& args, Feeder& fd, int stage,
                                  unsigned parity) {
  int it;
  while (true) {
    it = (int)atomicAdd(args.queue, 1u);
    if (it >= args.n_items) {
      it = -1;
      break;
    }
    if (args.jobs[args.items[it].job].state->status == 0) break;
  }
  fd.slot[stage] = it;
  if (it < 0) {
    mbar_arrive(&fd.full[stage]);
    return;
  }
  // testing hook of the bounded waits: no copy and no arrival, so the
  // buffer's phase never completes and every wait on it runs out
  if (it == args.withhold_item) return;
  const FrItem& item = args.items[it];
  const FrJob& job = args.jobs[item.job];
  const CUtensorMap* tm = &job.tmap;
  if (tm != fd.last) {
    tmap_acquire(tm);
    fd.last = tm;
  }
  const unsigned bytes = (unsigned)(job.box_x * job.box_y * job.box_z * 4);
  mbar_arrive_expect_tx(&fd.full[stage], bytes);
  tma_load_3d(fd.tiles + (size_t)stage * fd.tile_bytes, tm, item.bx - job.hx,
              item.by - job.r, item.bz - job.r, &fd.full[stage]);
  fd.pending[stage] = true;
  fd.ppar[stage] = parity;
}

// Voxel t of the item, or no voxel (has == false: the warp only keeps step).
// refill: this is the item's last round, so once every warp has gathered its
// window the feeder reloads buffer `stage` (next barrier phase `parity`).
template <bool DUMP>
__device__ __forceinline__ void map_voxel(const FrMapArgs& args, const FrJob& job,
                                          const FrItem& item, const uint32_t* tile, int t, bool has,
                                          Arena& A, char* smem_big, char* slab_big, int it, int nt,
                                          Feeder& fd, bool refill, int stage, unsigned parity,
                                          const FbPool& pool, unsigned char* arenas) {
  const int lane = lane_id();
  Win w;
  int col = 0;
  bool skip = false;
  int32_t *d_hist = nullptr, *d_glcm = nullptr, *d_glrlm = nullptr,
          *d_glszm = nullptr, *d_gldm = nullptr, *d_ngn = nullptr;
  long long* d_ngs = nullptr;
  if (has) {
    col = job.bcols[item.j0 + t];
    const int lin = job.voi[col];
    const int x = lin % job.nx;
    const int y = (lin / job.nx) % job.ny;
    const int z = lin / (job.nx * job.ny);
    w.r = job.r;
    w.s = 2 * job.r + 1;
    w.s2 = w.s * w.s;
    w.W = w.s2 * w.s;
    w.ms.init((unsigned)w.s);
    w.ms2.init((unsigned)w.s2);
    w.ng = job.state->ng;
    const int cx = (x - job.r) - (item.bx - job.hx);
    const int cy = y - item.by;
    const int cz = z - item.bz;
    w.nv = gather_window(w, A, tile, job.box_x, job.box_y, cx, cy, cz);
    // the big region is free until the families: the counting sort's bins
    const bool counting = w.nv > kCsortMinKeys && w.nv <= 32 * kRadixRounds;
    if (!counting || !warp_csort(A.kb, w.nv, (uint32_t*)smem_big, args.arena.big_bytes >> 2))
      warp_sort_x(A.kb, w.nv, (int*)(A.tmp + 32));
    if (DUMP) {
      const int ng = w.ng;
      int32_t* rec = args.dbg + (size_t)it * args.dbg_stride;
      d_hist = rec + 4;
      d_glcm = d_hist + ng;
      d_glrlm = d_glcm + (size_t)kNumDirs * ng * ng;
      d_glszm = d_glrlm + (size_t)kNumDirs * ng * w.s;
      d_gldm = d_glszm + (size_t)ng * w.W;
      d_ngn = d_gldm + (size_t)ng * 27;
      size_t o = (size_t)(d_ngn + ng - rec);
      o = (o + 1) & ~(size_t)1;
      d_ngs = (long long*)(rec + o);
      if (lane == 0) {
        rec[0] = ng;
        rec[1] = w.s;
        rec[2] = w.W;
        rec[3] = w.nv;
      }
    }
    first_order(w, A, job, d_hist);
    compact_levels(w, A);
    if (w.m > kMCap || w.R >= kBinCap) {
      if (slab_big == nullptr) {
        if (lane == 0) atomicCAS(args.status, 0, kStatusUnsupported);
        for (int f = lane; f < kNumFeatures; f += 32) A.fv[f] = kNaNf;
        __syncwarp();
        skip = true;
      } else {
        A.big = slab_big;
        A.mc = args.slab_ngc;
        A.bc = args.slab_ngc;
      }
    } else {
      A.big = smem_big;
      A.mc = kMCap;
      A.bc = kBinCap;
    }
    if (!skip) A.L = fr_big_layout(A.mc, A.bc, w.W);
  }
  const bool work = has && !skip;
  consumer_bar(nt);
  if (refill && threadIdx.x == 0) feed(args, fd, stage, parity);
  if (job.families & kFamGLCM) {
    const bool use_pool = args.fb != nullptr && (job.families & kFamMCC) != 0;
    if (work) glcm_family(w, A, job, d_glcm, use_pool ? &pool : nullptr);
    if (use_pool) {
      consumer_bar(nt);  // the task list is complete
      if (*(volatile int*)pool.count + *(volatile int*)pool.count_big > 0) {
        const int s = 2 * job.r + 1;
        fb_pool_work(pool, args, s * s * s, arenas, args.arena.bytes, args.arena.off_big, smem_big);
        consumer_bar(nt);  // every radius is in its owner's results
        if (threadIdx.x == 0) {
          *pool.count = 0;
          *pool.next = 0;
          *pool.count_big = 0;
          *pool.next_big = 0;
        }
      }
    }
    if (work) glcm_finish(A, job);
    consumer_bar(nt);
  }
  // GLRLM and GLSZM run without a barrier between them and GLDM: warps that
  // finish early go on (measured: the barriers after these two cost 1.5 %;
  // the ones after GLCM and GLDM keep the warps in the same code)
  if (job.families & kFamGLRLM) {
    if (work) glrlm_family(w, A, job.agg == 1, d_glrlm);
  }
  if (job.families & kFamGLSZM) {
    if (work) glszm_family(w, A, d_glszm);
  }
  if (job.families & (kFamGLDM | kFamNGTDM)) {
    if (work) gldm_ngtdm_family(w, A, job, d_gldm, d_ngn, d_ngs);
    consumer_bar(nt);
  }
  if (has) {
    float* out = (float*)args.run_ptrs[2 * item.job + 1];
    for (int f = lane; f < kNumFeatures; f += 32) {
      const int row = job.row_of[f];
      // maps are written once and never read here: streaming stores keep
      // them from evicting the MCC scratch from L2
      if (row >= 0) __stcs(&out[(size_t)row * job.n_voi + col], A.fv[f]);
    }
    __syncwarp();
  }
}

template <bool DUMP>
__global__ void __launch_bounds__(32 * kMaxConsumerWarps, 1)
    fr_map_kernel(const __grid_constant__ FrMapArgs args) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int S = args.stages, NW = args.consumer_warps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const CtaLayout cl = fr_cta_layout(S, args.tile_bytes, NW, args.arena.bytes);
  Feeder fd;
  fd.tiles = smem + cl.tiles;
  fd.full = (uint64_t*)(smem + cl.bars);
  fd.slot = (volatile int*)(smem + cl.slots);
  fd.tile_bytes = args.tile_bytes;
  fd.last = nullptr;
  for (int s = 0; s < kMaxStages; ++s) {
    fd.pending[s] = false;
    fd.ppar[s] = 0;
  }
  const volatile int* abort_flag = args.status;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&fd.full[s], 1);
    fence_mbar_init();
    int* fbc = (int*)(smem + cl.fb);
    for (int q = 0; q < 4; ++q) fbc[q] = 0;
  }
  // zero this warp's arena (the count matrices must start at zero)
  {
    uint4* a = (uint4*)(smem + cl.arenas + warp * args.arena.bytes);
    for (int i = lane; i < args.arena.bytes / 16; i += 32) a[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < S; ++s) feed(args, fd, s, 0u);

  unsigned char* ab = smem + cl.arenas + warp * args.arena.bytes;
  Arena A;
  A.kb = (uint32_t*)(ab + args.arena.off_kb);
  A.lvl = ab + args.arena.off_lvl;
  A.lut = ab + args.arena.off_lut;
  A.lev = ab + args.arena.off_lev;
  A.st = (uint16_t*)(ab + args.arena.off_st);
  A.fv = (float*)(ab + args.arena.off_fv);
  A.facc = (float*)(ab + args.arena.off_acc);
  A.nacc = (int*)(ab + args.arena.off_acc + 32 * 4);
  A.tmp = (float*)(ab + args.arena.off_tmp);
  A.fcomp = A.tmp;
  char* smem_big = (char*)(ab + args.arena.off_big);
  char* slab_big = args.slab ? args.slab + ((size_t)blockIdx.x * NW + warp) * args.slab_stride
                             : nullptr;
  const int nt = 32 * NW;
  FbPool pool;
  pool.count = (int*)(smem + cl.fb);
  pool.next = pool.count + 1;
  pool.count_big = pool.count + 2;
  pool.next_big = pool.count + 3;
  pool.tasks = pool.count + 4;
  pool.scratch = args.fb ? args.fb + ((size_t)blockIdx.x * NW + warp) * args.fb_stride : nullptr;
  pool.warp = warp;
  int stage = 0;
  unsigned phase = 0;
  while (true) {
    const bool ok = mbar_wait_bounded(&fd.full[stage], phase, args.timeout_ns, abort_flag);
    // every warp reaches this barrier; all leave together if any wait
    // failed, so none is left waiting at a later barrier
    if (consumer_any(!ok, nt)) {
      if (!ok && lane == 0) atomicCAS(args.status, 0, kStatusTimeout);
      if (threadIdx.x == 0) {
        // leave only after this CTA's own copies have landed
        const int zero = 0;
        for (int s = 0; s < S; ++s)
          if (fd.pending[s]) mbar_wait_bounded(&fd.full[s], fd.ppar[s], args.timeout_ns, &zero);
      }
      break;
    }
    if (threadIdx.x == 0) fd.pending[stage] = false;
    const int it = fd.slot[stage];
    if (it < 0) break;  // later buffers hold sentinels too: no copy in flight
    const FrItem item = args.items[it];
    const FrJob& job = args.jobs[item.job];
    const uint32_t* tile = (const uint32_t*)(smem + cl.tiles + (size_t)stage * args.tile_bytes);
    const int rounds = (item.n + NW - 1) / NW;
    for (int r = 0; r < rounds; ++r) {
      const int t = r * NW + warp;
      map_voxel<DUMP>(args, job, item, tile, t, t < item.n, A, smem_big, slab_big, it, nt, fd,
                      r == rounds - 1, stage, phase ^ 1u, pool, smem + cl.arenas);
    }
    if (++stage == S) {
      stage = 0;
      phase ^= 1u;
    }
  }
}

int fr_map_smem_bytes(int stages, int tile_bytes, int nw, int arena_bytes) {
  return fr_cta_layout(stages, tile_bytes, nw, arena_bytes).bytes;
}

cudaError_t fr_map_configure(bool dump, int smem_bytes) {
  const void* fn = dump ? (const void*)fr_map_kernel<true> : (const void*)fr_map_kernel<false>;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

cudaError_t fr_map_occupancy(bool dump, int threads, int smem_bytes, int* blocks) {
  const void* fn = dump ? (const void*)fr_map_kernel<true> : (const void*)fr_map_kernel<false>;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, threads, smem_bytes);
}

cudaError_t fr_map_launch(bool dump, const FrMapArgs& args, int grid, int smem_bytes,
                          cudaStream_t s) {
  const int threads = 32 * args.consumer_warps;
  if (dump)
    fr_map_kernel<true><<<grid, threads, smem_bytes, s>>>(args);
  else
    fr_map_kernel<false><<<grid, threads, smem_bytes, s>>>(args);
  return cudaGetLastError();
}

}  // namespace fr
