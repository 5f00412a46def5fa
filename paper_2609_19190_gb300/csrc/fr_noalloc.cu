// fr_noalloc.cu -- the VOI voxel list without any device allocation.
//
// Some callers cannot call cudaMalloc: their device memory already belongs to
// another allocator (a framework's caching pool that has reserved it, an
// application that hands all of it to its own arena at start-up), or they
// must not allocate once they are running (allocation-free service loops).
// fr_voxel_list_noalloc gives them the z-major VOI voxel list -- the output
// column order of every map -- from their own mask and output buffers, with
// its only scratch in the fixed array below, which every GPU that loads the
// library holds until the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/flashmap.h"
#include "fr_internal.h"

namespace fr {
cudaError_t fr_launch_row_count(const uint8_t* mask, int nx, int rows, int32_t* rowcnt,
                                cudaStream_t s);
cudaError_t fr_launch_scan(const int32_t* in, int32_t* out, int n, long long* tot,
                           cudaStream_t s);
cudaError_t fr_launch_voi_fill(const uint8_t* mask, int nx, int rows, const int32_t* rowoff,
                               int32_t* voi, cudaStream_t s);
}  // namespace fr

// Scratch: per-row mask counts, their exclusive prefix sums, and the total.
constexpr int kMaxRows = FR_NOALLOC_MAX_ROWS;
constexpr size_t kRowBytes = (size_t)kMaxRows * sizeof(int32_t);
constexpr size_t kScratchBytes = 2 * kRowBytes + 256;  // 2 MiB + 256 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices];  // device address of the scratch, per device

// The name g_noalloc_scratch in host code is only a stand-in for the device
// symbol; its device address is looked up once per device, with that device
// current, and cached.
fr_status scratch_for_device(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FR_ERR_CUDA;
    g_scratch_ptr[device] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[device];
  return FR_OK;
}

}  // namespace

extern "C" fr_status fr_voxel_list_noalloc(const uint8_t* mask, int32_t nx, int32_t ny,
                                           int32_t nz, int32_t* voi, int64_t capacity,
                                           int64_t* n_voi, int32_t device, fr_stream_t s) {
  if (!mask || !voi || !n_voi || nx < 1 || ny < 1 || nz < 1 || capacity < 0)
    return FR_ERR_INVALID_ARG;
  if ((long long)nx * ny * nz >= (1LL << 31)) return FR_ERR_UNSUPPORTED;
  if ((long long)ny * nz > kMaxRows) return FR_ERR_UNSUPPORTED;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev ||
      device >= kMaxDevices)
    return FR_ERR_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
  // an error left pending by earlier work of this thread is reported (and
  // cleared) here, so that a failure below belongs to this call's launches
  if (cudaGetLastError() != cudaSuccess) return FR_ERR_CUDA;
  unsigned char* base = nullptr;
  fr_status st = scratch_for_device(device, &base);
  if (st != FR_OK) return st;
  int32_t* rowcnt = (int32_t*)base;
  int32_t* rowoff = (int32_t*)(base + kRowBytes);
  long long* total = (long long*)(base + 2 * kRowBytes);
  cudaStream_t cs = (cudaStream_t)s;
  const int rows = ny * nz;
  // every scratch word read below is written first by this call: the row
  // counts by the count kernel, the offsets and the total by the scan
  if (fr::fr_launch_row_count(mask, nx, rows, rowcnt, cs) != cudaSuccess) return FR_ERR_CUDA;
  if (fr::fr_launch_scan(rowcnt, rowoff, rows, total, cs) != cudaSuccess) return FR_ERR_CUDA;
  long long n = 0;
  if (cudaMemcpyAsync(&n, total, sizeof(n), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return FR_ERR_CUDA;
  *n_voi = n;
  if (n > capacity) return FR_ERR_INVALID_ARG;
  if (n > 0 && fr::fr_launch_voi_fill(mask, nx, rows, rowoff, voi, cs) != cudaSuccess)
    return FR_ERR_CUDA;
  return FR_OK;
}
