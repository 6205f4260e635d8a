// Allocation-free entry point: db_rrl_iterate with its scratch taken from a
// fixed array compiled into the library instead of a caller workspace.  For
// callers that may not allocate device memory at run time (fixed-latency
// frame loops, plugins inside frameworks that own the GPU memory).  No
// cudaMalloc, cudaFree or allocating library call happens here.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.cuh"

namespace {

// The scratch.  Device code could name it directly; host code must not pass
// its name as a pointer (that is a host-side stand-in, not the device
// address), so the device address is looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DB_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device; the first call
// per device does the lookup (with that device current).  The address stays
// valid while the device's context lives: a cudaDeviceReset (which unloads
// the library's module) invalidates it.
db_status scratch_on_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DB_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DB_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
      return DB_ERR_CUDA;
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return DB_OK;
}

}  // namespace

extern "C" db_status db_rrl_iterate_noalloc(const float* f, float* u, int H, int W, int ld,
                                            const db_psf* psf, const db_params* p, int iters,
                                            int* dev_status, void* stream) {
  // only the iteration's regions: spatial mode needs no Wiener spectrum,
  // work rows or transform tables
  const size_t need = db::rrl_iterate_ws_bytes(H, W, psf, p);
  if (need == 0) return DB_ERR_ARG;
  if (need > DB_NOALLOC_SCRATCH_BYTES) return DB_ERR_WORKSPACE;
  void* ws = nullptr;
  const db_status st = scratch_on_current_device(&ws);
  if (st != DB_OK) return st;
  return db_rrl_iterate(f, u, H, W, ld, psf, p, iters, nullptr, 0, ws, DB_NOALLOC_SCRATCH_BYTES,
                        dev_status, stream);
}
