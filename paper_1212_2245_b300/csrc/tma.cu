// Host side of the TMA window staging: tensor maps of float images, encoded
// through the driver's cuTensorMapEncodeTiled (reached through the runtime's
// driver entry point, so the library links no driver library itself).
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "internal.cuh"
#include "tma.cuh"

namespace db {

static std::atomic<int> g_tma{1};
bool tma_enabled() { return g_tma.load() != 0; }

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool encode_window_map(CUtensorMap* out, const float* base, int W, int H, int ld, int nz, long long zstride,
                       int box_w, int box_h) {
  EncodeTiled fn = encode_fn();
  if (!fn || !out || !base || W < 1 || H < 1 || nz < 1 || ld < W) return false;
  if (((uintptr_t)base & 15u) != 0 || (ld & 3) != 0 || (nz > 1 && ((zstride & 3) != 0 || zstride < (long long)ld * H)))
    return false;
  if (box_w < 1 || box_w > 256 || box_h < 1 || box_h > 256 || ((size_t)box_w * sizeof(float)) % 16 != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * sizeof(float),
                                 (cuuint64_t)(nz > 1 ? zstride : (long long)ld * H) * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace db

using namespace db;

extern "C" db_status db_set_tma(int on) {
  if (on != 0 && on != 1) return DB_ERR_ARG;
  g_tma.store(on);
  bump_settings();
  return DB_OK;
}
