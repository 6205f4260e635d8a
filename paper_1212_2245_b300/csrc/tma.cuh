// Tensor-memory-accelerator (TMA) staging of image windows: a box of a
// float image copied from global to shared memory by one
// cp.async.bulk.tensor, its completion counted on a shared-memory mbarrier.
//
// The copy's rules, checked by the callers before they issue one:
//  - the tensor map (host, encode_window_map) describes a float image of
//    row stride ld (a multiple of 4 elements) at a 16-byte aligned address;
//  - the box's x coordinate is a multiple of 4 elements (16 bytes); x and y
//    may lie outside the image (a load fills those elements with zeros);
//  - the shared destination is 128-byte aligned.
// Every wait is bounded: a wait that runs out reports failure, and the
// caller raises DB_FLAG_TIMEOUT and leaves the tile.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace db {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the asynchronous proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this CTA's earlier generic-proxy accesses of shared memory (made
// visible to the calling thread by a CTA barrier) before a later TMA write.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of transaction to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait until the phase of parity `parity` has completed, for at most `limit`
// clock cycles; false if the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long limit) {
  if (mbar_test_parity(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test_parity(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// Box of a 3D tensor map (x, y, image) at (x, y, z) into shared memory dst,
// completing `bar`'s transaction count.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Bound of a TMA wait (clock cycles, about 2 s at 2 GHz): a box arrives in
// microseconds.
constexpr long long kTmaWaitLimit = 4000000000LL;

// Host: whether kernels stage windows by TMA (db_set_tma; default on).
bool tma_enabled();

// Host: a 3D tensor map of nz float images (W x H, row stride ld elements,
// image stride zstride elements) at base, with boxes of box_w x box_h x 1.
// False (map unusable) unless base is 16-byte aligned, ld and zstride are
// multiples of 4 and the driver encodes the map.
bool encode_window_map(CUtensorMap* out, const float* base, int W, int H, int ld, int nz, long long zstride,
                       int box_w, int box_h);

}  // namespace db
