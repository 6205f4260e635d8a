// All RRRL iterations of one image in one persistent launch, ordered by
// tile dependencies instead of launch boundaries (the split schedule's
// tiles, Sec. 2.3, Eq. 9-12; no counterpart in the paper).
//
// The work is the task list  (k, phase, tile)  for k = 0..iters-1, phase 0
// (q = (e, W) of a tile from u^k) and phase 1 (the update of a tile from q
// and u^k, writing u^{k+1}), numbered in that order and dealt round-robin to
// co-resident CTAs (cooperative launch): CTA c runs tasks c, c + G, c + 2G,
// ... in order.  A task waits only for the tiles whose output it reads:
//   q_k(T)      needs u^k     on T's blur footprint:  update_{k-1} done there
//   update_k(T) needs q_k     on T's correlation footprint
// Both footprints lie within ry tile rows and rx tile columns of T, with the
// radius taken symmetric and at least one tile.  Every tile publishes
// "iteration k done" in a per-tile counter (release: barrier, fence,
// atomic store), and waiters poll the counters of the neighbourhood
// (acquire: volatile polls, fence, barrier).  The ping-pong buffer that
// update_k(T) overwrites held u^{k-1}; its readers near T (q_{k-1} and
// update_{k-1} within one radius) finished before the q_k tiles that
// update_k(T) waited for could start, so write-after-read needs no extra
// wait, and likewise for the q buffer.  Every task waits only for tasks of
// lower number; the lowest unfinished task belongs to a resident CTA that has
// finished all its earlier (lower) tasks, so it runs and the run cannot
// deadlock.  Each wait is bounded all the same (time-out: DB_FLAG_TIMEOUT,
// the run aborts its waits and finishes).  One-axis PSFs run the one-axis
// tile bodies of the split schedule (box sums or register windows).
#include <cuda_runtime.h>

#include "internal.cuh"
#include "rrl_box.cuh"
#include "rrl_tiles.cuh"

namespace db {

constexpr int kFTH = 32, kFTW = 32, kFR = 8;  // tiles: 32 x 32, 128 threads

struct FlowArgs {
  const float* f; int ldf;
  float* A; int ldA;        // u^0; u^k for even k
  float* B; int ldB;        // u^k for odd k
  float2* q; int ldq;
  int H, W;
  const TapGroup* groups; const int* ngroups; int kh, kw, ng_max;
  RrlParams p;
  int tx, ty, rx, ry;       // tile grid and dependency radius (tiles)
  int iters;
  int* abort_;              // set on a time-out: later waits are skipped
  int* done_q; int* done_u; // per-tile counters: iterations completed
  int* status;
  long long spin_limit;
};

// Warp 0 polls the counters of the (2ry+1) x (2rx+1) tile neighbourhood of
// (bi, bj) until each is >= need.  Returns false on time-out.
__device__ bool flow_wait(const FlowArgs& a, const int* cnt, int bi, int bj, int need) {
  const int lane = threadIdx.x & 31;
  const int nw = 2 * a.rx + 1, n = (2 * a.ry + 1) * nw;
  bool ok = true;
  const long long t0 = clock64();
  const volatile int* ab = a.abort_;
  for (int idx = lane; idx < n; idx += 32) {
    const int ni = bi + idx / nw - a.ry, nj = bj + idx % nw - a.rx;
    if (ni < 0 || ni >= a.ty || nj < 0 || nj >= a.tx) continue;
    const volatile int* c = cnt + ni * a.tx + nj;
    // polled without a back-off: the waiting warp's CTA has nothing else to
    // do, and a 32 ns sleep between polls measured 1.3% slower on line1024
    while (*c < need) {
      if (*ab != 0) break;
      if (clock64() - t0 > a.spin_limit) { ok = false; break; }
    }
  }
  __threadfence();
  return __all_sync(0xffffffffu, ok);
}

// Dependency wait run inside a tile body (the tile's hook between the copies
// of what is ready anyway -- f, the tap records -- and of what the wait
// guards), so those copies overlap the wait.  Warp 0 polls; a time-out sets
// the abort flag and DB_FLAG_TIMEOUT.
struct FlowDep {
  const FlowArgs* a;
  const int* cnt;
  int bi, bj, need;
  __device__ void operator()() const {
    if (need > 0 && threadIdx.y == 0) {  // warp 0 (blockDim.x == 32)
      const bool ok = flow_wait(*a, cnt, bi, bj, need);
      if (!ok && threadIdx.x == 0) {
        atomicExch(a->abort_, 1);
        if (a->status) atomicOr(a->status, DB_FLAG_TIMEOUT);
      }
    }
    __syncthreads();
  }
};

// AX: 0 tap groups (halo class P); 1, 2 horizontal, vertical box; 3, 4
// horizontal, vertical one-axis PSF with register windows.
template <int P, int AX>
__global__ void __launch_bounds__((kFTH / kFR) * kFTW, 7) k_rrl_flow(FlowArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int ntiles = a.tx * a.ty;
  const int total = a.iters * 2 * ntiles;
  // tasks are dealt round-robin: CTA c runs c, c + G, c + 2G, ... in order
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    const int k = t / (2 * ntiles), rem = t - k * 2 * ntiles;
    const int phase = rem >= ntiles ? 1 : 0, T = rem - phase * ntiles;
    const int bi = T / a.tx, bj = T - bi * a.tx;
    // update tasks wait before their first copy (their u window is guarded
    // too); q tasks inside q_tile, after copying f and the tap records
    if (phase == 1) FlowDep{&a, a.done_q, bi, bj, k + 1}();
    const bool even = (k & 1) == 0;
    const float* src = even ? a.A : a.B;
    const int lds = even ? a.ldA : a.ldB;
    constexpr bool HORIZ = AX == 1 || AX == 3, BOX = AX <= 2;
    if (phase == 0) {
      const FlowDep dep{&a, a.done_u, bi, bj, k};  // k == 0: nothing to wait for (need 0)
      if constexpr (AX == 0)
        q_tile<kFTH, kFTW, kFR, P>(smem, a.f, a.ldf, src, lds, a.q, a.ldq, a.H, a.W, a.groups, a.ngroups, a.kh,
                                      a.kw, a.ng_max, a.p, bi * kFTH, bj * kFTW, dep);
      else
        q_tile_box<kFTH, kFTW, kFR, HORIZ, BOX>(smem, a.f, a.ldf, src, lds, a.q, a.ldq, a.H, a.W, a.ngroups, a.p,
                                                bi * kFTH, bj * kFTW, dep);
    } else {
      float* dst = even ? a.B : a.A;
      const int ldd = even ? a.ldB : a.ldA;
      if constexpr (AX == 0)
        update_tile<kFTH, kFTW, kFR, P>(smem, a.q, a.ldq, src, lds, dst, ldd, a.H, a.W, a.groups, a.ngroups,
                                           a.kh, a.kw, a.ng_max, a.p, a.status, bi * kFTH, bj * kFTW);
      else
        update_tile_box<kFTH, kFTW, kFR, HORIZ, BOX>(smem, a.q, a.ldq, src, lds, dst, ldd, a.H, a.W, a.ngroups,
                                                     a.p, a.status, bi * kFTH, bj * kFTW);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicExch((phase == 0 ? a.done_q : a.done_u) + T, k + 1);
    }
  }
}

size_t flow_smem(int kh, int kw, int ng_max, int axis) {
  const bool horiz = kh == 1;
  const int L = horiz ? kw : kh;
  const size_t sq = axis ? box_smem_q(kFTH, kFTW, L, horiz) : split_smem_q(kFTH, kFTW, kh, kw, ng_max);
  const size_t su = axis ? box_smem_update(kFTH, kFTW, L, horiz) : split_smem_update(kFTH, kFTW, kh, kw, ng_max);
  return sq > su ? sq : su;
}

int flow_tiles(int H, int W) { return ((H + kFTH - 1) / kFTH) * ((W + kFTW - 1) / kFTW); }

size_t flow_ws_bytes(int H, int W) { return (size_t)(2 * flow_tiles(H, W) + 64) * sizeof(int); }

static long long g_flow_spin = 4000000000LL;  // ~2 s at 2 GHz
void set_flow_spin_limit(long long cycles) { g_flow_spin = cycles; }

template <int P, int AX = 0>
static cudaError_t launch_flow_p(FlowArgs a, size_t smem, cudaStream_t s) {
  auto kern = k_rrl_flow<P, AX>;
  cudaError_t e;
  if (smem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int nthreads = (kFTH / kFR) * kFTW;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = a.tx * a.ty;
  int grid = sms * per_sm;
  if (grid > 2 * ntiles) grid = 2 * ntiles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32, nthreads / 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, kern, a)) != cudaSuccess) return e;
  count_launch();
  return cudaSuccess;
}

static cudaError_t launch_flow_groups(const FlowArgs& a, size_t smem, cudaStream_t s) {
  switch (split_halo_class(a.kw)) {
    case 8: return launch_flow_p<8>(a, smem, s);
    case 16: return launch_flow_p<16>(a, smem, s);
    case 32: return launch_flow_p<32>(a, smem, s);
    case 64: return launch_flow_p<64>(a, smem, s);
    case 128: return launch_flow_p<128>(a, smem, s);
    default: return launch_flow_p<256>(a, smem, s);
  }
}

cudaError_t launch_rrl_flow(const float* f, int ldf, float* u, int ldu, float* utmp, int ldt, float2* q, int H, int W,
                            const TapGroup* groups, const int* ngroups, int kh, int kw, int ng_bound,
                            const RrlParams& p, int iters, void* flow_ws, int* status, cudaStream_t s, int axis) {
  if (iters <= 0) return cudaSuccess;
  FlowArgs a = {};
  a.f = f; a.ldf = ldf;
  a.A = u; a.ldA = ldu; a.B = utmp; a.ldB = ldt;
  a.q = q; a.ldq = qpitch(W);
  a.H = H; a.W = W;
  a.groups = groups; a.ngroups = ngroups; a.kh = kh; a.kw = kw;
  a.ng_max = ng_bound > 0 ? ng_bound : max_tap_groups(kh, kw);
  a.p = p;
  a.tx = (W + kFTW - 1) / kFTW; a.ty = (H + kFTH - 1) / kFTH;
  // footprint half-widths: blur and correlation reach cy / kh-1-cy rows and
  // cx / kw-1-cx columns, the diffusion term 2; staging rounds the column
  // window out to 16-byte chunks (up to 4 more columns)
  const int cy = kh >> 1, cx = kw >> 1;
  int hy = kh - 1 - cy > cy ? kh - 1 - cy : cy;
  int hx = kw - 1 - cx > cx ? kw - 1 - cx : cx;
  hy = hy > 2 ? hy : 2;
  hx = (hx > 2 ? hx : 2) + 4;
  a.ry = (hy + kFTH - 1) / kFTH; a.rx = (hx + kFTW - 1) / kFTW;
  a.iters = iters;
  int* w = (int*)flow_ws;
  a.abort_ = w;
  a.done_q = w + 64; a.done_u = w + 64 + a.tx * a.ty;
  a.status = status;
  a.spin_limit = g_flow_spin;
  cudaError_t e;
  if ((e = cudaMemsetAsync(flow_ws, 0, flow_ws_bytes(H, W), s)) != cudaSuccess) return e;
  const size_t smem = flow_smem(kh, kw, a.ng_max, axis);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (axis) {
    const int ax = (axis == 1 ? 0 : 2) + (kh == 1 ? 1 : 2);
    switch (ax) {
      case 1: e = launch_flow_p<8, 1>(a, smem, s); break;
      case 2: e = launch_flow_p<8, 2>(a, smem, s); break;
      case 3: e = launch_flow_p<8, 3>(a, smem, s); break;
      default: e = launch_flow_p<8, 4>(a, smem, s); break;
    }
  } else {
    e = launch_flow_groups(a, smem, s);
  }
  if (e != cudaSuccess) (void)cudaGetLastError();
  return e;
}

}  // namespace db
