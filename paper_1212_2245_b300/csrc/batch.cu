// Batched WR3L: many images of uneven sizes, each with its own PSF and
// parameters, deblurred together (no counterpart in the paper; the closest is
// its persistent worker threads, Sec. 4.5).  The arithmetic per image is
// exactly the single-image pipeline's (same tile bodies, same transforms).
//
// Plan (host, once): per-axis transform tables, tap groups and PSF spectra
// for every image, the batched-Wiener job tables, a table of RRRL tiles over
// all images (sorted by cost), all uploaded into the caller's workspace.
// Run (capturable: stream-ordered launches and memsets only):
//   1. the batched Wiener launches (one per transform stage and column class);
//   2. one cooperative persistent launch that performs every RRRL iteration
//      of every image: per iteration a q-phase and an update-phase over all
//      tiles, tiles taken from an atomic work queue, phases separated by a
//      grid barrier (or, in the dependency order, per-image counters) whose
//      wait is bounded (on time-out it raises DB_FLAG_TIMEOUT and the kernel
//      returns).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "fft_df.cuh"
#include "internal.cuh"
#include "rrl_box.cuh"
#include "rrl_dense.cuh"
#include "rrl_fft_tile.cuh"
#include "rrl_tiles.cuh"

namespace db {

struct BatchImg {
  const float* f;
  float* A;      // holds u0; written by odd iterations
  float* B;      // written by even iterations
  float2* q;     // (e, W), pitch W
  const TapGroup* groups;
  const int* ngroups;
  int ldf, ldA, ldB, ldq;
  int H, W, kh, kw, ng_max, P;
  int box;       // 0: tap groups; 1, 2: horizontal, vertical box (sliding-window sums);
                 // 3, 4: other horizontal, vertical one-axis PSF (register windows)
  int kwd;       // dense-eligible 2D PSF: kw (the dense flag then picks the bodies); else 0
  int fft;       // 1: FFT tiles (rrl_fft_tile.cuh); the tile tables then hold that grid
  int nq, nu;    // the image's tiles in the q and the update tile table
  RrlParams p;
};

constexpr int kBTH = 32, kBTW = 64, kBR = 8;  // tiles of the split schedule

// Shared-memory slot of one queued tile: its index, (image, i0, j0, cost)
// and a copy of its image's descriptor.
struct TileSlot {
  BatchImg im;
  int4 T;
  int t;
  int k, phase;  // dependency-ordered kernel: the task's iteration and phase,
  int ready;     // and whether its wait was already satisfied when the slot was filled
};
constexpr int kImgWords = (int)(sizeof(BatchImg) / 4);
static_assert(sizeof(BatchImg) % 4 == 0 && kImgWords <= 64, "descriptor copied by one warp");

// Warp 0 fills a slot: tile t (from the work queue) and its descriptor.
__device__ __forceinline__ void fill_slot(TileSlot* slot, int t, const BatchImg* __restrict__ imgs,
                                          const int4* __restrict__ tiles, int ntiles) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) slot->t = t;
  if (t >= ntiles) return;
  const int4 T = tiles[t];
  if (lane == 0) slot->T = T;
  const unsigned* src = reinterpret_cast<const unsigned*>(imgs + T.x);
  unsigned* dst = reinterpret_cast<unsigned*>(&slot->im);
  for (int w = lane; w < kImgWords; w += 32) dst[w] = __ldg(src + w);
}

// Work-queue state of a CTA of the persistent kernel: two tile slots and
// the queue's tables (shared memory of the kernel, set up at its start).
struct QueueState {
  TileSlot slot[2];
  const BatchImg* imgs;
  const int4* tiles;
  int ntiles;
};
__shared__ __align__(16) QueueState g_queue;

// Warp 0 fills the other slot with the next tile of the queue, whose index
// thread 0 requested when the current tile began (so the atomic's latency
// is hidden behind the tile), and with its descriptor.  Done once the
// current tile's work is issued; the CTA's barrier then publishes it.
__device__ __forceinline__ void fetch_next(int slot, int next) {
  if (threadIdx.y == 0 && threadIdx.x < 32) {
    const int t = __shfl_sync(0xffffffffu, next, 0);
    fill_slot(&g_queue.slot[slot], t, g_queue.imgs, g_queue.tiles, g_queue.ntiles);
  }
}

template <int P>
__device__ __noinline__ void batch_q(unsigned char* smem, const BatchImg& im, const float* src, int lds,
                                     int i0, int j0) {
  q_tile<kBTH, kBTW, kBR, P>(smem, im.f, im.ldf, src, lds, im.q, im.ldq, im.H, im.W, im.groups,
                                im.ngroups, im.kh, im.kw, im.ng_max, im.p, i0, j0);
}

template <int P>
__device__ __noinline__ void batch_u(unsigned char* smem, const BatchImg& im, const float* src, int lds,
                                     float* dst, int ldd, int* status, int i0, int j0) {
  update_tile<kBTH, kBTW, kBR, P>(smem, im.q, im.ldq, src, lds, dst, ldd, im.H, im.W, im.groups,
                                     im.ngroups, im.kh, im.kw, im.ng_max, im.p, status, i0, j0);
}

template <bool HORIZ, bool BOX>
__device__ __noinline__ void batch_box(int phase, unsigned char* smem, const BatchImg& im, const float* src, int lds,
                                       float* dst, int ldd, int* status, int i0, int j0) {
  if (phase == 0)
    q_tile_box<kBTH, kBTW, kBR, HORIZ, BOX>(smem, im.f, im.ldf, src, lds, im.q, im.ldq, im.H, im.W, im.ngroups, im.p,
                                            i0, j0);
  else
    update_tile_box<kBTH, kBTW, kBR, HORIZ, BOX>(smem, im.q, im.ldq, src, lds, dst, ldd, im.H, im.W, im.ngroups,
                                                 im.p, status, i0, j0);
}

template <int KW>
__device__ __noinline__ void batch_dense(int phase, unsigned char* smem, const BatchImg& im, const float* src,
                                         int lds, float* dst, int ldd, int* status, int i0, int j0) {
  const int ldp = upitch(im.W);
  float* qe = reinterpret_cast<float*>(im.q);
  float* qw = qe + (size_t)im.H * ldp;
  const float* tab = dense_taps(im.groups, im.kh, im.kw);
  if (phase == 0)
    q_tile_dense<kBTH, kBTW, KW>(smem, im.f, im.ldf, src, lds, qe, qw, ldp, im.H, im.W, tab, im.kh, im.p, i0, j0);
  else
    update_tile_dense<kBTH, kBTW, KW>(smem, qe, qw, ldp, src, lds, dst, ldd, im.H, im.W, tab, im.kh, im.p, status,
                                      i0, j0);
}

// FFT tiles: a q-phase record holds the left tile of a horizontal pair.
__device__ __noinline__ void batch_fft(int phase, unsigned char* smem, const BatchImg& im, const float* src, int lds,
                                       float* dst, int ldd, int* status, int i0, int j0) {
  const int ldp = upitch(im.W);
  float* qe = reinterpret_cast<float*>(im.q);
  float* qw = qe + (size_t)im.H * ldp;
  const float2* spec = fft_tile_spec(im.groups, im.kh, im.kw);
  if (phase == 0)
    ftile::q_tile(smem, im.f, im.ldf, src, lds, qe, qw, ldp, im.H, im.W, spec, im.kh, im.kw, im.p, i0, j0);
  else
    ftile::update_tile(smem, qe, qw, ldp, src, lds, dst, ldd, im.H, im.W, spec, im.kh, im.kw, im.p, status, i0, j0);
}

__device__ __forceinline__ void batch_tile(int phase, unsigned char* smem, const BatchImg& im, const float* src,
                                           int lds, float* dst, int ldd, int* status, int i0, int j0) {
  if (im.kwd && __ldg(dense_flag(im.ngroups))) {
    switch (im.kwd) {
      case 3: batch_dense<3>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 5: batch_dense<5>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 7: batch_dense<7>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 9: batch_dense<9>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 11: batch_dense<11>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 13: batch_dense<13>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 15: batch_dense<15>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 17: batch_dense<17>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 19: batch_dense<19>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 21: batch_dense<21>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      case 23: batch_dense<23>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
      default: batch_dense<25>(phase, smem, im, src, lds, dst, ldd, status, i0, j0); return;
    }
  }
#define DB_BATCH_CASE(PV)                                           \
  case PV:                                                          \
    if (phase == 0) batch_q<PV>(smem, im, src, lds, i0, j0);        \
    else batch_u<PV>(smem, im, src, lds, dst, ldd, status, i0, j0); \
    break;
  switch (im.P) {
    DB_BATCH_CASE(8)
    DB_BATCH_CASE(16)
    DB_BATCH_CASE(32)
    DB_BATCH_CASE(64)
    DB_BATCH_CASE(128)
    default: DB_BATCH_CASE(256)
  }
#undef DB_BATCH_CASE
}

// Grid-wide barrier for a cooperatively launched grid.  bar[0] counts
// arrivals, bar[1] is the generation.  The wait is bounded by `limit` clock
// cycles; returns false (and raises DB_FLAG_TIMEOUT) if it gave up.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > limit) {
          ok = 0;
          if (status) atomicOr(status, DB_FLAG_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// tiles_q / tiles_u: the tile tables of the q and update phases (they
// differ for images with FFT tiles, whose q tiles go in pairs).
__global__ void __launch_bounds__(256, 3) k_rrl_batch(const BatchImg* __restrict__ imgs,
                                                   const int4* __restrict__ tiles_q, int ntiles_q,
                                                   const int4* __restrict__ tiles_u, int ntiles_u, int iters,
                                                   unsigned* bar, int* work, int* status,
                                                   long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid == 0) g_queue.imgs = imgs;
  for (int k = 0; k < iters; ++k) {
    const bool even = (k & 1) == 0;
    for (int phase = 0; phase < 2; ++phase) {
      int* queue = work + 2 * k + phase;
      const int4* tiles = phase == 0 ? tiles_q : tiles_u;
      const int ntiles = phase == 0 ? ntiles_q : ntiles_u;
      if (tid == 0) {
        g_queue.tiles = tiles;
        g_queue.ntiles = ntiles;
      }
      // the phase's first tile, then each tile prefetches the next one
      if (tid < 32) {
        int t = 0;
        if (tid == 0) t = atomicAdd(queue, 1);
        fill_slot(&g_queue.slot[0], __shfl_sync(0xffffffffu, t, 0), imgs, tiles, ntiles);
      }
      __syncthreads();
      int cur = 0;
      while (g_queue.slot[cur].t < ntiles) {
        int next = 0;
        if (tid == 0) next = atomicAdd(queue, 1);
        const BatchImg& im = g_queue.slot[cur].im;
        const int4 T = g_queue.slot[cur].T;
        const float* src = even ? im.A : im.B;
        const int lds = even ? im.ldA : im.ldB;
        float* dst = even ? im.B : im.A;
        const int ldd = even ? im.ldB : im.ldA;
        if (im.fft) batch_fft(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
        else if (im.box == 1) batch_box<true, true>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
        else if (im.box == 2) batch_box<false, true>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
        else if (im.box == 3) batch_box<true, false>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
        else if (im.box == 4) batch_box<false, false>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
        else batch_tile(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
        fetch_next(cur ^ 1, next);
        __syncthreads();
        cur ^= 1;
      }
      if (!grid_barrier(bar, gridDim.x, status, spin_limit)) return;
    }
  }
}

// ---------------------------------------------------------------------------
// Dependency-ordered form of the same run: one task list over all
// iterations, task t = k (nq + nu) + (q tile t' | nq + update tile t'), taken
// from one atomic counter in order.  A q task of image i in iteration k waits
// until all update tiles of image i in iterations < k are done (its u is
// complete), an update task until all q tiles of image i in iterations <= k
// are done (its q is complete); per-image counters count completed tiles.
// That also orders the ping-pong and q overwrites: every reader of the
// buffer a task overwrites belongs to an earlier phase of the same image,
// which the task's predecessors waited for.  The phases of different images
// overlap instead of meeting at grid barriers.
// No deadlock: a task waits only for lower-numbered tasks; the lowest
// unfinished task is the current task of a resident CTA (a CTA's prefetched
// next task is numbered above its current one), so it can always proceed.
// Waits are bounded by the spin limit (DB_FLAG_TIMEOUT, then the CTA stops).
// The arithmetic of every tile is unchanged, so both forms give the same bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Completed tiles a task needs of its image's counter (see k_rrl_batch_dep).
__device__ __forceinline__ int task_need(const BatchImg* __restrict__ imgs, int img, int k, int phase) {
  return phase == 0 ? k * __ldg(&imgs[img].nu) : (k + 1) * __ldg(&imgs[img].nq);
}

__device__ __forceinline__ void fill_task(TileSlot* slot, int t, int total, const BatchImg* __restrict__ imgs,
                                          const int4* __restrict__ tiles_q, int nq,
                                          const int4* __restrict__ tiles_u, int nu, const int* done, int n) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) slot->t = t;
  if (t >= total) return;
  const int per = nq + nu, k = t / per, r = t - k * per;
  const int phase = r >= nq ? 1 : 0;
  const int4 T = phase ? tiles_u[r - nq] : tiles_q[r];
  if (lane == 0) {
    slot->T = T;
    slot->k = k;
    slot->phase = phase;
    // acquire now: the CTA's barrier before the task orders its reads after it
    slot->ready = ld_acquire(done + (phase == 0 ? n : 0) + T.x) >= task_need(imgs, T.x, k, phase);
  }
  const unsigned* src = reinterpret_cast<const unsigned*>(imgs + T.x);
  unsigned* dst = reinterpret_cast<unsigned*>(&slot->im);
  for (int w = lane; w < kImgWords; w += 32) dst[w] = __ldg(src + w);
}

// done[0 .. n): completed q tiles per image, done[n .. 2n): update tiles.
__global__ void __launch_bounds__(256, 3) k_rrl_batch_dep(const BatchImg* __restrict__ imgs, int n,
                                                       const int4* __restrict__ tiles_q, int ntiles_q,
                                                       const int4* __restrict__ tiles_u, int ntiles_u,
                                                       int iters, int* work, int* done, int* status,
                                                       long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_ok;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int total = iters * (ntiles_q + ntiles_u);
  if (tid < 32) {
    int t = 0;
    if (tid == 0) t = atomicAdd(work, 1);
    fill_task(&g_queue.slot[0], __shfl_sync(0xffffffffu, t, 0), total, imgs, tiles_q, ntiles_q, tiles_u, ntiles_u,
              done, n);
  }
  __syncthreads();
  int cur = 0;
  while (g_queue.slot[cur].t < total) {
    int next = 0;
    if (tid == 0) next = atomicAdd(work, 1);
    const BatchImg& im = g_queue.slot[cur].im;
    const int4 T = g_queue.slot[cur].T;
    const int k = g_queue.slot[cur].k, phase = g_queue.slot[cur].phase;
    if (!g_queue.slot[cur].ready) {  // wait (bounded) for the image's previous phase
      if (tid == 0) {
        s_ok = 1;
        const int need = phase == 0 ? k * im.nu : (k + 1) * im.nq;
        const int* cnt = done + (phase == 0 ? n : 0) + T.x;
        const long long t0 = clock64();
        while (ld_acquire(cnt) < need) {
          if (clock64() - t0 > spin_limit) {
            s_ok = 0;
            if (status) atomicOr(status, DB_FLAG_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      if (!s_ok) return;
    }
    const bool even = (k & 1) == 0;
    const float* src = even ? im.A : im.B;
    const int lds = even ? im.ldA : im.ldB;
    float* dst = even ? im.B : im.A;
    const int ldd = even ? im.ldB : im.ldA;
    if (im.fft) batch_fft(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
    else if (im.box == 1) batch_box<true, true>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
    else if (im.box == 2) batch_box<false, true>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
    else if (im.box == 3) batch_box<true, false>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
    else if (im.box == 4) batch_box<false, false>(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
    else batch_tile(phase, smem, im, src, lds, dst, ldd, status, T.y, T.z);
    __syncthreads();  // the tile's outputs are written
    if (tid == 0) red_release_add(done + (phase == 0 ? 0 : n) + T.x, 1);
    if (threadIdx.y == 0 && threadIdx.x < 32)
      fill_task(&g_queue.slot[cur ^ 1], __shfl_sync(0xffffffffu, next, 0), total, imgs, tiles_q, ntiles_q, tiles_u,
                ntiles_u, done, n);
    __syncthreads();
    cur ^= 1;
  }
}

static std::atomic<long long> g_spin_limit{4000000000LL};  // ~2 s at 2 GHz
// Batch run order (db_set_batch_order): 0 dependency-ordered, 1 phases
// separated by grid barriers (the default: on batch512 56.7 against 59.4 ms
// per run; the dependency form pays a barrier, a release and an acquire per
// tile, about a million tiles per run, where the barrier form pays twenty
// grid barriers).
static std::atomic<int> g_batch_order{1};

// Largest dynamic shared memory k_rrl_batch has been allowed on each device.
static std::mutex g_smem_mutex;
static std::map<int, size_t> g_smem_limit;

static cudaError_t raise_batch_smem_limit(size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_smem_mutex);
  size_t& cur = g_smem_limit[dev];
  if (smem <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(k_rrl_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rrl_batch_dep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) cur = smem;
  return e;
}

void set_spin_limit(long long cycles) {
  g_spin_limit.store(cycles);
  set_flow_spin_limit(cycles);
}

// ---------------------------------------------------------------------------
// host plan
// ---------------------------------------------------------------------------
struct BatchPlan {
  int n = 0, iters = 0;
  WienerBatch* wb = nullptr;
  std::vector<BatchImg> imgs;
  std::vector<int4> tiles_q, tiles_u;
  BatchImg* d_imgs = nullptr;
  int4* d_tiles_q = nullptr;
  int4* d_tiles_u = nullptr;
  unsigned* d_bar = nullptr;
  int* d_work = nullptr;
  int* d_done = nullptr;  // per-image completed-tile counters (dependency order)
  int order = 1;          // 0 dependency-ordered, 1 grid barriers (db_set_batch_order at creation)
  size_t smem = 0;
  int grid = 0;
  // tunable forms (db_batch_autotune): per image the dense width of a
  // dense-eligible 2D PSF (else 0), the register-window code of a non-box
  // one-axis PSF (3 row, 4 column; else 0) and the code the size rule chose
  std::vector<int> dense_kw, window_box, rule_box;
  // per image: kh * kw when FFT tiles are possible (a 2D PSF of
  // fft_tile_shape), else 0; images with fft_taps >= fft_min use them
  std::vector<int> fft_taps;
  int fft_min = 0;
  ~BatchPlan() { if (wb) wiener_batch_delete(wb); }
};

// Per-image workspace regions, laid out in order.
struct ImgRegions {
  size_t groups, ngroups, utmp, q, spec, work, kspec, end;
};

static ImgRegions image_regions(size_t off, int H, int W, int kh, int kw) {
  ImgRegions r;
  r.groups = off;  off += tap_region_bytes(kh, kw);
  r.ngroups = off; off += kAuxBytes;
  r.utmp = off;    off += align256((size_t)H * upitch(W) * sizeof(float));
  r.q = off;       off += align256((size_t)H * upitch(W) * sizeof(float2));
  size_t spec = (kh == 1) ? (size_t)W : (kw == 1) ? (size_t)H : (size_t)H * W;
  r.spec = off;    off += align256(spec * sizeof(float4));
  r.work = off;    off += (kh > 1 && kw > 1) ? align256((size_t)H * W * sizeof(float4)) : 0;
  r.kspec = off;   off += align256(wiener_kspec_elems(H, W, kh, kw) * sizeof(float4));
  r.end = off;
  return r;
}

static size_t count_tiles(int H, int W) {
  return (size_t)((H + kBTH - 1) / kBTH) * ((W + kBTW - 1) / kBTW);
}
// Capacity of one tile table for an image: either grid may be chosen later
// (db_batch_autotune).
static size_t count_tiles_max(int H, int W, int kh, int kw) {
  size_t n = count_tiles(H, W);
  if (fft_tile_shape(kh, kw) && kh > 1 && kw > 1) {
    const size_t f = (size_t)((H + ftile::tile_oh(kh) - 1) / ftile::tile_oh(kh)) *
                     ((W + ftile::tile_ow(kw) - 1) / ftile::tile_ow(kw));
    n = std::max(n, f);
  }
  return n;
}

// Tile tables from the images' current forms: the split grid (kBTH x kBTW)
// in both phases, or for FFT tiles the (65-kh) x (65-kw) grid, whose q-phase
// tiles go in horizontal pairs.  Expensive tiles first (the work queue then
// ends on cheap ones); .w is a cost estimate (tap-group bound, or
// kFftTileCost for an FFT tile: about the time of a 25 x 25 dense tile's
// tap sums over 32 x 64 outputs scaled by 8k / 55k cycles).
constexpr int kFftTileCost = 48;
static void build_tiles(BatchPlan* P) {
  P->tiles_q.clear();
  P->tiles_u.clear();
  for (int i = 0; i < P->n; ++i) {
    BatchImg& bi = P->imgs[i];
    const size_t q0 = P->tiles_q.size(), u0 = P->tiles_u.size();
    if (bi.fft) {
      const int oh = ftile::tile_oh(bi.kh), ow = ftile::tile_ow(bi.kw);
      for (int i0 = 0; i0 < bi.H; i0 += oh) {
        for (int j0 = 0; j0 < bi.W; j0 += ow) P->tiles_u.push_back(make_int4(i, i0, j0, kFftTileCost));
        for (int j0 = 0; j0 < bi.W; j0 += 2 * ow) P->tiles_q.push_back(make_int4(i, i0, j0, kFftTileCost));
      }
    } else {
      for (int i0 = 0; i0 < bi.H; i0 += kBTH)
        for (int j0 = 0; j0 < bi.W; j0 += kBTW) {
          P->tiles_q.push_back(make_int4(i, i0, j0, bi.ng_max));
          P->tiles_u.push_back(make_int4(i, i0, j0, bi.ng_max));
        }
    }
    bi.nq = (int)(P->tiles_q.size() - q0);
    bi.nu = (int)(P->tiles_u.size() - u0);
  }
  auto by_cost = [](const int4& a, const int4& b) { return a.w > b.w; };
  std::stable_sort(P->tiles_q.begin(), P->tiles_q.end(), by_cost);
  std::stable_sort(P->tiles_u.begin(), P->tiles_u.end(), by_cost);
}

static cudaError_t upload_tiles(const BatchPlan* P, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(P->d_tiles_q, P->tiles_q.data(), P->tiles_q.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(P->d_tiles_u, P->tiles_u.data(), P->tiles_u.size() * sizeof(int4), cudaMemcpyHostToDevice,
                         s);
}

// Bytes of workspace the whole batch needs; 0 if any descriptor is invalid.
size_t batch_ws_bytes(const db_image_desc* d, int n, int iters, db_status* why) {
  *why = DB_OK;
  if (!d || n < 1 || iters < 0) { *why = DB_ERR_ARG; return 0; }
  size_t off = 0;
  std::map<int, bool> lens;
  size_t ntiles = 0, nitems = 0;
  for (int i = 0; i < n; ++i) {
    const db_image_desc& x = d[i];
    if (!x.f || !x.u || !x.psf.taps) { *why = DB_ERR_ARG; return 0; }
    if (x.H < 1 || x.W < 1 || x.H > kMaxSide || x.W > kMaxSide || x.ld < x.W) { *why = DB_ERR_SHAPE; return 0; }
    if (x.psf.kh < 1 || x.psf.kw < 1 || x.psf.kh > kMaxTapSide || x.psf.kw > kMaxTapSide ||
        x.psf.kh > x.H || x.psf.kw > x.W) { *why = DB_ERR_PSF; return 0; }
    if (x.psf.kind == DB_PSF_BOX && x.psf.kh != 1 && x.psf.kw != 1) { *why = DB_ERR_PSF; return 0; }
    if (x.psf.kind != DB_PSF_GENERAL && x.psf.kind != DB_PSF_BOX) { *why = DB_ERR_ARG; return 0; }
    if (!(x.p.K > 0.f) || !(x.p.alpha >= 0.f) || !(x.p.eps_phi > 0.f) || !(x.p.eps_psi > 0.f) ||
        !(x.p.pos_floor > 0.f) || (x.p.phi_robust != 0 && x.p.phi_robust != 1) ||
        (x.p.psi_tv != 0 && x.p.psi_tv != 1)) { *why = DB_ERR_ARG; return 0; }
    if (x.p.conv != DB_CONV_CLAMP) { *why = DB_ERR_UNSUPPORTED; return 0; }
    if (x.f == x.u) { *why = DB_ERR_ARG; return 0; }
    const int ngm = max_tap_groups(x.psf.kh, x.psf.kw);
    if (split_smem_q(kBTH, kBTW, x.psf.kh, x.psf.kw, ngm) > 227 * 1024 ||
        split_smem_update(kBTH, kBTW, x.psf.kh, x.psf.kw, ngm) > 227 * 1024) {
      *why = DB_ERR_UNSUPPORTED; return 0;
    }
    off = image_regions(off, x.H, x.W, x.psf.kh, x.psf.kw).end;
    if (x.psf.kw > 1 || x.psf.kh == 1) lens[x.W] = true;
    if (x.psf.kh > 1) lens[x.H] = true;
    ntiles += count_tiles_max(x.H, x.W, x.psf.kh, x.psf.kw);
    nitems += (size_t)2 * x.H + x.W;  // upper bound on Wiener work items
  }
  for (auto& kv : lens) off += align256(dft_table_elems(kv.first) * sizeof(float4));
  off += align256((size_t)n * sizeof(BatchImg));
  off += 2 * align256(ntiles * sizeof(int4));          // q and update tile tables
  off += 256;                                         // barrier
  off += align256((size_t)(2 * iters + 2) * sizeof(int));  // work counters
  off += align256((size_t)2 * n * sizeof(int));        // per-image tile counters
  // batched-Wiener job tables (8 stages x (jobs + 3 item classes) regions):
  // at most 3 jobs per image, one item per row
  // (pair) or column group (bounded by nitems), plus alignment slack
  off += 32 * 256 + (size_t)3 * n * wiener_job_bytes() + nitems * sizeof(int2);
  return off;
}

db_status batch_create(const db_image_desc* d, int n, int iters, void* ws, size_t ws_bytes,
                       int* status, cudaStream_t s, BatchPlan** out) {
  db_status why;
  const size_t need = batch_ws_bytes(d, n, iters, &why);
  if (need == 0) return why;
  if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < need) return DB_ERR_WORKSPACE;
  BatchPlan* P = new BatchPlan();
  P->n = n;
  P->iters = iters;
  P->wb = wiener_batch_new();
  char* base = (char*)ws;
  size_t off = 0;
  std::vector<ImgRegions> reg(n);
  for (int i = 0; i < n; ++i) {
    reg[i] = image_regions(off, d[i].H, d[i].W, d[i].psf.kh, d[i].psf.kw);
    off = reg[i].end;
  }
  // transform tables per distinct axis length
  std::map<int, std::pair<Dft1ff, Dft1>> dfts;
  std::vector<int> lens;
  for (int i = 0; i < n; ++i) {
    if (d[i].psf.kw > 1 || d[i].psf.kh == 1) lens.push_back(d[i].W);
    if (d[i].psf.kh > 1) lens.push_back(d[i].H);
  }
  std::sort(lens.begin(), lens.end());
  lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
  cudaError_t e = cudaSuccess;
  for (int N : lens) {
    Dft1ff ff;
    Dft1 f32;
    e = prepare_dft(N, (float4*)(base + off), &ff, &f32, s);
    if (e != cudaSuccess) { delete P; return DB_ERR_CUDA; }
    dfts[N] = std::make_pair(ff, f32);
    off += align256(dft_table_elems(N) * sizeof(float4));
  }
  // per image: tap groups, Wiener set-up, RRRL descriptor and tiles
  P->imgs.resize(n);
  size_t ntiles_cap = 0;
  for (int i = 0; i < n; ++i) {
    const db_image_desc& x = d[i];
    const ImgRegions& r = reg[i];
    const int kh = x.psf.kh, kw = x.psf.kw;
    TapGroup* groups = (TapGroup*)(base + r.groups);
    int* ngroups = (int*)(base + r.ngroups);
    if (launch_prepare_taps(x.psf.taps, kh, kw, x.psf.kind, groups, ngroups, status, s) != cudaSuccess) {
      delete P; return DB_ERR_CUDA;
    }
    float* utmp = (float*)(base + r.utmp);
    float* A = (iters % 2 == 1) ? utmp : x.u;
    const int ldA = (iters % 2 == 1) ? upitch(x.W) : x.ld;
    WienerImage wi = {};
    wi.f = x.f; wi.ld = x.ld; wi.u0 = A; wi.ldu = ldA; wi.H = x.H; wi.W = x.W;
    wi.taps = x.psf.taps; wi.kh = kh; wi.kw = kw; wi.K = x.p.K; wi.floor_ = x.p.pos_floor;
    wi.spec = (float4*)(base + r.spec);
    wi.work = (kh > 1 && kw > 1) ? (float4*)(base + r.work) : nullptr;
    wi.kspec = wiener_kspec_elems(x.H, x.W, kh, kw) ? (float4*)(base + r.kspec) : nullptr;
    wi.pDW = (kw > 1 || kh == 1) ? &dfts[x.W].first : nullptr;
    wi.pDH = (kh > 1) ? &dfts[x.H].first : nullptr;
    if (wiener_batch_add(P->wb, wi, s) != cudaSuccess) { delete P; return DB_ERR_CUDA; }
    BatchImg& bi = P->imgs[i];
    bi.f = x.f; bi.A = A; bi.ldA = ldA;
    bi.B = (iters % 2 == 1) ? x.u : utmp;
    bi.ldB = (iters % 2 == 1) ? x.ld : upitch(x.W);
    bi.ldq = qpitch(x.W);
    bi.q = (float2*)(base + r.q);
    bi.groups = groups; bi.ngroups = ngroups;
    bi.ldf = x.ld; bi.H = x.H; bi.W = x.W; bi.kh = kh; bi.kw = kw;
    bi.ng_max = max_tap_groups(kh, kw);
    bi.P = split_halo_class(kw);
    const int axis = axis_mode(x.psf.kind, kh, kw);
    bi.box = axis == 0 ? 0 : (axis == 1 ? 0 : 2) + (kh == 1 ? 1 : 2);
    bi.kwd = (axis == 0 && dense_eligible(kh, kw)) ? kw : 0;
    P->dense_kw.push_back(bi.kwd);
    P->fft_taps.push_back(axis == 0 && fft_tile_shape(kh, kw) ? kh * kw : 0);
    bi.fft = fft_tile_form(kh, kw) && axis == 0 ? 1 : 0;
    P->window_box.push_back((x.psf.kind != DB_PSF_BOX && (kh == 1 || kw == 1)) ? (kh == 1 ? 3 : 4) : 0);
    P->rule_box.push_back(bi.box);
    bi.p.alpha = x.p.alpha; bi.p.eps_phi = x.p.eps_phi; bi.p.eps_psi = x.p.eps_psi;
    bi.p.floor = x.p.pos_floor; bi.p.phi_robust = x.p.phi_robust; bi.p.psi_tv = x.p.psi_tv;
    bi.p.rf_lut = rf_lut_device();
    size_t sm = bi.box ? std::max(box_smem_q(kBTH, kBTW, kh == 1 ? kw : kh, kh == 1),
                                  box_smem_update(kBTH, kBTW, kh == 1 ? kw : kh, kh == 1))
                       : std::max(split_smem_q(kBTH, kBTW, kh, kw, bi.ng_max),
                                  split_smem_update(kBTH, kBTW, kh, kw, bi.ng_max));
    if (bi.kwd)
      sm = std::max(sm, std::max(dense_smem_q(kBTH, kBTW, kh, kw), dense_smem_update(kBTH, kBTW, kh, kw)));
    if (P->window_box.back()) {  // both one-axis forms may be chosen later (db_batch_autotune)
      const int L = kh == 1 ? kw : kh;
      sm = std::max(sm, std::max(box_smem_q(kBTH, kBTW, L, kh == 1), box_smem_update(kBTH, kBTW, L, kh == 1)));
      sm = std::max(sm, std::max(split_smem_q(kBTH, kBTW, kh, kw, bi.ng_max),
                                 split_smem_update(kBTH, kBTW, kh, kw, bi.ng_max)));
    }
    if (P->fft_taps.back()) sm = std::max(sm, ftile::smem_update(kh));
    if (sm > P->smem) P->smem = sm;
    ntiles_cap += count_tiles_max(x.H, x.W, kh, kw);
  }
  build_tiles(P);
  P->d_imgs = (BatchImg*)(base + off);
  off += align256((size_t)n * sizeof(BatchImg));
  P->d_tiles_q = (int4*)(base + off);
  off += align256(ntiles_cap * sizeof(int4));
  P->d_tiles_u = (int4*)(base + off);
  off += align256(ntiles_cap * sizeof(int4));
  P->d_bar = (unsigned*)(base + off);
  off += 256;
  P->d_work = (int*)(base + off);
  off += align256((size_t)(2 * iters + 2) * sizeof(int));
  P->d_done = (int*)(base + off);
  off += align256((size_t)2 * n * sizeof(int));
  P->order = g_batch_order.load();
  const size_t wtab = wiener_batch_table_bytes(P->wb);
  if (off + wtab > ws_bytes) { delete P; return DB_ERR_WORKSPACE; }
  if (wiener_batch_upload(P->wb, base + off, s) != cudaSuccess) { delete P; return DB_ERR_CUDA; }
  if (cudaMemcpyAsync(P->d_imgs, P->imgs.data(), (size_t)n * sizeof(BatchImg), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      upload_tiles(P, s) != cudaSuccess) {
    delete P; return DB_ERR_CUDA;
  }
  // persistent grid: every co-resident CTA.  The kernel's shared-memory
  // limit only ever grows (per device), so that plans made earlier with
  // larger tiles keep launching.
  if (P->smem > 48 * 1024 && raise_batch_smem_limit(P->smem) != cudaSuccess) {
    (void)cudaGetLastError();
    delete P; return DB_ERR_UNSUPPORTED;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      (P->order == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rrl_batch_dep, 256, P->smem)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rrl_batch, 256, P->smem)) !=
          cudaSuccess ||
      per_sm < 1) {
    (void)cudaGetLastError();
    delete P; return DB_ERR_CUDA;
  }
  P->grid = sms * per_sm;
  *out = P;
  return DB_OK;
}

db_status batch_run(const BatchPlan* P, int* status, cudaStream_t s) {
  if (!P) return DB_ERR_ARG;
  if (cudaMemsetAsync(P->d_bar, 0, 256, s) != cudaSuccess ||
      cudaMemsetAsync(P->d_work, 0, (size_t)(2 * P->iters + 2) * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(P->d_done, 0, (size_t)2 * P->n * sizeof(int), s) != cudaSuccess)
    return DB_ERR_CUDA;
  if (wiener_batch_run(P->wb, s) != cudaSuccess) return DB_ERR_CUDA;
  if (P->iters == 0) return DB_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P->grid);
  cfg.blockDim = dim3(64, 4);
  cfg.dynamicSmemBytes = P->smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const long long limit = g_spin_limit.load();
  const cudaError_t e =
      P->order == 0
          ? cudaLaunchKernelEx(&cfg, k_rrl_batch_dep, (const BatchImg*)P->d_imgs, P->n, (const int4*)P->d_tiles_q,
                               (int)P->tiles_q.size(), (const int4*)P->d_tiles_u, (int)P->tiles_u.size(), P->iters,
                               P->d_work, P->d_done, status, limit)
          : cudaLaunchKernelEx(&cfg, k_rrl_batch, (const BatchImg*)P->d_imgs, (const int4*)P->d_tiles_q,
                               (int)P->tiles_q.size(), (const int4*)P->d_tiles_u, (int)P->tiles_u.size(), P->iters,
                               P->d_bar, P->d_work, status, limit);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return DB_ERR_CUDA;
  }
  count_launch();
  return DB_OK;
}

void batch_destroy(BatchPlan* P) { delete P; }

// Set the tunable forms of every image (fft_min: FFT tiles for the 2D PSFs
// of their shape range with kh * kw >= fft_min, none if 0; dense: dense
// bodies for the dense-eligible 2D PSFs; windows for the non-box one-axis
// PSFs: 0 tap groups, 1 register windows, 2 the size rule's choice),
// rebuild the tile tables and upload them with the descriptors
// (synchronises the stream: the host tables are reused).
static db_status batch_set_forms(BatchPlan* P, int fft_min, bool dense, int windows, cudaStream_t s) {
  P->fft_min = fft_min;
  for (int i = 0; i < P->n; ++i) {
    P->imgs[i].fft = fft_min > 0 && P->fft_taps[i] >= fft_min ? 1 : 0;
    P->imgs[i].kwd = dense ? P->dense_kw[i] : 0;
    if (P->window_box[i]) P->imgs[i].box = windows == 2 ? P->rule_box[i] : windows == 1 ? P->window_box[i] : 0;
  }
  build_tiles(P);
  if (cudaMemcpyAsync(P->d_imgs, P->imgs.data(), (size_t)P->n * sizeof(BatchImg), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      upload_tiles(P, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return DB_ERR_CUDA;
  return DB_OK;
}

// ---------------------------------------------------------------------------
// streamed batch: host images in, results out, the copies overlapped with
// the runs of other sub-batches
// ---------------------------------------------------------------------------
// Partition of the images into `parts` groups by pixel count, in the order
// the groups are streamed: target shares w_k = 4^min(k, parts-1-k)
// (1, 4, 16, ..., 16, 4, 1).  The first group's upload and the last group's
// download, which no run overlaps, are then short, and each group's run
// still covers the next group's upload while a run takes at least four times
// as long as the upload of the same pixels (batch512: 56 ms of runs, 14 ms of
// uploads).  Every further group costs about 0.5 ms of run time (its own
// Wiener launches, grid barriers and tails).  Images are dealt largest first
// to the group with the least load relative to its share (ties to the lowest
// group); each group keeps ascending image order.
static std::vector<std::vector<int>> lpt_parts(const db_image_desc* d, int n, int parts) {
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)d[a].H * d[a].W > (long long)d[b].H * d[b].W;
  });
  std::vector<long long> load(parts, 0);
  std::vector<double> share(parts);
  for (int k = 0; k < parts; ++k) share[k] = std::ldexp(1.0, 2 * std::min(std::min(k, parts - 1 - k), 24));
  std::vector<std::vector<int>> out(parts);
  for (int i : order) {
    int k = 0;
    for (int j = 1; j < parts; ++j)
      if ((double)load[j] / share[j] < (double)load[k] / share[k]) k = j;
    load[k] += (long long)d[i].H * d[i].W;
    out[k].push_back(i);
  }
  for (auto& v : out) std::sort(v.begin(), v.end());
  out.erase(std::remove_if(out.begin(), out.end(), [](const std::vector<int>& v) { return v.empty(); }),
            out.end());
  return out;
}

struct BatchStream {
  std::vector<db_image_desc> descs;
  std::vector<std::vector<int>> idx;
  std::vector<BatchPlan*> plans;
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> ev_up, ev_done, ev_down;
  ~BatchStream() {
    for (BatchPlan* P : plans) delete P;
    for (auto* v : {&ev_up, &ev_done, &ev_down})
      for (cudaEvent_t e : *v)
        if (e) cudaEventDestroy(e);
    if (start) cudaEventDestroy(start);
    if (up) cudaStreamDestroy(up);
    if (down) cudaStreamDestroy(down);
  }
};

static size_t stream_ws_bytes(const db_image_desc* d, int n, int iters, int parts, db_status* why,
                              std::vector<std::vector<int>>* idx_out, std::vector<size_t>* sizes) {
  *why = DB_OK;
  if (!d || n < 1 || parts < 1 || iters < 0) { *why = DB_ERR_ARG; return 0; }
  if (batch_ws_bytes(d, n, iters, why) == 0) return 0;  // validates every descriptor
  std::vector<std::vector<int>> idx = lpt_parts(d, n, std::min(parts, n));
  size_t total = 0;
  for (const auto& v : idx) {
    std::vector<db_image_desc> sub;
    for (int i : v) sub.push_back(d[i]);
    const size_t b = batch_ws_bytes(sub.data(), (int)sub.size(), iters, why);
    if (b == 0) return 0;
    if (sizes) sizes->push_back(align256(b));
    total += align256(b);
  }
  if (idx_out) *idx_out = idx;
  return total;
}

}  // namespace db

using namespace db;

extern "C" {

size_t db_batch_workspace_bytes(const db_image_desc* descs, int n, int iters) {
  db_status why;
  return batch_ws_bytes(descs, n, iters, &why);
}

db_status db_batch_create(const db_image_desc* descs, int n, int iters, void* ws, size_t ws_bytes,
                          int* dev_status, void* stream, db_batch** out) {
  if (!out) return DB_ERR_ARG;
  *out = nullptr;
  BatchPlan* P = nullptr;
  const db_status st = batch_create(descs, n, iters, ws, ws_bytes, dev_status, (cudaStream_t)stream, &P);
  if (st == DB_OK) *out = (db_batch*)P;
  return st;
}

db_status db_batch_run(db_batch* b, int* dev_status, void* stream) {
  return batch_run((BatchPlan*)b, dev_status, (cudaStream_t)stream);
}

void db_batch_destroy(db_batch* b) { batch_destroy((BatchPlan*)b); }

db_status db_deblur_batch(const db_image_desc* descs, int n, int iters, void* ws, size_t ws_bytes,
                          int* dev_status, void* stream) {
  db_batch* b = nullptr;
  db_status st = db_batch_create(descs, n, iters, ws, ws_bytes, dev_status, stream, &b);
  if (st != DB_OK) return st;
  st = db_batch_run(b, dev_status, stream);
  // the plan's host tables were uploaded with copies that have already read
  // them, so the plan can go while the device work is still in flight
  db_batch_destroy(b);
  return st;
}

size_t db_batch_stream_workspace_bytes(const db_image_desc* descs, int n, int iters, int parts) {
  db_status why;
  return stream_ws_bytes(descs, n, iters, parts, &why, nullptr, nullptr);
}

db_status db_batch_stream_create(const db_image_desc* descs, int n, int iters, int parts, void* ws,
                                 size_t ws_bytes, int* dev_status, void* stream, db_batch_stream** out) {
  if (!out) return DB_ERR_ARG;
  *out = nullptr;
  db_status why;
  std::vector<std::vector<int>> idx;
  std::vector<size_t> sizes;
  const size_t need = stream_ws_bytes(descs, n, iters, parts, &why, &idx, &sizes);
  if (need == 0) return why;
  if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < need) return DB_ERR_WORKSPACE;
  BatchStream* B = new BatchStream();
  B->descs.assign(descs, descs + n);
  B->idx = idx;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  for (size_t k = 0; k < idx.size(); ++k) {
    std::vector<db_image_desc> sub;
    for (int i : idx[k]) sub.push_back(descs[i]);
    BatchPlan* P = nullptr;
    const db_status st = batch_create(sub.data(), (int)sub.size(), iters, base, sizes[k], dev_status, s, &P);
    if (st != DB_OK) { delete B; return st; }
    B->plans.push_back(P);
    base += sizes[k];
  }
  const size_t np = idx.size();
  B->ev_up.assign(np, nullptr);
  B->ev_done.assign(np, nullptr);
  B->ev_down.assign(np, nullptr);
  bool ok = cudaStreamCreateWithFlags(&B->up, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&B->down, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->start, cudaEventDisableTiming) == cudaSuccess;
  for (size_t k = 0; ok && k < np; ++k)
    ok = cudaEventCreateWithFlags(&B->ev_up[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->ev_done[k], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->ev_down[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) { (void)cudaGetLastError(); delete B; return DB_ERR_CUDA; }
  *out = (db_batch_stream*)B;
  return DB_OK;
}

db_status db_batch_stream_run_host(db_batch_stream* b, const float* const* f_host, float* const* u_host,
                                   int* dev_status, void* stream) {
  BatchStream* B = (BatchStream*)b;
  if (!B || !f_host || !u_host) return DB_ERR_ARG;
  const int n = (int)B->descs.size();
  for (int i = 0; i < n; ++i)
    if (!f_host[i] || !u_host[i]) return DB_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the copies in start after everything enqueued on `stream` before this call
  if (cudaEventRecord(B->start, s) != cudaSuccess || cudaStreamWaitEvent(B->up, B->start, 0) != cudaSuccess)
    return DB_ERR_CUDA;
  const size_t np = B->plans.size();
  auto upload = [&](size_t k) -> db_status {
    for (int i : B->idx[k]) {
      const db_image_desc& x = B->descs[i];
      if (copy_image_async((void*)x.f, (size_t)x.ld * sizeof(float), f_host[i], (size_t)x.W * sizeof(float), x.H,
                           x.W, cudaMemcpyHostToDevice, B->up) != cudaSuccess)
        return DB_ERR_CUDA;
    }
    return cudaEventRecord(B->ev_up[k], B->up) == cudaSuccess ? DB_OK : DB_ERR_CUDA;
  };
  // sub-batch k+1's copies are enqueued before sub-batch k's run, so that the
  // first run does not wait for the host to enqueue every upload
  db_status st = upload(0);
  for (size_t k = 0; k < np && st == DB_OK; ++k) {
    if (k + 1 < np && (st = upload(k + 1)) != DB_OK) break;
    if (cudaStreamWaitEvent(s, B->ev_up[k], 0) != cudaSuccess) return DB_ERR_CUDA;
    if ((st = batch_run(B->plans[k], dev_status, s)) != DB_OK) break;
    if (cudaEventRecord(B->ev_done[k], s) != cudaSuccess || cudaStreamWaitEvent(B->down, B->ev_done[k], 0) != cudaSuccess)
      return DB_ERR_CUDA;
    for (int i : B->idx[k]) {
      const db_image_desc& x = B->descs[i];
      if (copy_image_async(u_host[i], (size_t)x.W * sizeof(float), x.u, (size_t)x.ld * sizeof(float), x.H, x.W,
                           cudaMemcpyDeviceToHost, B->down) != cudaSuccess)
        return DB_ERR_CUDA;
    }
    if (cudaEventRecord(B->ev_down[k], B->down) != cudaSuccess) return DB_ERR_CUDA;
  }
  if (st != DB_OK) return st;
  // `stream` completes only after every result has reached the host
  for (size_t k = 0; k < np; ++k)
    if (cudaStreamWaitEvent(s, B->ev_down[k], 0) != cudaSuccess) return DB_ERR_CUDA;
  return DB_OK;
}

db_status db_batch_autotune(db_batch* b, int reps, int* dev_status, void* stream, int* dense_out,
                            int* windows_out, int* fft_out) {
  BatchPlan* P = (BatchPlan*)b;
  if (!P || reps < 1) return DB_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  bool has_dense = false, has_win = false;
  std::vector<int> fft_sizes;  // distinct kh * kw of the images that can take FFT tiles
  for (int i = 0; i < P->n; ++i) {
    has_dense |= P->dense_kw[i] != 0;
    has_win |= P->window_box[i] != 0;
    if (P->fft_taps[i]) fft_sizes.push_back(P->fft_taps[i]);
  }
  std::sort(fft_sizes.begin(), fft_sizes.end());
  fft_sizes.erase(std::unique(fft_sizes.begin(), fft_sizes.end()), fft_sizes.end());
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DB_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return DB_ERR_CUDA; }
  db_status st = DB_OK;
  // time of the whole batch under one combination of forms
  auto time_forms = [&](int fmin, bool dense, int windows, float* ms) -> db_status {
    db_status r;
    if ((r = batch_set_forms(P, fmin, dense, windows, s)) != DB_OK) return r;
    if ((r = batch_run(P, dev_status, s)) != DB_OK) return r;  // warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) return DB_ERR_CUDA;
    for (int k = 0; k < reps; ++k)
      if ((r = batch_run(P, dev_status, s)) != DB_OK) return r;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return DB_ERR_CUDA;
    return DB_OK;
  };
  // coordinate search from the size rules: the one-axis form, then the
  // dense sums, then the FFT-tile threshold (every distinct kh * kw of the
  // batch's 2D PSFs as a threshold, and none)
  int best_f = fft_tile_min(), best_w = 2;
  bool best_d = true;
  float best = -1.f, ms = 0.f;
  if ((st = time_forms(best_f, best_d, best_w, &ms)) == DB_OK) best = ms;
  for (int w : {1, 0}) {
    if (st != DB_OK || !has_win) break;
    if ((st = time_forms(best_f, best_d, w, &ms)) == DB_OK && ms < best) { best = ms; best_w = w; }
  }
  if (st == DB_OK && has_dense && (st = time_forms(best_f, false, best_w, &ms)) == DB_OK && ms < best) {
    best = ms;
    best_d = false;
  }
  // thresholds that change the set of FFT images: each distinct size, and
  // none (a threshold above every size)
  std::vector<int> cands(fft_sizes);
  if (!fft_sizes.empty()) cands.push_back(0);
  auto same_set = [&](int a, int c) {
    for (int v : fft_sizes)
      if ((a > 0 && v >= a) != (c > 0 && v >= c)) return false;
    return true;
  };
  for (int c : cands) {
    if (st != DB_OK) break;
    if (same_set(c, best_f)) continue;
    if ((st = time_forms(c, best_d, best_w, &ms)) == DB_OK && ms < best) { best = ms; best_f = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DB_OK) return st;
  if ((st = batch_set_forms(P, best_f, best_d, best_w, s)) != DB_OK) return st;
  if (dense_out) *dense_out = best_d ? 1 : 0;
  if (windows_out) *windows_out = best_w;
  if (fft_out) *fft_out = best_f;
  return DB_OK;
}

int db_batch_stream_parts(const db_batch_stream* b) {
  return b ? (int)((const BatchStream*)b)->plans.size() : 0;
}

void db_batch_stream_destroy(db_batch_stream* b) { delete (BatchStream*)b; }

db_status db_set_batch_order(int order) {
  if (order != 0 && order != 1) return DB_ERR_ARG;
  g_batch_order.store(order);
  bump_settings();
  return DB_OK;
}

db_status db_set_spin_limit(long long cycles) {
  if (cycles < 0) return DB_ERR_ARG;
  set_spin_limit(cycles);
  bump_settings();
  return DB_OK;
}

}  // extern "C"
