// Fused RRRL iteration with spatial (constant-continuation) blur and
// correlation: Sec. 2.3, Eq. 9-12, Sec. 4.1-4.2.
//
// One launch performs one whole iteration
//   b = u*h;  W = phi'(r_f(b));  q1 = W f/b;  q2 = W           (Eq. 7, 10)
//   A = q1*h*;  B = q2*h*;  D = div(psi'(|grad u|^2) grad u)  (Eq. 11)
//   u' = u (A + alpha [D]+) / (B - alpha [D]-)                (Eq. 9, 12)
// reading u and f once from global memory and writing u' once.  Each CTA
// owns a TH x TW output tile; it stages u with a halo of kh-1 rows / kw-1
// columns (at least 2, for the diffusion stencil) in shared memory, forms
// q1, q2 on the tile grown by the correlation footprint, then the outputs.
// Halo values are recomputed by neighbouring CTAs instead of exchanged.
//
// Boundary: shared-memory copies of u hold u(clamp(i), clamp(j)) for the
// virtual positions of the halo, so the blur sees constant continuation;
// q is formed at clamped positions, so the correlation sees the constant
// continuation of q (not the blur of continued u), as the operator
// definition requires.  Neighbour differences across the boundary vanish
// exactly, which gives the zero-flux diffusion term.
#include <cuda_runtime.h>

#include <cstring>

#include "internal.cuh"
#include "rrl_box.cuh"
#include "rrl_dense.cuh"
#include "rrl_fft_tile.cuh"
#include "rrl_tiles.cuh"

namespace db {

// ---------------------------------------------------------------------------
// tap preparation: validate the dense taps and build the tap groups.
//
// A group is a run of up to kMaxGroupH vertically adjacent rows of one PSF
// column, starting and ending on a non-zero tap: weights w[0..h-1] for
// offsets (dy0 + k, dx).  Within a column, a group starts at the first
// non-zero tap not yet covered.  The cluster from there (non-zero taps at
// most one zero row apart) becomes one group if it has at most kMaxGroupH
// rows, otherwise the first of ceil(n / kMaxGroupH) nearly equal parts
// (ending on its last non-zero tap).  Every non-zero tap lands in exactly
// one group, with its own weight; a column of kh rows yields at most
// ceil(kh / 3) groups (a group either spans at least 4 rows or ends a
// cluster, which is followed by at least 2 zero rows).  Groups are written
// sorted by height (then by column, then top to bottom), with the class
// starts next to the group count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool tap_nz(const float* __restrict__ taps, int kw, int r, int b) {
  return __ldg(taps + r * kw + b) != 0.f;
}

// The group of column b that starts after row `covered`: first row s and
// height h (h = 0: no non-zero tap left).
__device__ void next_group(const float* __restrict__ taps, int kh, int kw, int b, int covered, int* s_out,
                           int* h_out) {
  int s = -1;
  for (int r = covered + 1; r < kh; ++r)
    if (tap_nz(taps, kw, r, b)) { s = r; break; }
  *s_out = s;
  if (s < 0) { *h_out = 0; return; }
  int e = s;
  while (true) {
    int nxt = -1;
    for (int r = e + 1; r < kh && r <= e + 2; ++r)
      if (tap_nz(taps, kw, r, b)) { nxt = r; break; }
    if (nxt < 0) break;
    e = nxt;
  }
  const int n = e - s + 1;
  int h = n;
  if (n > kMaxGroupH) {
    const int parts = (n + kMaxGroupH - 1) / kMaxGroupH;
    h = (n + parts - 1) / parts;
    while (!tap_nz(taps, kw, s + h - 1, b)) --h;
  }
  *h_out = h;
}

__global__ void __launch_bounds__(256) k_prepare_taps(const float* __restrict__ taps, int kh, int kw,
                                                      int kind, int max_groups, int dense_pct,
                                                      TapGroup* __restrict__ groups,
                                                      int* __restrict__ ngroups, int* status) {
  __shared__ int scan[256];
  __shared__ int cstart[kMaxGroupH + 1];
  __shared__ float warp_sum[8];
  __shared__ int bad, s_nnz;
  const int n = kh * kw;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) { bad = 0; s_nnz = 0; }
  __syncthreads();
  // a box is uniform except possibly for its two end taps (non-integer
  // blur length, Sec. 4.3)
  const float t1 = n > 2 ? __ldg(taps + 1) : 0.f;
  float sum = 0.f;
  int nnz = 0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float w = __ldg(taps + k);
    if (!(w >= 0.f) || !isfinite(w)) atomicOr(&bad, DB_FLAG_TAPS);
    if (kind == DB_PSF_BOX && k >= 1 && k <= n - 2 && w != t1) atomicOr(&bad, DB_FLAG_BOX);
    sum += w;
    nnz += (w != 0.f);
  }
  // dense table of an eligible 2D PSF: kh rows of dense_tap_stride(kw)
  // floats, zero beyond column kw
  if (dense_eligible(kh, kw)) {
    float* tab = const_cast<float*>(dense_taps(groups, kh, kw));
    const int TS = dense_tap_stride(kw);
    for (int k = threadIdx.x; k < kh * TS; k += blockDim.x) {
      const int r = k / TS, c = k - r * TS;
      tab[k] = c < kw ? __ldg(taps + r * kw + c) : 0.f;
    }
  }
  for (int o = 16; o > 0; o >>= 1) nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
  if (lane == 0) atomicAdd(&s_nnz, nnz);
  // one-axis PSFs: (e0, w, e1, L) 16 bytes after the group count, the taps
  // themselves 32 bytes after it
  if ((kh == 1 || kw == 1) && threadIdx.x == 0)
    reinterpret_cast<float4*>(ngroups + 4)[0] = make_float4(__ldg(taps), t1, __ldg(taps + n - 1), __int_as_float(n));
  if (kh == 1 || kw == 1)
    for (int k = threadIdx.x; k < n; k += blockDim.x) reinterpret_cast<float*>(ngroups + 8)[k] = __ldg(taps + k);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) warp_sum[wid] = sum;
  // one thread per PSF column (kw <= 255): groups per height class, then
  // per class an exclusive scan over the columns
  const int b = threadIdx.x;
  int cnt[kMaxGroupH];
#pragma unroll
  for (int m = 0; m < kMaxGroupH; ++m) cnt[m] = 0;
  if (b < kw) {
    int covered = -1, s0, h;
    while (true) {
      next_group(taps, kh, kw, b, covered, &s0, &h);
      if (h == 0) break;
#pragma unroll
      for (int m = 0; m < kMaxGroupH; ++m) cnt[m] += (h == m + 1);
      covered = s0 + h - 1;
    }
  }
  int pos[kMaxGroupH];
  if (threadIdx.x == 0) cstart[0] = 0;
#pragma unroll
  for (int m = 0; m < kMaxGroupH; ++m) {
    __syncthreads();
    scan[threadIdx.x] = cnt[m];
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
      const int v = (threadIdx.x >= o) ? scan[threadIdx.x - o] : 0;
      __syncthreads();
      scan[threadIdx.x] += v;
      __syncthreads();
    }
    pos[m] = scan[threadIdx.x] - cnt[m];  // within the class
    if (threadIdx.x == 0) cstart[m + 1] = cstart[m] + scan[255];
    __syncthreads();
  }
  const int total = cstart[kMaxGroupH];
  if (total > max_groups) {
    if (threadIdx.x == 0) atomicOr(&bad, DB_FLAG_TAPS);
  } else if (b < kw) {
    const int cy = kh >> 1, cx = kw >> 1;
    int covered = -1, s0, h;
    while (true) {
      next_group(taps, kh, kw, b, covered, &s0, &h);
      if (h == 0) break;
      TapGroup g;
#pragma unroll
      for (int k = 0; k < kMaxGroupH; ++k) g.w[k] = k < h ? __ldg(taps + (s0 + k) * kw + b) : 0.f;
      g.dy0 = (int16_t)(s0 - cy);
      g.dx = (int16_t)(b - cx);
      int slot = 0;
#pragma unroll
      for (int m = 0; m < kMaxGroupH; ++m)
        if (h == m + 1) slot = cstart[m] + pos[m]++;
      groups[slot] = g;
      covered = s0 + h - 1;
    }
  }
  __syncthreads();
  if (threadIdx.x <= kMaxGroupH) group_class_starts(ngroups)[threadIdx.x] = total > max_groups ? 0 : cstart[threadIdx.x];
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < 8; ++i) s += warp_sum[i];
    if (!(s > 0.f)) bad |= DB_FLAG_TAPS;
    *ngroups = total > max_groups ? 0 : total;
    // dense sums when at least dense_pct percent (default half) of an
    // eligible PSF's taps are non-zero
    ngroups[1] = (dense_eligible(kh, kw) && 100 * s_nnz >= dense_pct * n) ? 1 : 0;
    if (bad && status) atomicOr(status, bad);
  }
}

// The 64 x 64 spectrum of the FFT tiles (rrl_fft_tile.cuh) for a PSF of
// fft_tile_shape, one CTA.  Raw taps: k_prepare_taps validates them.
__global__ void __launch_bounds__(256) k_prepare_fft_spec(const float* __restrict__ taps, int kh, int kw,
                                                         float2* __restrict__ spec) {
  __shared__ __align__(16) float2 tw[ftile::kTwSlots];  // read as float4
  __shared__ __align__(16) float2 A[ftile::kPos];
  ftile::psf_spectrum(A, tw, taps, kh, kw, spec);
}

cudaError_t launch_prepare_taps(const float* taps, int kh, int kw, int kind, TapGroup* groups,
                                int* ngroups, int* status, cudaStream_t s) {
  k_prepare_taps<<<1, 256, 0, s>>>(taps, kh, kw, kind, max_tap_groups(kh, kw), dense_min_pct(), groups, ngroups,
                                   status);
  count_launch();
  if (fft_tile_shape(kh, kw)) {
    k_prepare_fft_spec<<<1, 256, 0, s>>>(taps, kh, kw, const_cast<float2*>(fft_tile_spec(groups, kh, kw)));
    count_launch();
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// split schedule kernels (one tile per CTA), chained by programmatic
// dependent launch.  In the chain  ... update(k-1) -> q(k) -> update(k) ...
// each kernel lets its successor start only once it has itself passed the
// wait for its predecessor.  Hence when update(k) starts, update(k-1) (the
// writer of u) has completed, and the part of each tile that runs before
// the wait may read everything except its immediate predecessor's output:
// q(k) stages f and the tap groups, update(k) the tap groups and u; the
// wait then covers q(k)'s u and update(k)'s q.
// ---------------------------------------------------------------------------
struct PdlDep {
  __device__ void operator()() const {
    pdl_wait();
    pdl_trigger();
  }
};

// Equally sized images side by side: image z of a launch with gridDim.z > 1
// is at these element offsets times z (zero for one image).
struct ZStride {
  long long f, in, out, q;
};

template <int TH, int TW, int R, int P>
__global__ void __launch_bounds__((TH / R) * TW, 8) k_rrl_q(const float* __restrict__ f, int ldf,
                                               const float* __restrict__ uin, int ldin,
                                               float2* __restrict__ q, int ldq, int H, int W,
                                               const TapGroup* __restrict__ groups_g,
                                               const int* __restrict__ ngroups_g, int kh, int kw,
                                               int ng_max, RrlParams p, ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  q_tile<TH, TW, R, P>(smem_raw, f + z * zs.f, ldf, uin + z * zs.in, ldin, q + z * zs.q, ldq, H, W, groups_g,
                          ngroups_g, kh, kw, ng_max, p, blockIdx.y * TH, blockIdx.x * TW, PdlDep());
}

template <int TH, int TW, int R, int P>
__global__ void __launch_bounds__((TH / R) * TW, 7) k_rrl_update(const float2* __restrict__ q, int ldq,
                                                    const float* __restrict__ uin, int ldin,
                                                    float* __restrict__ uout, int ldout, int H, int W,
                                                    const TapGroup* __restrict__ groups_g,
                                                    const int* __restrict__ ngroups_g, int kh, int kw,
                                                    int ng_max, RrlParams p, int* status, ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  update_tile<TH, TW, R, P>(smem_raw, q + z * zs.q, ldq, uin + z * zs.in, ldin, uout + z * zs.out, ldout, H, W,
                               groups_g, ngroups_g, kh, kw, ng_max, p, status, blockIdx.y * TH, blockIdx.x * TW,
                               PdlDep());
}

// Dense-eligible 2D PSFs (odd sides 3..25): the split pair with the dense
// bodies when the prepared flag says so (at least half the taps non-zero),
// else the tap-group bodies; q is planar for the dense bodies.
template <int TH, int TW, int KW>
__global__ void __launch_bounds__((TH / kDR) * (TW / kDC), 6) k_rrl_q_dense(
    const float* __restrict__ f, int ldf, const float* __restrict__ uin, int ldin, float2* __restrict__ q, int ldq,
    int H, int W, const TapGroup* __restrict__ groups_g, const int* __restrict__ ngroups_g, int kh, int kw,
    int ng_max, RrlParams p, ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  if (__ldg(dense_flag(ngroups_g))) {
    float* qe = reinterpret_cast<float*>(q + z * zs.q);
    q_tile_dense<TH, TW, KW>(smem_raw, f + z * zs.f, ldf, uin + z * zs.in, ldin, qe, qe + (size_t)H * upitch(W),
                             upitch(W), H, W, dense_taps(groups_g, kh, kw), kh, p, blockIdx.y * TH, blockIdx.x * TW,
                             PdlDep());
  } else {
    constexpr int P = (KW + 2 <= 8) ? 8 : (KW + 2 <= 16) ? 16 : 32;
    q_tile<TH, TW, 8, P>(smem_raw, f + z * zs.f, ldf, uin + z * zs.in, ldin, q + z * zs.q, ldq, H, W, groups_g,
                         ngroups_g, kh, kw, ng_max, p, blockIdx.y * TH, blockIdx.x * TW, PdlDep());
  }
}

template <int TH, int TW, int KW>
__global__ void __launch_bounds__((TH / kDR) * (TW / kDC), 6) k_rrl_update_dense(
    const float2* __restrict__ q, int ldq, const float* __restrict__ uin, int ldin, float* __restrict__ uout,
    int ldout, int H, int W, const TapGroup* __restrict__ groups_g, const int* __restrict__ ngroups_g, int kh, int kw,
    int ng_max, RrlParams p, int* status, ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  if (__ldg(dense_flag(ngroups_g))) {
    const float* qe = reinterpret_cast<const float*>(q + z * zs.q);
    update_tile_dense<TH, TW, KW>(smem_raw, qe, qe + (size_t)H * upitch(W), upitch(W), uin + z * zs.in, ldin,
                                  uout + z * zs.out, ldout, H, W, dense_taps(groups_g, kh, kw), kh, p, status,
                                  blockIdx.y * TH, blockIdx.x * TW, PdlDep());
  } else {
    constexpr int P = (KW + 2 <= 8) ? 8 : (KW + 2 <= 16) ? 16 : 32;
    update_tile<TH, TW, 8, P>(smem_raw, q + z * zs.q, ldq, uin + z * zs.in, ldin, uout + z * zs.out, ldout, H, W,
                              groups_g, ngroups_g, kh, kw, ng_max, p, status, blockIdx.y * TH, blockIdx.x * TW,
                              PdlDep());
  }
}

// FFT tiles (rrl_fft_tile.cuh): the q kernel takes two horizontally
// adjacent tiles per CTA (blockIdx.x pairs), the update kernel one; q is
// planar as for the dense bodies.
// umap (use_tma): the 3D tensor map of uin's images for the TMA-staged
// windows (encode_window_map; kBoxW x kN boxes).
__global__ void __launch_bounds__(256, 4) k_rrl_q_fft(const float* __restrict__ f, int ldf, const float* uin,
                                                     int ldin, float2* q, int H, int W,
                                                     const TapGroup* __restrict__ groups_g, int kh, int kw,
                                                     RrlParams p, ZStride zs,
                                                     const __grid_constant__ CUtensorMap umap, int use_tma,
                                                     int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned long long bar;
  if (use_tma) {
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
  }
  const long long z = blockIdx.z;
  float* qe = reinterpret_cast<float*>(q + z * zs.q);
  const ftile::WinTma tma = {&umap, (int)blockIdx.z, &bar, 0u, kTmaWaitLimit, status};
  ftile::q_tile(smem_raw, f + z * zs.f, ldf, uin + z * zs.in, ldin, qe, qe + (size_t)H * upitch(W), upitch(W), H, W,
                fft_tile_spec(groups_g, kh, kw), kh, kw, p, blockIdx.y * ftile::tile_oh(kh),
                2 * blockIdx.x * ftile::tile_ow(kw), PdlDep(), use_tma ? &tma : nullptr);
}

__global__ void __launch_bounds__(256, 4) k_rrl_update_fft(const float2* q, const float* uin, int ldin,
                                                          float* __restrict__ uout, int ldout, int H, int W,
                                                          const TapGroup* __restrict__ groups_g, int kh, int kw,
                                                          RrlParams p, int* status, ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  const float* qe = reinterpret_cast<const float*>(q + z * zs.q);
  ftile::update_tile(smem_raw, qe, qe + (size_t)H * upitch(W), upitch(W), uin + z * zs.in, ldin, uout + z * zs.out,
                     ldout, H, W, fft_tile_spec(groups_g, kh, kw), kh, kw, p, status,
                     blockIdx.y * ftile::tile_oh(kh), blockIdx.x * ftile::tile_ow(kw), PdlDep());
}

// one-axis PSFs: the same split pair with sliding-window sums (box) or
// register-window tap sums (rrl_box.cuh)
// Tiles of TH x 32 outputs (TH = 32, or 16 for images with fewer 32 x 32
// tiles than SMs), 128 threads with strips of TH / 4 rows.
template <bool HORIZ, bool BOX, int TH>
__global__ void __launch_bounds__(128) k_rrl_q_box(const float* __restrict__ f, int ldf,
                                                  const float* __restrict__ uin, int ldin, float2* __restrict__ q,
                                                  int ldq, int H, int W, const int* __restrict__ ngroups_g,
                                                  RrlParams p, ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  q_tile_box<TH, 32, TH / 4, HORIZ, BOX>(smem_raw, f + z * zs.f, ldf, uin + z * zs.in, ldin, q + z * zs.q, ldq, H,
                                         W, ngroups_g, p, blockIdx.y * TH, blockIdx.x * 32, PdlDep());
}

template <bool HORIZ, bool BOX, int TH>
__global__ void __launch_bounds__(128) k_rrl_update_box(const float2* __restrict__ q, int ldq,
                                                       const float* __restrict__ uin, int ldin,
                                                       float* __restrict__ uout, int ldout, int H, int W,
                                                       const int* __restrict__ ngroups_g, RrlParams p, int* status,
                                                       ZStride zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long z = blockIdx.z;
  update_tile_box<TH, 32, TH / 4, HORIZ, BOX>(smem_raw, q + z * zs.q, ldq, uin + z * zs.in, ldin, uout + z * zs.out,
                                              ldout, H, W, ngroups_g, p, status, blockIdx.y * TH, blockIdx.x * 32,
                                              PdlDep());
}

// ---------------------------------------------------------------------------
// host side: shared-memory sizes and launches.  The halo class P is the
// smallest of 8, 16, 32, 64, 128, 256 that holds kw - 1 (and 2).
// ---------------------------------------------------------------------------
constexpr int kTH = 64, kTW = 64, kR = 8;        // fused tiles
// split tiles: 32 x 32 outputs, 128 threads (one 8-row strip each).  Small
// tiles keep 7-8 CTAs resident per SM, so a 1024^2 image (1024 tiles) is
// one balanced wave.
constexpr int kQTH = 32, kQTW = 32;
constexpr int kUTH = 32, kUTW = 32;

static int halo_class(int kw) {
  const int need = kw - 1 > 2 ? kw - 1 : 2;
  int P = 8;
  while (P < need) P *= 2;
  return P;
}

size_t rrl_spatial_smem(int kh, int kw) {
  const int ng_max = max_tap_groups(kh, kw), P = halo_class(kw);
  const int Ry = kh - 1 > 2 ? kh - 1 : 2;
  const int QHp = ((kTH + kh - 1 + kR - 1) / kR) * kR;
  const int UH = Ry + (QHp > kTH + 2 ? QHp : kTH + 2);
  const size_t us = (size_t)(UH * (kTW + 2 * P) + 1) & ~size_t(1);
  return 32 + (size_t)2 * ng_max * kGroupRecordBytes + us * sizeof(float) + (size_t)QHp * (kTW + P) * sizeof(float2);
}
static size_t split_smem_q_single(int kh, int kw, int ng_max) {
  return split_smem_q(kQTH, kQTW, kh, kw, ng_max);
}
static size_t split_smem_update_single(int kh, int kw, int ng_max) {
  return split_smem_update(kUTH, kUTW, kh, kw, ng_max);
}
size_t rrl_fft_tile_smem(int kh) { return ftile::smem_update(kh); }
size_t rrl_split_smem(int kh, int kw) {
  size_t a = split_smem_q_single(kh, kw, max_tap_groups(kh, kw));
  size_t b = split_smem_update_single(kh, kw, max_tap_groups(kh, kw));
  if (dense_eligible(kh, kw)) {
    a = a > dense_smem_q(kQTH, kQTW, kh, kw) ? a : dense_smem_q(kQTH, kQTW, kh, kw);
    b = b > dense_smem_update(kUTH, kUTW, kh, kw) ? b : dense_smem_update(kUTH, kUTW, kh, kw);
  }
  return a > b ? a : b;
}

template <typename K>
static cudaError_t set_smem(K kern, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

struct IterArgs {
  const float* f; int ldf; const float* uin; int ldin; float* uout; int ldout; float2* q;
  int H, W; const TapGroup* groups; const int* ngroups; int kh, kw; RrlParams p; int* status;
  int ng_bound;  // known upper bound of the group count (0: use max_tap_groups)
  int axis;      // axis_mode(): one-axis form of the split schedule (1 box, 2 general taps)
  int nz;        // images per launch (split schedule), offsets zs
  ZStride zs;
};

template <int P>
static cudaError_t launch_fused_p(const IterArgs& a, cudaStream_t s) {
  const int ng_max = max_tap_groups(a.kh, a.kw);
  const size_t smem = rrl_spatial_smem(a.kh, a.kw);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = k_rrl_spatial<kTH, kTW, kR, P>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3((a.W + kTW - 1) / kTW, (a.H + kTH - 1) / kTH), dim3(64, 4), smem, s>>>(
      a.f, a.ldf, a.uin, a.ldin, a.uout, a.ldout, a.H, a.W, a.groups, a.ngroups, a.kh, a.kw, ng_max,
      a.p, a.status);
  count_launch();
  return cudaGetLastError();
}

template <typename KQ, typename KU>
static cudaError_t launch_split_pair(const IterArgs& a, KQ kq, KU ku, int ng_max, size_t sq, size_t su,
                                     cudaStream_t s);

template <int P>
static cudaError_t launch_split_p(const IterArgs& a, cudaStream_t s) {
  const int ng_max = a.ng_bound > 0 ? a.ng_bound : max_tap_groups(a.kh, a.kw);
  const size_t sq = split_smem_q_single(a.kh, a.kw, ng_max), su = split_smem_update_single(a.kh, a.kw, ng_max);
  if (sq > 227 * 1024 || su > 227 * 1024) return cudaErrorInvalidValue;
  return launch_split_pair(a, k_rrl_q<kQTH, kQTW, kR, P>, k_rrl_update<kUTH, kUTW, kR, P>, ng_max, sq, su, s);
}

template <int KW>
static cudaError_t launch_split_dense(const IterArgs& a, cudaStream_t s) {
  static_assert(kQTH == kUTH && kQTW == kUTW, "one tile shape");
  const int ng_max = a.ng_bound > 0 ? a.ng_bound : max_tap_groups(a.kh, a.kw);
  size_t sq = split_smem_q_single(a.kh, a.kw, ng_max), su = split_smem_update_single(a.kh, a.kw, ng_max);
  const size_t dq = dense_smem_q(kQTH, kQTW, a.kh, a.kw), du = dense_smem_update(kUTH, kUTW, a.kh, a.kw);
  sq = sq > dq ? sq : dq;
  su = su > du ? su : du;
  if (sq > 227 * 1024 || su > 227 * 1024) return cudaErrorInvalidValue;
  return launch_split_pair(a, k_rrl_q_dense<kQTH, kQTW, KW>, k_rrl_update_dense<kUTH, kUTW, KW>, ng_max, sq, su, s);
}

template <typename KQ, typename KU>
static cudaError_t launch_split_pair(const IterArgs& a, KQ kq, KU ku, int ng_max, size_t sq, size_t su,
                                     cudaStream_t s) {
  cudaError_t e;
  if ((e = set_smem(kq, sq)) != cudaSuccess) return e;
  if ((e = set_smem(ku, su)) != cudaSuccess) return e;
  // all of L1 as shared memory: 7-8 tiles resident per SM
  if ((e = cudaFuncSetAttribute(kq, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(ku, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(32, 4);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((a.W + kQTW - 1) / kQTW, (a.H + kQTH - 1) / kQTH, a.nz);
  cfg.dynamicSmemBytes = sq;
  if ((e = cudaLaunchKernelEx(&cfg, kq, a.f, a.ldf, a.uin, a.ldin, a.q, qpitch(a.W), a.H, a.W, a.groups, a.ngroups,
                              a.kh, a.kw, ng_max, a.p, a.zs)) != cudaSuccess)
    return e;
  count_launch();
  cfg.gridDim = dim3((a.W + kUTW - 1) / kUTW, (a.H + kUTH - 1) / kUTH, a.nz);
  cfg.dynamicSmemBytes = su;
  if ((e = cudaLaunchKernelEx(&cfg, ku, (const float2*)a.q, qpitch(a.W), a.uin, a.ldin, a.uout, a.ldout, a.H, a.W, a.groups,
                              a.ngroups, a.kh, a.kw, ng_max, a.p, a.status, a.zs)) != cudaSuccess)
    return e;
  count_launch();
  return cudaSuccess;
}

static cudaError_t launch_split_fft(const IterArgs& a, cudaStream_t s) {
  const size_t sq = ftile::smem_q(), su = ftile::smem_update(a.kh);
  cudaError_t e;
  if ((e = set_smem(k_rrl_q_fft, sq)) != cudaSuccess) return e;
  if ((e = set_smem(k_rrl_update_fft, su)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_rrl_q_fft, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_rrl_update_fft, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) !=
      cudaSuccess)
    return e;
  const int tx = (a.W + ftile::tile_ow(a.kw) - 1) / ftile::tile_ow(a.kw);
  const int ty = (a.H + ftile::tile_oh(a.kh) - 1) / ftile::tile_oh(a.kh);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((tx + 1) / 2, ty, a.nz);
  cfg.dynamicSmemBytes = sq;
  CUtensorMap umap;
  const int use_tma = tma_enabled() &&
                      encode_window_map(&umap, a.uin, a.W, a.H, a.ldin, a.nz, a.zs.in, ftile::kBoxW, ftile::kN);
  if (!use_tma) memset(&umap, 0, sizeof(umap));
  if ((e = cudaLaunchKernelEx(&cfg, k_rrl_q_fft, a.f, a.ldf, a.uin, a.ldin, a.q, a.H, a.W, a.groups, a.kh, a.kw,
                              a.p, a.zs, umap, use_tma, a.status)) != cudaSuccess)
    return e;
  count_launch();
  cfg.gridDim = dim3(tx, ty, a.nz);
  cfg.dynamicSmemBytes = su;
  if ((e = cudaLaunchKernelEx(&cfg, k_rrl_update_fft, (const float2*)a.q, a.uin, a.ldin, a.uout, a.ldout, a.H, a.W,
                              a.groups, a.kh, a.kw, a.p, a.status, a.zs)) != cudaSuccess)
    return e;
  count_launch();
  return cudaSuccess;
}

// SM count of the current device (per call: devices may differ).
static int sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
    return v;
  return 148;
}

template <bool HORIZ, bool BOX, int TH>
static cudaError_t launch_split_box_th(const IterArgs& a, cudaStream_t s) {
  const int L = HORIZ ? a.kw : a.kh;
  const size_t sq = box_smem_q(TH, 32, L, HORIZ), su = box_smem_update(TH, 32, L, HORIZ);
  if (sq > 227 * 1024 || su > 227 * 1024) return cudaErrorInvalidValue;
  auto kq = k_rrl_q_box<HORIZ, BOX, TH>;
  auto ku = k_rrl_update_box<HORIZ, BOX, TH>;
  cudaError_t e;
  if ((e = set_smem(kq, sq)) != cudaSuccess) return e;
  if ((e = set_smem(ku, su)) != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(32, 4);
  cfg.gridDim = dim3((a.W + 31) / 32, (a.H + TH - 1) / TH, a.nz);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.dynamicSmemBytes = sq;
  if ((e = cudaLaunchKernelEx(&cfg, kq, a.f, a.ldf, a.uin, a.ldin, a.q, qpitch(a.W), a.H, a.W, a.ngroups, a.p,
                              a.zs)) != cudaSuccess)
    return e;
  count_launch();
  cfg.dynamicSmemBytes = su;
  if ((e = cudaLaunchKernelEx(&cfg, ku, (const float2*)a.q, qpitch(a.W), a.uin, a.ldin, a.uout, a.ldout, a.H, a.W,
                              a.ngroups, a.p, a.status, a.zs)) != cudaSuccess)
    return e;
  count_launch();
  return cudaSuccess;
}

template <bool HORIZ, bool BOX>
static cudaError_t launch_split_box(const IterArgs& a, cudaStream_t s) {
  const long long tiles = (long long)((a.W + 31) / 32) * ((a.H + 31) / 32) * a.nz;
  return tiles < sm_count() ? launch_split_box_th<HORIZ, BOX, 16>(a, s) : launch_split_box_th<HORIZ, BOX, 32>(a, s);
}

__global__ void k_copy_images(const float* __restrict__ src, int lds, long long zsrc, float* __restrict__ dst,
                              int ldd, long long zdst, int H, int W) {
  const int z = blockIdx.z;
  for (int i = blockIdx.y; i < H; i += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < W; j += gridDim.x * blockDim.x)
      dst[z * zdst + (long long)i * ldd + j] = src[z * zsrc + (long long)i * lds + j];
}

cudaError_t copy_images(const float* src, int lds, long long zsrc, float* dst, int ldd, long long zdst, int H, int W,
                        int n, cudaStream_t s) {
  const dim3 grid((W + 255) / 256, H < 256 ? H : 256, n);
  k_copy_images<<<grid, 256, 0, s>>>(src, lds, zsrc, dst, ldd, zdst, H, W);
  count_launch();
  return cudaGetLastError();
}

size_t rrl_box_smem(int kh, int kw) {
  const bool horiz = kh == 1;
  const int L = horiz ? kw : kh;
  const size_t a = box_smem_q(32, 32, L, horiz), b = box_smem_update(32, 32, L, horiz);
  return a > b ? a : b;
}

static cudaError_t dispatch_dense(const IterArgs& a, cudaStream_t s) {
  switch (a.kw) {
    case 3: return launch_split_dense<3>(a, s);
    case 5: return launch_split_dense<5>(a, s);
    case 7: return launch_split_dense<7>(a, s);
    case 9: return launch_split_dense<9>(a, s);
    case 11: return launch_split_dense<11>(a, s);
    case 13: return launch_split_dense<13>(a, s);
    case 15: return launch_split_dense<15>(a, s);
    case 17: return launch_split_dense<17>(a, s);
    case 19: return launch_split_dense<19>(a, s);
    case 21: return launch_split_dense<21>(a, s);
    case 23: return launch_split_dense<23>(a, s);
    default: return launch_split_dense<25>(a, s);
  }
}

template <bool SPLIT>
static cudaError_t dispatch(const IterArgs& a, cudaStream_t s) {
  if (SPLIT && dense_eligible(a.kh, a.kw)) return dispatch_dense(a, s);
  switch (SPLIT ? split_halo_class(a.kw) : halo_class(a.kw)) {
    case 8: return SPLIT ? launch_split_p<8>(a, s) : launch_fused_p<8>(a, s);
    case 16: return SPLIT ? launch_split_p<16>(a, s) : launch_fused_p<16>(a, s);
    case 32: return SPLIT ? launch_split_p<32>(a, s) : launch_fused_p<32>(a, s);
    case 64: return SPLIT ? launch_split_p<64>(a, s) : launch_fused_p<64>(a, s);
    case 128: return SPLIT ? launch_split_p<128>(a, s) : launch_fused_p<128>(a, s);
    default: return SPLIT ? launch_split_p<256>(a, s) : launch_fused_p<256>(a, s);
  }
}

cudaError_t launch_rrl_spatial(const float* f, int ldf, const float* uin, int ldin, float* uout,
                               int ldout, int H, int W, const TapGroup* groups, const int* ngroups,
                               int kh, int kw, const RrlParams& p, int* status, cudaStream_t s) {
  const IterArgs a = {f, ldf, uin, ldin, uout, ldout, nullptr, H, W, groups, ngroups, kh, kw, p, status, 0, 0, 1, {}};
  return dispatch<false>(a, s);
}

cudaError_t launch_rrl_split(const float* f, int ldf, const float* uin, int ldin, float* uout,
                             int ldout, float2* q, int H, int W, const TapGroup* groups,
                             const int* ngroups, int kh, int kw, const RrlParams& p, int* status,
                             int ng_bound, int axis, cudaStream_t s, int nz, long long zf, long long zin,
                             long long zout, long long zq) {
  const IterArgs a = {f, ldf, uin, ldin, uout, ldout, q, H, W, groups, ngroups, kh, kw, p, status, ng_bound, axis,
                      nz, {zf, zin, zout, zq}};
  if (axis == 1) return kh == 1 ? launch_split_box<true, true>(a, s) : launch_split_box<false, true>(a, s);
  if (axis == 2) return kh == 1 ? launch_split_box<true, false>(a, s) : launch_split_box<false, false>(a, s);
  if (axis == 3) return launch_split_fft(a, s);
  return dispatch<true>(a, s);
}

}  // namespace db
