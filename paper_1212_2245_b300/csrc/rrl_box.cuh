// One-axis PSFs (Sec. 4.3, "Uniform linear motion" and "Non-uniform linear
// motion"): the PSF lies on one row or one column.
//
// Box PSFs -- uniform linear motion along a coordinate axis: the blur b = u*h and both correlations e*h*,
// W*h* by sliding-window sums instead of tap sums.  The taps are
// [e0, w, ..., w, e1] in tap order: a plain box (e0 = e1 = w) or a box of
// non-integer length with lighter end pixels.  Along the blur axis each
// thread owns a run of kBoxSeg outputs: the first output's interior window
// is summed directly, then for every further output one pixel enters and one
// leaves the window, and the two end pixels are added with their own
// weights.  The rest of the iteration (robust weight, diffusion, update) is
// the split schedule's, on the same 32 x 32 tiles.
//
// Layout: shared tiles hold u (or q) over the tile plus the window along the
// blur axis, with constant continuation.  For a horizontal box a thread's
// run lies along a row and the lanes of a warp take 32 different rows, so
// the row stride is odd (bank-conflict free) and the staging copies single
// elements; for a vertical box the lanes take adjacent columns.  The sums go
// to a shared result tile, from which the vertical strips of the split
// schedule finish the pixels.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"
#include "rrl_tiles.cuh"

namespace db {

constexpr int kBoxSeg = 8;  // outputs per sliding-window run

// Box weights as k_prepare_taps stores them, 16 bytes after the group count:
// (e0, w, e1, L as int bits).
__device__ __forceinline__ float4 load_box_weights(const int* ngroups) {
  return __ldg(reinterpret_cast<const float4*>(ngroups + 4));
}

__device__ __forceinline__ float bx_zero(float) { return 0.f; }
__device__ __forceinline__ float2 bx_zero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float bx_add(float a, float b) { return a + b; }
__device__ __forceinline__ float2 bx_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float bx_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float2 bx_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// w S + eL a + eR b
__device__ __forceinline__ float bx_out(float w, float S, float eL, float a, float eR, float b) {
  return fmaf(eR, b, fmaf(eL, a, w * S));
}
__device__ __forceinline__ float2 bx_out(float w, float2 S, float eL, float2 a, float eR, float2 b) {
  return make_float2(bx_out(w, S.x, eL, a.x, eR, b.x), bx_out(w, S.y, eL, a.y, eR, b.y));
}

// kBoxSeg outputs of a box of length L.  src points at the first pixel of the
// first output's window; pixels along the blur axis are `step` apart.  The
// window of output s is src[s .. s+L-1] (in steps): weight eL on its first
// pixel, eR on its last, w on the interior.
template <typename T>
__device__ __forceinline__ void box_run(const T* src, int step, int L, float eL, float w, float eR, T* dst,
                                        int dstep) {
  if (L == 1) {
#pragma unroll
    for (int s = 0; s < kBoxSeg; ++s) {
      const T a = src[s * step];
      dst[s * dstep] = bx_out(0.f, a, eL, a, 0.f, a);
    }
    return;
  }
  T S = bx_zero(T());
  for (int k = 1; k < L - 1; ++k) S = bx_add(S, src[k * step]);
  const int last = (L - 1) * step;
#pragma unroll
  for (int s = 0; s < kBoxSeg; ++s) {
    const T* p = src + s * step;
    const T a = p[0], b = p[last];
    dst[s * dstep] = bx_out(w, S, eL, a, eR, b);
    if (L > 2) S = bx_add(S, bx_sub(b, p[step]));  // p[last] enters, p[step] leaves
  }
}

// Any other one-axis PSF (non-uniform linear motion): the same runs of
// kBoxSeg outputs, each a plain tap sum.  The kBoxSeg window pixels live in a
// register ring: output s at tap m needs pixel m + s, so after tap m the slot
// of pixel m (no longer needed) takes pixel m + kBoxSeg.  Unrolled over
// blocks of kBoxSeg taps the ring indices are compile-time constants.  Full
// blocks (all taps and all pixel loads present) run without conditions, with
// their weights read as two 16-byte words; the last block checks each tap.
// wts[m] is the weight of window pixel m + s for output s: the taps reversed
// for the convolution, in tap order for the correlation (16-byte aligned,
// shared).  The largest pixel read is L - 2 + kBoxSeg.
__device__ __forceinline__ float ax_fma(float w, float a, float acc) { return fmaf(w, a, acc); }
__device__ __forceinline__ float2 ax_fma(float w, float2 a, float2 acc) {
  return make_float2(fmaf(w, a.x, acc.x), fmaf(w, a.y, acc.y));
}
static_assert(kBoxSeg == 8, "two float4 weight words per block");
template <typename T>
__device__ __forceinline__ void axis_run(const T* src, int step, int L, const float* __restrict__ wts, T* dst,
                                         int dstep) {
  T acc[kBoxSeg], x[kBoxSeg];
#pragma unroll
  for (int s = 0; s < kBoxSeg; ++s) { acc[s] = bx_zero(T()); x[s] = src[s * step]; }
  int mb = 0;
  for (; mb + kBoxSeg < L; mb += kBoxSeg) {
    const float4 w0 = *reinterpret_cast<const float4*>(wts + mb);
    const float4 w1 = *reinterpret_cast<const float4*>(wts + mb + 4);
    const float w[kBoxSeg] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int t = 0; t < kBoxSeg; ++t) {
#pragma unroll
      for (int s = 0; s < kBoxSeg; ++s) acc[s] = ax_fma(w[t], x[(t + s) % kBoxSeg], acc[s]);
      x[t] = src[(mb + t + kBoxSeg) * step];
    }
  }
#pragma unroll
  for (int t = 0; t < kBoxSeg; ++t) {
    const int m = mb + t;
    if (m < L) {
      const float w = wts[m];
#pragma unroll
      for (int s = 0; s < kBoxSeg; ++s) acc[s] = ax_fma(w, x[(t + s) % kBoxSeg], acc[s]);
      if (m + 1 < L) x[t] = src[(m + kBoxSeg) * step];
    }
  }
#pragma unroll
  for (int s = 0; s < kBoxSeg; ++s) dst[s * dstep] = acc[s];
}

// Shared copy of a one-axis PSF's taps for axis_run: REV (convolution) holds
// them reversed.
template <bool REV>
__device__ __forceinline__ void load_axis_weights(float* wts, const float* __restrict__ taps, int L) {
  for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < L; k += blockDim.x * blockDim.y)
    wts[k] = __ldg(taps + (REV ? L - 1 - k : k));
}

// The taps of a one-axis PSF as k_prepare_taps stores them, 32 bytes after the
// group count (tap order, L = kh * kw of them).
__device__ __forceinline__ const float* axis_taps(const int* ngroups) {
  return reinterpret_cast<const float*>(ngroups + 8);
}

// Copy rows y0.. (nrows) x columns x0.. (ncols) of a T image into shared rows
// of stride S elements, one element per copy, with clamped indices.
template <typename T>
__device__ __forceinline__ void stage_elems(T* dst, int S, const T* __restrict__ src, int ld, int H, int W, int y0,
                                            int nrows, int x0, int ncols) {
  for (int r = threadIdx.y; r < nrows; r += blockDim.y) {
    const T* srow = src + (size_t)min(max(y0 + r, 0), H - 1) * ld;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
      if constexpr (sizeof(T) == 4) cp_async4(dst + r * S + c, srow + min(max(x0 + c, 0), W - 1));
      else cp_async8(dst + r * S + c, srow + min(max(x0 + c, 0), W - 1));
    }
  }
}

__host__ __device__ inline int box_window_stride(int TW, int L, bool horiz, int elem_pad) {
  return horiz ? ((TW + L - 1) | 1) : TW + elem_pad;
}
__host__ __device__ inline size_t round16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared memory of the one-axis tiles (L: PSF length along its axis); the
// tap array (general taps) comes first.
constexpr int kAxisTapsSmem = 1024;  // 256 floats
__host__ __device__ inline size_t box_smem_q(int TH, int TW, int L, bool horiz) {
  const size_t fs = (size_t)TH * TW * 4 + kAxisTapsSmem, bs = round16((size_t)TH * (TW + 1) * 4);
  const size_t us = horiz ? (size_t)TH * box_window_stride(TW, L, true, 4) * 4
                          : (size_t)(TH + L - 1) * box_window_stride(TW, L, false, 4) * 4;
  return fs + bs + us;
}
__host__ __device__ inline size_t box_smem_update(int TH, int TW, int L, bool horiz) {
  const size_t ds = round16((size_t)TH * (TW + 1) * 8) + kAxisTapsSmem, ud = (size_t)(TH + 4) * (TW + 8) * 4;
  const size_t qs = horiz ? (size_t)TH * box_window_stride(TW, L, true, 2) * 8
                          : (size_t)(TH + L - 1) * box_window_stride(TW, L, false, 2) * 8;
  return ds + ud + qs;
}

// q = (e, W) on the TH x TW tile at (i0, j0) for a one-axis PSF: box (BOX,
// sliding-window sums) or general taps (register windows).
template <int TH, int TW, int R, bool HORIZ, bool BOX = true, typename Dep = NoDep>
__device__ __forceinline__ void q_tile_box(unsigned char* smem_raw, const float* __restrict__ f, int ldf,
                                           const float* __restrict__ uin, int ldin, float2* __restrict__ q, int ldq,
                                           int H, int W, const int* __restrict__ ngroups_g, const RrlParams& p,
                                           int i0, int j0, Dep dep = Dep()) {
  static_assert(TH % R == 0 && TW % 4 == 0 && TW % kBoxSeg == 0 && TH % kBoxSeg == 0, "tile shape");
  const float4 bw = load_box_weights(ngroups_g);
  const int L = __float_as_int(bw.w), before = L - 1 - (L >> 1);  // conv window: L-1-c before, c after
  constexpr int BS = TW + 1;
  const int US = box_window_stride(TW, L, HORIZ, 4);
  float* taps = (float*)smem_raw;  // general taps, reversed (kAxisTapsSmem bytes)
  float* fs = taps + kAxisTapsSmem / 4;
  float* bs = fs + TH * TW;
  float* us = (float*)((unsigned char*)bs + round16((size_t)TH * BS * 4));
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  if (!BOX) load_axis_weights<true>(taps, axis_taps(ngroups_g), L);
  stage_tile<float, TW>(fs, f, ldf, H, W, i0, TH, j0, TW / 4, rows_aligned16(f, ldf));
  dep();
  if (HORIZ) stage_elems<float>(us, US, uin, ldin, H, W, i0, TH, j0 - before, TW + L - 1);
  else stage_tile<float, TW + 4>(us, uin, ldin, H, W, i0 - before, TH + L - 1, j0, TW / 4, rows_aligned16(uin, ldin));
  cp_async_wait_all();
  __syncthreads();
  // convolution: the window's first pixel carries tap L-1, its last tap 0
  for (int item = tid; item < TH * TW / kBoxSeg; item += nth) {
    if (HORIZ) {
      const int r = item % TH, x0 = (item / TH) * kBoxSeg;
      if (BOX) box_run<float>(us + r * US + x0, 1, L, bw.z, bw.y, bw.x, bs + r * BS + x0, 1);
      else axis_run<float>(us + r * US + x0, 1, L, taps, bs + r * BS + x0, 1);
    } else {
      const int c = item % TW, y0 = (item / TW) * kBoxSeg;
      if (BOX) box_run<float>(us + y0 * US + c, US, L, bw.z, bw.y, bw.x, bs + y0 * BS + c, BS);
      else axis_run<float>(us + y0 * US + c, US, L, taps, bs + y0 * BS + c, BS);
    }
  }
  __syncthreads();
  const bool full = i0 + TH <= H && j0 + TW <= W;
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, c = item - s * TW;
    const int r0 = s * R, j = j0 + c;
    float2* qo = q + (size_t)(i0 + r0) * ldq + j;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (full || (j < W && i0 + r0 + r < H))
        qo[(size_t)r * ldq] = weighted_residual(bs[(r0 + r) * BS + c], fmaxf(fs[(r0 + r) * TW + c], p.floor), p);
  }
}

// Delta, B (one-axis sums of q), D and the update on the TH x TW tile at (i0, j0).
template <int TH, int TW, int R, bool HORIZ, bool BOX = true, typename Dep = NoDep>
__device__ __forceinline__ void update_tile_box(unsigned char* smem_raw, const float2* __restrict__ q, int ldq,
                                                const float* __restrict__ uin, int ldin, float* __restrict__ uout,
                                                int ldout, int H, int W, const int* __restrict__ ngroups_g,
                                                const RrlParams& p, int* status, int i0, int j0, Dep dep = Dep()) {
  static_assert(TH % R == 0 && TW % 4 == 0 && TW % kBoxSeg == 0 && TH % kBoxSeg == 0, "tile shape");
  const float4 bw = load_box_weights(ngroups_g);
  const int L = __float_as_int(bw.w), c0 = L >> 1;  // correlation window: c before, L-1-c after
  constexpr int DS = TW + 1, UH = TH + 4, US = TW + 8;
  const int QS = box_window_stride(TW, L, HORIZ, 2);
  float* taps = (float*)smem_raw;  // general taps (kAxisTapsSmem bytes)
  float2* ds = (float2*)(smem_raw + kAxisTapsSmem);
  float* us = (float*)((unsigned char*)ds + round16((size_t)TH * DS * 8));
  float2* qs = (float2*)(us + UH * US);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  if (!BOX) load_axis_weights<false>(taps, axis_taps(ngroups_g), L);
  stage_tile<float, US>(us, uin, ldin, H, W, i0 - 2, UH, j0 - 4, TW / 4 + 2, rows_aligned16(uin, ldin));
  dep();
  if (HORIZ) stage_elems<float2>(qs, QS, q, ldq, H, W, i0, TH, j0 - c0, TW + L - 1);
  else stage_tile<float2, TW + 2>(qs, q, ldq, H, W, i0 - c0, TH + L - 1, j0, TW / 2, rows_aligned16(q, ldq));
  cp_async_wait_all();
  __syncthreads();
  // correlation: the window's first pixel carries tap 0, its last tap L-1
  for (int item = tid; item < TH * TW / kBoxSeg; item += nth) {
    if (HORIZ) {
      const int r = item % TH, x0 = (item / TH) * kBoxSeg;
      if (BOX) box_run<float2>(qs + r * QS + x0, 1, L, bw.x, bw.y, bw.z, ds + r * DS + x0, 1);
      else axis_run<float2>(qs + r * QS + x0, 1, L, taps, ds + r * DS + x0, 1);
    } else {
      const int c = item % TW, y0 = (item / TW) * kBoxSeg;
      if (BOX) box_run<float2>(qs + y0 * QS + c, QS, L, bw.x, bw.y, bw.z, ds + y0 * DS + c, DS);
      else axis_run<float2>(qs + y0 * QS + c, QS, L, taps, ds + y0 * DS + c, DS);
    }
  }
  __syncthreads();
  const bool full = i0 + TH <= H && j0 + TW <= W;
  bool bad = false;
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, oj = item - s * TW;
    const int oi0 = s * R, j = j0 + oj;
    float D[R], c[R];
    diffusion_strip<R, US>(us + (oi0 + 2) * US + (oj + 4), p, D, c);
    float* uo = uout + (size_t)(i0 + oi0) * ldout + j;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float2 dB = ds[(oi0 + r) * DS + oj];
      const float un = rrl_update(c[r], dB.x, dB.y, D[r], p);
      bad |= !isfinite(un);
      if (full || (j < W && i0 + oi0 + r < H)) uo[(size_t)r * ldout] = un;
    }
  }
  if (bad && status) atomicOr(status, DB_FLAG_NONFINITE);
}

}  // namespace db
