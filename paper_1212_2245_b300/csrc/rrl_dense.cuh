// Dense 2D PSFs (Sec. 4.1 "Convolution", Sec. 4.3 general 2D variant): tile
// bodies of the split schedule for PSFs whose taps are mostly non-zero
// (Gaussian mixtures and the like), register blocked in two dimensions.
//
// Each thread owns a block of R = 2 rows x C = 4 columns of outputs.  It
// walks the tap rows in order; at each it loads the one staged input row
// (C + kw - 1 values, 16-byte shared loads; consecutive lanes own
// consecutive column blocks, so a warp's loads are conflict-free) that the
// tap row maps onto its first output row, keeps the previous one (which the
// same tap row maps onto its second output row) in registers, and reads the
// tap row once: a weight (a broadcast 16-byte load of four taps) feeds
// R x C FMAs and an input value up to R x C x kw / (C + kw - 1), so the tap
// sums are bound by the FMA pipe rather than by shared-memory wavefronts.
//
// Per output the sums run in a fixed order independent of the tile and of
// the block shape (convolution: tap rows from 0 up to kh-1, correlation:
// from kh-1 down to 0; taps of a row from 0 up to kw-1), so every schedule
// and the batched kernel that use these bodies give the same bits.
//
// q = (e, W) goes through global memory in planar form for these PSFs: the
// e plane (pitch upitch(W) floats) followed by the W plane, each staged with
// 16-byte copies.  The weights are read from the dense tap table that
// k_prepare_taps writes after the tap groups (kh rows, dense_tap_stride(kw)
// floats each); its flag word selects these bodies on the device, so a PSF
// of an eligible shape but with many zero taps keeps the tap groups.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"
#include "rrl_tiles.cuh"

namespace db {

constexpr int kDR = 2, kDC = 4;  // output block of one thread

// Columns the staged window of the dense bodies is shifted by: the window of
// a tile starts at a 4-column boundary at or left of the first column read.
template <int KW>
struct DenseGeom {
  static constexpr int cx = (KW - 1) / 2;
  static constexpr int OXB = (4 - (cx & 3)) & 3;      // convolution (u window starts cx left of j0)
  static constexpr int OXC = (4 - (cx & 3)) & 3;      // correlation (q window starts cx left of j0)
  static constexpr int NB = ((kDC + KW - 1 + OXB) + 3) & ~3;  // window floats (convolution)
  static constexpr int NC = ((kDC + KW - 1 + OXC) + 3) & ~3;  // window floats (correlation)
  static constexpr int KW4 = (KW + 3) / 4;
};

__device__ __forceinline__ void load_row(float* v, const float* __restrict__ src, int n4) {
#pragma unroll
  for (int k = 0; k < n4; ++k) {
    const float4 t = reinterpret_cast<const float4*>(src)[k];
    v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
  }
}

// acc0[c] += sum_b w[b] va[c + OFF(b)], acc1[c] += sum_b w[b] vb[c + OFF(b)]
// for one tap row w (KW taps, 16-byte aligned): every weight read once
// feeds 2 C FMAs.  CONV: OFF(b) = KW-1-b + OX, else b + OX.
template <int KW, int OX, bool CONV>
__device__ __forceinline__ void dense_row_taps2(const float* __restrict__ w, const float* va, const float* vb,
                                                float (&acc0)[kDC], float (&acc1)[kDC]) {
#pragma unroll
  for (int g = 0; g < DenseGeom<KW>::KW4; ++g) {
    const float4 w4 = reinterpret_cast<const float4*>(w)[g];
    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int b = 4 * g + t;
      if (b < KW) {
#pragma unroll
        for (int c = 0; c < kDC; ++c) {
          acc0[c] = fmaf(wv[t], va[c + (CONV ? KW - 1 - b : b) + OX], acc0[c]);
          acc1[c] = fmaf(wv[t], vb[c + (CONV ? KW - 1 - b : b) + OX], acc1[c]);
        }
      }
    }
  }
}

// Tap sums at the 2 x C block whose first output sits at row r0, column c0
// of the tile, over the staged plane `base` (row stride S; row 0 = image row
// i0 - (kh-1)/2, column 0 = the window start).  Output row o meets staged
// row s = o + kh - 1 - a of tap row a (convolution, b = u*h) or s = o + a
// (correlation with h*).  Step k = 0 .. kh-1 applies tap row a = k
// (convolution) or a = kh-1-k (correlation): in both cases output row 0
// reads staged row kh-1-k, loaded at this step, and output row 1 the row
// loaded one step earlier, so each staged row is loaded once and each tap
// row read once.  Per output the taps are summed by tap row in step order,
// within a row from b = 0 up.
template <int KW, int S, bool CONV>
__device__ __forceinline__ void dense_sum(const float* __restrict__ base, const float* __restrict__ tab, int TS,
                                          int kh, int r0, int c0, float (&acc)[kDR][kDC]) {
  static_assert(kDR == 2, "two output rows per block");
  using G = DenseGeom<KW>;
  constexpr int OX = CONV ? G::OXB : G::OXC;
  constexpr int NV = CONV ? G::NB : G::NC;
#pragma unroll
  for (int o = 0; o < kDR; ++o)
#pragma unroll
    for (int c = 0; c < kDC; ++c) acc[o][c] = 0.f;
  float v0[NV], v1[NV];
  const float* rowp = base + (r0 + kh) * S + c0;  // staged row kh: output row 1 at step 0
  load_row(v1, rowp, NV / 4);
#pragma unroll 1
  for (int k = 0; k < kh; k += 2) {
    rowp -= S;  // staged row kh-1-k
    load_row(v0, rowp, NV / 4);
    dense_row_taps2<KW, OX, CONV>(tab + (CONV ? k : kh - 1 - k) * TS, v0, v1, acc[0], acc[1]);
    if (k + 1 < kh) {
      rowp -= S;  // staged row kh-2-k
      load_row(v1, rowp, NV / 4);
      dense_row_taps2<KW, OX, CONV>(tab + (CONV ? k + 1 : kh - 2 - k) * TS, v1, v0, acc[0], acc[1]);
    }
  }
}

// Row stride (floats) of the staged windows: TW + P with P >= kw + 2, as
// the tap-group bodies use.
__host__ __device__ inline size_t dense_smem_q(int TH, int TW, int kh, int kw) {
  return (size_t)kh * dense_tap_stride(kw) * 4 + (size_t)TH * TW * 4 +
         (size_t)(TH + kh - 1) * (TW + split_halo_class(kw)) * 4;
}
__host__ __device__ inline size_t dense_smem_update(int TH, int TW, int kh, int kw) {
  return (size_t)kh * dense_tap_stride(kw) * 4 + (size_t)2 * (TH + kh - 1) * (TW + split_halo_class(kw)) * 4 +
         (size_t)(TH + 4) * (TW + 8) * 4;
}

// Copy the dense tap table (kh rows of TS floats) into shared memory.
__device__ __forceinline__ void stage_dense_taps(float* dst, const float* __restrict__ tab_g, int kh, int TS) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  for (int k = tid; k < kh * TS / 4; k += nth) cp_async16(dst + 4 * k, tab_g + 4 * k);
}

// q = (e, W) on the TH x TW tile at (i0, j0), planar: qe, qw (pitch ldqp).
// smem_raw: dense_smem_q bytes.
template <int TH, int TW, int KW, typename Dep = NoDep>
__device__ __forceinline__ void q_tile_dense(unsigned char* smem_raw, const float* __restrict__ f, int ldf,
                                             const float* __restrict__ uin, int ldin, float* __restrict__ qe,
                                             float* __restrict__ qw, int ldqp, int H, int W,
                                             const float* __restrict__ tab_g, int kh, const RrlParams& p, int i0,
                                             int j0, Dep dep = Dep()) {
  static_assert(TH % kDR == 0 && TW % kDC == 0, "tile shape");
  using G = DenseGeom<KW>;
  constexpr int P = (KW + 2 <= 8) ? 8 : (KW + 2 <= 16) ? 16 : 32;
  static_assert(KW + 2 <= P, "halo class");
  constexpr int US = TW + P, TS = (KW + 3) & ~3;
  const int cy = (kh - 1) / 2;
  const int UH = TH + kh - 1;
  const int xs = j0 - G::cx - G::OXB;  // a multiple of 4: j0 is
  const int nc = (G::OXB + TW + KW - 1 + 3) >> 2;
  float* tab = (float*)smem_raw;
  float* fs = tab + kh * TS;  // TH x TW
  float* us = fs + TH * TW;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  stage_dense_taps(tab, tab_g, kh, TS);
  stage_tile<float, TW>(fs, f, ldf, H, W, i0, TH, j0, TW / 4, rows_aligned16(f, ldf));
  dep();
  stage_tile<float, US>(us, uin, ldin, H, W, i0 - cy, UH, xs, nc, rows_aligned16(uin, ldin));
  cp_async_wait_all();
  __syncthreads();
  const bool vec = rows_aligned16(qe, ldqp) && rows_aligned16(qw, ldqp);
  for (int item = tid; item < (TH / kDR) * (TW / kDC); item += nth) {
    const int br = item / (TW / kDC), bc = item - br * (TW / kDC);
    const int r0 = br * kDR, c0 = bc * kDC;
    float b[kDR][kDC];
    dense_sum<KW, US, true>(us, tab, TS, kh, r0, c0, b);
    const int j = j0 + c0;
#pragma unroll
    for (int o = 0; o < kDR; ++o) {
      const int i = i0 + r0 + o;
      if (i >= H) continue;
      const float4 f4 = *reinterpret_cast<const float4*>(fs + (r0 + o) * TW + c0);
      const float fv[kDC] = {f4.x, f4.y, f4.z, f4.w};
      float e4[kDC], w4[kDC];
#pragma unroll
      for (int c = 0; c < kDC; ++c) {
        const float2 q = weighted_residual(b[o][c], fmaxf(fv[c], p.floor), p);
        e4[c] = q.x; w4[c] = q.y;
      }
      float* pe = qe + (size_t)i * ldqp + j;
      float* pw = qw + (size_t)i * ldqp + j;
      if (vec && j + kDC <= W) {
        *reinterpret_cast<float4*>(pe) = make_float4(e4[0], e4[1], e4[2], e4[3]);
        *reinterpret_cast<float4*>(pw) = make_float4(w4[0], w4[1], w4[2], w4[3]);
      } else {
#pragma unroll
        for (int c = 0; c < kDC; ++c)
          if (j + c < W) { pe[c] = e4[c]; pw[c] = w4[c]; }
      }
    }
  }
}

// Delta, B from planar q, the diffusion term and the update on the TH x TW
// tile at (i0, j0).  smem_raw: dense_smem_update bytes.
template <int TH, int TW, int KW, typename Dep = NoDep>
__device__ __forceinline__ void update_tile_dense(unsigned char* smem_raw, const float* __restrict__ qe,
                                                  const float* __restrict__ qw, int ldqp,
                                                  const float* __restrict__ uin, int ldin, float* __restrict__ uout,
                                                  int ldout, int H, int W, const float* __restrict__ tab_g, int kh,
                                                  const RrlParams& p, int* status, int i0, int j0, Dep dep = Dep()) {
  static_assert(TH % kDR == 0 && TW % kDC == 0, "tile shape");
  using G = DenseGeom<KW>;
  constexpr int P = (KW + 2 <= 8) ? 8 : (KW + 2 <= 16) ? 16 : 32;
  constexpr int QS = TW + P, US = TW + 8, TS = (KW + 3) & ~3;
  const int cy = (kh - 1) / 2;
  const int QH = TH + kh - 1, UH = TH + 4;
  const int xq = j0 - G::cx - G::OXC;  // a multiple of 4
  const int ncq = (G::OXC + TW + KW - 1 + 3) >> 2;
  float* tab = (float*)smem_raw;
  float* es = tab + kh * TS;
  float* ws = es + QH * QS;
  float* us = ws + QH * QS;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  stage_dense_taps(tab, tab_g, kh, TS);
  stage_tile<float, US>(us, uin, ldin, H, W, i0 - 2, UH, j0 - 4, TW / 4 + 2, rows_aligned16(uin, ldin));
  dep();
  const bool qa = rows_aligned16(qe, ldqp) && rows_aligned16(qw, ldqp);
  stage_tile<float, QS>(es, qe, ldqp, H, W, i0 - cy, QH, xq, ncq, qa);
  stage_tile<float, QS>(ws, qw, ldqp, H, W, i0 - cy, QH, xq, ncq, qa);
  cp_async_wait_all();
  __syncthreads();
  const bool vec = rows_aligned16(uout, ldout);
  bool bad = false;
  for (int item = tid; item < (TH / kDR) * (TW / kDC); item += nth) {
    const int br = item / (TW / kDC), bc = item - br * (TW / kDC);
    const int r0 = br * kDR, c0 = bc * kDC;
    float dl[kDR][kDC], B[kDR][kDC];
    dense_sum<KW, QS, false>(es, tab, TS, kh, r0, c0, dl);
    dense_sum<KW, QS, false>(ws, tab, TS, kh, r0, c0, B);
    float un[kDR][kDC];
#pragma unroll
    for (int c = 0; c < kDC; ++c) {
      float D[kDR], ctr[kDR];
      diffusion_strip<kDR, US>(us + (r0 + 2) * US + (c0 + c + 4), p, D, ctr);
#pragma unroll
      for (int o = 0; o < kDR; ++o) {
        un[o][c] = rrl_update(ctr[o], dl[o][c], B[o][c], D[o], p);
        bad |= !isfinite(un[o][c]);
      }
    }
    const int j = j0 + c0;
#pragma unroll
    for (int o = 0; o < kDR; ++o) {
      const int i = i0 + r0 + o;
      if (i >= H) continue;
      float* po = uout + (size_t)i * ldout + j;
      if (vec && j + kDC <= W) {
        *reinterpret_cast<float4*>(po) = make_float4(un[o][0], un[o][1], un[o][2], un[o][3]);
      } else {
#pragma unroll
        for (int c = 0; c < kDC; ++c)
          if (j + c < W) po[c] = un[o][c];
      }
    }
  }
  if (bad && status) atomicOr(status, DB_FLAG_NONFINITE);
}

}  // namespace db
