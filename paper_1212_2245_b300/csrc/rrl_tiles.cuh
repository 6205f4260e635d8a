// Device pieces of the spatial RRRL iteration (Sec. 2.3, Eq. 9-12; spatial
// sums with constant continuation, Sec. 4.1-4.2): pointwise formulas, the
// register-blocked strip sums, and the tile bodies of the fused and split
// schedules.  Shared by the single-image kernels and the batched persistent
// kernel.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace db {

// ---------------------------------------------------------------------------
// pointwise pieces
//
// The update of Eq. 9 is evaluated in increment form.  With
//   e = W (f - b)/b   (so that W f/b = W + e),
//   Delta = e*h*,  B = W*h*   (hence A = B + Delta),
// the update u (A + alpha[D]+)/(B - alpha[D]-) equals exactly
//   u + u (Delta + alpha D) / (B - alpha [D]-),
// because [D]+ + [D]- = D.  In FP32 this keeps the correlation sums and the
// final rounding on the small increment instead of on values near 1 and on
// the full product, which cuts the rounding drift of 20 iterations about
// sixfold against the FP64 reference.
// ---------------------------------------------------------------------------
// W = phi'(r_f(b)) (Eq. 7, 10), r_f by rf_divergence.
__device__ __forceinline__ float robust_weight(float b, float f, const RrlParams& p) {
  if (!p.phi_robust) return 1.0f;
  const float r = rf_divergence(b, f, p);
  return p.eps_phi * rsqrtf(fmaf(p.eps_phi, p.eps_phi, fmaxf(r, 0.0f)));  // explicit FMA: same rounding in every kernel shape
}

// (e, W) for one pixel: W = phi'(r_f(b)), e = W (f - b)/b.
__device__ __forceinline__ float2 weighted_residual(float b, float f, const RrlParams& p) {
  const float w = robust_weight(b, f, p);
  return make_float2(__fdividef(w * (f - b), b), w);
}

// ---------------------------------------------------------------------------
// tap groups in shared memory
//
// Each group is staged as two float4: (w0, w1, w2, offset of its first load
// as int bits) and (w3 .. w6).  Groups are sorted by height, so the strip
// sums run one loop per height class with compile-time height M: a group
// loaded once from shared memory feeds M*R (blur) or 2*M*R (correlation)
// FMAs from R+M-1 shared loads.  `cls` holds the class starts (kMaxGroupH+1
// ints, staged next to the records).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void stage_group(float4* dst, const TapGroup& t, int off) {
  dst[0] = make_float4(t.w[0], t.w[1], t.w[2], __int_as_float(off));
  dst[1] = make_float4(t.w[3], t.w[4], t.w[5], t.w[6]);
}

// Height of group g (classes delimited by cls).
__device__ __forceinline__ int group_height(const int* cls, int g) {
  int m = 1;
  while (m < kMaxGroupH && g >= cls[m]) ++m;
  return m;
}

// Stage the class starts and the records of all groups; off(t, m) gives a
// group's offset from its tap group and height.
template <typename Off>
__device__ __forceinline__ void stage_groups(int* cls_s, float4* rec, const TapGroup* __restrict__ groups_g,
                                             const int* __restrict__ ngroups_g, Off off) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const int* cls_g = group_class_starts(ngroups_g);
  if (tid <= kMaxGroupH) cls_s[tid] = __ldg(cls_g + tid);
  const int ng = __ldg(ngroups_g);
  for (int g = tid; g < ng; g += nth) {
    const TapGroup t = groups_g[g];
    int m = 1;
    while (m < kMaxGroupH && g >= __ldg(cls_g + m)) ++m;
    stage_group(rec + 2 * g, t, off(t, m));
  }
}

template <int M>
__device__ __forceinline__ void group_weights(const float4* __restrict__ rec, float (&w)[kMaxGroupH], int& off) {
  const float4 A = rec[0];
  w[0] = A.x; w[1] = A.y; w[2] = A.z;
  off = __float_as_int(A.w);
  if (M > 3) {
    const float4 B = rec[1];
    w[3] = B.x; w[4] = B.y; w[5] = B.z;
    if (kMaxGroupH > 6) w[6] = B.w;
  }
}

// b[r] += (u*h) over the groups g0..g1-1 of height M, at R vertically
// adjacent pixels; `base` points at the u value the first pixel's strip
// starts from.
template <int R, int M, int STRIDE>
__device__ __forceinline__ void blur_class(const float* __restrict__ base, const float4* __restrict__ rec, int g0,
                                           int g1, float (&b)[R]) {
#pragma unroll(M > 3 ? 1 : 2)
  for (int g = g0; g < g1; ++g) {
    float w[kMaxGroupH];
    int off;
    group_weights<M>(rec + 2 * g, w, off);
    const float* pu = base + off;
    float v[R + M - 1];
#pragma unroll
    for (int t = 0; t < R + M - 1; ++t) v[t] = pu[t * STRIDE];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < M; ++k) b[r] = fmaf(w[k], v[r + M - 1 - k], b[r]);
  }
}

template <int R, int STRIDE>
__device__ __forceinline__ void blur_strip(const float* __restrict__ base, const float4* __restrict__ rec,
                                           const int* __restrict__ cls, float (&b)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) b[r] = 0.f;
  blur_class<R, 1, STRIDE>(base, rec, cls[0], cls[1], b);
  blur_class<R, 2, STRIDE>(base, rec, cls[1], cls[2], b);
  blur_class<R, 3, STRIDE>(base, rec, cls[2], cls[3], b);
  blur_class<R, 4, STRIDE>(base, rec, cls[3], cls[4], b);
  blur_class<R, 5, STRIDE>(base, rec, cls[4], cls[5], b);
  if constexpr (kMaxGroupH >= 6) blur_class<R, 6, STRIDE>(base, rec, cls[5], cls[6], b);
  if constexpr (kMaxGroupH >= 7) blur_class<R, 7, STRIDE>(base, rec, cls[6], cls[7], b);
}

// Delta[r] += (e*h*), B[r] += (W*h*) over the groups of height M.
template <int R, int M, int STRIDE>
__device__ __forceinline__ void correlate_class(const float2* __restrict__ base, const float4* __restrict__ rec,
                                                int g0, int g1, float (&dl)[R], float (&B)[R]) {
#pragma unroll(M > 3 ? 1 : 2)
  for (int g = g0; g < g1; ++g) {
    float w[kMaxGroupH];
    int off;
    group_weights<M>(rec + 2 * g, w, off);
    const float2* pq = base + off;
    float2 v[R + M - 1];
#pragma unroll
    for (int t = 0; t < R + M - 1; ++t) v[t] = pq[t * STRIDE];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < M; ++k) {
        dl[r] = fmaf(w[k], v[r + k].x, dl[r]);
        B[r] = fmaf(w[k], v[r + k].y, B[r]);
      }
  }
}

template <int R, int STRIDE>
__device__ __forceinline__ void correlate_strip(const float2* __restrict__ base, const float4* __restrict__ rec,
                                                const int* __restrict__ cls, float (&dl)[R], float (&B)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) { dl[r] = 0.f; B[r] = 0.f; }
  correlate_class<R, 1, STRIDE>(base, rec, cls[0], cls[1], dl, B);
  correlate_class<R, 2, STRIDE>(base, rec, cls[1], cls[2], dl, B);
  correlate_class<R, 3, STRIDE>(base, rec, cls[2], cls[3], dl, B);
  correlate_class<R, 4, STRIDE>(base, rec, cls[3], cls[4], dl, B);
  correlate_class<R, 5, STRIDE>(base, rec, cls[4], cls[5], dl, B);
  if constexpr (kMaxGroupH >= 6) correlate_class<R, 6, STRIDE>(base, rec, cls[5], cls[6], dl, B);
  if constexpr (kMaxGroupH >= 7) correlate_class<R, 7, STRIDE>(base, rec, cls[6], cls[7], dl, B);
}

// Diffusion term D = div(psi'(|grad u|^2) grad u) (Eq. 11) at R vertically
// adjacent pixels.  uc points at the first pixel in a shared-memory copy of
// u(clamp(.)) with at least 2 pixels of halo on every side.  Diffusivities
// and vertical fluxes shared by neighbouring rows of the strip are formed
// once.  Across the image boundary the clamped copy makes every difference
// vanish exactly: zero flux.
template <int R, int S0, bool TV>
__device__ __forceinline__ void diffusion_strip_t(const float* __restrict__ uc, const RrlParams& p,
                                                  float (&D)[R], float (&c)[R], int s_rt) {
  const int S = S0 > 0 ? S0 : s_rt;  // row stride: compile-time, or given at run time (S0 = 0)
  // With g = psi'(|grad u|^2) and central differences, g = 2 g2 where
  // g2 = 1/sqrt(dx^2 + dy^2 + 4 eps^2) on the undivided differences dx, dy;
  // a flux 1/2 (g_a + g_b)(u_b - u_a) is then (g2_a + g2_b)(u_b - u_a).
  // (Linear diffusion, psi' = 1: g2 = 1/2.)
  const float e4 = 4.0f * p.eps_psi * p.eps_psi;
  auto g2 = [&](float dx, float dy) { return TV ? rsqrtf(fmaf(dx, dx, fmaf(dy, dy, e4))) : 0.5f; };
  float m[R + 4], e1[R + 2], w1[R + 2];
#pragma unroll
  for (int t = 0; t < R + 4; ++t) m[t] = uc[(t - 2) * S];
#pragma unroll
  for (int t = 0; t < R + 2; ++t) { e1[t] = uc[(t - 1) * S + 1]; w1[t] = uc[(t - 1) * S - 1]; }
  float gC[R + 2];
#pragma unroll
  for (int t = 0; t < R + 2; ++t)  // rows -1..R
    gC[t] = g2(e1[t] - w1[t], m[t + 2] - m[t]);
  float Fv[R + 1];
#pragma unroll
  for (int t = 0; t < R + 1; ++t)  // flux between rows t-1 and t (rounded on its own, so that
    // no FMA contraction at a strip's ends makes the result depend on the strip height)
    Fv[t] = __fmul_rn(gC[t + 1] + gC[t], m[t + 2] - m[t + 1]);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float e2 = uc[r * S + 2], w2 = uc[r * S - 2];
    const float ctr = m[r + 2];
    const float gE = g2(e2 - ctr, e1[r + 2] - e1[r]);
    const float gW = g2(ctr - w2, w1[r + 2] - w1[r]);
    const float fe = (gE + gC[r + 1]) * (e1[r + 1] - ctr);
    const float fw = (gC[r + 1] + gW) * (ctr - w1[r + 1]);
    D[r] = (fe - fw) + (Fv[r + 1] - Fv[r]);
    c[r] = ctr;
  }
}

template <int R, int S>
__device__ __forceinline__ void diffusion_strip(const float* __restrict__ uc, const RrlParams& p,
                                                float (&D)[R], float (&c)[R], int s_rt = 0) {
  if (p.psi_tv) diffusion_strip_t<R, S, true>(uc, p, D, c, s_rt);
  else diffusion_strip_t<R, S, false>(uc, p, D, c, s_rt);
}

// u' = u + u (Delta + alpha D) / (B - alpha [D]-)
__device__ __forceinline__ float rrl_update(float u, float dl, float B, float D, const RrlParams& p) {
  const float den = B - p.alpha * fminf(D, 0.f);
  return fmaf(u, __fdividef(fmaf(p.alpha, D, dl), den), u);
}

// ---------------------------------------------------------------------------
// fused iteration, register blocked.
//
// Each thread owns a vertical strip of R q-points (phase 1) or R outputs
// (phase 2) in one column, so a tap group of height M loaded once from
// shared memory feeds M*R (phase 1) or 2*M*R (phase 2) FMAs from R+M-1
// shared loads.  Lanes of a warp own adjacent columns: shared accesses are
// conflict-free.
//
// Geometry (virtual rows/cols may lie outside the image):
//   q tile : rows i0-cy .. i0-cy+QHp-1, cols j0-cx .. j0-cx+QW-1
//   u tile : rows i0-Ry .. i0-Ry+UH-1,  cols j0-Rx .. j0-Rx+US-1
// u is staged as u(clamp(.)); q = (e, W) is first formed at every virtual
// position from the clamped u and then, at virtual positions outside the
// image, replaced by q at the clamped position.
// ---------------------------------------------------------------------------
template <int TH, int TW, int R, int P>
__global__ void __launch_bounds__(256, 2) k_rrl_spatial(const float* __restrict__ f, int ldf,
                                                     const float* __restrict__ uin, int ldin,
                                                     float* __restrict__ uout, int ldout, int H, int W,
                                                     const TapGroup* __restrict__ groups_g,
                                                     const int* __restrict__ ngroups_g, int kh, int kw,
                                                     int ng_max, RrlParams p, int* status) {
  static_assert(TH % R == 0, "output strips must tile TH");
  // row strides padded to the halo class P >= kw - 1 (compile-time strides
  // let every strip load use an immediate offset)
  constexpr int US = TW + 2 * P, QS = TW + P;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cy = kh >> 1, cx = kw >> 1;
  const int Ry = max(kh - 1, 2), Rx = P;
  const int QH = TH + kh - 1, QW = TW + kw - 1;
  const int NQS = (QH + R - 1) / R, QHp = NQS * R;
  const int UH = Ry + max(QHp, TH + 2);
  int* cls = (int*)smem_raw;
  float4* gu = (float4*)(smem_raw + 32);
  float4* gq = gu + 2 * ng_max;
  float* us = (float*)(gq + 2 * ng_max);
  float2* qs = (float2*)(us + ((UH * US + 1) & ~1));
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;

  stage_groups(cls, gu, groups_g, ngroups_g,
               [&](const TapGroup& t, int m) { return (Ry - cy - t.dy0 - (m - 1)) * US + (Rx - cx - t.dx); });
  stage_groups(cls, gq, groups_g, ngroups_g,
               [&](const TapGroup& t, int m) { return (cy + t.dy0) * QS + (cx + t.dx); });
  for (int r = threadIdx.y; r < UH; r += blockDim.y) {
    const int gi = min(max(i0 - Ry + r, 0), H - 1);
    const float* src = uin + (size_t)gi * ldin;
    for (int c = threadIdx.x; c < US; c += blockDim.x)
      cp_async4(us + r * US + c, src + min(max(j0 - Rx + c, 0), W - 1));
  }
  cp_async_wait_all();
  __syncthreads();

  // phase 1: (e, W) on the q tile (virtual positions)
  for (int item = tid; item < NQS * QW; item += nth) {
    const int s = item / QW, qc = item - s * QW;
    const int qr0 = s * R;
    const int aj = min(max(j0 - cx + qc, 0), W - 1);
    float fv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int ai = min(max(i0 - cy + qr0 + r, 0), H - 1);
      fv[r] = fmaxf(__ldg(f + (size_t)ai * ldf + aj), p.floor);
    }
    float b[R];
    blur_strip<R, US>(us + qr0 * US + qc, gu, cls, b);
#pragma unroll
    for (int r = 0; r < R; ++r) qs[(qr0 + r) * QS + qc] = weighted_residual(b[r], fv[r], p);
  }
  __syncthreads();
  const bool border = (i0 - cy < 0) || (j0 - cx < 0) || (i0 - cy + QH > H) || (j0 - cx + QW > W);
  if (border) {
    // writes only positions outside the image, reads only positions inside
    // it: no ordering between threads is needed within this pass
    for (int idx = tid; idx < QH * QW; idx += nth) {
      const int qr = idx / QW, qc = idx - qr * QW;
      const int vi = i0 - cy + qr, vj = j0 - cx + qc;
      const int ci = min(max(vi, 0), H - 1), cj = min(max(vj, 0), W - 1);
      if (ci != vi || cj != vj) qs[qr * QS + qc] = qs[(ci - (i0 - cy)) * QS + (cj - (j0 - cx))];
    }
    __syncthreads();
  }

  // phase 2: Delta = e*h*, B = W*h*, diffusion, update
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, oj = item - s * TW;
    const int oi0 = s * R, j = j0 + oj;
    float dl[R], B[R], D[R], c[R];
    correlate_strip<R, QS>(qs + oi0 * QS + oj, gq, cls, dl, B);
    diffusion_strip<R, US>(us + (oi0 + Ry) * US + (oj + Rx), p, D, c);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + oi0 + r;
      const float un = rrl_update(c[r], dl[r], B[r], D[r], p);
      if (i < H && j < W) {
        if (!isfinite(un) && status) atomicOr(status, DB_FLAG_NONFINITE);
        uout[(size_t)i * ldout + j] = un;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// split schedule: the same iteration as two launches.
//   k_rrl_q      : q = (e, W) once per pixel into a global float2 buffer
//   k_rrl_update : Delta, B from q (clamped reads), diffusion from u, update
// Used when the image (u, f, q: 16 bytes per pixel) stays resident in L2, so
// the extra round trip of q costs no HBM traffic while the halo recompute of
// the fused kernel disappears.
//
// Tiles are staged in 16-byte chunks.  The staged window starts at a column
// rounded down to a chunk boundary; the few extra columns are absorbed by
// the tap offsets.  A chunk that lies inside the image (and a source whose
// rows are 16-byte aligned) is one cp.async of 16 bytes; any other chunk is
// copied element by element with clamped indices (constant continuation).
// ---------------------------------------------------------------------------
// Halo class of the split tiles: the smallest of 8, 16, ..., 256 that holds
// kw + 2 (the kw - 1 halo columns plus up to 3 columns of chunk alignment).
__host__ __device__ inline int split_halo_class(int kw) {
  int P = 8;
  while (P < kw + 2) P *= 2;
  return P;
}
// Shared memory of one split tile of TH x TW outputs (class starts, group
// records, staged images).
__host__ __device__ inline size_t groups_smem(int ng_max) { return 32 + (size_t)ng_max * kGroupRecordBytes; }
__host__ __device__ inline size_t split_smem_q(int TH, int TW, int kh, int kw, int ng_max) {
  return groups_smem(ng_max) + (size_t)TH * TW * sizeof(float) +
         (size_t)(TH + kh - 1) * (TW + split_halo_class(kw)) * sizeof(float);
}
__host__ __device__ inline size_t split_smem_update(int TH, int TW, int kh, int kw, int ng_max) {
  return groups_smem(ng_max) + (size_t)(TH + kh - 1) * (TW + split_halo_class(kw)) * 8 +
         (size_t)(TH + 4) * (TW + 8) * sizeof(float);
}

// Stage rows y0 .. y0+nrows-1 and the nc chunks of EPC = 16/sizeof(T)
// elements starting at column x0 (a multiple of EPC) of a T image into
// shared rows of stride S elements.  Positions outside the image read the
// clamped position.  vec: rows of src are 16-byte aligned.
template <typename T, int S>
__device__ __forceinline__ void stage_tile(T* dst, const T* __restrict__ src, int ld, int H, int W, int y0,
                                           int nrows, int x0, int nc, bool vec) {
  constexpr int EPC = 16 / (int)sizeof(T);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const int lg = nc <= 1 ? 0 : min(5, 32 - __clz(nc - 1));  // 2^lg chunk slots per row
  const int slots = 1 << lg;
  const int cs = tid & (slots - 1);
  if (vec && x0 >= 0 && x0 + EPC * nc <= W) {
    // the whole window lies inside the image horizontally: 16-byte copies,
    // rows clamped
    for (int r = tid >> lg; r < nrows; r += nth >> lg) {
      const T* srow = src + (size_t)min(max(y0 + r, 0), H - 1) * ld + x0;
      T* drow = dst + r * S;
      for (int c = cs; c < nc; c += slots) cp_async16(drow + EPC * c, srow + EPC * c);
    }
    return;
  }
  for (int r = tid >> lg; r < nrows; r += nth >> lg) {
    const T* srow = src + (size_t)min(max(y0 + r, 0), H - 1) * ld;
    T* drow = dst + r * S;
    for (int c = cs; c < nc; c += slots) {
      const int x = x0 + EPC * c;
      if (vec && x >= 0 && x + EPC <= W) {
        cp_async16(drow + EPC * c, srow + x);
      } else {
#pragma unroll
        for (int k = 0; k < EPC; ++k) {
          if constexpr (sizeof(T) == 4) cp_async4(drow + EPC * c + k, srow + min(max(x + k, 0), W - 1));
          else cp_async8(drow + EPC * c + k, srow + min(max(x + k, 0), W - 1));
        }
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ bool rows_aligned16(const T* p, int ld) {
  return (((uintptr_t)p) & 15) == 0 && ((size_t)ld * sizeof(T)) % 16 == 0;
}

// Ordering hook of the split tiles.  Each tile body first stages what does
// not depend on the preceding launch (tap groups, f, and in the update
// tile u), then calls `dep()`, then stages the data the preceding launch
// wrote.  Under programmatic dependent launch dep() waits for the preceding
// grid; in the batched kernel it is empty.
struct NoDep {
  __device__ void operator()() const {}
};

// q = (e, W) on the TH x TW tile at (i0, j0).  smem_raw: split_smem_q bytes.
template <int TH, int TW, int R, int P, typename Dep = NoDep>
__device__ __forceinline__ void q_tile(unsigned char* smem_raw, const float* __restrict__ f, int ldf,
                                       const float* __restrict__ uin, int ldin,
                                       float2* __restrict__ q, int ldq, int H, int W,
                                       const TapGroup* __restrict__ groups_g,
                                       const int* __restrict__ ngroups_g, int kh, int kw,
                                       int ng_max, const RrlParams& p, int i0, int j0, Dep dep = Dep()) {
  static_assert(TH % R == 0 && TW % 4 == 0, "tile shape");
  const int cy = kh >> 1, cx = kw >> 1;
  const int Ty = kh - 1 - cy, Tx = kw - 1 - cx;  // u rows/cols needed above/left of a pixel
  constexpr int US = TW + P;                      // row stride, P >= kw + 2
  const int UH = TH + kh - 1;
  const int xs = (j0 - Tx) & ~3, ox = (j0 - Tx) - xs;  // staged window starts at column xs
  const int nc = (TW + kw - 1 + ox + 3) >> 2;
  int* cls = (int*)smem_raw;
  float4* gu = (float4*)(smem_raw + 32);
  float* fs = (float*)(gu + 2 * ng_max);  // TH x TW
  float* us = fs + TH * TW;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  stage_groups(cls, gu, groups_g, ngroups_g,
               [&](const TapGroup& t, int m) { return (Ty - t.dy0 - (m - 1)) * US + (Tx + ox - t.dx); });
  stage_tile<float, TW>(fs, f, ldf, H, W, i0, TH, j0, TW / 4, rows_aligned16(f, ldf));
  dep();
  stage_tile<float, US>(us, uin, ldin, H, W, i0 - Ty, UH, xs, nc, rows_aligned16(uin, ldin));
  cp_async_wait_all();
  __syncthreads();
  const bool full = i0 + TH <= H && j0 + TW <= W;
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, c = item - s * TW;
    const int r0 = s * R, j = j0 + c;
    float b[R];
    blur_strip<R, US>(us + r0 * US + c, gu, cls, b);
    float2* qo = q + (size_t)(i0 + r0) * ldq + j;
    if (full) {
#pragma unroll
      for (int r = 0; r < R; ++r) qo[(size_t)r * ldq] = weighted_residual(b[r], fmaxf(fs[(r0 + r) * TW + c], p.floor), p);
    } else if (j < W) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i0 + r0 + r < H) qo[(size_t)r * ldq] = weighted_residual(b[r], fmaxf(fs[(r0 + r) * TW + c], p.floor), p);
    }
  }
}

// Delta, B, D and the update on the TH x TW tile at (i0, j0).
// smem_raw: split_smem_update bytes.
template <int TH, int TW, int R, int P, typename Dep = NoDep>
__device__ __forceinline__ void update_tile(unsigned char* smem_raw, const float2* __restrict__ q, int ldq,
                                            const float* __restrict__ uin, int ldin,
                                            float* __restrict__ uout, int ldout, int H, int W,
                                            const TapGroup* __restrict__ groups_g,
                                            const int* __restrict__ ngroups_g, int kh, int kw,
                                            int ng_max, const RrlParams& p, int* status, int i0, int j0,
                                            Dep dep = Dep()) {
  static_assert(TH % R == 0 && TW % 4 == 0, "tile shape");
  const int cy = kh >> 1, cx = kw >> 1;
  const int QH = TH + kh - 1;
  constexpr int QS = TW + P, UH = TH + 4, US = TW + 8;  // row strides, P >= kw + 2
  const int xq = (j0 - cx) & ~1, oq = (j0 - cx) - xq;    // q window starts at column xq
  const int ncq = (TW + kw - 1 + oq + 1) >> 1;
  int* cls = (int*)smem_raw;
  float4* gq = (float4*)(smem_raw + 32);
  float2* qs = (float2*)(gq + 2 * ng_max);
  float* us = (float*)(qs + QH * QS);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  stage_groups(cls, gq, groups_g, ngroups_g,
               [&](const TapGroup& t, int m) { return (cy + t.dy0) * QS + (cx + oq + t.dx); });
  // u(clamp) with a 2-pixel halo (staged from column j0 - 4 so that every
  // chunk is aligned), then q(clamp) over the correlation footprint
  stage_tile<float, US>(us, uin, ldin, H, W, i0 - 2, UH, j0 - 4, TW / 4 + 2, rows_aligned16(uin, ldin));
  dep();
  stage_tile<float2, QS>(qs, q, ldq, H, W, i0 - cy, QH, xq, ncq, rows_aligned16(q, ldq));
  cp_async_wait_all();
  __syncthreads();
  const bool full = i0 + TH <= H && j0 + TW <= W;
  bool bad = false;
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, oj = item - s * TW;
    const int oi0 = s * R, j = j0 + oj;
    float dl[R], B[R], D[R], c[R];
    correlate_strip<R, QS>(qs + oi0 * QS + oj, gq, cls, dl, B);
    diffusion_strip<R, US>(us + (oi0 + 2) * US + (oj + 4), p, D, c);
    float* uo = uout + (size_t)(i0 + oi0) * ldout + j;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float un = rrl_update(c[r], dl[r], B[r], D[r], p);
      bad |= !isfinite(un);
      if (full || (j < W && i0 + oi0 + r < H)) uo[(size_t)r * ldout] = un;
    }
  }
  if (bad && status) atomicOr(status, DB_FLAG_NONFINITE);
}

}  // namespace db
