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

#include "internal.cuh"

namespace db {

// ---------------------------------------------------------------------------
// tap list: validate the dense taps and keep the non-zero ones (row-major)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_compact_taps(const float* __restrict__ taps, int kh, int kw,
                                                      int kind, Tap* __restrict__ out,
                                                      int* __restrict__ nout, int* status) {
  __shared__ int warp_cnt[8];
  __shared__ float warp_sum[8];
  __shared__ int base;
  __shared__ int bad;
  const int n = kh * kw, cy = kh >> 1, cx = kw >> 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) { base = 0; bad = 0; }
  __syncthreads();
  const float t0 = __ldg(taps);
  float sum = 0.f;
  for (int c0 = 0; c0 < n; c0 += 256) {
    const int k = c0 + threadIdx.x;
    float w = 0.f;
    if (k < n) {
      w = __ldg(taps + k);
      if (!(w >= 0.f) || !isfinite(w)) atomicOr(&bad, DB_FLAG_TAPS);
      if (kind == DB_PSF_BOX && w != t0) atomicOr(&bad, DB_FLAG_BOX);
      sum += w;
    }
    const bool keep = (k < n) && (w != 0.f);
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_cnt[wid] = __popc(m);
    __syncthreads();
    int off = base;
    for (int i = 0; i < wid; ++i) off += warp_cnt[i];
    off += __popc(m & ((1u << lane) - 1u));
    if (keep) {
      Tap t;
      t.w = w;
      t.dy = (int16_t)(k / kw - cy);
      t.dx = (int16_t)(k % kw - cx);
      out[off] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int i = 0; i < 8; ++i) tot += warp_cnt[i];
      base += tot;
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) warp_sum[wid] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < 8; ++i) s += warp_sum[i];
    if (!(s > 0.f)) bad |= DB_FLAG_TAPS;
    *nout = base;
    if (bad && status) atomicOr(status, bad);
  }
}

cudaError_t launch_compact_taps(const float* taps, int kh, int kw, int kind, Tap* out, int* nout,
                                int* status, cudaStream_t s) {
  k_compact_taps<<<1, 256, 0, s>>>(taps, kh, kw, kind, out, nout, status);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pointwise pieces
// ---------------------------------------------------------------------------
// W = phi'(r_f(b)) (Eq. 7, 10) with r_f(b) = f (t - log(1+t)), t = (b - f)/f:
// the same quantity as b - f - f ln(b/f) without its cancellation near b = f.
__device__ __forceinline__ float robust_weight(float b, float f, const RrlParams& p) {
  if (!p.phi_robust) return 1.0f;
  const float t = (b - f) / f;
  const float r = f * (t - log1pf(t));
  return p.eps_phi * rsqrtf(fmaxf(r, 0.0f) + p.eps_phi * p.eps_phi);
}

__device__ __forceinline__ float diffusivity(float gx, float gy, const RrlParams& p) {
  if (!p.psi_tv) return 1.0f;
  return rsqrtf(fmaf(gx, gx, fmaf(gy, gy, p.eps_psi * p.eps_psi)));
}

// ---------------------------------------------------------------------------
// fused iteration
// ---------------------------------------------------------------------------
template <int TH, int TW>
__global__ void __launch_bounds__(256) k_rrl_spatial(const float* __restrict__ f, int ldf,
                                                     const float* __restrict__ uin, int ldin,
                                                     float* __restrict__ uout, int ldout, int H, int W,
                                                     const Tap* __restrict__ taps_g,
                                                     const int* __restrict__ ntaps_g, int kh, int kw,
                                                     RrlParams p, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cy = kh >> 1, cx = kw >> 1;
  const int Ry = max(kh - 1, 2), Rx = max(kw - 1, 2);
  const int US = TW + 2 * Rx;             // u tile row stride
  const int UH = TH + 2 * Ry;
  const int QW = TW + kw - 1, QH = TH + kh - 1;
  const int ntaps = *ntaps_g;
  Tap* taps = (Tap*)smem_raw;
  float* us = (float*)(smem_raw + (size_t)kh * kw * sizeof(Tap));
  float2* qs = (float2*)(us + ((UH * US + 1) & ~1));
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;

  for (int t = threadIdx.x; t < ntaps; t += blockDim.x) taps[t] = taps_g[t];
  // u(clamp) over the halo region
  for (int idx = threadIdx.x; idx < UH * US; idx += blockDim.x) {
    const int r = idx / US, c = idx - r * US;
    const int gi = min(max(i0 - Ry + r, 0), H - 1);
    const int gj = min(max(j0 - Rx + c, 0), W - 1);
    us[idx] = __ldg(uin + (size_t)gi * ldin + gj);
  }
  __syncthreads();

  // q1 = W f / b, q2 = W at clamped positions of the correlation footprint
  for (int idx = threadIdx.x; idx < QH * QW; idx += blockDim.x) {
    const int qr = idx / QW, qc = idx - qr * QW;
    const int ai = min(max(i0 - cy + qr, 0), H - 1);
    const int aj = min(max(j0 - cx + qc, 0), W - 1);
    const float* ub = us + (ai - i0 + Ry) * US + (aj - j0 + Rx);
    float b = 0.f;
    for (int t = 0; t < ntaps; ++t) {
      const Tap tp = taps[t];
      b = fmaf(tp.w, ub[-tp.dy * US - tp.dx], b);
    }
    const float fv = fmaxf(__ldg(f + (size_t)ai * ldf + aj), p.floor);
    const float w = robust_weight(b, fv, p);
    qs[idx] = make_float2(w * fv / b, w);
  }
  __syncthreads();

  // outputs
  for (int idx = threadIdx.x; idx < TH * TW; idx += blockDim.x) {
    const int oi = idx / TW, oj = idx - oi * TW;
    const int i = i0 + oi, j = j0 + oj;
    if (i >= H || j >= W) continue;
    const float2* qb = qs + (oi + cy) * QW + (oj + cx);
    float A = 0.f, B = 0.f;
    for (int t = 0; t < ntaps; ++t) {
      const Tap tp = taps[t];
      const float2 q = qb[tp.dy * QW + tp.dx];
      A = fmaf(tp.w, q.x, A);
      B = fmaf(tp.w, q.y, B);
    }
    // diffusion term on the diamond of radius 2 around (i, j)
    const float* uc = us + (oi + Ry) * US + (oj + Rx);
    const float c = uc[0];
    const float e = uc[1], w_ = uc[-1], n = uc[-US], s = uc[US];
    const float gc = diffusivity(0.5f * (e - w_), 0.5f * (s - n), p);
    const float ge = diffusivity(0.5f * (uc[2] - c), 0.5f * (uc[US + 1] - uc[-US + 1]), p);
    const float gw = diffusivity(0.5f * (c - uc[-2]), 0.5f * (uc[US - 1] - uc[-US - 1]), p);
    const float gs = diffusivity(0.5f * (uc[US + 1] - uc[US - 1]), 0.5f * (uc[2 * US] - c), p);
    const float gn = diffusivity(0.5f * (uc[-US + 1] - uc[-US - 1]), 0.5f * (c - uc[-2 * US]), p);
    const float D = 0.5f * ((ge + gc) * (e - c) - (gc + gw) * (c - w_) + (gs + gc) * (s - c) -
                            (gc + gn) * (c - n));
    const float num = A + p.alpha * fmaxf(D, 0.f);
    const float den = B - p.alpha * fminf(D, 0.f);
    const float un = c * num / den;
    if (!isfinite(un) && status) atomicOr(status, DB_FLAG_NONFINITE);
    uout[(size_t)i * ldout + j] = un;
  }
}

static size_t rrl_smem_bytes(int TH, int TW, int kh, int kw) {
  const int Ry = kh - 1 > 2 ? kh - 1 : 2, Rx = kw - 1 > 2 ? kw - 1 : 2;
  const size_t us = (size_t)((TH + 2 * Ry) * (TW + 2 * Rx) + 1) & ~size_t(1);
  const size_t q = (size_t)(TH + kh - 1) * (TW + kw - 1);
  return (size_t)kh * kw * sizeof(Tap) + us * sizeof(float) + q * sizeof(float2);
}

cudaError_t launch_rrl_spatial(const float* f, int ldf, const float* uin, int ldin, float* uout,
                               int ldout, int H, int W, const Tap* taps, const int* ntaps, int kh,
                               int kw, const RrlParams& p, int* status, cudaStream_t s) {
  constexpr int TH = 32, TW = 64;
  const size_t smem = rrl_smem_bytes(TH, TW, kh, kw);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rrl_spatial<TH, TW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH);
  k_rrl_spatial<TH, TW><<<grid, 256, smem, s>>>(f, ldf, uin, ldin, uout, ldout, H, W, taps, ntaps,
                                                 kh, kw, p, status);
  count_launch();
  return cudaGetLastError();
}

}  // namespace db
