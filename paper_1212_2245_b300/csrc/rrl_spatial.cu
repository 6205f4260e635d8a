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
// tap preparation: validate the dense taps and build the tap groups.
//
// A group is a run of up to M vertically adjacent taps of one PSF column:
// weights w[0..M-1] for offsets (dy0 + k, dx).  Within a column, a group
// starts at the first non-zero tap not yet covered (moved up so that it ends
// inside the PSF) and taps it covers twice get weight 0 in the later group.
// Every non-zero tap lands in exactly one group, with its own weight.
// ---------------------------------------------------------------------------
template <bool WRITE>
__device__ int column_groups(const float* __restrict__ taps, int kh, int kw, int b, int M,
                             TapGroup* out) {
  const int cy = kh >> 1, cx = kw >> 1;
  int covered = -1, n = 0;
  while (true) {
    int s = -1;
    for (int r = covered + 1; r < kh; ++r)
      if (__ldg(taps + r * kw + b) != 0.f) { s = r; break; }
    if (s < 0) break;
    const int st = min(s, kh - M);
    if (WRITE) {
      TapGroup g;
      for (int k = 0; k < 3; ++k) {
        const int r = st + k;
        g.w[k] = (k < M && r > covered && r < kh) ? __ldg(taps + r * kw + b) : 0.f;
      }
      g.dy0 = (int16_t)(st - cy);
      g.dx = (int16_t)(b - cx);
      out[n] = g;
    }
    ++n;
    covered = st + M - 1;
  }
  return n;
}

__global__ void __launch_bounds__(256) k_prepare_taps(const float* __restrict__ taps, int kh, int kw,
                                                      int kind, int M, TapGroup* __restrict__ groups,
                                                      int* __restrict__ ngroups, int* status) {
  __shared__ int scan[256];
  __shared__ float warp_sum[8];
  __shared__ int bad;
  const int n = kh * kw;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const float t0 = __ldg(taps);
  float sum = 0.f;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float w = __ldg(taps + k);
    if (!(w >= 0.f) || !isfinite(w)) atomicOr(&bad, DB_FLAG_TAPS);
    if (kind == DB_PSF_BOX && w != t0) atomicOr(&bad, DB_FLAG_BOX);
    sum += w;
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) warp_sum[wid] = sum;
  // one thread per PSF column (kw <= 255): count, exclusive scan, write
  const int b = threadIdx.x;
  const int cnt = (b < kw) ? column_groups<false>(taps, kh, kw, b, M, nullptr) : 0;
  scan[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const int v = (threadIdx.x >= o) ? scan[threadIdx.x - o] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  if (b < kw) column_groups<true>(taps, kh, kw, b, M, groups + scan[threadIdx.x] - cnt);
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < 8; ++i) s += warp_sum[i];
    if (!(s > 0.f)) bad |= DB_FLAG_TAPS;
    *ngroups = scan[255];
    if (bad && status) atomicOr(status, bad);
  }
}

int tap_group_height(int kh) { return kh < 3 ? kh : 3; }

int max_tap_groups(int kh, int kw) {
  const int M = tap_group_height(kh);
  return kw * ((kh + M - 1) / M);
}

cudaError_t launch_prepare_taps(const float* taps, int kh, int kw, int kind, TapGroup* groups,
                                int* ngroups, int* status, cudaStream_t s) {
  k_prepare_taps<<<1, 256, 0, s>>>(taps, kh, kw, kind, tap_group_height(kh), groups, ngroups, status);
  count_launch();
  return cudaGetLastError();
}

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
// W = phi'(r_f(b)) (Eq. 7, 10) with r_f(b) = f (t - log(1+t)), t = (b - f)/f:
// the same quantity as b - f - f ln(b/f) without its cancellation near b = f.
__device__ __forceinline__ float robust_weight(float b, float f, const RrlParams& p) {
  if (!p.phi_robust) return 1.0f;
  const float t = __fdividef(b - f, f);
  const float r = f * (t - log1pf(t));
  return p.eps_phi * rsqrtf(fmaxf(r, 0.0f) + p.eps_phi * p.eps_phi);
}

// (e, W) for one pixel: W = phi'(r_f(b)), e = W (f - b)/b.
__device__ __forceinline__ float2 weighted_residual(float b, float f, const RrlParams& p) {
  const float w = robust_weight(b, f, p);
  return make_float2(__fdividef(w * (f - b), b), w);
}

__device__ __forceinline__ float diffusivity(float gx, float gy, const RrlParams& p) {
  if (!p.psi_tv) return 1.0f;
  return rsqrtf(fmaf(gx, gx, fmaf(gy, gy, p.eps_psi * p.eps_psi)));
}

// b[r] = (u*h) at R vertically adjacent pixels.  `base` points at the u
// value that the first pixel's strip starts from; each group record holds
// three weights and the shared-memory offset of its first load.
template <int R, int M, int STRIDE>
__device__ __forceinline__ void blur_strip(const float* __restrict__ base,
                                           const float4* __restrict__ grp, int ng, float (&b)[R]) {
  constexpr int stride = STRIDE;
#pragma unroll
  for (int r = 0; r < R; ++r) b[r] = 0.f;
#pragma unroll 2
  for (int g = 0; g < ng; ++g) {
    const float4 G = grp[g];
    const float* pu = base + __float_as_int(G.w);
    float v[R + M - 1];
#pragma unroll
    for (int t = 0; t < R + M - 1; ++t) v[t] = pu[t * stride];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      b[r] = fmaf(G.x, v[r + M - 1], b[r]);
      if (M > 1) b[r] = fmaf(G.y, v[r + M - 2], b[r]);
      if (M > 2) b[r] = fmaf(G.z, v[r + M - 3], b[r]);
    }
  }
}

// Delta[r] = (e*h*), B[r] = (W*h*) at R vertically adjacent pixels.
template <int R, int M, int STRIDE>
__device__ __forceinline__ void correlate_strip(const float2* __restrict__ base,
                                                const float4* __restrict__ grp, int ng, float (&dl)[R],
                                                float (&B)[R]) {
  constexpr int stride = STRIDE;
#pragma unroll
  for (int r = 0; r < R; ++r) { dl[r] = 0.f; B[r] = 0.f; }
#pragma unroll 2
  for (int g = 0; g < ng; ++g) {
    const float4 G = grp[g];
    const float2* pq = base + __float_as_int(G.w);
    float2 v[R + M - 1];
#pragma unroll
    for (int t = 0; t < R + M - 1; ++t) v[t] = pq[t * stride];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      dl[r] = fmaf(G.x, v[r].x, dl[r]);
      B[r] = fmaf(G.x, v[r].y, B[r]);
      if (M > 1) { dl[r] = fmaf(G.y, v[r + 1].x, dl[r]); B[r] = fmaf(G.y, v[r + 1].y, B[r]); }
      if (M > 2) { dl[r] = fmaf(G.z, v[r + 2].x, dl[r]); B[r] = fmaf(G.z, v[r + 2].y, B[r]); }
    }
  }
}

// Diffusion term D = div(psi'(|grad u|^2) grad u) (Eq. 11) at R vertically
// adjacent pixels.  uc points at the first pixel in a shared-memory copy of
// u(clamp(.)) with at least 2 pixels of halo on every side.  Diffusivities
// and vertical fluxes shared by neighbouring rows of the strip are formed
// once.  Across the image boundary the clamped copy makes every difference
// vanish exactly: zero flux.
template <int R, int S>
__device__ __forceinline__ void diffusion_strip(const float* __restrict__ uc, const RrlParams& p,
                                                float (&D)[R], float (&c)[R]) {
  float m[R + 4], e1[R + 2], w1[R + 2];
#pragma unroll
  for (int t = 0; t < R + 4; ++t) m[t] = uc[(t - 2) * S];
#pragma unroll
  for (int t = 0; t < R + 2; ++t) { e1[t] = uc[(t - 1) * S + 1]; w1[t] = uc[(t - 1) * S - 1]; }
  float gC[R + 2];
#pragma unroll
  for (int t = 0; t < R + 2; ++t)  // rows -1..R
    gC[t] = diffusivity(0.5f * (e1[t] - w1[t]), 0.5f * (m[t + 2] - m[t]), p);
  float Fv[R + 1];
#pragma unroll
  for (int t = 0; t < R + 1; ++t)  // flux between rows t-1 and t
    Fv[t] = 0.5f * (gC[t + 1] + gC[t]) * (m[t + 2] - m[t + 1]);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float e2 = uc[r * S + 2], w2 = uc[r * S - 2];
    const float ctr = m[r + 2];
    const float gE = diffusivity(0.5f * (e2 - ctr), 0.5f * (e1[r + 2] - e1[r]), p);
    const float gW = diffusivity(0.5f * (ctr - w2), 0.5f * (w1[r + 2] - w1[r]), p);
    const float fe = 0.5f * (gE + gC[r + 1]) * (e1[r + 1] - ctr);
    const float fw = 0.5f * (gC[r + 1] + gW) * (ctr - w1[r + 1]);
    D[r] = (fe - fw) + (Fv[r + 1] - Fv[r]);
    c[r] = ctr;
  }
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
// (phase 2) in one column, so a tap group loaded once from shared memory
// feeds M*R (phase 1) or 2*M*R (phase 2) FMAs from R+M-1 shared loads.
// Lanes of a warp own adjacent columns: shared accesses are conflict-free.
//
// Geometry (virtual rows/cols may lie outside the image):
//   q tile : rows i0-cy .. i0-cy+QHp-1, cols j0-cx .. j0-cx+QW-1
//   u tile : rows i0-Ry .. i0-Ry+UH-1,  cols j0-Rx .. j0-Rx+US-1
// u is staged as u(clamp(.)); q = (e, W) is first formed at every virtual
// position from the clamped u and then, at virtual positions outside the
// image, replaced by q at the clamped position.
// ---------------------------------------------------------------------------
template <int TH, int TW, int R, int M, int P>
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
  const int ng = *ngroups_g;
  float4* gu = (float4*)smem_raw;
  float4* gq = gu + ng_max;
  float* us = (float*)(gq + ng_max);
  float2* qs = (float2*)(us + ((UH * US + 1) & ~1));
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;

  for (int g = tid; g < ng; g += nth) {
    const TapGroup t = groups_g[g];
    const int offu = (Ry - cy - t.dy0 - (M - 1)) * US + (Rx - cx - t.dx);
    const int offq = (cy + t.dy0) * QS + (cx + t.dx);
    gu[g] = make_float4(t.w[0], t.w[1], t.w[2], __int_as_float(offu));
    gq[g] = make_float4(t.w[0], t.w[1], t.w[2], __int_as_float(offq));
  }
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
    blur_strip<R, M, US>(us + qr0 * US + qc, gu, ng, b);
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
    correlate_strip<R, M, QS>(qs + oi0 * QS + oj, gq, ng, dl, B);
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
// ---------------------------------------------------------------------------
template <int TH, int TW, int R, int M, int P>
__global__ void __launch_bounds__(256, 4) k_rrl_q(const float* __restrict__ f, int ldf,
                                               const float* __restrict__ uin, int ldin,
                                               float2* __restrict__ q, int ldq, int H, int W,
                                               const TapGroup* __restrict__ groups_g,
                                               const int* __restrict__ ngroups_g, int kh, int kw,
                                               int ng_max, RrlParams p) {
  static_assert(TH % R == 0, "strips must tile TH");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cy = kh >> 1, cx = kw >> 1;
  const int Ty = kh - 1 - cy, Tx = kw - 1 - cx;  // u rows/cols needed above/left of a pixel
  constexpr int US = TW + P;                      // row stride, P >= kw - 1
  const int UH = TH + kh - 1, UW = TW + kw - 1;
  const int ng = *ngroups_g;
  float4* gu = (float4*)smem_raw;
  float* us = (float*)(gu + ng_max);
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  for (int g = tid; g < ng; g += nth) {
    const TapGroup t = groups_g[g];
    const int offu = (Ty - t.dy0 - (M - 1)) * US + (Tx - t.dx);
    gu[g] = make_float4(t.w[0], t.w[1], t.w[2], __int_as_float(offu));
  }
  for (int r = threadIdx.y; r < UH; r += blockDim.y) {
    const int gi = min(max(i0 - Ty + r, 0), H - 1);
    const float* src = uin + (size_t)gi * ldin;
    for (int c = threadIdx.x; c < UW; c += blockDim.x)
      cp_async4(us + r * US + c, src + min(max(j0 - Tx + c, 0), W - 1));
  }
  cp_async_wait_all();
  __syncthreads();
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, c = item - s * TW;
    const int r0 = s * R, j = j0 + c;
    if (j >= W || i0 + r0 >= H) continue;
    float fv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = min(i0 + r0 + r, H - 1);
      fv[r] = fmaxf(__ldg(f + (size_t)i * ldf + j), p.floor);
    }
    float b[R];
    blur_strip<R, M, US>(us + r0 * US + c, gu, ng, b);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r0 + r;
      if (i < H) q[(size_t)i * ldq + j] = weighted_residual(b[r], fv[r], p);
    }
  }
}

template <int TH, int TW, int R, int M, int P>
__global__ void __launch_bounds__(256, 4) k_rrl_update(const float2* __restrict__ q, int ldq,
                                                    const float* __restrict__ uin, int ldin,
                                                    float* __restrict__ uout, int ldout, int H, int W,
                                                    const TapGroup* __restrict__ groups_g,
                                                    const int* __restrict__ ngroups_g, int kh, int kw,
                                                    int ng_max, RrlParams p, int* status) {
  static_assert(TH % R == 0, "strips must tile TH");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cy = kh >> 1, cx = kw >> 1;
  const int QH = TH + kh - 1, QW = TW + kw - 1;
  constexpr int QS = TW + P, UH = TH + 4, US = TW + 4;  // row strides, P >= kw - 1
  const int ng = *ngroups_g;
  float4* gq = (float4*)smem_raw;
  float2* qs = (float2*)(gq + ng_max);
  float* us = (float*)(qs + QH * QS);
  const int i0 = blockIdx.y * TH, j0 = blockIdx.x * TW;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  for (int g = tid; g < ng; g += nth) {
    const TapGroup t = groups_g[g];
    const int offq = (cy + t.dy0) * QS + (cx + t.dx);
    gq[g] = make_float4(t.w[0], t.w[1], t.w[2], __int_as_float(offq));
  }
  // q(clamp) over the correlation footprint, u(clamp) with a 2-pixel halo
  for (int r = threadIdx.y; r < QH; r += blockDim.y) {
    const int gi = min(max(i0 - cy + r, 0), H - 1);
    const float2* src = q + (size_t)gi * ldq;
    for (int c = threadIdx.x; c < QW; c += blockDim.x)
      cp_async8(qs + r * QS + c, src + min(max(j0 - cx + c, 0), W - 1));
  }
  for (int r = threadIdx.y; r < UH; r += blockDim.y) {
    const int gi = min(max(i0 - 2 + r, 0), H - 1);
    const float* src = uin + (size_t)gi * ldin;
    for (int c = threadIdx.x; c < US; c += blockDim.x)
      cp_async4(us + r * US + c, src + min(max(j0 - 2 + c, 0), W - 1));
  }
  cp_async_wait_all();
  __syncthreads();
  for (int item = tid; item < (TH / R) * TW; item += nth) {
    const int s = item / TW, oj = item - s * TW;
    const int oi0 = s * R, j = j0 + oj;
    if (j >= W || i0 + oi0 >= H) continue;
    float dl[R], B[R], D[R], c[R];
    correlate_strip<R, M, QS>(qs + oi0 * QS + oj, gq, ng, dl, B);
    diffusion_strip<R, US>(us + (oi0 + 2) * US + (oj + 2), p, D, c);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + oi0 + r;
      const float un = rrl_update(c[r], dl[r], B[r], D[r], p);
      if (i < H) {
        if (!isfinite(un) && status) atomicOr(status, DB_FLAG_NONFINITE);
        uout[(size_t)i * ldout + j] = un;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side: shared-memory sizes and launches.  The halo class P is the
// smallest of 8, 16, 32, 64, 128, 256 that holds kw - 1 (and 2).
// ---------------------------------------------------------------------------
constexpr int kTH = 64, kTW = 64, kR = 8;        // fused tiles
constexpr int kQTH = 32, kQTW = 64;              // split: q tiles
constexpr int kUTH = 32, kUTW = 64;              // split: update tiles

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
  return (size_t)2 * ng_max * sizeof(float4) + us * sizeof(float) + (size_t)QHp * (kTW + P) * sizeof(float2);
}
size_t rrl_split_smem_q(int kh, int kw) {
  return (size_t)max_tap_groups(kh, kw) * sizeof(float4) +
         (size_t)(kQTH + kh - 1) * (kQTW + halo_class(kw)) * sizeof(float);
}
size_t rrl_split_smem_update(int kh, int kw) {
  return (size_t)max_tap_groups(kh, kw) * sizeof(float4) +
         (size_t)(kUTH + kh - 1) * (kUTW + halo_class(kw)) * sizeof(float2) +
         (size_t)(kUTH + 4) * (kUTW + 4) * sizeof(float);
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
};

template <int M, int P>
static cudaError_t launch_fused_mp(const IterArgs& a, cudaStream_t s) {
  const int ng_max = max_tap_groups(a.kh, a.kw);
  const size_t smem = rrl_spatial_smem(a.kh, a.kw);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  auto kern = k_rrl_spatial<kTH, kTW, kR, M, P>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3((a.W + kTW - 1) / kTW, (a.H + kTH - 1) / kTH), dim3(64, 4), smem, s>>>(
      a.f, a.ldf, a.uin, a.ldin, a.uout, a.ldout, a.H, a.W, a.groups, a.ngroups, a.kh, a.kw, ng_max,
      a.p, a.status);
  count_launch();
  return cudaGetLastError();
}

template <int M, int P>
static cudaError_t launch_split_mp(const IterArgs& a, cudaStream_t s) {
  const int ng_max = max_tap_groups(a.kh, a.kw);
  const size_t sq = rrl_split_smem_q(a.kh, a.kw), su = rrl_split_smem_update(a.kh, a.kw);
  if (sq > 227 * 1024 || su > 227 * 1024) return cudaErrorInvalidValue;
  auto kq = k_rrl_q<kQTH, kQTW, kR, M, P>;
  auto ku = k_rrl_update<kUTH, kUTW, kR, M, P>;
  cudaError_t e;
  if ((e = set_smem(kq, sq)) != cudaSuccess) return e;
  if ((e = set_smem(ku, su)) != cudaSuccess) return e;
  kq<<<dim3((a.W + kQTW - 1) / kQTW, (a.H + kQTH - 1) / kQTH), dim3(64, 4), sq, s>>>(
      a.f, a.ldf, a.uin, a.ldin, a.q, a.W, a.H, a.W, a.groups, a.ngroups, a.kh, a.kw, ng_max, a.p);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ku<<<dim3((a.W + kUTW - 1) / kUTW, (a.H + kUTH - 1) / kUTH), dim3(64, 4), su, s>>>(
      a.q, a.W, a.uin, a.ldin, a.uout, a.ldout, a.H, a.W, a.groups, a.ngroups, a.kh, a.kw, ng_max,
      a.p, a.status);
  count_launch();
  return cudaGetLastError();
}

template <bool SPLIT, int M>
static cudaError_t dispatch_p(const IterArgs& a, cudaStream_t s) {
  switch (halo_class(a.kw)) {
    case 8: return SPLIT ? launch_split_mp<M, 8>(a, s) : launch_fused_mp<M, 8>(a, s);
    case 16: return SPLIT ? launch_split_mp<M, 16>(a, s) : launch_fused_mp<M, 16>(a, s);
    case 32: return SPLIT ? launch_split_mp<M, 32>(a, s) : launch_fused_mp<M, 32>(a, s);
    case 64: return SPLIT ? launch_split_mp<M, 64>(a, s) : launch_fused_mp<M, 64>(a, s);
    case 128: return SPLIT ? launch_split_mp<M, 128>(a, s) : launch_fused_mp<M, 128>(a, s);
    default: return SPLIT ? launch_split_mp<M, 256>(a, s) : launch_fused_mp<M, 256>(a, s);
  }
}

template <bool SPLIT>
static cudaError_t dispatch(const IterArgs& a, cudaStream_t s) {
  switch (tap_group_height(a.kh)) {
    case 1: return dispatch_p<SPLIT, 1>(a, s);
    case 2: return dispatch_p<SPLIT, 2>(a, s);
    default: return dispatch_p<SPLIT, 3>(a, s);
  }
}

cudaError_t launch_rrl_spatial(const float* f, int ldf, const float* uin, int ldin, float* uout,
                               int ldout, int H, int W, const TapGroup* groups, const int* ngroups,
                               int kh, int kw, const RrlParams& p, int* status, cudaStream_t s) {
  const IterArgs a = {f, ldf, uin, ldin, uout, ldout, nullptr, H, W, groups, ngroups, kh, kw, p, status};
  return dispatch<false>(a, s);
}

cudaError_t launch_rrl_split(const float* f, int ldf, const float* uin, int ldin, float* uout,
                             int ldout, float2* q, int H, int W, const TapGroup* groups,
                             const int* ngroups, int kh, int kw, const RrlParams& p, int* status,
                             cudaStream_t s) {
  const IterArgs a = {f, ldf, uin, ldin, uout, ldout, q, H, W, groups, ngroups, kh, kw, p, status};
  return dispatch<true>(a, s);
}

}  // namespace db
