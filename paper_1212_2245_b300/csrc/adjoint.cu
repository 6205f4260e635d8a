// Reverse mode (adjoint) of the WR3L chain for gradient-based tuning of the
// PSF taps, alpha and K (no counterpart in the paper; it differentiates the
// operators of Sec. 2.1, Eq. 2 and Sec. 2.3, Eq. 7-12 as evaluated here).
//
// Forward step (spatial mode, constant continuation), per pixel:
//   b = C u,  r = r_f(b),  W = phi'(r),  q1 = W f/b,  q2 = W,
//   A = C' q1,  B = C' q2,  D = div(psi'(|grad u|^2) grad u),
//   u' = u (A + alpha [D]+) / (B - alpha [D]-)
// with C the clamped convolution and C' the clamped correlation.  Neither is
// the transpose of the other at the image border, so the reverse step uses
// the exact transposes: (C^T y)(j) = sum_d h(d) sum_{i: clip(i-d) = j} y(i)
// and (C'^T z)(j) = sum_d h(d) sum_{i: clip(i+d) = j} z(i); at border pixels
// the inner sums run over a range of i.
//
// Reverse step, given the adjoint U' of u':
//   num = A + alpha[D]+, den = B - alpha[D]-
//   U   = U' num/den              Abar = U' u/den      Bbar = -U' u num/den^2
//   Dbar = alpha (Abar 1[D>0] - Bbar 1[D<0]);  alpha_bar += Abar [D]+ - Bbar [D]-
//   q1bar = C'^T Abar,  q2bar = C'^T Bbar
//   Wbar = q1bar f/b + q2bar;  rbar = Wbar phi''(r)
//   bbar = -q1bar W f/b^2 + rbar (1 - f/b);  fbar += q1bar W/b - rbar ln(b/f)
//   U  += C^T bbar + (diffusion adjoint of Dbar)
//   hbar(d) += sum_i Abar(i) q1(clip(i+d)) + Bbar(i) q2(clip(i+d)) + bbar(i) u(clip(i-d))
// Derivative conventions at kinks: d[z]+/dz = 1[z>0], d[z]-/dz = 1[z<0],
// d max(z, delta)/dz = 1[z>delta].
//
// Reductions (alpha, taps, K) are two-level and deterministic: per-CTA
// partial sums in fixed order, then one CTA sums the partials in double.
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "fft_df.cuh"
#include "internal.cuh"

namespace db {

constexpr int kAdjThreads = 256;
constexpr int kAdjMaxTaps = 1024;  // kh * kw limit of the reverse pass

struct AdjImage {
  int N, H, W;     // N images of H x W, packed (pitch W, image stride H*W) internally
  const float* taps; int kh, kw;
  RrlParams p;
};

// Pixel loop over all N images, row by row (rows of all images packed, one
// CTA per row, grid-stride; threads across the row): idx is the packed pixel
// index; ADJ_DECOMPOSE gives the image offset `o`, row i and column j.
#define ADJ_PIXELS(im)                                                                        \
  for (int R_ = blockIdx.x; R_ < (im).N * (im).H; R_ += gridDim.x)                            \
    for (int j_ = threadIdx.x, idx = R_ * (im).W + j_; j_ < (im).W; j_ += blockDim.x, idx += blockDim.x)
#define ADJ_DECOMPOSE(im)                                    \
  const int img_ = R_ / (im).H;                              \
  const int o = img_ * (im).H * (im).W;                      \
  const int i = R_ - img_ * (im).H, j = j_;

// ---------------------------------------------------------------------------
// forward recompute of the intermediates of one iteration
// ---------------------------------------------------------------------------
__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

__device__ __forceinline__ float phi_w(float b, float f, const RrlParams& p, float* r_out) {
  const float t = (b - f) / f;
  const float r = fmaxf(f * (t - log1pf(t)), 0.f);
  *r_out = r;
  if (!p.phi_robust) return 1.0f;
  return p.eps_phi * rsqrtf(r + p.eps_phi * p.eps_phi);
}

// b = C u and q = (W f/b, W)
__global__ void k_adj_fwd_q(const float* __restrict__ u, const float* __restrict__ f0, AdjImage im,
                            float* __restrict__ b_out, float2* __restrict__ q_out) {
  __shared__ float taps[kAdjMaxTaps];
  const int nt = im.kh * im.kw, cy = im.kh >> 1, cx = im.kw >> 1;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) taps[t] = im.taps[t];
  __syncthreads();
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    float b = 0.f;
    for (int a = 0; a < im.kh; ++a) {
      const int ii = clampi(i - (a - cy), im.H);
      for (int c = 0; c < im.kw; ++c) {
        const float w = taps[a * im.kw + c];
        if (w != 0.f) b = fmaf(w, u[o + ii * im.W + clampi(j - (c - cx), im.W)], b);
      }
    }
    const float fv = f0[idx];
    float r;
    const float w = phi_w(b, fv, im.p, &r);
    b_out[idx] = b;
    q_out[idx] = make_float2(w * fv / b, w);
  }
}

__device__ __forceinline__ float psi_g(float gx, float gy, const RrlParams& p) {
  if (!p.psi_tv) return 1.0f;
  return rsqrtf(fmaf(gx, gx, fmaf(gy, gy, p.eps_psi * p.eps_psi)));
}

// A, B = C' q;  g = psi'(|grad u|^2);  D = div(g grad u)  (zero flux)
__global__ void k_adj_fwd_ab(const float* __restrict__ u, const float2* __restrict__ q, AdjImage im,
                             float2* __restrict__ ab_out, float* __restrict__ g_out) {
  __shared__ float taps[kAdjMaxTaps];
  const int nt = im.kh * im.kw, cy = im.kh >> 1, cx = im.kw >> 1;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) taps[t] = im.taps[t];
  __syncthreads();
  const int W = im.W, H = im.H;
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    float A = 0.f, B = 0.f;
    for (int a = 0; a < im.kh; ++a) {
      const int ii = clampi(i + (a - cy), H);
      for (int c = 0; c < im.kw; ++c) {
        const float w = taps[a * im.kw + c];
        if (w != 0.f) {
          const float2 v = q[o + ii * W + clampi(j + (c - cx), W)];
          A = fmaf(w, v.x, A);
          B = fmaf(w, v.y, B);
        }
      }
    }
    ab_out[idx] = make_float2(A, B);
    const float gx = 0.5f * (u[o + i * W + clampi(j + 1, W)] - u[o + i * W + clampi(j - 1, W)]);
    const float gy = 0.5f * (u[o + clampi(i + 1, H) * W + j] - u[o + clampi(i - 1, H) * W + j]);
    g_out[idx] = psi_g(gx, gy, im.p);
  }
}

// D from u and g (in-image neighbours only: zero flux across the border);
// u and g point at the image's first pixel.
__device__ __forceinline__ float diffusion_at(const float* u, const float* g, int i, int j, int H, int W) {
  const int p = i * W + j;
  const float up = u[p], gp = g[p];
  float D = 0.f;
  if (j + 1 < W) D += 0.5f * (g[p + 1] + gp) * (u[p + 1] - up);
  if (j > 0) D += 0.5f * (g[p - 1] + gp) * (u[p - 1] - up);
  if (i + 1 < H) D += 0.5f * (g[p + W] + gp) * (u[p + W] - up);
  if (i > 0) D += 0.5f * (g[p - W] + gp) * (u[p - W] - up);
  return D;
}

// Forward step output (used to rebuild checkpoint segments).  A CTA takes
// kFuRows rows of one image and a thread one column of them: the loads of
// u, g and (A, B) for the column go out together and the rows share them
// (D as diffusion_at forms it).
constexpr int kFuRows = 8;
__global__ void __launch_bounds__(kAdjThreads) k_adj_fwd_update(const float* __restrict__ u,
                                                                const float2* __restrict__ ab,
                                                                const float* __restrict__ g, AdjImage im,
                                                                float* __restrict__ u_out) {
  const int H = im.H, W = im.W;
  const int nblk = (H + kFuRows - 1) / kFuRows;
  for (int blk = blockIdx.x; blk < im.N * nblk; blk += gridDim.x) {
    const int n = blk / nblk, i0 = (blk - n * nblk) * kFuRows, i1 = min(i0 + kFuRows, H);
    const size_t o = (size_t)n * H * W;
    const float* ui = u + o;
    const float* gi = g + o;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
      const int jw = clampi(j - 1, W), je = clampi(j + 1, W);
      float Uc[kFuRows + 2], Gc[kFuRows + 2], Uw[kFuRows], Ue[kFuRows], Gw[kFuRows], Ge[kFuRows];
      float2 abv[kFuRows];
#pragma unroll
      for (int t = 0; t < kFuRows + 2; ++t) {
        const size_t row = (size_t)clampi(i0 - 1 + t, H) * W;
        Uc[t] = ui[row + j];
        Gc[t] = gi[row + j];
      }
#pragma unroll
      for (int r = 0; r < kFuRows; ++r) {
        const size_t row = (size_t)min(i0 + r, H - 1) * W;
        Uw[r] = ui[row + jw]; Ue[r] = ui[row + je];
        Gw[r] = gi[row + jw]; Ge[r] = gi[row + je];
        abv[r] = ab[o + row + j];
      }
#pragma unroll
      for (int r = 0; r < kFuRows; ++r) {
        const int i = i0 + r;
        if (i >= i1) continue;
        const float up = Uc[r + 1], gp = Gc[r + 1];
        float D = 0.f;
        if (j + 1 < W) D += 0.5f * (Ge[r] + gp) * (Ue[r] - up);
        if (j > 0) D += 0.5f * (Gw[r] + gp) * (Uw[r] - up);
        if (i + 1 < H) D += 0.5f * (Gc[r + 2] + gp) * (Uc[r + 2] - up);
        if (i > 0) D += 0.5f * (Gc[r] + gp) * (Uc[r] - up);
        const float2 v = abv[r];
        const float num = v.x + im.p.alpha * fmaxf(D, 0.f);
        const float den = v.y - im.p.alpha * fminf(D, 0.f);
        u_out[o + (size_t)i * W + j] = up * num / den;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// reverse step
// ---------------------------------------------------------------------------
__device__ void block_reduce_add(float* partial_out, float v) {
  __shared__ float red[kAdjThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < kAdjThreads / 32; ++k) s += red[k];
    *partial_out = s;
  }
  __syncthreads();
}

// U = U' num/den; Abar, Bbar; Dbar; partial alpha_bar per CTA
__global__ void __launch_bounds__(kAdjThreads) k_adj_rev_update(
    const float* __restrict__ Ubar_next, const float* __restrict__ u, const float2* __restrict__ ab,
    const float* __restrict__ g, AdjImage im, float* __restrict__ Uacc, float2* __restrict__ abbar,
    float* __restrict__ Dbar, float* __restrict__ alpha_partial) {
  float asum = 0.f;
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    const float D = diffusion_at(u + o, g + o, i, j, im.H, im.W);
    const float2 v = ab[idx];
    const float Dp = fmaxf(D, 0.f), Dm = fminf(D, 0.f);
    const float num = v.x + im.p.alpha * Dp;
    const float den = v.y - im.p.alpha * Dm;
    const float ub = Ubar_next[idx], uu = u[idx];
    const float Ab = ub * uu / den;
    const float Bb = -ub * uu * num / (den * den);
    Uacc[idx] = ub * num / den;
    abbar[idx] = make_float2(Ab, Bb);
    Dbar[idx] = im.p.alpha * ((D > 0.f ? Ab : 0.f) - (D < 0.f ? Bb : 0.f));
    asum += Ab * Dp - Bb * Dm;
  }
  block_reduce_add(alpha_partial + blockIdx.x, asum);
}

// Index range {i in [0,n): clip(i + s) == j} for shift s (s = +d for the
// correlation transpose, s = -d for the convolution transpose).
__device__ __forceinline__ void preimage(int j, int s, int n, int* lo, int* hi) {
  if (n == 1) { *lo = 0; *hi = 0; return; }
  if (j == 0) { *lo = 0; *hi = min(-s, n - 1); return; }              // i + s <= 0
  if (j == n - 1) { *lo = max(n - 1 - s, 0); *hi = n - 1; return; }   // i + s >= n-1
  const int i = j - s;
  *lo = i; *hi = (i >= 0 && i < n) ? i : i - 1;                        // empty if out of range
}

// qbar = C'^T (Abar, Bbar);  tap partials of Abar q1(clip(i+d)) + Bbar q2(clip(i+d)).
// Tap sums: for at most kAdjRegTaps taps each thread keeps one partial per
// tap in registers over its pixels (one pass); otherwise one pass per tap.
constexpr int kAdjRegTaps = 32;

__global__ void __launch_bounds__(kAdjThreads) k_adj_rev_corrT(const float2* __restrict__ abbar,
                                                                const float2* __restrict__ q, AdjImage im,
                                                                float2* __restrict__ qbar,
                                                                float* __restrict__ tap_partial) {
  __shared__ float taps[kAdjMaxTaps];
  const int nt = im.kh * im.kw, cy = im.kh >> 1, cx = im.kw >> 1;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) taps[t] = im.taps[t];
  __syncthreads();
  const int H = im.H, W = im.W;
  float acc[kAdjRegTaps];
#pragma unroll
  for (int t = 0; t < kAdjRegTaps; ++t) acc[t] = 0.f;
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    float s1 = 0.f, s2 = 0.f;
    for (int a = 0; a < im.kh; ++a) {
      int ilo, ihi;
      preimage(i, a - cy, H, &ilo, &ihi);
      for (int c = 0; c < im.kw; ++c) {
        const float w = taps[a * im.kw + c];
        int jlo, jhi;
        preimage(j, c - cx, W, &jlo, &jhi);
        float z1 = 0.f, z2 = 0.f;
        for (int ii = ilo; ii <= ihi; ++ii)
          for (int jj = jlo; jj <= jhi; ++jj) {
            const float2 v = abbar[o + ii * W + jj];
            z1 += v.x;
            z2 += v.y;
          }
        s1 = fmaf(w, z1, s1);
        s2 = fmaf(w, z2, s2);
      }
    }
    qbar[idx] = make_float2(s1, s2);
    if (nt <= kAdjRegTaps) {
      const float2 v = abbar[idx];
#pragma unroll
      for (int t = 0; t < kAdjRegTaps; ++t) {
        if (t < nt) {
          const float2 qq = q[o + clampi(i + t / im.kw - cy, H) * W + clampi(j + t % im.kw - cx, W)];
          acc[t] = fmaf(v.x, qq.x, fmaf(v.y, qq.y, acc[t]));
        }
      }
    }
  }
  if (nt <= kAdjRegTaps) {
    for (int t = 0; t < nt; ++t) block_reduce_add(tap_partial + (size_t)t * gridDim.x + blockIdx.x, acc[t]);
    return;
  }
  for (int t = 0; t < nt; ++t) {
    const int dy = t / im.kw - cy, dx = t % im.kw - cx;
    float a2 = 0.f;
    ADJ_PIXELS(im) {
      ADJ_DECOMPOSE(im)
      const float2 v = abbar[idx];
      const float2 qq = q[o + clampi(i + dy, H) * W + clampi(j + dx, W)];
      a2 = fmaf(v.x, qq.x, fmaf(v.y, qq.y, a2));
    }
    block_reduce_add(tap_partial + (size_t)t * gridDim.x + blockIdx.x, a2);
  }
}

// bbar and the f0 contribution from qbar
__global__ void k_adj_rev_weight(const float2* __restrict__ qbar, const float* __restrict__ b,
                                 const float* __restrict__ f0, AdjImage im, float* __restrict__ bbar,
                                 float* __restrict__ f0bar) {
  ADJ_PIXELS(im) {
    const float bv = b[idx], fv = f0[idx];
    float r;
    const float w = phi_w(bv, fv, im.p, &r);
    const float2 qb = qbar[idx];
    const float Wbar = qb.x * fv / bv + qb.y;
    // phi''(r) = -phi'(r)^3 / (2 eps^2) for the regularised L1 penaliser
    const float rbar = im.p.phi_robust ? Wbar * (-w * w * w / (2.f * im.p.eps_phi * im.p.eps_phi)) : 0.f;
    bbar[idx] = -qb.x * w * fv / (bv * bv) + rbar * (1.f - fv / bv);
    f0bar[idx] += qb.x * w / bv - rbar * logf(bv / fv);
  }
}

// U += C^T bbar;  tap partials of bbar(i) u(clip(i-d))
__global__ void __launch_bounds__(kAdjThreads) k_adj_rev_convT(const float* __restrict__ bbar,
                                                                const float* __restrict__ u, AdjImage im,
                                                                float* __restrict__ Uacc,
                                                                float* __restrict__ tap_partial) {
  __shared__ float taps[kAdjMaxTaps];
  const int nt = im.kh * im.kw, cy = im.kh >> 1, cx = im.kw >> 1;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) taps[t] = im.taps[t];
  __syncthreads();
  const int H = im.H, W = im.W;
  float acc[kAdjRegTaps];
#pragma unroll
  for (int t = 0; t < kAdjRegTaps; ++t) acc[t] = 0.f;
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    float s = 0.f;
    for (int a = 0; a < im.kh; ++a) {
      int ilo, ihi;
      preimage(i, -(a - cy), H, &ilo, &ihi);
      for (int c = 0; c < im.kw; ++c) {
        const float w = taps[a * im.kw + c];
        int jlo, jhi;
        preimage(j, -(c - cx), W, &jlo, &jhi);
        float z = 0.f;
        for (int ii = ilo; ii <= ihi; ++ii)
          for (int jj = jlo; jj <= jhi; ++jj) z += bbar[o + ii * W + jj];
        s = fmaf(w, z, s);
      }
    }
    Uacc[idx] += s;
    if (nt <= kAdjRegTaps) {
      const float bv = bbar[idx];
#pragma unroll
      for (int t = 0; t < kAdjRegTaps; ++t) {
        if (t < nt) acc[t] = fmaf(bv, u[o + clampi(i - (t / im.kw - cy), H) * W + clampi(j - (t % im.kw - cx), W)], acc[t]);
      }
    }
  }
  if (nt <= kAdjRegTaps) {
    for (int t = 0; t < nt; ++t) block_reduce_add(tap_partial + (size_t)t * gridDim.x + blockIdx.x, acc[t]);
    return;
  }
  for (int t = 0; t < nt; ++t) {
    const int dy = t / im.kw - cy, dx = t % im.kw - cx;
    float a2 = 0.f;
    ADJ_PIXELS(im) {
      ADJ_DECOMPOSE(im)
      a2 = fmaf(bbar[idx], u[o + clampi(i - dy, H) * W + clampi(j - dx, W)], a2);
    }
    block_reduce_add(tap_partial + (size_t)t * gridDim.x + blockIdx.x, a2);
  }
}

// Diffusion adjoint, pass 1: flux part of U and the per-pixel terms
// ah = sbar (u_E - u_W)/2, av = sbar (u_S - u_N)/2 with sbar = gbar psi''(s).
__global__ void k_adj_rev_diff1(const float* __restrict__ Dbar, const float* __restrict__ u,
                                const float* __restrict__ g, AdjImage im, float* __restrict__ Uacc,
                                float2* __restrict__ a_out) {
  const int H = im.H, W = im.W;
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    const int p = idx;
    const float up = u[p], gp = g[p], dp = Dbar[p];
    float ub = 0.f, gb = 0.f;
    if (j + 1 < W) { const int q = p + 1; ub -= 0.5f * (dp - Dbar[q]) * (gp + g[q]); gb += 0.5f * (dp - Dbar[q]) * (u[q] - up); }
    if (j > 0)     { const int q = p - 1; ub -= 0.5f * (dp - Dbar[q]) * (gp + g[q]); gb += 0.5f * (dp - Dbar[q]) * (u[q] - up); }
    if (i + 1 < H) { const int q = p + W; ub -= 0.5f * (dp - Dbar[q]) * (gp + g[q]); gb += 0.5f * (dp - Dbar[q]) * (u[q] - up); }
    if (i > 0)     { const int q = p - W; ub -= 0.5f * (dp - Dbar[q]) * (gp + g[q]); gb += 0.5f * (dp - Dbar[q]) * (u[q] - up); }
    Uacc[p] += ub;
    // psi''(s) = -psi'(s)^3 / 2 for TV; 0 for linear diffusion
    const float sbar = im.p.psi_tv ? gb * (-0.5f * gp * gp * gp) : 0.f;
    const float dxu = 0.5f * (u[o + i * W + clampi(j + 1, W)] - u[o + i * W + clampi(j - 1, W)]);
    const float dyu = 0.5f * (u[o + clampi(i + 1, H) * W + j] - u[o + clampi(i - 1, H) * W + j]);
    a_out[p] = make_float2(sbar * dxu, sbar * dyu);
  }
}

// Diffusion adjoint, pass 2: gather of the neighbour-difference terms
// (s_p depends on u at clip(p +- e_x), clip(p +- e_y)).
__global__ void k_adj_rev_diff2(const float2* __restrict__ a, AdjImage im, float* __restrict__ Uacc) {
  const int H = im.H, W = im.W;
  ADJ_PIXELS(im) {
    ADJ_DECOMPOSE(im)
    (void)o;
    const int p = idx;
    float s = 0.f;
    // east neighbour of (i, j-1) is (i, j); of (i, W-1) itself
    if (j >= 1) s += a[p - 1].x;
    if (j == W - 1) s += a[p].x;
    // west neighbour of (i, j+1) is (i, j); of (i, 0) itself
    if (j <= W - 2) s -= a[p + 1].x;
    if (j == 0) s -= a[p].x;
    if (i >= 1) s += a[p - W].y;
    if (i == H - 1) s += a[p].y;
    if (i <= H - 2) s -= a[p + W].y;
    if (i == 0) s -= a[p].y;
    Uacc[p] += s;
  }
}

// Both diffusion passes in one launch: a CTA takes kDiffRows rows of one
// image, forms pass 1 (flux part of U, and (ah, av)) on those rows and the
// row above and below into shared memory, then pass 2 on its own rows, and
// adds both parts to U once.  The halo rows are formed twice (by both
// neighbouring CTAs) instead of going through global memory.
constexpr int kDiffRows = 4;
__host__ __device__ inline size_t diff_smem(int W) { return (size_t)W * (8 * (kDiffRows + 2) + 4 * kDiffRows); }

__global__ void __launch_bounds__(kAdjThreads) k_adj_rev_diff(const float* __restrict__ Dbar,
                                                             const float* __restrict__ u,
                                                             const float* __restrict__ g, AdjImage im,
                                                             float* __restrict__ Uacc) {
  extern __shared__ __align__(16) unsigned char diff_sm[];
  const int H = im.H, W = im.W;
  float2* sa = (float2*)diff_sm;                    // rows i0-1 .. i0+kDiffRows of (ah, av)
  float* sub = (float*)(sa + (kDiffRows + 2) * W);  // rows i0 .. of the flux part
  const int nblk = (H + kDiffRows - 1) / kDiffRows;
  for (int blk = blockIdx.x; blk < im.N * nblk; blk += gridDim.x) {
    const int n = blk / nblk, i0 = (blk - n * nblk) * kDiffRows, i1 = min(i0 + kDiffRows, H);
    const float* ui = u + (size_t)n * H * W;
    const float* gi = g + (size_t)n * H * W;
    const float* di = Dbar + (size_t)n * H * W;
    __syncthreads();  // the previous block's reads of sa and sub are done
    // pass 1 on rows i0-1 .. i1 (those in the image), one column per thread:
    // u, g and Dbar of rows i0-2 .. i1+1 and columns j-1 .. j+1 are loaded
    // together (clamped indices; the in-image tests below decide which
    // enter), so the loads of a column are in flight at once
    constexpr int NR = kDiffRows + 4;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
      const int jw = clampi(j - 1, W), je = clampi(j + 1, W);
      float U[NR][3], G[NR][3], Dd[NR][3];
#pragma unroll
      for (int t = 0; t < NR; ++t) {
        const int row = clampi(i0 - 2 + t, H) * W;
        U[t][0] = ui[row + jw]; U[t][1] = ui[row + j]; U[t][2] = ui[row + je];
        G[t][0] = gi[row + jw]; G[t][1] = gi[row + j]; G[t][2] = gi[row + je];
        Dd[t][0] = di[row + jw]; Dd[t][1] = di[row + j]; Dd[t][2] = di[row + je];
      }
#pragma unroll
      for (int t = 1; t < NR - 1; ++t) {
        const int i = i0 - 2 + t;
        if (i < 0 || i >= H || i > i1) continue;
        const float up = U[t][1], gp = G[t][1], dp = Dd[t][1];
        float ub = 0.f, gb = 0.f;
        if (j + 1 < W) { ub -= 0.5f * (dp - Dd[t][2]) * (gp + G[t][2]); gb += 0.5f * (dp - Dd[t][2]) * (U[t][2] - up); }
        if (j > 0)     { ub -= 0.5f * (dp - Dd[t][0]) * (gp + G[t][0]); gb += 0.5f * (dp - Dd[t][0]) * (U[t][0] - up); }
        if (i + 1 < H) { ub -= 0.5f * (dp - Dd[t + 1][1]) * (gp + G[t + 1][1]); gb += 0.5f * (dp - Dd[t + 1][1]) * (U[t + 1][1] - up); }
        if (i > 0)     { ub -= 0.5f * (dp - Dd[t - 1][1]) * (gp + G[t - 1][1]); gb += 0.5f * (dp - Dd[t - 1][1]) * (U[t - 1][1] - up); }
        // psi''(s) = -psi'(s)^3 / 2 for TV; 0 for linear diffusion
        const float sbar = im.p.psi_tv ? gb * (-0.5f * gp * gp * gp) : 0.f;
        const float dxu = 0.5f * (U[t][2] - U[t][0]);
        const float dyu = 0.5f * (U[t + 1][1] - U[t - 1][1]);  // rows clamped at the image's edges
        sa[(i - i0 + 1) * W + j] = make_float2(sbar * dxu, sbar * dyu);
        if (i >= i0 && i < i1) sub[(i - i0) * W + j] = ub;
      }
    }
    __syncthreads();
    // pass 2: the accumulations of a column issued together
    float* Ub = Uacc + (size_t)n * H * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
      float acc[kDiffRows];
#pragma unroll
      for (int r = 0; r < kDiffRows; ++r) acc[r] = i0 + r < i1 ? Ub[(size_t)(i0 + r) * W + j] : 0.f;
#pragma unroll
      for (int r = 0; r < kDiffRows; ++r) {
        const int i = i0 + r;
        if (i >= i1) continue;
        const float2* a = sa + (i - i0 + 1) * W;  // row i; a - W: row i-1, a + W: row i+1
        float s = 0.f;
        // east neighbour of (i, j-1) is (i, j); of (i, W-1) itself
        if (j >= 1) s += a[j - 1].x;
        if (j == W - 1) s += a[j].x;
        // west neighbour of (i, j+1) is (i, j); of (i, 0) itself
        if (j <= W - 2) s -= a[j + 1].x;
        if (j == 0) s -= a[j].x;
        if (i >= 1) s += a[j - W].y;
        if (i == H - 1) s += a[j].y;
        if (i <= H - 2) s -= a[j + W].y;
        if (i == 0) s -= a[j].y;
        Ub[(size_t)i * W + j] = acc[r] + (sub[(i - i0) * W + j] + s);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Row kernels for one-row PSFs with kw <= kAdjRowTaps.  With kh == 1 the
// blur, the correlation and their transposes act along rows only, so a CTA
// stages whole rows in shared memory, padded by kAdjRowPad columns on each
// side: constant continuation for u and q, zeros for the adjoint images.  The
// exact transposes of the clamped sums equal the zero-padded sums except at
// the two end pixels of a row, where the preimage ranges of the clamp are
// summed explicitly.  Per pixel the arithmetic is that of the generic
// kernels above, term for term.
//
// The tap loops run over runs of RUN adjacent outputs per thread (8 in the
// forward kernel, 4 in the reverse kernel, which keeps the tap partials in
// registers and needs the occupancy): a run slides a register window over the
// KWB + RUN - 1 staged values its taps reach, so each value is read from
// shared memory once per run instead of once per output and tap, and each
// tap weight once per run.  Each output still sums its taps in tap order.
//
// Shared layout of a staged row: logical element e sits at e + floor(e/RUN),
// one pad word after every RUN, so that lanes whose runs start RUN elements
// apart hit distinct banks.  Column j of an array staged with shift sh in
// [0, RUN) is element kAdjRowPad + sh + j.  The shift makes the first element
// of every run's window a multiple of RUN -- sh = -cx mod RUN for the arrays
// read at j + cx - c (u, Abar/Bbar), cx mod RUN for those read at j - cx + c
// (q, bbar) -- so that every offset within the window is a compile-time
// constant m + floor(m/RUN).
// ---------------------------------------------------------------------------
constexpr int kAdjRowTaps = 32, kAdjRowPad = 32;
constexpr int kAdjRowBlock = 4;  // rows staged per CTA and step
constexpr int kAdjRunFwd = 8, kAdjRunRev = 4;  // outputs per thread in the tap loops

__device__ __forceinline__ float zero_of(float) { return 0.f; }
__device__ __forceinline__ float2 zero_of(float2) { return make_float2(0.f, 0.f); }

template <int RUN>
__host__ __device__ __forceinline__ int pidx(int e) {
  static_assert(RUN == 4 || RUN == 8, "run length");
  return e + (e >> (RUN == 8 ? 3 : 2));
}
// Elements per staged row (shifted logical range: kAdjRowPad + RUN-1 + W + kAdjRowPad).
template <int RUN>
__host__ __device__ inline int adj_row_pitch(int W) {
  const int L = W + 2 * kAdjRowPad + RUN;
  return pidx<RUN>(L) + 1;
}

// Stage rows R0..R0+nr-1 (pitch W, packed) with shift sh: row r at s + r*P,
// columns -kAdjRowPad .. W+kAdjRowPad-1, constant continuation or zeros.
template <int RUN, typename T, bool CLAMP>
__device__ __forceinline__ void stage_rows(T* s, const T* __restrict__ src, int R0, int nr, int W, int sh) {
  const int P = adj_row_pitch<RUN>(W), L = W + 2 * kAdjRowPad, total = nr * L;
  constexpr int B = 4;  // loads in flight per thread before their shared stores
  for (int base = threadIdx.x; base < total; base += B * blockDim.x) {
    T v[B];
    int at[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int k = base + b * blockDim.x;
      at[b] = -1;
      v[b] = zero_of(T());
      if (k < total) {
        const int r = k / L, kk = k - r * L, j = kk - kAdjRowPad;
        const T* row = src + (size_t)(R0 + r) * W;
        if (CLAMP) v[b] = row[clampi(j, W)];
        else if (j >= 0 && j < W) v[b] = row[j];
        at[b] = r * P + pidx<RUN>(kk + sh);
      }
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
      if (at[b] >= 0) s[at[b]] = v[b];
  }
}

// Column of pad slot t (0 .. 2 kAdjRowPad - 1) of a row: -1-t left, W+t' right.
__device__ __forceinline__ int pad_column(int t, int W) {
  return t < kAdjRowPad ? -1 - t : W + (t - kAdjRowPad);
}

// The taps of a one-row PSF, zero beyond kw up to KWB (the tap loops below
// run over KWB taps with compile-time offsets; a zero tap adds exactly zero
// to a finite sum).
template <int KWB>
__device__ __forceinline__ void load_row_taps(float* taps, const AdjImage& im) {
  if ((int)threadIdx.x < KWB) taps[threadIdx.x] = (int)threadIdx.x < im.kw ? im.taps[threadIdx.x] : 0.f;
}

// A tap weight read from shared memory at each use (volatile: the weights
// stay out of registers, which the row kernels need for occupancy).
__device__ __forceinline__ float tap_at(const float* taps, int c) { return *((volatile const float*)taps + c); }

// Exact transpose of a clamped one-row sum at a row end (j = 0: first, or
// j = n - 1): sum over taps c of w[c] times the sum of x over the clamp's
// preimage of the shift sgn (c - cx).  At j = 0 the preimage of a shift s
// is [0, min(-s, n-1)] (empty for s > 0), at j = n - 1 it is
// [max(n-1-s, 0), n-1] (empty for s < 0).  With d = |s| the preimages of
// the taps with nonempty ranges are nested, so one running prefix (suffix)
// sum visits every x once: O(kw) per end pixel.  x(d) reads column d.
__device__ __forceinline__ float2 x_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float x_add(float a, float b) { return a + b; }
__device__ __forceinline__ float2 x_fma(float w, float2 a, float2 acc) {
  return make_float2(fmaf(w, a.x, acc.x), fmaf(w, a.y, acc.y));
}
__device__ __forceinline__ float x_fma(float w, float a, float acc) { return fmaf(w, a, acc); }
template <typename T, typename X>
__device__ T row_end_transpose(X x, const float* taps, int kw, int cx, int n, bool first, int sgn) {
  T out = zero_of(T());
  if (n == 1) {
    for (int c = 0; c < kw; ++c) out = x_fma(taps[c], x(0), out);
    return out;
  }
  const int dmax = (first == (sgn > 0)) ? cx : kw - 1 - cx;
  const int e = first ? -sgn : sgn;  // tap c = cx + e d
  T run = zero_of(T());
  for (int d = 0; d <= dmax; ++d) {
    if (d < n) run = x_add(run, x(first ? d : n - 1 - d));
    out = x_fma(taps[cx + e * d], run, out);
  }
  return out;
}

// Smallest tap-loop length of the row kernels that holds kw taps.
inline int row_taps_bucket(int kw) { return kw <= 8 ? 8 : kw <= 16 ? 16 : kw <= 24 ? 24 : 32; }

// A run's values from / to global memory: n valid; vec: 16-byte aligned and
// the run is full.
__device__ __forceinline__ bool al16(const void* p) { return (((uintptr_t)p) & 15) == 0; }
template <int RUN>
__device__ __forceinline__ void run_load(float (&v)[RUN], const float* __restrict__ src, int n, bool vec) {
  if (vec) {
#pragma unroll
    for (int k = 0; k < RUN / 4; ++k) {
      const float4 a = reinterpret_cast<const float4*>(src)[k];
      v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int s = 0; s < RUN; ++s) v[s] = s < n ? src[s] : 0.f;
  }
}
template <int RUN>
__device__ __forceinline__ void run_store(float* dst, const float (&v)[RUN], int n, bool vec) {
  if (vec) {
#pragma unroll
    for (int k = 0; k < RUN / 4; ++k)
      reinterpret_cast<float4*>(dst)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  } else {
#pragma unroll
    for (int s = 0; s < RUN; ++s)
      if (s < n) dst[s] = v[s];
  }
}
template <int RUN>
__device__ __forceinline__ void run_store(float2* dst, const float2 (&v)[RUN], int n, bool vec) {
  if (vec) {
#pragma unroll
    for (int k = 0; k < RUN / 2; ++k)
      reinterpret_cast<float4*>(dst)[k] = make_float4(v[2 * k].x, v[2 * k].y, v[2 * k + 1].x, v[2 * k + 1].y);
  } else {
#pragma unroll
    for (int s = 0; s < RUN; ++s)
      if (s < n) dst[s] = v[s];
  }
}

// Sliding window over a run's tap reach: for c = 0..KWB-1 in order, f(c, win)
// with win[s] = x[pidx(s + c)] (SGN > 0) or x[pidx(s - c)] (SGN < 0).  Every
// value is read from shared memory once and then moves through the window
// (register renaming once unrolled).
template <int KWB, int SGN, int RUN, typename T, typename F>
__device__ __forceinline__ void run_window(const T* x, F f) {
  T win[RUN];
#pragma unroll
  for (int s = 0; s < RUN; ++s) win[s] = x[pidx<RUN>(s)];
#pragma unroll
  for (int c = 0; c < KWB; ++c) {
    f(c, win);
    if (c + 1 < KWB) {
      if (SGN > 0) {
#pragma unroll
        for (int s = 0; s + 1 < RUN; ++s) win[s] = win[s + 1];
        win[RUN - 1] = x[pidx<RUN>(c + RUN)];
      } else {
#pragma unroll
        for (int s = RUN - 1; s > 0; --s) win[s] = win[s - 1];
        win[0] = x[pidx<RUN>(-c - 1)];
      }
    }
  }
}

// (row, column) of a loop index over rows of n columns that starts at
// `start` and advances by `stride`, kept without a division per step.
struct RowCol {
  int r, c, dr, dc, n;
  __device__ __forceinline__ RowCol(int start, int stride, int n_) : n(n_) {
    r = start / n;
    c = start - r * n;
    dr = stride / n;
    dc = stride - dr * n;
  }
  __device__ __forceinline__ void next() {
    r += dr;
    c += dc;
    if (c >= n) { c -= n; ++r; }
  }
};

// Row within its image of row r of the block starting at stacked row R0
// (ib = R0 mod H).
__device__ __forceinline__ int image_row(int ib, int r, int H) {
  int i = ib + r;
  while (i >= H) i -= H;
  return i;
}

// Row-block loop: the CTA takes kAdjRowBlock rows at a time (grid-stride).
#define ADJ_ROW_BLOCKS(rows)                                                                       \
  for (int R0 = blockIdx.x * kAdjRowBlock; R0 < (rows); R0 += gridDim.x * kAdjRowBlock)
// Pixel loop over nr rows of W: row rc_.r, column rc_.c.
#define ADJ_ROW_ITEMS(nr, W)                                                                       \
  for (RowCol rc_(threadIdx.x, blockDim.x, (W)); rc_.r < (nr); rc_.next())
// Run loop: run rc_.c of row r starts at column j0 and holds n outputs.
#define ADJ_ROW_RUNS(nr, nrun, W)                                                                  \
  for (RowCol rc_(threadIdx.x, blockDim.x, (nrun)); rc_.r < (nr); rc_.next())
#define ADJ_RUN_DECOMPOSE(nrun, W)                                                                 \
  const int r = rc_.r, j0 = rc_.c * RUN, n = min(RUN, (W) - j0);

// Forward recompute of one iteration for one-row PSFs, fused: b = C u and
// q = (W f/b, W) into a shared row, then A, B = C' q and g from it.
template <int KWB>
__global__ void __launch_bounds__(kAdjThreads) k_adj_fwd_rows(const float* __restrict__ u,
                                                                  const float* __restrict__ f0, AdjImage im,
                                                                  float* __restrict__ b_out,
                                                                  float2* __restrict__ q_out,
                                                                  float2* __restrict__ ab_out,
                                                                  float* __restrict__ g_out) {
  extern __shared__ __align__(16) unsigned char adj_sm[];
  __shared__ float taps[KWB];
  constexpr int RUN = kAdjRunFwd;
  const int kw = im.kw, cx = kw >> 1, W = im.W, H = im.H, rows = im.N * im.H;
  const int P = adj_row_pitch<RUN>(W), nrun = (W + RUN - 1) / RUN;
  const int shu = (-cx) & (RUN - 1), shq = cx & (RUN - 1);  // u read at j + cx - c, q at j - cx + c
  float2* sq = (float2*)adj_sm;
  float* su = (float*)(sq + kAdjRowBlock * P);
  const bool vec = (W & 3) == 0 && al16(u) && al16(f0) && al16(b_out) && al16(q_out) && al16(ab_out) && al16(g_out);
  load_row_taps<KWB>(taps, im);
  ADJ_ROW_BLOCKS(rows) {
    const int nr = min(kAdjRowBlock, rows - R0), ib = R0 % H;
    __syncthreads();
    stage_rows<RUN, float, true>(su, u, R0, nr, W, shu);
    __syncthreads();
    ADJ_ROW_RUNS(nr, nrun, W) {
      ADJ_RUN_DECOMPOSE(nrun, W)
      const bool full = vec && n == RUN;
      const float* ub = su + r * P + pidx<RUN>(kAdjRowPad + shu + j0 + cx);  // ub[pidx<RUN>(m)] = u(j0 + cx + m)
      float bb[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) bb[s] = 0.f;
      run_window<KWB, -1, RUN>(ub, [&](int c, const float(&win)[RUN]) {
        const float w = tap_at(taps, c);
#pragma unroll
        for (int s = 0; s < RUN; ++s) bb[s] = fmaf(w, win[s], bb[s]);
      });
      const size_t idx0 = (size_t)(R0 + r) * W + j0;
      float fv[RUN];
      run_load(fv, f0 + idx0, n, full);
      float2 qv[RUN];
      float2* qrow = sq + r * P;
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        float rr;
        const float w = phi_w(bb[s], fv[s], im.p, &rr);
        qv[s] = make_float2(w * fv[s] / bb[s], w);
        if (s < n) qrow[pidx<RUN>(kAdjRowPad + shq + j0 + s)] = qv[s];
      }
      run_store(b_out + idx0, bb, n, full);
      run_store(q_out + idx0, qv, n, full);
    }
    __syncthreads();
    // constant continuation of q beyond the row ends
    for (int k = threadIdx.x; k < nr * 2 * kAdjRowPad; k += blockDim.x) {
      const int r = k / (2 * kAdjRowPad), t = k - r * 2 * kAdjRowPad;
      const int jj = pad_column(t, W), js = t < kAdjRowPad ? 0 : W - 1;
      sq[r * P + pidx<RUN>(kAdjRowPad + shq + jj)] = sq[r * P + pidx<RUN>(kAdjRowPad + shq + js)];
    }
    __syncthreads();
    ADJ_ROW_RUNS(nr, nrun, W) {
      ADJ_RUN_DECOMPOSE(nrun, W)
      const bool full = vec && n == RUN;
      const float2* qb = sq + r * P + pidx<RUN>(kAdjRowPad + shq + j0 - cx);  // qb[pidx<RUN>(m)] = q(j0 - cx + m)
      float A[RUN], B[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) { A[s] = 0.f; B[s] = 0.f; }
      run_window<KWB, 1, RUN>(qb, [&](int c, const float2(&win)[RUN]) {
        const float w = tap_at(taps, c);
#pragma unroll
        for (int s = 0; s < RUN; ++s) {
          A[s] = fmaf(w, win[s].x, A[s]);
          B[s] = fmaf(w, win[s].y, B[s]);
        }
      });
      const int Rr = R0 + r, i = image_row(ib, r, H);
      const float* ip = u + (size_t)(Rr - i) * W + j0;
      const float* ur = su + r * P;
      float up[RUN], dn[RUN];
      run_load(up, ip + (size_t)clampi(i - 1, H) * W, n, full);
      run_load(dn, ip + (size_t)clampi(i + 1, H) * W, n, full);
      const size_t idx0 = (size_t)Rr * W + j0;
      float2 abv[RUN];
      float gv[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        const int j = j0 + s;
        abv[s] = make_float2(A[s], B[s]);
        const float gx = 0.5f * (ur[pidx<RUN>(kAdjRowPad + shu + j + 1)] - ur[pidx<RUN>(kAdjRowPad + shu + j - 1)]);
        const float gy = 0.5f * (dn[s] - up[s]);
        gv[s] = psi_g(gx, gy, im.p);
      }
      run_store(ab_out + idx0, abv, n, full);
      run_store(g_out + idx0, gv, n, full);
    }
  }
}

// One reverse step for one-row PSFs, fused row by row:
//   U = U' num/den, Abar, Bbar, Dbar          (as k_adj_rev_update)
//   qbar = C'^T (Abar, Bbar)                  (as k_adj_rev_corrT)
//   bbar, f0bar                               (as k_adj_rev_weight)
//   U += C^T bbar                             (as k_adj_rev_convT)
// with the alpha partial in part[0 .. G) and the tap partials (both
// transposes, summed per tap) in part[G + t G ...].  The diffusion adjoint
// (k_adj_rev_diff) follows: it needs Dbar of the neighbouring rows.
template <int KWB>
__global__ void __launch_bounds__(kAdjThreads, KWB <= 24 ? 3 : 2) k_adj_rev_rows(
    const float* __restrict__ Ubar_next, const float* __restrict__ u, const float2* __restrict__ ab,
    const float* __restrict__ g, const float2* __restrict__ q, const float* __restrict__ b,
    const float* __restrict__ f0, AdjImage im, float* __restrict__ Uacc, float* __restrict__ Dbar,
    float* __restrict__ f0bar, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char adj_sm[];
  __shared__ float taps[KWB];
  constexpr int RUN = kAdjRunRev;
  const int kw = im.kw, cx = kw >> 1, W = im.W, H = im.H, rows = im.N * im.H;
  const int P = adj_row_pitch<RUN>(W), nrun = (W + RUN - 1) / RUN;
  const int shm = (-cx) & (RUN - 1), shp = cx & (RUN - 1);  // read at j + cx - c: u, Abar/Bbar; at j - cx + c: q, bbar
  float2* sa = (float2*)adj_sm;
  float2* sq = sa + kAdjRowBlock * P;
  float* sb = (float*)(sq + kAdjRowBlock * P);
  float* su = sb + kAdjRowBlock * P;
  const bool vec = (W & 3) == 0 && al16(b) && al16(f0) && al16(f0bar) && al16(Uacc);
  load_row_taps<KWB>(taps, im);
  float acc[KWB];  // tap partials (entries from kw on are never reduced)
#pragma unroll
  for (int t = 0; t < KWB; ++t) acc[t] = 0.f;
  float asum = 0.f;
  ADJ_ROW_BLOCKS(rows) {
    const int nr = min(kAdjRowBlock, rows - R0);
    __syncthreads();
    stage_rows<RUN, float2, true>(sq, q, R0, nr, W, shp);
    stage_rows<RUN, float, true>(su, u, R0, nr, W, shm);
    for (int k = threadIdx.x; k < nr * 2 * kAdjRowPad; k += blockDim.x) {  // zero pads of abar, bbar
      const int r = k / (2 * kAdjRowPad), jj = pad_column(k - r * 2 * kAdjRowPad, W);
      sa[r * P + pidx<RUN>(kAdjRowPad + shm + jj)] = make_float2(0.f, 0.f);
      sb[r * P + pidx<RUN>(kAdjRowPad + shp + jj)] = 0.f;
    }
    // U = U' num/den, Abar, Bbar, Dbar
    const int ib = R0 % H;
    ADJ_ROW_ITEMS(nr, W) {
      const int r = rc_.r, j = rc_.c;
      const int R = R0 + r, i = image_row(ib, r, H);
      const size_t o = (size_t)(R - i) * W, idx = (size_t)R * W + j;
      const float D = diffusion_at(u + o, g + o, i, j, H, W);
      const float2 v = ab[idx];
      const float Dp = fmaxf(D, 0.f), Dm = fminf(D, 0.f);
      const float num = v.x + im.p.alpha * Dp;
      const float den = v.y - im.p.alpha * Dm;
      const float ub = Ubar_next[idx], uu = u[idx];
      const float rd = __fdividef(1.f, den);  // den >= B > 0
      const float Ab = ub * uu * rd;
      const float Bb = -ub * uu * num * (rd * rd);
      Uacc[idx] = ub * num * rd;
      sa[r * P + pidx<RUN>(kAdjRowPad + shm + j)] = make_float2(Ab, Bb);
      Dbar[idx] = im.p.alpha * ((D > 0.f ? Ab : 0.f) - (D < 0.f ? Bb : 0.f));
      asum += Ab * Dp - Bb * Dm;
    }
    __syncthreads();
    // qbar = C'^T (Abar, Bbar); bbar and f0bar; correlation tap partials
    ADJ_ROW_RUNS(nr, nrun, W) {
      ADJ_RUN_DECOMPOSE(nrun, W)
      const bool full = vec && n == RUN;
      const size_t idx0 = (size_t)(R0 + r) * W + j0;
      float bv[RUN], fv[RUN], fb[RUN];  // issued ahead of the tap loops
      run_load(bv, b + idx0, n, full);
      run_load(fv, f0 + idx0, n, full);
      run_load(fb, f0bar + idx0, n, full);
      const float2* ar = sa + r * P;
      const float2* a8 = ar + pidx<RUN>(kAdjRowPad + shm + j0 + cx);  // a8[pidx<RUN>(m)] = abar(j0 + cx + m)
      float s1[RUN], s2[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) { s1[s] = 0.f; s2[s] = 0.f; }
      run_window<KWB, -1, RUN>(a8, [&](int c, const float2(&win)[RUN]) {
        const float w = tap_at(taps, c);
#pragma unroll
        for (int s = 0; s < RUN; ++s) {
          s1[s] = fmaf(w, win[s].x, s1[s]);
          s2[s] = fmaf(w, win[s].y, s2[s]);
        }
      });
      // the two row-end pixels: exact transposes over the clamp's preimages
      auto acol = [&](int d) { return ar[pidx<RUN>(kAdjRowPad + shm + d)]; };
      const float2 z0 = j0 == 0 ? row_end_transpose<float2>(acol, taps, kw, cx, W, true, +1) : make_float2(0.f, 0.f);
      const float2 z1 = j0 + n == W ? row_end_transpose<float2>(acol, taps, kw, cx, W, W == 1, +1)
                                    : make_float2(0.f, 0.f);
      float2 v[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        const int j = j0 + s;
        if (j == 0) { s1[s] = z0.x; s2[s] = z0.y; }
        else if (j == W - 1) { s1[s] = z1.x; s2[s] = z1.y; }
        v[s] = ar[pidx<RUN>(kAdjRowPad + shm + j)];  // zero beyond the row
      }
      const float2* q8 = sq + r * P + pidx<RUN>(kAdjRowPad + shp + j0 - cx);  // q8[pidx<RUN>(m)] = q(j0 - cx + m)
      run_window<KWB, 1, RUN>(q8, [&](int t, const float2(&win)[RUN]) {
#pragma unroll
        for (int s = 0; s < RUN; ++s) acc[t] = fmaf(v[s].x, win[s].x, fmaf(v[s].y, win[s].y, acc[t]));
      });
      float* brow = sb + r * P;
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        if (s < n) {
          float rr;
          const float w = phi_w(bv[s], fv[s], im.p, &rr);
          const float rb = __fdividef(1.f, bv[s]);  // b >= the floor > 0
          const float Wbar = s1[s] * fv[s] * rb + s2[s];
          // phi''(r) = -phi'(r)^3 / (2 eps^2) for the regularised L1 penaliser
          const float rbar = im.p.phi_robust ? Wbar * (-w * w * w / (2.f * im.p.eps_phi * im.p.eps_phi)) : 0.f;
          brow[pidx<RUN>(kAdjRowPad + shp + j0 + s)] = -s1[s] * w * fv[s] * (rb * rb) + rbar * (1.f - fv[s] * rb);
          fb[s] += s1[s] * w * rb - rbar * __logf(bv[s] * __fdividef(1.f, fv[s]));
        }
      }
      run_store(f0bar + idx0, fb, n, full);
    }
    __syncthreads();
    // U += C^T bbar; convolution tap partials
    ADJ_ROW_RUNS(nr, nrun, W) {
      ADJ_RUN_DECOMPOSE(nrun, W)
      const bool full = vec && n == RUN;
      const size_t idx0 = (size_t)(R0 + r) * W + j0;
      float ua[RUN];  // issued ahead of the tap loops
      run_load(ua, Uacc + idx0, n, full);
      const float* br = sb + r * P;
      const float* b8 = br + pidx<RUN>(kAdjRowPad + shp + j0 - cx);  // b8[pidx<RUN>(m)] = bbar(j0 - cx + m)
      float sacc[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) sacc[s] = 0.f;
      run_window<KWB, 1, RUN>(b8, [&](int c, const float(&win)[RUN]) {
        const float w = tap_at(taps, c);
#pragma unroll
        for (int s = 0; s < RUN; ++s) sacc[s] = fmaf(w, win[s], sacc[s]);
      });
      auto bcol = [&](int d) { return br[pidx<RUN>(kAdjRowPad + shp + d)]; };
      const float z0 = j0 == 0 ? row_end_transpose<float>(bcol, taps, kw, cx, W, true, -1) : 0.f;
      const float z1 = j0 + n == W ? row_end_transpose<float>(bcol, taps, kw, cx, W, W == 1, -1) : 0.f;
      float bvv[RUN];
#pragma unroll
      for (int s = 0; s < RUN; ++s) {
        const int j = j0 + s;
        if (j == 0) sacc[s] = z0;
        else if (j == W - 1) sacc[s] = z1;
        bvv[s] = br[pidx<RUN>(kAdjRowPad + shp + j)];  // zero beyond the row
      }
#pragma unroll
      for (int s = 0; s < RUN; ++s) ua[s] += sacc[s];
      run_store(Uacc + idx0, ua, n, full);
      const float* u8 = su + r * P + pidx<RUN>(kAdjRowPad + shm + j0 + cx);  // u8[pidx<RUN>(m)] = u(j0 + cx + m)
      run_window<KWB, -1, RUN>(u8, [&](int t, const float(&win)[RUN]) {
#pragma unroll
        for (int s = 0; s < RUN; ++s) acc[t] = fmaf(bvv[s], win[s], acc[t]);
      });
    }
  }
  block_reduce_add(part + blockIdx.x, asum);
#pragma unroll
  for (int t = 0; t < KWB; ++t)
    if (t < kw) block_reduce_add(part + (size_t)(1 + t) * gridDim.x + blockIdx.x, acc[t]);
}

// Sum `nparts` partials of each of `nsum` sums in fixed order, in double,
// and add them into out[k].
__global__ void k_adj_reduce(const float* __restrict__ partials, int nsum, int nparts, double* __restrict__ out) {
  const int k = blockIdx.x;
  if (k >= nsum) return;
  __shared__ double red[kAdjThreads];
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += blockDim.x) s += (double)partials[(size_t)k * nparts + t];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] += red[0];
}

__global__ void k_copy_pitched(const float* __restrict__ src, int lds, float* __restrict__ dst, int ldd,
                               int H, int W, const float* __restrict__ mask_src, float mask_floor) {
  const size_t n = (size_t)H * W;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / W), j = (int)(idx - (size_t)i * W);
    float v = src[(size_t)i * lds + j];
    if (mask_src) v = (mask_src[(size_t)i * lds + j] > mask_floor) ? v : 0.f;
    dst[(size_t)i * ldd + j] = v;
  }
}

// Two real rows per CTA (rows 2b and 2b+1).  For each row z = u0bar + i f0
// gives both spectra from one transform -- U(k) = (Z(k) + conj Z(-k))/2,
// F(k) = (Z(k) - conj Z(-k))/(2i) -- and the inverse of the Hermitian G_a +
// i G_b (G = U S/(|S|^2 + K)) returns row a's result in its real part and
// row b's in its imaginary part: three transforms for two rows instead of
// six.  Spectra are in the transform's storage order (bit-reversed for a
// power of two, natural under Bluestein).
__global__ void __launch_bounds__(256) k_adj_wiener_rows2(const float* __restrict__ u0bar,
                                                          const float* __restrict__ f0, int W, int rows,
                                                          const float4* __restrict__ spec, Dft1ff D, float K,
                                                          float2 invN, float* __restrict__ f0bar,
                                                          float2* __restrict__ prow) {
  extern __shared__ float4 sm[];
  const int M = dft_len(D);
  const bool pow2 = D.c == nullptr;
  float4* x = sm;      // row a: Z, then the packed G_a + i G_b
  float4* y = sm + M;  // row b: Z
  const int ra = 2 * blockIdx.x, rb = ra + 1;
  const bool has_b = rb < rows;
  for (int c = threadIdx.x; c < W; c += blockDim.x) {
    x[c] = mkc(make_float2(u0bar[(size_t)ra * W + c], 0.f), make_float2(f0[(size_t)ra * W + c], 0.f));
    y[c] = has_b ? mkc(make_float2(u0bar[(size_t)rb * W + c], 0.f), make_float2(f0[(size_t)rb * W + c], 0.f))
                 : zzero();
  }
  __syncthreads();
  dft_fwd_ff(x, 1, 1, M, D, false);
  dft_fwd_ff(y, 1, 1, M, D, false);
  const float2 half = make_float2(0.5f, 0.f);
  for (int si = threadIdx.x; si < W; si += blockDim.x) {
    const int k = pow2 ? (D.logM ? (int)(__brev((unsigned)si) >> (32 - D.logM)) : 0) : si;
    const int kn = k ? W - k : 0;
    const int sn = pow2 ? (D.logM ? (int)(__brev((unsigned)kn) >> (32 - D.logM)) : 0) : kn;
    if (si > sn) continue;  // each pair (k, -k) once, by the thread of its lower storage index
    const float4 S0 = __ldg(spec + si), S1 = __ldg(spec + sn);
    const float2 den0 = ff_add(ff_add(ff_mul(re_(S0), re_(S0)), ff_mul(im_(S0), im_(S0))), make_float2(K, 0.f));
    const float2 den1 = ff_add(ff_add(ff_mul(re_(S1), re_(S1)), ff_mul(im_(S1), im_(S1))), make_float2(K, 0.f));
    float4 G0[2], G1[2];
    for (int row = 0; row < 2; ++row) {
      const float4* z = row ? y : x;
      const float4 Za = z[si], Zb = z[sn];
      // U(k), F(k) and U(-k) = conj U(k), F(-k) = conj F(k) (real rows)
      const float4 U0 = zscale(zadd(Za, zconj(Zb)), half);
      const float4 dz = zsub(Za, zconj(Zb));
      const float4 F0 = zscale(mkc(im_(dz), ff_neg(re_(dz))), half);  // dz / (2i)
      const float4 U1 = zconj(U0), F1 = zconj(F0);
      const int r = row ? rb : ra;
      if (row == 0 || has_b) {
        const float4 P0 = zmulc(F0, U0), P1 = zmulc(F1, U1);  // P(k) = conj(U) F
        prow[(size_t)r * W + si] = make_float2(P0.x + P0.y, P0.z + P0.w);
        prow[(size_t)r * W + sn] = make_float2(P1.x + P1.y, P1.z + P1.w);
      }
      const float4 t0 = zmul(U0, S0), t1 = zmul(U1, S1);
      G0[row] = mkc(ff_div(re_(t0), den0), ff_div(im_(t0), den0));
      G1[row] = mkc(ff_div(re_(t1), den1), ff_div(im_(t1), den1));
    }
    // packed Q = G_a + i G_b at k and -k (each pair is read and written by
    // this thread only)
    x[si] = mkc(ff_sub(re_(G0[0]), im_(G0[1])), ff_add(im_(G0[0]), re_(G0[1])));
    x[sn] = mkc(ff_sub(re_(G1[0]), im_(G1[1])), ff_add(im_(G1[0]), re_(G1[1])));
  }
  __syncthreads();
  dft_inv_ff(x, 1, 1, M, D, false);
  for (int c = threadIdx.x; c < W; c += blockDim.x) {
    const float2 va = ff_mul(re_(x[c]), invN), vb = ff_mul(im_(x[c]), invN);
    f0bar[(size_t)ra * W + c] += va.x + va.y;
    if (has_b) f0bar[(size_t)rb * W + c] += vb.x + vb.y;
  }
}

// ---------------------------------------------------------------------------
// Wiener adjoint for a PSF on one row (float-float transforms; two real rows
// per CTA share three transforms, k_adj_wiener_rows2):
//   U0 = DFT(u0bar_row) (masked by 1[w > delta]),  F0 = DFT(f0_row)
//   f0bar_row += Re IDFT(U0 conj(M)) / N          (transpose of the filter)
//   P(k) = conj(U0(k)) F0(k)  (summed over rows)  for the K and tap gradients
// ---------------------------------------------------------------------------

// Column sums of prow (rows x W complex) in double: P(k), in two levels of
// fixed order: chunks of kPsumRows rows (one thread per column and chunk),
// then the chunk sums in chunk order.
constexpr int kPsumRows = 256;
__global__ void k_adj_psum_part(const float2* __restrict__ prow, int rows, int W, double2* __restrict__ part) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
  if (k >= W) return;
  double sr = 0.0, si = 0.0;
  const int r1 = min(rows, (ch + 1) * kPsumRows);
  for (int r = ch * kPsumRows; r < r1; ++r) {
    const float2 v = prow[(size_t)r * W + k];
    sr += v.x;
    si += v.y;
  }
  part[(size_t)ch * W + k] = make_double2(sr, si);
}
__global__ void k_adj_psum(const double2* __restrict__ part, int nch, int W, double2* __restrict__ P) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= W) return;
  double sr = 0.0, si = 0.0;
  for (int c = 0; c < nch; ++c) {
    const double2 v = part[(size_t)c * W + k];
    sr += v.x;
    si += v.y;
  }
  P[k] = make_double2(sr, si);
}

// K and tap gradients of the Wiener step from P(k):
//   M = conj(S)/(|S|^2+K);  dM/dK = -conj(S)/(|S|^2+K)^2
//   dM/dS = -conj(S)^2/(|S|^2+K)^2,  dM/dconj(S) = K/(|S|^2+K)^2
//   d(loss) = Re sum_k P(k) dM(k) / N,  dS(k)/dh(d) = E_d(k) (spectrum of a
//   unit tap at offset d, same storage order as S).
// One CTA; thread t < kw handles tap t, thread kw handles K.
// One CTA per output (taps 0..kw-1, then K): the sum over frequencies in
// double, each thread a strided share, combined by a fixed-order tree.
__global__ void __launch_bounds__(256) k_adj_wiener_params(const double2* __restrict__ P,
                                                           const float4* __restrict__ spec,
                                                           const float4* __restrict__ unit_spec, int W, int kw,
                                                           float K, double* __restrict__ grad_taps,
                                                           double* __restrict__ grad_K) {
  __shared__ double red[256];
  const int t = blockIdx.x;
  double acc = 0.0;
  for (int k = threadIdx.x; k < W; k += blockDim.x) {
    const float4 Sf = spec[k];
    const double sr = (double)Sf.x + (double)Sf.y, si = (double)Sf.z + (double)Sf.w;
    const double den = sr * sr + si * si + (double)K;
    const double pr = P[k].x, pi = P[k].y;
    if (t == kw) {
      // Re P * (-conj(S)/den^2)
      acc += -(pr * sr + pi * si) / (den * den);
    } else {
      const float4 Ef = unit_spec[(size_t)t * W + k];
      const double er = (double)Ef.x + (double)Ef.y, ei = (double)Ef.z + (double)Ef.w;
      // dM/dS * E + dM/dconj(S) * conj(E)
      const double c2r = sr * sr - si * si, c2i = -2.0 * sr * si;           // conj(S)^2
      const double ar = -(c2r * er - c2i * ei) / (den * den);
      const double ai = -(c2r * ei + c2i * er) / (den * den);
      const double br = (double)K * er / (den * den), bi = -(double)K * ei / (den * den);
      const double mr = ar + br, mi = ai + bi;
      acc += pr * mr - pi * mi;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = red[0] / (double)W;
    if (t == kw) *grad_K += v;
    else grad_taps[t] += v;
  }
}

// Spectra of unit taps at each offset of a one-row PSF: row t holds the
// wrapped unit impulse at column (t - kw/2) mod W.
__global__ void k_unit_taps(float* __restrict__ out, int kw) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kw * kw; t += gridDim.x * blockDim.x)
    out[t] = ((t / kw) == (t % kw)) ? 1.f : 0.f;
}

}  // namespace db

namespace db {

constexpr int kAdjBlocks = 592;  // 4 x 148 SMs, grid-stride

struct AdjLayout {
  size_t f0, seg, b, q, ab, g, ubar, uacc, abbar, dbar, qbar, bbar, f0bar, a, part, wraw, prow, ppart, psum,
      spec, unit_taps, unit_spec, tabs, kspec, total;
};

static AdjLayout adj_layout(int N, int H, int W, int kw, int ntaps, int every) {
  AdjLayout L = {};
  const size_t n = (size_t)N * H * W;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += align256(bytes); return o; };
  L.f0 = take(n * 4);
  L.seg = take(n * 4 * (size_t)(every + 1));
  // forward intermediates of every iterate of a segment (computed while the
  // segment is rebuilt, read again by its reverse steps)
  L.b = take(n * 4 * (size_t)every);
  L.q = take(n * 8 * (size_t)every);
  L.ab = take(n * 8 * (size_t)every);
  L.g = take(n * 4 * (size_t)every);
  L.ubar = take(n * 4);
  L.uacc = take(n * 4);
  L.abbar = take(n * 8);
  L.dbar = take(n * 4);
  L.qbar = take(n * 8);
  L.bbar = take(n * 4);
  L.f0bar = take(n * 4);
  L.a = take(n * 8);
  L.part = take((size_t)(ntaps + 1) * kAdjBlocks * 4);
  L.wraw = take(n * 4);
  L.prow = take(n * 8);  // (N*H) x W
  L.ppart = take((size_t)((N * H + kPsumRows - 1) / kPsumRows) * W * 16);
  L.psum = take((size_t)W * 16);
  L.spec = take((size_t)W * 16);
  L.unit_taps = take((size_t)kw * kw * 4);
  L.unit_spec = take((size_t)kw * W * 16);
  L.tabs = take(dft_table_elems(W) * 16);
  L.kspec = take(wiener_kspec_elems(1, W, 1, kw) * 16);  // the forward Wiener's filter spectrum
  L.total = off;
  return L;
}

size_t adj_ws_bytes(int N, int H, int W, int kh, int kw, int every) {
  return adj_layout(N, H, W, kw, kh * kw, every).total;
}

__global__ void k_floor_pack(const float* __restrict__ f, int ld, int H, int W, float delta, float* __restrict__ f0) {
  const size_t n = (size_t)H * W;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / W), j = (int)(idx - (size_t)i * W);
    f0[idx] = fmaxf(f[(size_t)i * ld + j], delta);
  }
}

__global__ void k_grad_f_out(const float* __restrict__ f0bar, const float* __restrict__ f, int ld, int H, int W,
                             float delta, float* __restrict__ grad_f) {
  const size_t n = (size_t)H * W;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / W), j = (int)(idx - (size_t)i * W);
    grad_f[(size_t)i * ld + j] = (f[(size_t)i * ld + j] > delta) ? f0bar[idx] : 0.f;
  }
}

#define ADJ_CHECK(x) do { if ((x) != cudaSuccess) { (void)cudaGetLastError(); return DB_ERR_CUDA; } } while (0)
#define ADJ_LAUNCH(...) do { __VA_ARGS__; count_launch(); ADJ_CHECK(cudaGetLastError()); } while (0)

db_status adj_backward(const float* f, int ld, int N, const float* ckpt, int iters, int every,
                       const float* grad_u, int H, int W, const db_psf* psf, const db_params* p, float* grad_f,
                       double* grad_taps, double* grad_alpha, double* grad_K, void* ws, size_t ws_bytes,
                       int* status, cudaStream_t s) {
  const int kh = psf->kh, kw = psf->kw, ntaps = kh * kw;
  if (ntaps > kAdjMaxTaps || kh != 1) return DB_ERR_UNSUPPORTED;
  if ((size_t)N * H * W >= (size_t)1 << 31) return DB_ERR_SHAPE;
  const AdjLayout L = adj_layout(N, H, W, kw, ntaps, every);
  if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < L.total) return DB_ERR_WORKSPACE;
  char* base = (char*)ws;
  const size_t n = (size_t)N * H * W;  // all images, packed
  float* f0 = (float*)(base + L.f0);
  float* seg = (float*)(base + L.seg);
  float* b = (float*)(base + L.b);      // every x n (per iterate of a segment)
  float2* q = (float2*)(base + L.q);
  float2* ab = (float2*)(base + L.ab);
  float* g = (float*)(base + L.g);
  float* const L_b = b;
  float2* const L_q = q;
  float2* const L_ab = ab;
  float* const L_g = g;
  float* ubar = (float*)(base + L.ubar);
  float* uacc = (float*)(base + L.uacc);
  float2* abbar = (float2*)(base + L.abbar);
  float* dbar = (float*)(base + L.dbar);
  float2* qbar = (float2*)(base + L.qbar);
  float* bbar = (float*)(base + L.bbar);
  float* f0bar = (float*)(base + L.f0bar);
  float2* av = (float2*)(base + L.a);
  float* part = (float*)(base + L.part);
  float* wraw = (float*)(base + L.wraw);
  float2* prow = (float2*)(base + L.prow);
  double2* psum = (double2*)(base + L.psum);
  float4* spec = (float4*)(base + L.spec);
  float* unit_taps = (float*)(base + L.unit_taps);
  float4* unit_spec = (float4*)(base + L.unit_spec);
  float4* tabs = (float4*)(base + L.tabs);

  AdjImage im;
  im.N = N; im.H = H; im.W = W; im.taps = psf->taps; im.kh = kh; im.kw = kw;
  im.p.alpha = p->alpha; im.p.eps_phi = p->eps_phi; im.p.eps_psi = p->eps_psi; im.p.floor = p->pos_floor;
  im.p.phi_robust = p->phi_robust; im.p.psi_tv = p->psi_tv;
  im.p.rf_lut = nullptr;  // the reverse pass differentiates the log form
  const int G = kAdjBlocks, T = kAdjThreads;
  // row kernels (kw <= kAdjRowTaps): shared memory of the staged rows
  const size_t smab = (size_t)adj_row_pitch<kAdjRunFwd>(W) * kAdjRowBlock * 12;
  const size_t smrev = (size_t)adj_row_pitch<kAdjRunRev>(W) * kAdjRowBlock * 24;
  const bool rowk = kw <= kAdjRowTaps && smrev <= 227 * 1024;
  auto fwd_rows = k_adj_fwd_rows<32>;
  auto rev_rows = k_adj_rev_rows<32>;
  switch (row_taps_bucket(kw)) {
    case 8: fwd_rows = k_adj_fwd_rows<8>; rev_rows = k_adj_rev_rows<8>; break;
    case 16: fwd_rows = k_adj_fwd_rows<16>; rev_rows = k_adj_rev_rows<16>; break;
    case 24: fwd_rows = k_adj_fwd_rows<24>; rev_rows = k_adj_rev_rows<24>; break;
    default: break;
  }
  // row kernels: one wave of resident CTAs (their grid-stride loops give every
  // CTA the same number of row blocks; a partial second wave would run at a
  // fraction of the occupancy)
  int Gfwd = G, Grev = G;
  if (rowk) {
    if (smrev > 48 * 1024)
      ADJ_CHECK(cudaFuncSetAttribute(rev_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smrev));
    if (smab > 48 * 1024)
      ADJ_CHECK(cudaFuncSetAttribute(fwd_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smab));
    int dev = 0, sms = 0, of = 0, orv = 0;
    ADJ_CHECK(cudaGetDevice(&dev));
    ADJ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ADJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, fwd_rows, T, smab));
    ADJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&orv, rev_rows, T, smrev));
    if (of > 0) Gfwd = std::min(G, of * sms);
    if (orv > 0) Grev = std::min(G, orv * sms);
  }

  const size_t smdiff = diff_smem(W);
  if (smdiff > 48 * 1024 && smdiff <= 227 * 1024)
    ADJ_CHECK(cudaFuncSetAttribute(k_adj_rev_diff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smdiff));
  int Gfu = G;    // one resident wave, as for the row kernels
  {
    int dev = 0, sms = 0, ou = 0;
    ADJ_CHECK(cudaGetDevice(&dev));
    ADJ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ADJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ou, k_adj_fwd_update, T, 0));
    if (ou > 0) Gfu = std::min(G, ou * sms);
  }
  int Gdiff = G;  // one resident wave, as for the row kernels
  if (smdiff <= 227 * 1024) {
    int dev = 0, sms = 0, od = 0;
    ADJ_CHECK(cudaGetDevice(&dev));
    ADJ_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ADJ_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&od, k_adj_rev_diff, T, smdiff));
    if (od > 0) Gdiff = std::min(G, od * sms);
  }

  // pointwise copies treat the batch as one image of N*H rows (image stride H*ld)
  ADJ_LAUNCH(k_floor_pack<<<G, T, 0, s>>>(f, ld, N * H, W, p->pos_floor, f0));
  ADJ_LAUNCH(k_copy_pitched<<<G, T, 0, s>>>(grad_u, ld, ubar, W, N * H, W, nullptr, 0.f));
  ADJ_CHECK(cudaMemsetAsync(f0bar, 0, n * 4, s));

  const int nseg = iters > 0 ? (iters - 1) / every + 1 : 0;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * every, k1 = (k0 + every < iters) ? k0 + every : iters;
    // checkpoint sg of every image (ckpt is N x nseg x H x W)
    const size_t hw = (size_t)H * W;
    ADJ_CHECK(cudaMemcpy2DAsync(seg, hw * 4, ckpt + (size_t)sg * hw, (size_t)nseg * hw * 4, hw * 4, N,
                                cudaMemcpyDeviceToDevice, s));
    // the segment's iterates u_k and their intermediates b, q, (A, B), g
    for (int k = k0; k < k1; ++k) {
      float* uk = seg + (size_t)(k - k0) * n;
      const size_t z = (size_t)(k - k0) * n;
      if (rowk) {
        ADJ_LAUNCH(fwd_rows<<<Gfwd, T, smab, s>>>(uk, f0, im, b + z, q + z, ab + z, g + z));
      } else {
        ADJ_LAUNCH(k_adj_fwd_q<<<G, T, 0, s>>>(uk, f0, im, b + z, q + z));
        ADJ_LAUNCH(k_adj_fwd_ab<<<G, T, 0, s>>>(uk, q + z, im, ab + z, g + z));
      }
      if (k + 1 < k1) ADJ_LAUNCH(k_adj_fwd_update<<<Gfu, T, 0, s>>>(uk, ab + z, g + z, im, uk + n));
    }
    for (int k = k1 - 1; k >= k0; --k) {  // reverse steps
      const float* uk = seg + (size_t)(k - k0) * n;
      const size_t z = (size_t)(k - k0) * n;
      const float* b = L_b + z;
      const float2* q = L_q + z;
      const float2* ab = L_ab + z;
      const float* g = L_g + z;
      if (rowk) {
        ADJ_LAUNCH(rev_rows<<<Grev, T, smrev, s>>>(ubar, uk, ab, g, q, b, f0, im, uacc, dbar, f0bar, part));
        ADJ_LAUNCH(k_adj_reduce<<<1, T, 0, s>>>(part, 1, Grev, grad_alpha));
        ADJ_LAUNCH(k_adj_reduce<<<ntaps, T, 0, s>>>(part + Grev, ntaps, Grev, grad_taps));
      } else {
        ADJ_LAUNCH(k_adj_rev_update<<<G, T, 0, s>>>(ubar, uk, ab, g, im, uacc, abbar, dbar, part));
        ADJ_LAUNCH(k_adj_reduce<<<1, T, 0, s>>>(part, 1, G, grad_alpha));
        ADJ_LAUNCH(k_adj_rev_corrT<<<G, T, 0, s>>>(abbar, q, im, qbar, part));
        ADJ_LAUNCH(k_adj_reduce<<<ntaps, T, 0, s>>>(part, ntaps, G, grad_taps));
        ADJ_LAUNCH(k_adj_rev_weight<<<G, T, 0, s>>>(qbar, b, f0, im, bbar, f0bar));
        ADJ_LAUNCH(k_adj_rev_convT<<<G, T, 0, s>>>(bbar, uk, im, uacc, part));
        ADJ_LAUNCH(k_adj_reduce<<<ntaps, T, 0, s>>>(part, ntaps, G, grad_taps));
      }
      if (smdiff <= 227 * 1024) {
        ADJ_LAUNCH(k_adj_rev_diff<<<Gdiff, T, smdiff, s>>>(dbar, uk, g, im, uacc));
      } else {
        ADJ_LAUNCH(k_adj_rev_diff1<<<G, T, 0, s>>>(dbar, uk, g, im, uacc, av));
        ADJ_LAUNCH(k_adj_rev_diff2<<<G, T, 0, s>>>(av, im, uacc));
      }
      float* t = ubar; ubar = uacc; uacc = t;
    }
  }
  // Wiener step (row PSF): raw output w for the floor mask, then the adjoint
  Dft1ff D;
  ADJ_CHECK(prepare_dft(W, tabs, &D, nullptr, s));
  {
    WsLayout WL = {};
    // run_wiener needs spec and table regions: the spectrum region (W
    // float4) and the table region of this layout
    WL.spec = L.spec;
    WL.work = L.spec;  // not used for a one-row PSF
    WL.tw = L.tabs;
    WL.kspec = L.kspec;
    // a one-row PSF filters every row on its own: the batch is N*H rows
    ADJ_CHECK(run_wiener(f0, wraw, N * H, W, W, psf->taps, kh, kw, p->K, -FLT_MAX, ws, WL, status, s));
  }
  ADJ_LAUNCH(k_copy_pitched<<<G, T, 0, s>>>(ubar, W, uacc, W, N * H, W, wraw, p->pos_floor));
  ADJ_CHECK(psf_row_spectrum(psf->taps, kw, D, spec, s));
  ADJ_LAUNCH(k_unit_taps<<<(kw * kw + 255) / 256, 256, 0, s>>>(unit_taps, kw));
  for (int t = 0; t < kw; ++t) ADJ_CHECK(psf_row_spectrum(unit_taps + (size_t)t * kw, kw, D, unit_spec + (size_t)t * W, s));
  const int M = dft_len(D);
  const size_t smem = (size_t)2 * M * sizeof(float4);
  if (smem > 227 * 1024) return DB_ERR_UNSUPPORTED;
  const double invN = 1.0 / (double)W;
  const float2 invNf = make_float2((float)invN, (float)(invN - (double)(float)invN));
  if (smem > 48 * 1024) ADJ_CHECK(cudaFuncSetAttribute(k_adj_wiener_rows2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ADJ_LAUNCH(k_adj_wiener_rows2<<<(N * H + 1) / 2, 256, smem, s>>>(uacc, f0, W, N * H, spec, D, p->K, invNf, f0bar,
                                                                  prow));
  {
    const int nch = (N * H + kPsumRows - 1) / kPsumRows;
    double2* ppart = (double2*)(base + L.ppart);
    ADJ_LAUNCH(k_adj_psum_part<<<dim3((W + 255) / 256, nch), 256, 0, s>>>(prow, N * H, W, ppart));
    ADJ_LAUNCH(k_adj_psum<<<(W + 255) / 256, 256, 0, s>>>(ppart, nch, W, psum));
  }
  ADJ_LAUNCH(k_adj_wiener_params<<<kw + 1, 256, 0, s>>>(psum, spec, unit_spec, W, kw, p->K, grad_taps, grad_K));
  ADJ_LAUNCH(k_grad_f_out<<<G, T, 0, s>>>(f0bar, f, ld, N * H, W, p->pos_floor, grad_f));
  return DB_OK;
}

}  // namespace db

using namespace db;

extern "C" {

size_t db_backward_workspace_bytes(int H, int W, int batch, const db_psf* psf, int ckpt_every) {
  if (!psf || H < 1 || W < 1 || H > kMaxSide || W > kMaxSide || ckpt_every < 1 || batch < 1) return 0;
  if (psf->kh < 1 || psf->kw < 1 || psf->kh > H || psf->kw > W) return 0;
  return adj_ws_bytes(batch, H, W, psf->kh, psf->kw, ckpt_every);
}

db_status db_rrl_backward(const float* f, const float* ckpt, const float* grad_u, int H, int W, int ld,
                          int batch, const db_psf* psf, const db_params* p, int iters, int ckpt_every,
                          float* grad_f, double* grad_taps, double* grad_alpha, double* grad_K, void* ws,
                          size_t ws_bytes, int* dev_status, void* stream) {
  if (!f || !ckpt || !grad_u || !psf || !psf->taps || !p || !grad_f || !grad_taps || !grad_alpha || !grad_K)
    return DB_ERR_ARG;
  if (batch < 1) return DB_ERR_ARG;
  if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide || ld < W) return DB_ERR_SHAPE;
  if (psf->kh < 1 || psf->kw < 1 || psf->kh > H || psf->kw > W) return DB_ERR_PSF;
  if (iters < 0 || ckpt_every < 1) return DB_ERR_ARG;
  if (!(p->K > 0.f) || !(p->alpha >= 0.f) || !(p->eps_phi > 0.f) || !(p->eps_psi > 0.f) || !(p->pos_floor > 0.f))
    return DB_ERR_ARG;
  if (rf_mode() != DB_RF_LOG1P) return DB_ERR_UNSUPPORTED;  // table form has no derivative here
  if (p->conv != DB_CONV_CLAMP) return DB_ERR_UNSUPPORTED;
  return adj_backward(f, ld, batch, ckpt, iters, ckpt_every, grad_u, H, W, psf, p, grad_f, grad_taps,
                      grad_alpha, grad_K, ws, ws_bytes, dev_status, (cudaStream_t)stream);
}

}  // extern "C"
