// RRRL iteration with Fourier-domain (periodic) blur and correlation:
// Sec. 2.3, Eq. 9-12, with the convolutions of Sec. 4.1 ("Convolution")
// realised through the Fourier domain and periodic continuation (Sec. 4.2),
// the paper's general 2D variant (Sec. 4.3).
//
// Per iteration, with S = h^ (bit-reversed order, from the same transforms):
//   b      = IDFT(DFT(u) S)                      blur
//   e, W   = W (f - b)/b, W = phi'(r_f(b))       weighted residual (Eq. 7, 10)
//   Delta + iB = IDFT(DFT(e + iW) conj(S))       both correlations at once:
//                                                 h is real, so the real and
//                                                 imaginary parts stay apart
//   D      = div(psi' grad u)                    spatial, zero flux (Eq. 11)
//   u'     = u + u (Delta + alpha D)/(B - alpha [D]-)   (Eq. 9 in increment form)
// as four passes over complex buffers X, Z (H x W, row pitch W):
//   C1: columns of X: DIF, x S, DIT                 (X = row DIF of u)
//   R2: rows of X: DIT -> b; (e, W); DIF -> Z
//   C3: columns of Z: DIF, x conj(S), DIT
//   R4: rows of Z: DIT -> Delta, B; D from 5 rows of u; update -> u';
//       DIF of u' -> X for the next iteration
// plus one initial row pass R0 (DIF of u -> X).
#include <cuda_runtime.h>

#include "fft.cuh"
#include "fft8.cuh"
#include "internal.cuh"

namespace db {

enum FRowMode { FR_U = 0, FR_MID = 1, FR_FIN = 2 };

struct FourierArgs {
  const float* f; int ldf;
  const float* uin; int ldin;
  float* uout; int ldout;
  float2* X; float2* Z;      // complex buffers, pitch W
  const float2* S;           // PSF spectrum, column by column (element (k, c) at c H + k)
  const float2* twW;         // twiddle table for length W
  int H, W, logW, logH;
  float scale;               // 1/(H W)
  int write_next;            // R4: also produce X for the next iteration
  RrlParams p;
  int* status;
};

__device__ __forceinline__ float robust_weight_f(float b, float f, const RrlParams& p) {
  if (!p.phi_robust) return 1.0f;
  const float r = rf_divergence(b, f, p);
  return p.eps_phi * rsqrtf(fmaf(p.eps_phi, p.eps_phi, fmaxf(r, 0.0f)));  // explicit FMA: same rounding in every kernel shape
}

__device__ __forceinline__ float diffusivity_f(float gx, float gy, const RrlParams& p) {
  if (!p.psi_tv) return 1.0f;
  return rsqrtf(fmaf(gx, gx, fmaf(gy, gy, p.eps_psi * p.eps_psi)));
}

// One row of length W per CTA.  Every global input is staged with
// asynchronous copies before the transform.
template <int MODE>
__global__ void __launch_bounds__(256, 4) k_fourier_rows(FourierArgs a) {
  extern __shared__ float2 smem[];
  const int W = a.W;
  const float2* tw = a.twW;
  float2* x = smem;                            // padded layout: element c at x[fft_pad(c)]
  float* rs = (float*)(x + fft_padded(W));     // real rows: FR_U/FR_MID one row, FR_FIN rows i-2..i+2 of u
  const int i = blockIdx.x;
  if (MODE == FR_U) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) cp_async4(rs + c, a.uin + (size_t)i * a.ldin + c);
  } else if (MODE == FR_MID) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
      cp_async8(x + fft_pad(c), a.X + (size_t)i * W + c);
      cp_async4(rs + c, a.f + (size_t)i * a.ldf + c);
    }
  } else {
    for (int c = threadIdx.x; c < W; c += blockDim.x) cp_async8(x + fft_pad(c), a.Z + (size_t)i * W + c);
    for (int r = 0; r < 5; ++r) {
      const int gi = min(max(i - 2 + r, 0), a.H - 1);
      for (int c = threadIdx.x; c < W; c += blockDim.x) cp_async4(rs + r * W + c, a.uin + (size_t)gi * a.ldin + c);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (MODE == FR_U) {
    for (int c = threadIdx.x; c < W; c += blockDim.x) x[fft_pad(c)] = make_float2(rs[c], 0.f);
    __syncthreads();
    fft_dif_blk(x, a.logW, 1, 1, 0, tw, false);
    for (int c = threadIdx.x; c < W; c += blockDim.x) a.X[(size_t)i * W + c] = x[fft_pad(c)];
    return;
  }
  if (MODE == FR_MID) {
    fft_dit_inv_blk(x, a.logW, 1, 1, 0, tw, false);
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
      const float b = x[fft_pad(c)].x * a.scale;
      const float fv = fmaxf(rs[c], a.p.floor);
      const float w = robust_weight_f(b, fv, a.p);
      x[fft_pad(c)] = make_float2(__fdividef(w * (fv - b), b), w);
    }
    __syncthreads();
    fft_dif_blk(x, a.logW, 1, 1, 0, tw, false);
    for (int c = threadIdx.x; c < W; c += blockDim.x) a.Z[(size_t)i * W + c] = x[fft_pad(c)];
    return;
  }
  // FR_FIN
  fft_dit_inv_blk(x, a.logW, 1, 1, 0, tw, false);
  const RrlParams& p = a.p;
  for (int c = threadIdx.x; c < W; c += blockDim.x) {
    const int cw = max(c - 1, 0), ce = min(c + 1, W - 1);
    const int cww = max(c - 2, 0), cee = min(c + 2, W - 1);
    const float* n2 = rs;
    const float* n1 = rs + W;
    const float* m0 = rs + 2 * W;
    const float* s1 = rs + 3 * W;
    const float* s2 = rs + 4 * W;
    const float ctr = m0[c], e = m0[ce], w_ = m0[cw], n = n1[c], s = s1[c];
    const float gc = diffusivity_f(0.5f * (e - w_), 0.5f * (s - n), p);
    const float ge = diffusivity_f(0.5f * (m0[cee] - ctr), 0.5f * (s1[ce] - n1[ce]), p);
    const float gw = diffusivity_f(0.5f * (ctr - m0[cww]), 0.5f * (s1[cw] - n1[cw]), p);
    const float gs = diffusivity_f(0.5f * (s1[ce] - s1[cw]), 0.5f * (s2[c] - ctr), p);
    const float gn = diffusivity_f(0.5f * (n1[ce] - n1[cw]), 0.5f * (ctr - n2[c]), p);
    const float D = 0.5f * ((ge + gc) * (e - ctr) - (gc + gw) * (ctr - w_) + (gs + gc) * (s - ctr) -
                            (gc + gn) * (ctr - n));
    const float2 xv = x[fft_pad(c)];
    const float dl = xv.x * a.scale, B = xv.y * a.scale;
    const float den = B - p.alpha * fminf(D, 0.f);
    const float un = fmaf(ctr, __fdividef(fmaf(p.alpha, D, dl), den), ctr);
    if (!isfinite(un) && a.status) atomicOr(a.status, DB_FLAG_NONFINITE);
    a.uout[(size_t)i * a.ldout + c] = un;
    x[fft_pad(c)] = make_float2(un, 0.f);
  }
  if (!a.write_next) return;
  __syncthreads();
  fft_dif_blk(x, a.logW, 1, 1, 0, tw, false);
  for (int c = threadIdx.x; c < W; c += blockDim.x) a.X[(size_t)i * W + c] = x[fft_pad(c)];
}

// C adjacent columns per CTA: DIF, multiply by S (or conj S), DIT, in place.
// Shared layout: element k of column c at x[fft_pad(k) * C + c].
template <bool CONJ, int C>
__global__ void __launch_bounds__(256, 4) k_fourier_cols(float2* __restrict__ buf, const float2* __restrict__ S,
                                                      const float2* __restrict__ twH, int H, int W, int logH) {
  extern __shared__ float2 smem[];
  const float2* tw = twH;
  float2* x = smem;
  const int c0 = blockIdx.x * C;
  for (int idx = threadIdx.x; idx < H * C; idx += blockDim.x) {
    const int k = idx / C, c = idx - k * C;
    float2* d = x + fft_pad(k) * C + c;
    if (c0 + c < W) cp_async8(d, buf + (size_t)k * W + c0 + c);
    else *d = make_float2(0.f, 0.f);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_dif_blk(x, logH, C, C, 1, tw, true);
  // the spectrum in batches of kSBatch loads per thread, issued together
  constexpr int kSBatch = 8;
  for (int base = threadIdx.x; base < H * C; base += kSBatch * blockDim.x) {
    float2 sv[kSBatch];
#pragma unroll
    for (int t = 0; t < kSBatch; ++t) {
      const int idx = base + t * blockDim.x, k = idx / C, c = idx - k * C;
      sv[t] = (idx < H * C && c0 + c < W) ? __ldg(S + (size_t)(c0 + c) * H + k) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kSBatch; ++t) {
      const int idx = base + t * blockDim.x, k = idx / C, c = idx - k * C;
      if (idx < H * C && c0 + c < W) {
        float2* d = x + fft_pad(k) * C + c;
        *d = CONJ ? cmulc(*d, sv[t]) : cmul(*d, sv[t]);
      }
    }
  }
  __syncthreads();
  fft_dit_inv_blk(x, logH, C, C, 1, tw, true);
  for (int idx = threadIdx.x; idx < H * C; idx += blockDim.x) {
    const int k = idx / C, c = idx - k * C;
    if (c0 + c < W) buf[(size_t)k * W + c0 + c] = x[fft_pad(k) * C + c];
  }
}

// ---------------------------------------------------------------------------
// Register-resident passes (fft8.cuh) for sides 64..4096: the same four
// passes, with each transform's data in registers between shared-memory
// exchanges, the pointwise work done on the registers of the last inverse
// pass, and the column spectrum product between the forward and inverse
// bottom passes.  C = f8::seqs(L) rows or columns per CTA, thread t C + c.
//
// Layout of X and Z when both sides take these passes (PAIRS): column pairs,
// element (i, k) at float2 index ((k >> 1) H + i) 2 + (k & 1).  A column
// pass then reads and writes each pair of columns as one contiguous block,
// and a row pass moves 16 bytes per pair and row, which the CTA's other row
// completes to a full 32-byte sector.  Otherwise (one side below 64, whose
// passes are the shared-memory ones above) plain row-major, pitch W.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tv_pad(int C) { return C >= 32 ? 1 : 32 / C; }

// FR_U and FR_FIN (FR_MID runs in k_fourier_mid8 below)
template <int L, int MODE, bool PAIRS>
__global__ void __launch_bounds__(f8::threads(L), L >= 12 ? 1 : 2) k_fourier_rows8(FourierArgs a) {
  static_assert(MODE != FR_MID, "FR_MID runs in k_fourier_mid8");
  constexpr int C = f8::seqs(L), N = 1 << L, T = N / 8;
  constexpr int P = N + tv_pad(C);  // staged u rows (FR_FIN): conflict-free row pitch
  extern __shared__ float2 smem[];
  const int q = threadIdx.x % C, t = threadIdx.x / C;
  const int i0 = blockIdx.x * C, i = i0 + q;
  const bool ok = i < a.H;
  const int ic = ok ? i : a.H - 1;  // rows past the image load the last row and store nothing
  // float2 offset of elements (ic, 8t + 2u), (ic, 8t + 2u + 1): u_off(u)
  const size_t rbase = PAIRS ? ((size_t)(4 * t) * a.H + ic) * 2 : (size_t)ic * N + 8 * t;
  const size_t ustep = PAIRS ? (size_t)2 * a.H : 2;
  float* ust = (float*)(smem + C * f8::padded(N));  // FR_FIN: rows i0-2 .. i0+C+1 of u
  float2 v[8];
  if (MODE == FR_FIN) {
    const bool al = (a.ldin % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.uin) & 15) == 0);
    for (int rr = 0; rr < C + 4; ++rr) {
      const int gi = min(max(i0 - 2 + rr, 0), a.H - 1);
      const float* src = a.uin + (size_t)gi * a.ldin;
      float* dst = ust + rr * P;
      if (al && P % 4 == 0) {
        for (int c = 4 * threadIdx.x; c < N; c += 4 * blockDim.x) cp_async16(dst + c, src + c);
      } else {
        for (int c = threadIdx.x; c < N; c += blockDim.x) cp_async4(dst + c, src + c);
      }
    }
  }
  if (MODE == FR_U) {
    const float* ur = a.uin + (size_t)ic * a.ldin;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = make_float2(ur[t + T * r], 0.f);
  } else {
    const float2* src = a.Z + rbase;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 x = *(const float4*)(src + u * ustep);
      v[2 * u] = make_float2(x.x, x.y);
      v[2 * u + 1] = make_float2(x.z, x.w);
    }
    f8::dit_chain<L, f8::bottom_hb(L), C>(v, smem, t, q, a.twW);
    // v[r]: element t + T r, natural order
    const RrlParams& p = a.p;
    {
      cp_async_wait_all();
      __syncthreads();
      // rows ic-2 .. ic+2 of u: staged row rr holds image row
      // clamp(i0 - 2 + rr), so the edge rows repeat by themselves
      const float* m0 = ust + (ic - i0 + 2) * P;
      const float* n2 = m0 - 2 * P;
      const float* n1 = m0 - P;
      const float* s1 = m0 + P;
      const float* s2 = m0 + 2 * P;
      float* out = a.uout + (size_t)ic * a.ldout;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int c = t + T * r;
        const int cw = max(c - 1, 0), ce = min(c + 1, N - 1);
        const int cww = max(c - 2, 0), cee = min(c + 2, N - 1);
        const float ctr = m0[c], e = m0[ce], w_ = m0[cw], n = n1[c], s = s1[c];
        const float s1e = s1[ce], s1w = s1[cw], n1e = n1[ce], n1w = n1[cw];
        const float gc = diffusivity_f(0.5f * (e - w_), 0.5f * (s - n), p);
        const float ge = diffusivity_f(0.5f * (m0[cee] - ctr), 0.5f * (s1e - n1e), p);
        const float gw = diffusivity_f(0.5f * (ctr - m0[cww]), 0.5f * (s1w - n1w), p);
        const float gs = diffusivity_f(0.5f * (s1e - s1w), 0.5f * (s2[c] - ctr), p);
        const float gn = diffusivity_f(0.5f * (n1e - n1w), 0.5f * (ctr - n2[c]), p);
        const float D = 0.5f * ((ge + gc) * (e - ctr) - (gc + gw) * (ctr - w_) + (gs + gc) * (s - ctr) -
                                (gc + gn) * (ctr - n));
        const float dl = v[r].x * a.scale, B = v[r].y * a.scale;
        const float den = B - p.alpha * fminf(D, 0.f);
        const float un = fmaf(ctr, __fdividef(fmaf(p.alpha, D, dl), den), ctr);
        if (ok) {
          if (!isfinite(un) && a.status) atomicOr(a.status, DB_FLAG_NONFINITE);
          out[c] = un;
        }
        v[r] = make_float2(un, 0.f);
      }
      if (!a.write_next) return;  // the same for every thread of the launch
    }
  }
  int t2 = t;
  asm volatile("" : "+r"(t2));  // recompute the per-pass indices (keeps them out of the registers above)
  f8::dif_chain<L, L - 1, C>(v, smem, t2, q, a.twW);
  if (!ok) return;
  float2* dst = a.X + rbase;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *(float4*)(dst + u * ustep) = make_float4(v[2 * u].x, v[2 * u].y, v[2 * u + 1].x, v[2 * u + 1].y);
}

// FR_MID as a persistent kernel: CTA b takes row blocks b, b + gridDim.x, ...
// While a block is transformed, the next block's row spectra and rows of f
// are copied into shared memory, each thread copying exactly the elements
// it will read itself (so no barrier guards the buffer).
template <int L, bool PAIRS>
__global__ void __launch_bounds__(f8::threads(L), L >= 12 ? 1 : 2) k_fourier_mid8(FourierArgs a) {
  constexpr int C = f8::seqs(L), N = 1 << L, T = N / 8, NT = f8::threads(L);
  extern __shared__ float2 smem[];
  float4* pfx = (float4*)(smem + C * f8::padded(N));  // [4][NT]: the thread's 8 spectrum elements
  float* pff = (float*)(pfx + 4 * NT);                 // [8][NT]: the thread's 8 values of f
  const int tid = threadIdx.x, q = tid % C, t = tid / C;
  const int nrb = (a.H + C - 1) / C;
  const size_t ustep = PAIRS ? (size_t)2 * a.H : 2;
  // float2 offset of elements (ic, 8t), (ic, 8t + 1); + u ustep for 8t + 2u
  auto rowbase = [&](int ic) -> size_t {
    return PAIRS ? ((size_t)(4 * t) * a.H + ic) * 2 : (size_t)ic * N + 8 * t;
  };
  auto prefetch = [&](int rb) {
    const int ic = min(rb * C + q, a.H - 1);
    const float2* src = a.X + rowbase(ic);
#pragma unroll
    for (int u = 0; u < 4; ++u) cp_async16(pfx + u * NT + tid, src + u * ustep);
    const float* fr = a.f + (size_t)ic * a.ldf;
#pragma unroll
    for (int r = 0; r < 8; ++r) cp_async4(pff + r * NT + tid, fr + t + T * r);
  };
  int rb = blockIdx.x;
  if (rb < nrb) prefetch(rb);
  const RrlParams& p = a.p;
  for (; rb < nrb; rb += gridDim.x) {
    const int i = rb * C + q;
    cp_async_wait_all();
    float2 v[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float4 x = pfx[u * NT + tid];
      v[2 * u] = make_float2(x.x, x.y);
      v[2 * u + 1] = make_float2(x.z, x.w);
    }
    f8::dit_chain<L, f8::bottom_hb(L), C>(v, smem, t, q, a.twW);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const float b = v[r].x * a.scale;
      const float fv = fmaxf(pff[r * NT + tid], p.floor);
      const float w = robust_weight_f(b, fv, p);
      v[r] = make_float2(__fdividef(w * (fv - b), b), w);
    }
    if (rb + (int)gridDim.x < nrb) prefetch(rb + gridDim.x);
    int t2 = t;
    asm volatile("" : "+r"(t2));  // recompute the per-pass indices
    f8::dif_chain<L, L - 1, C>(v, smem, t2, q, a.twW);
    if (i < a.H) {
      float2* dst = a.Z + rowbase(i);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        *(float4*)(dst + u * ustep) = make_float4(v[2 * u].x, v[2 * u].y, v[2 * u + 1].x, v[2 * u + 1].y);
    }
  }
}

// C = f8::seqs(L) columns of length H = 2^L per CTA: DIF, x S (or conj S)
// on the bottom pass's registers, DIT, in place.
template <int L, bool CONJ, bool PAIRS>
__global__ void __launch_bounds__(f8::threads(L), L >= 12 ? 1 : 2)
    k_fourier_cols8(float2* __restrict__ buf, const float2* __restrict__ S, const float2* __restrict__ twH, int W) {
  constexpr int C = f8::seqs(L), H = 1 << L, T = H / 8;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % C, t = threadIdx.x / C;
  const int col = blockIdx.x * C + c;
  const bool ok = col < W;
  const int cc = ok ? col : W - 1;
  // element (k, cc) at off + k kstep; 32-bit offsets (H W <= 2^24), so that
  // no 64-bit address has to live across the transforms
  int off = PAIRS ? (cc >> 1) * 2 * H + 2 * t + (cc & 1) : t * W + cc;
  const int kstep = PAIRS ? 2 * T : T * W;
  float2 v[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = buf[off + r * kstep];
  f8::dif_chain<L, L - 1, C>(v, smem, t, c, twH);
  const float4* s4 = (const float4*)(S + (size_t)cc * H + 8 * t);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 sv = __ldg(s4 + u);
    const float2 s0 = make_float2(sv.x, sv.y), s1 = make_float2(sv.z, sv.w);
    v[2 * u] = CONJ ? cmulc(v[2 * u], s0) : cmul(v[2 * u], s0);
    v[2 * u + 1] = CONJ ? cmulc(v[2 * u + 1], s1) : cmul(v[2 * u + 1], s1);
  }
  int t2 = t;
  asm volatile("" : "+r"(t2));  // recompute the per-pass indices (keeps them out of the registers above)
  f8::dit_chain<L, f8::bottom_hb(L), C>(v, smem, t2, c, twH);
  if (!ok) return;
  asm volatile("" : "+r"(off));  // recompute the addresses rather than keep the loads' ones live
#pragma unroll
  for (int r = 0; r < 8; ++r) buf[off + r * kstep] = v[r];
}

template <typename K>
static cudaError_t set_smem_f(K kern, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <int L, int MODE, bool PAIRS>
static cudaError_t launch_frow8(const FourierArgs& a, cudaStream_t s) {
  constexpr int C = f8::seqs(L), N = 1 << L;
  size_t smem = (size_t)C * f8::padded(N) * sizeof(float2);
  if (MODE == FR_FIN) smem += (size_t)(C + 4) * (N + tv_pad(C)) * sizeof(float);
  cudaError_t e = set_smem_f(k_fourier_rows8<L, MODE, PAIRS>, smem);
  if (e != cudaSuccess) return e;
  k_fourier_rows8<L, MODE, PAIRS><<<(a.H + C - 1) / C, f8::threads(L), smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

// grid of a persistent kernel: as many CTAs as fit on the device at once
// (at most `items`); the occupancy query is made once per kernel
template <typename K>
static cudaError_t persistent_grid(K kern, int threads, size_t smem, int items, int* cache, int* grid) {
  if (*cache == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess)
      return e;
    *cache = max(1, sms * per_sm);
  }
  *grid = min(items, *cache);
  return cudaSuccess;
}

template <int L, bool PAIRS>
static cudaError_t launch_fmid8(const FourierArgs& a, cudaStream_t s) {
  constexpr int C = f8::seqs(L), N = 1 << L, NT = f8::threads(L);
  const size_t smem = (size_t)C * f8::padded(N) * sizeof(float2) + (size_t)NT * (4 * sizeof(float4) + 8 * sizeof(float));
  static int cache = 0;
  cudaError_t e = set_smem_f(k_fourier_mid8<L, PAIRS>, smem);
  int grid = 0;
  if (e == cudaSuccess) e = persistent_grid(k_fourier_mid8<L, PAIRS>, NT, smem, (a.H + C - 1) / C, &cache, &grid);
  if (e != cudaSuccess) return e;
  k_fourier_mid8<L, PAIRS><<<grid, NT, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int L, bool CONJ, bool PAIRS>
static cudaError_t launch_fcol8(float2* buf, const float2* S, const float2* twH, int W, cudaStream_t s) {
  constexpr int C = f8::seqs(L);
  const size_t smem = (size_t)C * f8::padded(1 << L) * sizeof(float2);
  cudaError_t e = set_smem_f(k_fourier_cols8<L, CONJ, PAIRS>, smem);
  if (e != cudaSuccess) return e;
  k_fourier_cols8<L, CONJ, PAIRS><<<(W + C - 1) / C, f8::threads(L), smem, s>>>(buf, S, twH, W);
  count_launch();
  return cudaGetLastError();
}

// both sides take the register-resident passes: X and Z in column pairs
static bool fourier_pairs(int H, int W) { return ilog2(H) >= 6 && ilog2(W) >= 6; }

template <int L, int MODE>
static cudaError_t launch_frow8p(const FourierArgs& a, cudaStream_t s) {
  if constexpr (MODE == FR_MID)
    return fourier_pairs(a.H, a.W) ? launch_fmid8<L, true>(a, s) : launch_fmid8<L, false>(a, s);
  else
    return fourier_pairs(a.H, a.W) ? launch_frow8<L, MODE, true>(a, s) : launch_frow8<L, MODE, false>(a, s);
}
template <int L, bool CONJ>
static cudaError_t launch_fcol8p(float2* buf, const float2* S, const float2* twH, int H, int W, cudaStream_t s) {
  return fourier_pairs(H, W) ? launch_fcol8<L, CONJ, true>(buf, S, twH, W, s)
                             : launch_fcol8<L, CONJ, false>(buf, S, twH, W, s);
}

template <int MODE>
static cudaError_t launch_frow(const FourierArgs& a, cudaStream_t s) {
  switch (a.logW) {
    case 6: return launch_frow8p<6, MODE>(a, s);
    case 7: return launch_frow8p<7, MODE>(a, s);
    case 8: return launch_frow8p<8, MODE>(a, s);
    case 9: return launch_frow8p<9, MODE>(a, s);
    case 10: return launch_frow8p<10, MODE>(a, s);
    case 11: return launch_frow8p<11, MODE>(a, s);
    case 12: return launch_frow8p<12, MODE>(a, s);
    default: break;
  }
  const size_t smem = (size_t)fft_padded(a.W) * sizeof(float2) + (size_t)(MODE == FR_FIN ? 5 : 1) * a.W * sizeof(float);
  cudaError_t e = set_smem_f(k_fourier_rows<MODE>, smem);
  if (e != cudaSuccess) return e;
  k_fourier_rows<MODE><<<a.H, 256, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <bool CONJ>
static cudaError_t launch_fcol(float2* buf, const float2* S, const float2* twH, int H, int W, cudaStream_t s) {
  const int logH = ilog2(H);
  switch (logH) {
    case 6: return launch_fcol8p<6, CONJ>(buf, S, twH, H, W, s);
    case 7: return launch_fcol8p<7, CONJ>(buf, S, twH, H, W, s);
    case 8: return launch_fcol8p<8, CONJ>(buf, S, twH, H, W, s);
    case 9: return launch_fcol8p<9, CONJ>(buf, S, twH, H, W, s);
    case 10: return launch_fcol8p<10, CONJ>(buf, S, twH, H, W, s);
    case 11: return launch_fcol8p<11, CONJ>(buf, S, twH, H, W, s);
    case 12: return launch_fcol8p<12, CONJ>(buf, S, twH, H, W, s);
    default: break;
  }
  if (H <= 1024) {
    constexpr int C = 4;
    const size_t smem = (size_t)C * fft_padded(H) * sizeof(float2);
    cudaError_t e = set_smem_f(k_fourier_cols<CONJ, C>, smem);
    if (e != cudaSuccess) return e;
    k_fourier_cols<CONJ, C><<<(W + C - 1) / C, 256, smem, s>>>(buf, S, twH, H, W, logH);
  } else {
    constexpr int C = 2;
    const size_t smem = (size_t)C * fft_padded(H) * sizeof(float2);
    cudaError_t e = set_smem_f(k_fourier_cols<CONJ, C>, smem);
    if (e != cudaSuccess) return e;
    k_fourier_cols<CONJ, C><<<(W + C - 1) / C, 256, smem, s>>>(buf, S, twH, H, W, logH);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t run_rrl_fourier(const float* f, int ldf, float* u, int ld, float* utmp, int H, int W,
                            float2* X, float2* Z, const float2* S, const float2* twW,
                            const float2* twH, const RrlParams& p, int iters, float* ckpt,
                            int ckpt_every, int* status, cudaStream_t s) {
  FourierArgs a = {};
  a.f = f; a.ldf = ldf; a.X = X; a.Z = Z; a.S = S; a.twW = twW;
  a.H = H; a.W = W; a.logW = ilog2(W); a.logH = ilog2(H);
  a.scale = 1.0f / ((float)H * (float)W);
  a.p = p; a.status = status;
  cudaError_t e;
  a.uin = u; a.ldin = ld;
  if ((e = launch_frow<FR_U>(a, s)) != cudaSuccess) return e;
  const float* src = u;
  int ld_src = ld;
  for (int k = 0; k < iters; ++k) {
    if (ckpt && k % ckpt_every == 0) {
      float* dst = ckpt + (size_t)(k / ckpt_every) * H * W;
      if ((e = cudaMemcpy2DAsync(dst, (size_t)W * sizeof(float), src, (size_t)ld_src * sizeof(float),
                                 (size_t)W * sizeof(float), H, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    }
    float* dst = (k % 2 == 0) ? utmp : u;
    const int ld_dst = (k % 2 == 0) ? W : ld;
    if ((e = launch_fcol<false>(X, S, twH, H, W, s)) != cudaSuccess) return e;
    a.uin = src; a.ldin = ld_src;
    if ((e = launch_frow<FR_MID>(a, s)) != cudaSuccess) return e;
    if ((e = launch_fcol<true>(Z, S, twH, H, W, s)) != cudaSuccess) return e;
    a.uout = dst; a.ldout = ld_dst; a.write_next = (k + 1 < iters);
    if ((e = launch_frow<FR_FIN>(a, s)) != cudaSuccess) return e;
    src = dst;
    ld_src = ld_dst;
  }
  if (src != u) {
    if ((e = cudaMemcpy2DAsync(u, (size_t)ld * sizeof(float), src, (size_t)W * sizeof(float),
                               (size_t)W * sizeof(float), H, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace db
