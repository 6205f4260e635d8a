// Shared-memory FP32 FFT building blocks (power-of-two lengths, and
// Bluestein's chirp-z form for other lengths).
//
// The Wiener filter (Sec. 2.1, Eq. 2) and the Fourier-mode blur/correlation
// (Sec. 4.1, "Fourier transform"; Sec. 4.3) only ever use a transform to
// multiply by a spectrum and transform back.  The forward transform is
// therefore a decimation-in-frequency (DIF) sweep that leaves its output in
// bit-reversed order, and the inverse a decimation-in-time (DIT) sweep that
// takes bit-reversed input and returns natural order: no reordering pass is
// ever needed, provided the spectrum multiplied in between went through the
// same forward sweep (it does: PSF spectra are computed with these routines).
//
// Pairs of radix-2 stages are fused into one radix-2^2 butterfly held in
// registers, halving the shared-memory sweeps.  Twiddles come from a table
// tw[k] = exp(-2 pi i k / NT) in global memory (computed once per call in
// double precision), read through the read-only cache.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace db {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
// multiply by +i
__device__ __forceinline__ float2 cmul_pi(float2 a) { return make_float2(-a.y, a.x); }

// Work item -> (sequence q, item b) with shifts: nseq = 2^lns sequences of
// 2^lnb items each (both powers of two in every sweep below).
__device__ __forceinline__ void split_item(int it, int lns, int lnb, bool seq_fast, int& q, int& b) {
  if (seq_fast) { q = it & ((1 << lns) - 1); b = it >> lns; }
  else { q = it >> lnb; b = it & ((1 << lnb) - 1); }
}

// Forward DIF transform of `nseq` sequences of length N = 2^logN held in
// shared memory: element k of sequence q is x[q*ss + k*es].  Output is in
// bit-reversed order.  `seq_fast` chooses the thread->work mapping: true when
// sequences are interleaved element-wise (columns), false when each sequence
// is contiguous (rows).  tw is a table for length NT = N << tw_shift.
// Ends with __syncthreads().
__device__ inline void fft_dif(float2* x, int logN, int nseq, int es, int ss, const float2* tw,
                               int tw_shift, bool seq_fast) {
  const int N = 1 << logN, lns = 31 - __clz(nseq);  // nseq: a power of two
  const int nb = N >> 2;  // radix-4 butterflies per sequence
  int logLen = logN;
  while (logLen >= 2) {
    const int len = 1 << logLen, m = len >> 2, logm = logLen - 2;
    const int tstep = 1 << (logN - logLen + tw_shift);  // NT / len
    const int items = nseq * nb;
    if (m == 1) {  // blocks of 4: every twiddle is 1
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int q, b;
        split_item(it, lns, logN - 2, seq_fast, q, b);
        float2* p = x + q * ss + (b * 4) * es;
        float2 x0 = p[0], x1 = p[es], x2 = p[2 * es], x3 = p[3 * es];
        float2 y0 = cadd(x0, x2), y2 = csub(x0, x2);
        float2 y1 = cadd(x1, x3), y3 = cmul_mi(csub(x1, x3));
        p[0] = cadd(y0, y1);
        p[es] = csub(y0, y1);
        p[2 * es] = cadd(y2, y3);
        p[3 * es] = csub(y2, y3);
      }
      __syncthreads();
      logLen -= 2;
      continue;
    }
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      int q, b;
      split_item(it, lns, logN - 2, seq_fast, q, b);
      const int blk = b >> logm, j = b & (m - 1);
      float2* p = x + q * ss + (blk * len + j) * es;
      const int sm = m * es;
      float2 x0 = p[0], x1 = p[sm], x2 = p[2 * sm], x3 = p[3 * sm];
      const float2 w1 = __ldg(tw + j * tstep), w2 = __ldg(tw + 2 * j * tstep);
      float2 y0 = cadd(x0, x2), y2 = cmul(csub(x0, x2), w1);
      float2 y1 = cadd(x1, x3), y3 = cmul_mi(cmul(csub(x1, x3), w1));
      p[0] = cadd(y0, y1);
      p[sm] = cmul(csub(y0, y1), w2);
      p[2 * sm] = cadd(y2, y3);
      p[3 * sm] = cmul(csub(y2, y3), w2);
    }
    __syncthreads();
    logLen -= 2;
  }
  if (logLen == 1) {  // last radix-2 stage, blocks of length 2, twiddle 1
    const int items = nseq * (N >> 1);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      int q, b;
      split_item(it, lns, logN - 1, seq_fast, q, b);
      float2* p = x + q * ss + (2 * b) * es;
      float2 a = p[0], c = p[es];
      p[0] = cadd(a, c);
      p[es] = csub(a, c);
    }
    __syncthreads();
  }
}

// Inverse DIT transform (unnormalised: returns N times the inverse DFT),
// taking bit-reversed input to natural order.  Exactly mirrors fft_dif.
// Ends with __syncthreads().
__device__ inline void fft_dit_inv(float2* x, int logN, int nseq, int es, int ss, const float2* tw,
                                   int tw_shift, bool seq_fast) {
  const int N = 1 << logN, lns = 31 - __clz(nseq);  // nseq: a power of two
  const int nb = N >> 2;
  int logLen = (logN & 1) ? 1 : 0;
  if (logLen == 1) {
    const int items = nseq * (N >> 1);
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      int q, b;
      split_item(it, lns, logN - 1, seq_fast, q, b);
      float2* p = x + q * ss + (2 * b) * es;
      float2 a = p[0], c = p[es];
      p[0] = cadd(a, c);
      p[es] = csub(a, c);
    }
    __syncthreads();
  }
  for (logLen += 2; logLen <= logN; logLen += 2) {
    const int len = 1 << logLen, m = len >> 2, logm = logLen - 2;
    const int tstep = 1 << (logN - logLen + tw_shift);
    const int items = nseq * nb;
    if (m == 1) {  // blocks of 4: every twiddle is 1
      for (int it = threadIdx.x; it < items; it += blockDim.x) {
        int q, b;
        split_item(it, lns, logN - 2, seq_fast, q, b);
        float2* p = x + q * ss + (b * 4) * es;
        float2 z0 = p[0], z1 = p[es], z2 = p[2 * es], z3 = p[3 * es];
        float2 y0 = cadd(z0, z1), y1 = csub(z0, z1);
        float2 y2 = cadd(z2, z3), u3 = cmul_pi(csub(z2, z3));
        p[0] = cadd(y0, y2);
        p[2 * es] = csub(y0, y2);
        p[es] = cadd(y1, u3);
        p[3 * es] = csub(y1, u3);
      }
      __syncthreads();
      continue;
    }
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      int q, b;
      split_item(it, lns, logN - 2, seq_fast, q, b);
      const int blk = b >> logm, j = b & (m - 1);
      float2* p = x + q * ss + (blk * len + j) * es;
      const int sm = m * es;
      float2 z0 = p[0], z1 = p[sm], z2 = p[2 * sm], z3 = p[3 * sm];
      const float2 w1 = __ldg(tw + j * tstep), w2 = __ldg(tw + 2 * j * tstep);
      float2 t1 = cmulc(z1, w2), t3 = cmulc(z3, w2);
      float2 y0 = cadd(z0, t1), y1 = csub(z0, t1);
      float2 y2 = cadd(z2, t3), y3 = csub(z2, t3);
      float2 u2 = cmulc(y2, w1), u3 = cmul_pi(cmulc(y3, w1));
      p[0] = cadd(y0, u2);
      p[2 * sm] = csub(y0, u2);
      p[sm] = cadd(y1, u3);
      p[3 * sm] = csub(y1, u3);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Register-blocked form of the same transforms.  The radix-2 stages are taken
// in blocks of up to four: a work item loads the 2^NB elements whose indices
// differ only in the block's bits, runs the block's stages in registers and
// stores them back, so a length-2048 transform makes three shared-memory
// sweeps.  Each stage is the plain radix-2 DIF butterfly
//   a' = a + c,  c' = (a - c) w^e,  e = (i mod h) 2^s   (stage s, span h),
// and the inverse runs the mirrored butterflies a + c conj(w^e), a - c conj(w^e)
// in the reverse stage order (unnormalised inverse): storage orders are those
// of fft_dif / fft_dit_inv (bit-reversed spectra).
//
// Shared layout: element k of a sequence sits at fft_pad(k) = k + k/16 (one
// gap every 16 elements), so the strided loads of every block spread over
// the banks.  A sequence of length N needs fft_padded(N) slots.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int fft_pad(int k) { return k + (k >> 4); }
constexpr int kFftBlock = 3;  // stages per shared sweep (register block of 2^3 elements)
__host__ __device__ __forceinline__ int fft_padded(int n) { return n + (n >> 4); }

template <int NB, bool INV>
__device__ __forceinline__ void fft_block(float2* x, int logN, int hb, int nseq, int es, int ss,
                                          const float2* __restrict__ tw, bool seq_fast) {
  constexpr int R = 1 << NB;
  const int lo = hb - NB + 1, lowmask = (1 << lo) - 1;
  const int lns = 31 - __clz(nseq), lng = logN - NB;
  const int items = nseq << lng;
  const int s0 = logN - 1 - hb;  // stage of the block's top bit
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    int q, g;
    split_item(it, lns, lng, seq_fast, q, g);
    const int base = ((g >> lo) << (hb + 1)) | (g & lowmask);
    float2* p = x + q * ss;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = p[fft_pad(base + (r << lo)) * es];
    const int bl = base & lowmask;
    if (!INV) {
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        const int rb = NB - 1 - k, s = s0 + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r & (1 << rb)) continue;
          const float2 a = v[r], c = v[r + (1 << rb)];
          const int e = (bl + ((r & ((1 << rb) - 1)) << lo)) << s;
          v[r] = cadd(a, c);
          v[r + (1 << rb)] = cmul(csub(a, c), __ldg(tw + e));
        }
      }
    } else {
#pragma unroll
      for (int k = NB - 1; k >= 0; --k) {
        const int rb = NB - 1 - k, s = s0 + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r & (1 << rb)) continue;
          const float2 a = v[r];
          const int e = (bl + ((r & ((1 << rb) - 1)) << lo)) << s;
          const float2 t = cmulc(v[r + (1 << rb)], __ldg(tw + e));
          v[r] = cadd(a, t);
          v[r + (1 << rb)] = csub(a, t);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) p[fft_pad(base + (r << lo)) * es] = v[r];
  }
  __syncthreads();
}

// Forward DIF (output bit-reversed) on the padded layout: element k of
// sequence q at x[q*ss + fft_pad(k)*es].  nseq: a power of two.  Ends with a
// barrier.
__device__ inline void fft_dif_blk(float2* x, int logN, int nseq, int es, int ss, const float2* __restrict__ tw,
                                   bool seq_fast) {
  for (int hb = logN - 1; hb >= 0;) {
    const int nb = hb + 1 < kFftBlock ? hb + 1 : kFftBlock;
    switch (nb) {
      case 4: fft_block<4, false>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
      case 3: fft_block<3, false>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
      case 2: fft_block<2, false>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
      default: fft_block<1, false>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
    }
    hb -= nb;
  }
}

// Inverse (unnormalised) from bit-reversed to natural order, padded layout.
__device__ inline void fft_dit_inv_blk(float2* x, int logN, int nseq, int es, int ss,
                                       const float2* __restrict__ tw, bool seq_fast) {
  for (int lo = 0; lo < logN;) {
    const int nb = logN - lo < kFftBlock ? logN - lo : kFftBlock;
    const int hb = lo + nb - 1;
    switch (nb) {
      case 4: fft_block<4, true>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
      case 3: fft_block<3, true>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
      case 2: fft_block<2, true>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
      default: fft_block<1, true>(x, logN, hb, nseq, es, ss, tw, seq_fast); break;
    }
    lo += nb;
  }
}

}  // namespace db
