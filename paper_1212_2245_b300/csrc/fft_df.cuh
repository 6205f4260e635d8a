// Float-float ("double-single") FFT building blocks for the Wiener filter.
//
// The RRRL update is multiplicative, so a pixel whose Wiener value is small
// carries its relative error through every iteration while its value grows.
// An FP32 transform leaves absolute errors of ~1e-4 grey levels everywhere,
// which dark pixels turn into relative errors of 1e-4..1e-3.  Carrying every
// value of the Wiener transforms as an unevaluated sum hi + lo of two floats
// (about 44 significant bits) and rounding once at the end makes the output
// error relative (half an FP32 ulp) instead.
//
// A complex value is a float4 (re.hi, re.lo, im.hi, im.lo).  Addition uses
// Knuth's two-sum, multiplication the FMA-based exact product (Dekker/Knuth
// error-free transformations), each followed by a renormalising fast
// two-sum.  The sweep structure (DIF forward to bit-reversed order, DIT
// inverse back, radix-4 butterflies, Bluestein for other lengths) is the
// same as in fft.cuh.  Twiddle and chirp tables are float-float too and are
// read from global memory (they stay in L1/L2).
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace db {

// ---- real float-float arithmetic (value = x + y, |y| <= ulp(x)/2) ----------
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return make_float2(s, b - (s - a));
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float s = a.x + b.x;
  const float bb = s - a.x;
  const float e = (a.x - (s - bb)) + (b.x - bb) + (a.y + b.y);
  return ff_fast_two_sum(s, e);
}
__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return ff_fast_two_sum(p, e);
}
// a / b, one Newton-style correction of the float quotient
__device__ __forceinline__ float2 ff_div(float2 a, float2 b) {
  const float q1 = a.x / b.x;
  const float2 r = ff_sub(a, ff_mul(b, make_float2(q1, 0.f)));
  const float q2 = r.x / b.x;
  return ff_fast_two_sum(q1, q2);
}

// ---- complex float-float ---------------------------------------------------
__device__ __forceinline__ float2 re_(float4 z) { return make_float2(z.x, z.y); }
__device__ __forceinline__ float2 im_(float4 z) { return make_float2(z.z, z.w); }
__device__ __forceinline__ float4 mkc(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float4 zadd(float4 a, float4 b) { return mkc(ff_add(re_(a), re_(b)), ff_add(im_(a), im_(b))); }
__device__ __forceinline__ float4 zsub(float4 a, float4 b) { return mkc(ff_sub(re_(a), re_(b)), ff_sub(im_(a), im_(b))); }
// a0 b0 + a1 b1 for float-float a0, b0, a1, b1 with one renormalisation:
// the two high products and their exact rounding errors (FMA), Knuth's
// two-sum of the high products, and the cross terms a.hi b.lo + a.lo b.hi
// gathered by FMA into the low word (the lo * lo terms, below 2^-48 of the
// products, are dropped, as in ff_mul).  About 18 operations against 25 for
// ff_add(ff_mul, ff_mul) at the same accuracy class (a few units of 2^-46).
__device__ __forceinline__ float2 ff_dot2(float2 a0, float2 b0, float2 a1, float2 b1) {
  const float p0 = a0.x * b0.x, p1 = a1.x * b1.x;
  const float e0 = fmaf(a0.x, b0.x, -p0), e1 = fmaf(a1.x, b1.x, -p1);
  const float s = p0 + p1;
  const float bb = s - p0;
  float lo = (p0 - (s - bb)) + (p1 - bb);
  lo += e0 + e1;
  lo = fmaf(a0.x, b0.y, lo);
  lo = fmaf(a0.y, b0.x, lo);
  lo = fmaf(a1.x, b1.y, lo);
  lo = fmaf(a1.y, b1.x, lo);
  return ff_fast_two_sum(s, lo);
}
__device__ __forceinline__ float4 zmul(float4 a, float4 b) {
  return mkc(ff_dot2(re_(a), re_(b), ff_neg(im_(a)), im_(b)), ff_dot2(re_(a), im_(b), im_(a), re_(b)));
}
// a * conj(b)
__device__ __forceinline__ float4 zmulc(float4 a, float4 b) {
  return mkc(ff_dot2(re_(a), re_(b), im_(a), im_(b)), ff_dot2(im_(a), re_(b), ff_neg(re_(a)), im_(b)));
}
__device__ __forceinline__ float4 zmul_mi(float4 a) { return make_float4(a.z, a.w, -a.x, -a.y); }  // * (-i)
__device__ __forceinline__ float4 zmul_pi(float4 a) { return make_float4(-a.z, -a.w, a.x, a.y); }  // * (+i)
__device__ __forceinline__ float4 zconj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 zscale(float4 a, float2 s) { return mkc(ff_mul(re_(a), s), ff_mul(im_(a), s)); }
__device__ __forceinline__ float4 zzero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
// a / 2: exact on both words (no renormalisation needed)
__device__ __forceinline__ float4 zhalf(float4 a) { return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w); }

// A 1D DFT of length N in float-float.  A power of two N is transformed
// directly (M = N); any other N by Bluestein's chirp-z form as a circular
// convolution of length M = 2^logM 3^M3 >= 2N - 1 (the smallest such number,
// so that the convolution is at most about 1.125 times longer than needed;
// a power of two alone would be up to twice as long).
struct Dft1ff {
  int N, logM, M3;   // M = 2^logM * 3^M3 (M3 = 0 for power-of-two N)
  float2 invM;       // 1/M, float-float
  const float4* tw;  // exp(-2 pi i k / M), k < M
  const float4* c;   // chirp, nullptr for power-of-two N
  const float4* Bf;  // transform of the circular chirp
};
__host__ __device__ inline int pow3i(int b) {
  int r = 1;
  while (b-- > 0) r *= 3;
  return r;
}
// Transform length M of D (the capacity every sequence needs).
__host__ __device__ inline int dft_len(const Dft1ff& D) { return (1 << D.logM) * pow3i(D.M3); }

// Host-side state of a prepared Wiener filter (tables and spectrum live in
// the workspace).
struct WienerState {
  int H, W, kh, kw;
  Dft1ff DW, DH;
  const float4* kspec = nullptr;  // filter spectra of the filtering passes (non-power-of-two axis), or null
};

// Quotient and remainder of 0 <= n < 2^24 by a divisor 1 <= d < 2^24 fixed
// for a loop, through a float reciprocal formed once: the product n (1/d)
// is within one of n / d, and one step on the remainder makes it exact.
// Here n counts the items of one CTA's sequences, which live in its shared
// memory (at most 227 KB / 16 B per float-float element), so n < 2^24.
struct DivBy {
  float r;
  int d;
};
__device__ __forceinline__ DivBy div_by(int d) { return DivBy{__frcp_rn((float)d), d}; }
__device__ __forceinline__ int div_q(int n, const DivBy& v, int& rem) {
  int q = __float2int_rz((float)n * v.r);
  rem = n - q * v.d;
  if (rem < 0) { --q; rem += v.d; }
  else if (rem >= v.d) { ++q; rem -= v.d; }
  return q;
}

// Item `it` of nseq sequences of len items: sequence q, item k (seq_fast:
// consecutive items in consecutive sequences; the column kernels' nseq is a
// compile-time power of two there).  dv = div_by(len).
__device__ __forceinline__ void seq_item_ff(int it, int nseq, const DivBy& dv, bool seq_fast, int& q, int& k) {
  if (seq_fast) { q = it % nseq; k = it / nseq; }
  else q = div_q(it, dv, k);
}
// The same with shifts: nseq = 2^lns sequences of 2^lnb items each.
__device__ __forceinline__ void split_item_ff(int it, int lns, int lnb, bool seq_fast, int& q, int& b) {
  if (seq_fast) { q = it & ((1 << lns) - 1); b = it >> lns; }
  else { q = it >> lnb; b = it & ((1 << lnb) - 1); }
}

// Item `it` of nseq (a power of two, 2^lns) sequences x nsub contiguous
// sub-blocks x 2^lnb items: sequence q, sub-block u, item b.
// dv = div_by(nsub << lnb) (used when nsub > 1 and not seq_fast).
__device__ __forceinline__ void sub_item_ff(int it, int lns, int nsub, int lnb, bool seq_fast, const DivBy& dv,
                                            int& q, int& u, int& b) {
  int r;
  if (seq_fast) { q = it & ((1 << lns) - 1); r = it >> lns; }
  else if (nsub == 1) { q = it >> lnb; r = it - (q << lnb); }
  else q = div_q(it, dv, r);
  u = r >> lnb;
  b = r & ((1 << lnb) - 1);
}

// Forward DIF sweep (output bit-reversed) of length 2^logN on each of nsub
// contiguous sub-blocks of every sequence; the twiddle of exponent e is
// tw[e * twmul] (tw: a table for length 2^logN * twmul).  Ends with a barrier.
__device__ inline void fft_dif_ff(float4* x, int logN, int nseq, int es, int ss, const float4* __restrict__ tw,
                                  bool seq_fast, int nsub = 1, int twmul = 1) {
  const int N = 1 << logN, lns = 31 - __clz(nseq);  // nseq: a power of two
  const DivBy dv2 = div_by(logN >= 2 ? nsub << (logN - 2) : 1), dv1 = div_by(logN >= 1 ? nsub << (logN - 1) : 1);
  const int nb = N >> 2;
  int logLen = logN;
  while (logLen >= 2) {
    const int len = 1 << logLen, m = len >> 2, logm = logLen - 2;
    const int tstep = (1 << (logN - logLen)) * twmul;
    if (m == 1) {  // blocks of 4: every twiddle is 1
      for (int it = threadIdx.x; it < nseq * nsub * nb; it += blockDim.x) {
        int q, u, b;
        sub_item_ff(it, lns, nsub, logN - 2, seq_fast, dv2, q, u, b);
        float4* p = x + q * ss + ((u << logN) + b * 4) * es;
        const float4 x0 = p[0], x1 = p[es], x2 = p[2 * es], x3 = p[3 * es];
        const float4 y0 = zadd(x0, x2), y2 = zsub(x0, x2);
        const float4 y1 = zadd(x1, x3), y3 = zmul_mi(zsub(x1, x3));
        p[0] = zadd(y0, y1);
        p[es] = zsub(y0, y1);
        p[2 * es] = zadd(y2, y3);
        p[3 * es] = zsub(y2, y3);
      }
      __syncthreads();
      logLen -= 2;
      continue;
    }
    for (int it = threadIdx.x; it < nseq * nsub * nb; it += blockDim.x) {
      int q, u, b;
      sub_item_ff(it, lns, nsub, logN - 2, seq_fast, dv2, q, u, b);
      const int blk = b >> logm, j = b & (m - 1);
      float4* p = x + q * ss + ((u << logN) + blk * len + j) * es;
      const int sm = m * es;
      const float4 x0 = p[0], x1 = p[sm], x2 = p[2 * sm], x3 = p[3 * sm];
      // the two radix-2 stages as one radix-4 butterfly: the 4-point DFT
      // Y of (x0..x3), slots in bit-reversed order, Y_s times w^(s j)
      // (three products instead of the four of two separate stages)
      const float4 w1 = __ldg(tw + j * tstep), w2 = __ldg(tw + 2 * j * tstep), w3 = __ldg(tw + 3 * j * tstep);
      const float4 t0 = zadd(x0, x2), t1 = zsub(x0, x2);
      const float4 t2 = zadd(x1, x3), t3 = zmul_mi(zsub(x1, x3));
      p[0] = zadd(t0, t2);
      p[sm] = zmul(zsub(t0, t2), w2);
      p[2 * sm] = zmul(zadd(t1, t3), w1);
      p[3 * sm] = zmul(zsub(t1, t3), w3);
    }
    __syncthreads();
    logLen -= 2;
  }
  if (logLen == 1) {
    for (int it = threadIdx.x; it < nseq * nsub * (N >> 1); it += blockDim.x) {
      int q, u, b;
      sub_item_ff(it, lns, nsub, logN - 1, seq_fast, dv1, q, u, b);
      float4* p = x + q * ss + ((u << logN) + 2 * b) * es;
      const float4 a = p[0], c = p[es];
      p[0] = zadd(a, c);
      p[es] = zsub(a, c);
    }
    __syncthreads();
  }
}

// Inverse DIT sweep (unnormalised), mirror of fft_dif_ff.  Ends with a barrier.
__device__ inline void fft_dit_inv_ff(float4* x, int logN, int nseq, int es, int ss,
                                      const float4* __restrict__ tw, bool seq_fast, int nsub = 1, int twmul = 1) {
  const int N = 1 << logN, lns = 31 - __clz(nseq);  // nseq: a power of two
  const DivBy dv2 = div_by(logN >= 2 ? nsub << (logN - 2) : 1), dv1 = div_by(logN >= 1 ? nsub << (logN - 1) : 1);
  const int nb = N >> 2;
  int logLen = (logN & 1) ? 1 : 0;
  if (logLen == 1) {
    for (int it = threadIdx.x; it < nseq * nsub * (N >> 1); it += blockDim.x) {
      int q, u, b;
      sub_item_ff(it, lns, nsub, logN - 1, seq_fast, dv1, q, u, b);
      float4* p = x + q * ss + ((u << logN) + 2 * b) * es;
      const float4 a = p[0], c = p[es];
      p[0] = zadd(a, c);
      p[es] = zsub(a, c);
    }
    __syncthreads();
  }
  for (logLen += 2; logLen <= logN; logLen += 2) {
    const int len = 1 << logLen, m = len >> 2, logm = logLen - 2;
    const int tstep = (1 << (logN - logLen)) * twmul;
    if (m == 1) {  // blocks of 4: every twiddle is 1
      for (int it = threadIdx.x; it < nseq * nsub * nb; it += blockDim.x) {
        int q, u, b;
        sub_item_ff(it, lns, nsub, logN - 2, seq_fast, dv2, q, u, b);
        float4* p = x + q * ss + ((u << logN) + b * 4) * es;
        const float4 z0 = p[0], z1 = p[es], z2 = p[2 * es], z3 = p[3 * es];
        const float4 y0 = zadd(z0, z1), y1 = zsub(z0, z1);
        const float4 y2 = zadd(z2, z3), u3 = zmul_pi(zsub(z2, z3));
        p[0] = zadd(y0, y2);
        p[2 * es] = zsub(y0, y2);
        p[es] = zadd(y1, u3);
        p[3 * es] = zsub(y1, u3);
      }
      __syncthreads();
      continue;
    }
    for (int it = threadIdx.x; it < nseq * nsub * nb; it += blockDim.x) {
      int q, u, b;
      sub_item_ff(it, lns, nsub, logN - 2, seq_fast, dv2, q, u, b);
      const int blk = b >> logm, j = b & (m - 1);
      float4* p = x + q * ss + ((u << logN) + blk * len + j) * es;
      const int sm = m * es;
      const float4 z0 = p[0], z1 = p[sm], z2 = p[2 * sm], z3 = p[3 * sm];
      // inverse of the radix-4 butterfly of fft_dif_ff: conjugate twiddles
      // (three products), then the 4-point inverse DFT
      const float4 w1 = __ldg(tw + j * tstep), w2 = __ldg(tw + 2 * j * tstep), w3 = __ldg(tw + 3 * j * tstep);
      const float4 Y2 = zmulc(z1, w2), Y1 = zmulc(z2, w1), Y3 = zmulc(z3, w3);
      const float4 t0 = zadd(z0, Y2), t2 = zsub(z0, Y2);
      const float4 t1 = zadd(Y1, Y3), t3 = zmul_pi(zsub(Y1, Y3));
      p[0] = zadd(t0, t1);
      p[2 * sm] = zsub(t0, t1);
      p[sm] = zadd(t2, t3);
      p[3 * sm] = zsub(t2, t3);
    }
    __syncthreads();
  }
}

// sqrt(3)/2 as float-float: hi = the float nearest to it, lo = the float
// nearest to the rest (sqrt(3)/2 = 0.86602540378443864676...)
__device__ __forceinline__ float2 ff_sqrt3_half() { return make_float2(0x1.bb67aep-1f, 0x1.0b0996p-26f); }

// Radix-3 stages of a length-M = 2^logM 3^M3 transform, spans M, M/3, ...,
// 3 * 2^logM (decimation in frequency: the DFT of three points m apart,
// then the twiddles exp(-2 pi i j k / len), k = 1, 2).  After them every
// sequence consists of 3^M3 contiguous sub-blocks of length 2^logM that the
// power-of-two sweep finishes.  With w = exp(-2 pi i / 3):
//   y0 = x0 + x1 + x2,  y1,2 = (x0 - (x1 + x2)/2) -/+ i (sqrt 3 / 2)(x1 - x2).
// Ends with a barrier.
__device__ inline void fft3_dif_ff(float4* x, const Dft1ff& D, int nseq, int es, int ss, bool seq_fast) {
  const int M = dft_len(D), nt = M / 3;  // triples per sequence and stage
  const float2 s3 = ff_sqrt3_half();
  int len = M;
  for (int st = 0; st < D.M3; ++st, len /= 3) {
    const int m = len / 3, tstep = M / len;
    const DivBy dvs = div_by(nt), dvm = div_by(m);
    for (int it = threadIdx.x; it < nseq * nt; it += blockDim.x) {
      int q, b, j;
      seq_item_ff(it, nseq, dvs, seq_fast, q, b);
      const int blk = div_q(b, dvm, j);
      float4* p = x + q * ss + (blk * len + j) * es;
      const int sm = m * es;
      const float4 x0 = p[0], x1 = p[sm], x2 = p[2 * sm];
      const float4 t1 = zadd(x1, x2);
      const float4 t2 = zsub(x0, zhalf(t1));
      const float4 d = zsub(x1, x2);
      const float4 t3 = zmul_mi(zscale(d, s3));  // -i sqrt(3)/2 (x1 - x2)
      p[0] = zadd(x0, t1);
      p[sm] = zmul(zadd(t2, t3), __ldg(D.tw + j * tstep));
      p[2 * sm] = zmul(zsub(t2, t3), __ldg(D.tw + 2 * j * tstep));
    }
    __syncthreads();
  }
}

// The inverse of fft3_dif_ff's stages (unnormalised), spans 3 * 2^logM up to
// M: conjugate twiddles first, then the DFT of three points with
// w = exp(+2 pi i / 3).  Ends with a barrier.
__device__ inline void fft3_dit_inv_ff(float4* x, const Dft1ff& D, int nseq, int es, int ss, bool seq_fast) {
  const int M = dft_len(D), nt = M / 3;
  const float2 s3 = ff_sqrt3_half();
  int len = 3 << D.logM;
  for (int st = 0; st < D.M3; ++st, len *= 3) {
    const int m = len / 3, tstep = M / len;
    const DivBy dvs = div_by(nt), dvm = div_by(m);
    for (int it = threadIdx.x; it < nseq * nt; it += blockDim.x) {
      int q, b, j;
      seq_item_ff(it, nseq, dvs, seq_fast, q, b);
      const int blk = div_q(b, dvm, j);
      float4* p = x + q * ss + (blk * len + j) * es;
      const int sm = m * es;
      const float4 z0 = p[0];
      const float4 z1 = zmulc(p[sm], __ldg(D.tw + j * tstep));
      const float4 z2 = zmulc(p[2 * sm], __ldg(D.tw + 2 * j * tstep));
      const float4 t1 = zadd(z1, z2);
      const float4 t2 = zsub(z0, zhalf(t1));
      const float4 t3 = zmul_pi(zscale(zsub(z1, z2), s3));  // +i sqrt(3)/2 (z1 - z2)
      p[0] = zadd(z0, t1);
      p[sm] = zadd(t2, t3);
      p[2 * sm] = zsub(t2, t3);
    }
    __syncthreads();
  }
}

// The whole length-M forward sweep (radix-3 stages, then the power-of-two
// sweep on every sub-block) and its inverse.  Both end with a barrier.
__device__ inline void fft_fwd_m_ff(float4* x, const Dft1ff& D, int nseq, int es, int ss, bool seq_fast) {
  if (D.M3 > 0) fft3_dif_ff(x, D, nseq, es, ss, seq_fast);
  fft_dif_ff(x, D.logM, nseq, es, ss, D.tw, seq_fast, pow3i(D.M3), pow3i(D.M3));
}
__device__ inline void fft_inv_m_ff(float4* x, const Dft1ff& D, int nseq, int es, int ss, bool seq_fast) {
  fft_dit_inv_ff(x, D.logM, nseq, es, ss, D.tw, seq_fast, pow3i(D.M3), pow3i(D.M3));
  if (D.M3 > 0) fft3_dit_inv_ff(x, D, nseq, es, ss, seq_fast);
}

// Forward DFT of nseq sequences (capacity dft_len(D) each, data in the first
// D.N elements, element k of sequence q at x[q*ss + k*es]).  Power-of-two N:
// the DIF sweep, output bit-reversed.  Otherwise Bluestein: premultiply by
// conj(c), circular convolution with the chirp through the length-M sweeps
// and the chirp's precomputed spectrum, post-multiply by conj(c) and 1/M;
// output in natural order in the first N elements.  Ends with a barrier.
__device__ inline void dft_fwd_ff(float4* x, int nseq, int es, int ss, const Dft1ff& D, bool seq_fast) {
  if (D.c == nullptr) {
    fft_fwd_m_ff(x, D, nseq, es, ss, seq_fast);
    return;
  }
  const int N = D.N, M = dft_len(D);
  const DivBy dv1_ = div_by(M);
  for (int it = threadIdx.x; it < nseq * M; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv1_, seq_fast, q, k);
    float4* p = x + q * ss + k * es;
    *p = (k < N) ? zmulc(*p, __ldg(D.c + k)) : zzero();
  }
  __syncthreads();
  fft_fwd_m_ff(x, D, nseq, es, ss, seq_fast);
  const DivBy dv2_ = div_by(M);
  for (int it = threadIdx.x; it < nseq * M; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv2_, seq_fast, q, k);
    float4* p = x + q * ss + k * es;
    *p = zmul(*p, __ldg(D.Bf + k));
  }
  __syncthreads();
  fft_inv_m_ff(x, D, nseq, es, ss, seq_fast);
  const DivBy dv3_ = div_by(N);
  for (int it = threadIdx.x; it < nseq * N; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv3_, seq_fast, q, k);
    float4* p = x + q * ss + k * es;
    *p = zscale(zmulc(*p, __ldg(D.c + k)), D.invM);
  }
  __syncthreads();
}

// Inverse DFT, unnormalised (N times the inverse), taking the storage order
// dft_fwd_ff produces back to natural order; Bluestein as conj(DFT(conj(.))).
// Ends with a barrier.
__device__ inline void dft_inv_ff(float4* x, int nseq, int es, int ss, const Dft1ff& D, bool seq_fast) {
  if (D.c == nullptr) {
    fft_inv_m_ff(x, D, nseq, es, ss, seq_fast);
    return;
  }
  const int N = D.N;
  const DivBy dv4_ = div_by(N);
  for (int it = threadIdx.x; it < nseq * N; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv4_, seq_fast, q, k);
    float4* p = x + q * ss + k * es;
    *p = zconj(*p);
  }
  __syncthreads();
  dft_fwd_ff(x, nseq, es, ss, D, seq_fast);
  const DivBy dv5_ = div_by(N);
  for (int it = threadIdx.x; it < nseq * N; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv5_, seq_fast, q, k);
    float4* p = x + q * ss + k * es;
    *p = zconj(*p);
  }
  __syncthreads();
}

}  // namespace db
