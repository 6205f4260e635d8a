// Register-resident FP32 FFT for power-of-two lengths N = 2^L (L = 6..12),
// used by the Fourier-mode iteration (Sec. 4.1 "Fourier transform", Sec. 4.3).
//
// Same transforms as fft.cuh (forward DIF with bit-reversed output, inverse
// DIT from bit-reversed input, unnormalised), so spectra computed by either
// are interchangeable.  The difference is where the data lives: each thread
// keeps 8 elements of a sequence in registers for the whole transform, and
// the radix-2 stages go in passes of three (one radix-8 butterfly per thread
// and pass) with a shared-memory exchange between passes only.  A length-2048
// transform is 4 passes and 3 exchanges; the first pass takes its elements
// straight from global memory and the last one leaves them in registers.
//
// Pass with top bit HB (bits HB..LO, LO = HB - 2; the remainder of L mod 3
// bits is the bottom pass, LO = 0): the thread's group is j = t mod 2^LO,
// hi = t >> LO, elements hi 2^(HB+1) + j + r 2^LO, r = 0..7.  Forward, the
// 8-point DFT of the group (natural order in, bit-reversed order out) is
// followed by the twiddle w_{2^(HB+1)}^(j e) on output e; the inverse applies
// the conjugate twiddles first and runs the mirrored butterflies.  The
// bottom pass holds 8 consecutive elements 8t..8t+7 (one group of 8, two of
// 4 or four of 2); there j = 0 and no twiddle is needed.
//
// Shared layout: C sequences per CTA interleaved, element k of sequence c at
// (k + k/8) C + c, with the sequence index fastest among the threads
// (thread = t C + c).  A bank model over every pass of L = 6..12 and
// C = 2..64 finds no conflict for 8-byte accesses.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace db {
namespace f8 {

__host__ __device__ constexpr int pass_lo(int hb) { return hb >= 2 ? hb - 2 : 0; }
// top bit of the bottom pass
__host__ __device__ constexpr int bottom_hb(int L) { return L % 3 == 0 ? 2 : L % 3 - 1; }
__host__ __device__ constexpr int padded(int n) { return n + (n >> 3); }
__device__ __forceinline__ int spos(int k) { return k + (k >> 3); }
// sequences per CTA: 512 threads (1024 for N = 4096)
__host__ __device__ constexpr int seqs(int L) { return L >= 11 ? 2 : 512 >> (L - 3); }
__host__ __device__ constexpr int threads(int L) { return seqs(L) * ((1 << L) >> 3); }

// element index held in register r by thread t in the pass with top bit HB
template <int HB>
__device__ __forceinline__ int elem(int t, int r) {
  constexpr int LO = pass_lo(HB), NB = HB - LO + 1;
  if constexpr (NB == 3) return ((t >> LO) << (HB + 1)) + (t & ((1 << LO) - 1)) + (r << LO);
  else return 8 * t + r;
}

// spos(elem(t, r)) = spos(elem(t, 0)) + spos(r 2^LO): the group's base has
// no bits in LO..HB and its part below 2^LO never carries into bit 3 when
// r 2^LO is added, so every register's position is the base plus a constant.
template <int HB>
__host__ __device__ constexpr int reg_off(int r) {
  return HB - pass_lo(HB) == 2 ? (r << pass_lo(HB)) + ((r << pass_lo(HB)) >> 3) : r;
}
template <int HB, int C>
__device__ __forceinline__ void store(const float2 (&v)[8], float2* sm, int t, int c) {
  float2* p = sm + spos(elem<HB>(t, 0)) * C + c;
#pragma unroll
  for (int r = 0; r < 8; ++r) p[reg_off<HB>(r) * C] = v[r];
}
template <int HB, int C>
__device__ __forceinline__ void load(float2 (&v)[8], const float2* sm, int t, int c) {
  const float2* p = sm + spos(elem<HB>(t, 0)) * C + c;
#pragma unroll
  for (int r = 0; r < 8; ++r) v[r] = p[reg_off<HB>(r) * C];
}

__device__ __forceinline__ void bfly(float2& a, float2& b) {
  const float2 x = a;
  a = cadd(x, b);
  b = csub(x, b);
}
constexpr float kR2 = 0.70710678118654752f;  // 1/sqrt(2)
// x w8, w8 = (1 - i)/sqrt(2)
__device__ __forceinline__ float2 mul_w8(float2 x) { return make_float2((x.x + x.y) * kR2, (x.y - x.x) * kR2); }
// x w8^3, w8^3 = (-1 - i)/sqrt(2)
__device__ __forceinline__ float2 mul_w83(float2 x) { return make_float2((x.y - x.x) * kR2, -(x.x + x.y) * kR2); }
// x conj(w8)
__device__ __forceinline__ float2 mul_cw8(float2 x) { return make_float2((x.x - x.y) * kR2, (x.x + x.y) * kR2); }
// x conj(w8^3)
__device__ __forceinline__ float2 mul_cw83(float2 x) { return make_float2(-(x.x + x.y) * kR2, (x.x - x.y) * kR2); }

// 8-point DIF on v[o..o+7]: natural order in, bit-reversed order out
__device__ __forceinline__ void dif8(float2 (&v)[8]) {
  float2 d;
  d = csub(v[0], v[4]); v[0] = cadd(v[0], v[4]); v[4] = d;
  d = csub(v[1], v[5]); v[1] = cadd(v[1], v[5]); v[5] = mul_w8(d);
  d = csub(v[2], v[6]); v[2] = cadd(v[2], v[6]); v[6] = cmul_mi(d);
  d = csub(v[3], v[7]); v[3] = cadd(v[3], v[7]); v[7] = mul_w83(d);
#pragma unroll
  for (int h = 0; h < 8; h += 4) {
    d = csub(v[h], v[h + 2]); v[h] = cadd(v[h], v[h + 2]); v[h + 2] = d;
    d = csub(v[h + 1], v[h + 3]); v[h + 1] = cadd(v[h + 1], v[h + 3]); v[h + 3] = cmul_mi(d);
  }
#pragma unroll
  for (int q = 0; q < 8; q += 2) bfly(v[q], v[q + 1]);
}
// inverse of dif8 (times 8): bit-reversed order in, natural order out
__device__ __forceinline__ void dit8_inv(float2 (&v)[8]) {
#pragma unroll
  for (int q = 0; q < 8; q += 2) bfly(v[q], v[q + 1]);
#pragma unroll
  for (int h = 0; h < 8; h += 4) {
    bfly(v[h], v[h + 2]);
    const float2 t = cmul_pi(v[h + 3]);
    v[h + 3] = csub(v[h + 1], t);
    v[h + 1] = cadd(v[h + 1], t);
  }
  float2 t;
  t = v[4];           v[4] = csub(v[0], t); v[0] = cadd(v[0], t);
  t = mul_cw8(v[5]);  v[5] = csub(v[1], t); v[1] = cadd(v[1], t);
  t = cmul_pi(v[6]);  v[6] = csub(v[2], t); v[2] = cadd(v[2], t);
  t = mul_cw83(v[7]); v[7] = csub(v[3], t); v[3] = cadd(v[3], t);
}
// 4-point DIF / inverse on v[o..o+3]
template <int O>
__device__ __forceinline__ void dif4(float2 (&v)[8]) {
  float2 d;
  d = csub(v[O], v[O + 2]); v[O] = cadd(v[O], v[O + 2]); v[O + 2] = d;
  d = csub(v[O + 1], v[O + 3]); v[O + 1] = cadd(v[O + 1], v[O + 3]); v[O + 3] = cmul_mi(d);
  bfly(v[O], v[O + 1]);
  bfly(v[O + 2], v[O + 3]);
}
template <int O>
__device__ __forceinline__ void dit4_inv(float2 (&v)[8]) {
  bfly(v[O], v[O + 1]);
  bfly(v[O + 2], v[O + 3]);
  bfly(v[O], v[O + 2]);
  const float2 t = cmul_pi(v[O + 3]);
  v[O + 3] = csub(v[O + 1], t);
  v[O + 1] = cadd(v[O + 1], t);
}

// Twiddles w^(j e), e = 1..7, of one group from three table loads (e = 1, 2,
// 4) and four products; slot s of the 8-point output holds DFT index
// bitrev3(s): 0,4,2,6,1,5,3,7.
template <int L, int HB>
__device__ __forceinline__ void twiddles(int t, const float2* __restrict__ tw, float2 (&w)[8]) {
  constexpr int LO = pass_lo(HB), SH = L - HB - 1;
  const int j = t & ((1 << LO) - 1);
  // an opaque copy of the table pointer per pass: the forward and inverse
  // passes of one bit range use the same twiddles, and sharing the loads
  // would keep them live across the whole transform (register spills)
  asm volatile("" : "+l"(tw));
  const float2 w1 = __ldg(tw + (j << SH)), w2 = __ldg(tw + ((2 * j) << SH)), w4 = __ldg(tw + ((4 * j) << SH));
  const float2 w3 = cmul(w1, w2);
  w[1] = w4;              // e = 4
  w[2] = w2;              // e = 2
  w[3] = cmul(w2, w4);    // e = 6
  w[4] = w1;              // e = 1
  w[5] = cmul(w1, w4);    // e = 5
  w[6] = w3;              // e = 3
  w[7] = cmul(w3, w4);    // e = 7
}

template <int L, int HB>
__device__ __forceinline__ void dif_pass(float2 (&v)[8], int t, const float2* __restrict__ tw) {
  constexpr int LO = pass_lo(HB), NB = HB - LO + 1;
  if constexpr (NB == 3) {
    dif8(v);
    if constexpr (LO > 0) {
      float2 w[8];
      twiddles<L, HB>(t, tw, w);
#pragma unroll
      for (int s = 1; s < 8; ++s) v[s] = cmul(v[s], w[s]);
    }
  } else if constexpr (NB == 2) {
    dif4<0>(v);
    dif4<4>(v);
  } else {
#pragma unroll
    for (int q = 0; q < 8; q += 2) bfly(v[q], v[q + 1]);
  }
}

template <int L, int HB>
__device__ __forceinline__ void dit_pass(float2 (&v)[8], int t, const float2* __restrict__ tw) {
  constexpr int LO = pass_lo(HB), NB = HB - LO + 1;
  if constexpr (NB == 3) {
    if constexpr (LO > 0) {
      float2 w[8];
      twiddles<L, HB>(t, tw, w);
#pragma unroll
      for (int s = 1; s < 8; ++s) v[s] = cmulc(v[s], w[s]);
    }
    dit8_inv(v);
  } else if constexpr (NB == 2) {
    dit4_inv<0>(v);
    dit4_inv<4>(v);
  } else {
#pragma unroll
    for (int q = 0; q < 8; q += 2) bfly(v[q], v[q + 1]);
  }
}

// Forward DIF from the pass with top bit HB down to the bottom pass.  On entry
// v holds pass HB's elements; on exit the bottom pass's (8t..8t+7, output in
// bit-reversed storage order).  Exchanges through sm; every thread of the
// CTA must call it.
template <int L, int HB, int C>
__device__ __forceinline__ void dif_chain(float2 (&v)[8], float2* sm, int t, int c, const float2* __restrict__ tw) {
  dif_pass<L, HB>(v, t, tw);
  constexpr int LO = pass_lo(HB);
  if constexpr (LO > 0) {
    store<HB, C>(v, sm, t, c);
    __syncthreads();
    load<LO - 1, C>(v, sm, t, c);
    dif_chain<L, LO - 1, C>(v, sm, t, c, tw);
  }
}

// Inverse DIT from the pass with top bit HB up to the top pass (HB = L - 1).
// On exit v holds elements t + (N/8) r in natural order.
template <int L, int HB, int C>
__device__ __forceinline__ void dit_chain(float2 (&v)[8], float2* sm, int t, int c, const float2* __restrict__ tw) {
  dit_pass<L, HB>(v, t, tw);
  if constexpr (HB < L - 1) {
    store<HB, C>(v, sm, t, c);
    __syncthreads();
    load<HB + 3, C>(v, sm, t, c);
    dit_chain<L, HB + 3, C>(v, sm, t, c, tw);
  }
}

}  // namespace f8
}  // namespace db
