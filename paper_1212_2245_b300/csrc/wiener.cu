// Wiener filter (Sec. 2.1, Eq. 2) with the positivity floor of Sec. 3.2.
//
//   u0 = max( Re IDFT( DFT(f0) * conj(h^) / (|h^|^2 + K) ), delta ),  f0 = max(f, delta)
//
// h^ is the DFT of the PSF wrapped periodically with its origin at (0,0), at
// the native image size.  A PSF on one row (column) is filtered with 1D
// transforms along rows (columns), the paper's 1D variant (Sec. 4.3); the
// general case uses a row pass and a column pass of 1D transforms.  Two real
// rows (columns) are packed into one complex sequence wherever the operator
// is applied to each of them independently: multiplying by the spectrum of a
// real filter is real-linear, so real and imaginary parts stay separate.
//
// All transform arithmetic is float-float (fft_df.cuh); the output is rounded
// to float once.  Transform lengths: a power of two uses bit-reversed DIF/DIT
// sweeps; any other length N uses Bluestein's chirp-z form of the same DFT,
//   X_k = conj(c_k) sum_n (x_n conj(c_n)) c_{k-n},   c_m = exp(i pi m^2 / N),
// evaluated as a circular convolution of length M >= 2N-1 (a power of two)
// with the precomputed spectrum of the chirp.  Both produce the spectrum in
// a fixed storage order (bit-reversed, resp. natural) and every spectrum
// multiplied in goes through the same routine, so orders always match.
#include <cuda_runtime.h>

#include <vector>

#include "fft_df.cuh"
#include "internal.cuh"

namespace db {

// ---------------------------------------------------------------------------
// per-axis transform tables (workspace, float4 units):
//   [tw_ff (M) | c_ff (N) | Bf_ff (M) | tw32 (M float2 = M/2 float4)]
// (c_ff and Bf_ff only for lengths that are not powers of two)
// ---------------------------------------------------------------------------
// Transform length of an axis of N points: N itself for a power of two,
// else the smallest M = 2^logM 3^M3 >= 2N - 1 for Bluestein's convolution.
void dft_plan(int N, int* logM, int* M3) {
  if (is_pow2(N)) { *logM = ilog2(N); *M3 = 0; return; }
  long long best = -1;
  for (int b = 0, p3 = 1; p3 < 4 * N; ++b, p3 *= 3) {
    int a = 0;
    while (((long long)p3 << a) < 2LL * N - 1) ++a;
    const long long M = (long long)p3 << a;
    if (best < 0 || M < best) { best = M; *logM = a; *M3 = b; }
  }
}

int dft_len_n(int N) {
  int a, b;
  dft_plan(N, &a, &b);
  return (1 << a) * pow3i(b);
}

size_t dft_table_elems(int N) {  // in float4 units
  const size_t M = (size_t)dft_len_n(N);
  return (is_pow2(N) ? M : M + N + M) + (M + 1) / 2;
}

__device__ __forceinline__ float2 split_double(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// tw_ff[k] = exp(-2 pi i k / M) as float-float; tw32[k] the same rounded to
// float (both from double).
__global__ void k_twiddles(float4* __restrict__ tw_ff, float2* __restrict__ tw32, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < M) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)M, &s, &c);
    const float2 re = split_double(c), im = split_double(s);
    tw_ff[k] = make_float4(re.x, re.y, im.x, im.y);
    tw32[k] = make_float2((float)c, (float)s);
  }
}

// Chirp c_m = exp(i pi m^2/N) for m < N (m^2 reduced mod 2N exactly), and
// the circular sequence b of length M whose spectrum the convolution uses:
// b_j = c_j (0 <= j < N), b_{M-j} = c_j (0 < j < N), 0 elsewhere.
__global__ void k_chirp(float4* __restrict__ c, float4* __restrict__ b, int N, int M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < N) {
    const long long r = ((long long)m * m) % (2LL * N);
    double s, co;
    sincospi((double)r / (double)N, &s, &co);
    const float2 re = split_double(co), im = split_double(s);
    c[m] = make_float4(re.x, re.y, im.x, im.y);
  }
  if (m < M) {
    int j = -1;
    if (m < N) j = m;
    else if (m > M - N) j = M - m;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j >= 0) {
      const long long r = ((long long)j * j) % (2LL * N);
      double s, co;
      sincospi((double)r / (double)N, &s, &co);
      const float2 re = split_double(co), im = split_double(s);
      v = make_float4(re.x, re.y, im.x, im.y);
    }
    b[m] = v;
  }
}

enum RowMode { ROW_PSF = 0, ROW_FWD_REAL = 1, ROW_INV_REAL = 2, ROW_WIENER_1D = 3, ROW_FWD_CPLX = 4,
               ROW_FWD_R2C = 5, ROW_PSF_R2C = 6, ROW_INV_C2R = 7, ROW_FILTER_1D = 8, ROW_KSPEC = 9 };
enum ColMode { COL_FWD = 0, COL_WIENER = 1, COL_WIENER_1D_REAL = 2, COL_FILTER = 3, COL_FILTER_1D_REAL = 4,
               COL_KSPEC = 5 };

struct FftArgs {
  const float* fin; int ldf;   // real input image
  float* uout; int ldu;        // real output image
  float4* cbuf; int ldc;       // complex float-float rows (row pitch ldc elements)
  const float4* spec;          // spectrum (storage order of the transform)
  int ldspec;
  const float4* kspec;         // filter spectra (the *_FILTER* modes), pitch ldk between columns
  int ldk;
  const float* taps; int kh, kw;
  Dft1ff D;                    // transform along the kernel's axis
  int nrows;                   // rows (row kernels) or columns (column kernels) of data
  int img_rows;                // image rows (packed row-pair Wiener)
  int seqs_per_cta;            // batched row passes: sequences per CTA (items step by it)
  float K, floor_;
  float2 scale;                // 1/(transform size), float-float
};

// X conj(S) / (|S|^2 + K) in float-float
__device__ __forceinline__ float4 wiener_gain(float4 S, float4 X, float K) {
  const float2 den = ff_add(ff_add(ff_mul(re_(S), re_(S)), ff_mul(im_(S), im_(S))), make_float2(K, 0.f));
  const float4 t = zmulc(X, S);
  return mkc(ff_div(re_(t), den), ff_div(im_(t), den));
}

__device__ __forceinline__ float ff_round(float2 v) { return v.x + v.y; }

// ---------------------------------------------------------------------------
// Filtering passes along a non-power-of-two axis of N points.  The filter
// Y = IDFT(G . DFT(x)) is the circular convolution of x with the impulse
// response g' = IDFT(G) (unnormalised, as the inverse sweeps are).  With b
// the circular sequence of length M >= 2N - 1 that holds g'(d) at d and
// g'(N - d) at M - d (0 < d < N), zero elsewhere, the zero-padded
// circular convolution of length M reproduces it exactly at k < N:
//   (x_pad (*)_M b)(k) = sum_j x_j b((k - j) mod M) = sum_j x_j g'((k - j) mod N),
// since k - j lies in (-N, N).  Its spectrum FFT_M(b)/M (the filter
// spectrum) is computed once per image when the filter is prepared, so a
// pass is two length-M transforms instead of the four of Bluestein's forward
// and inverse DFTs.
// ---------------------------------------------------------------------------
// In place on nseq sequences (element k of sequence q at x[q*ss + k*es],
// capacity M): g' at k < N becomes the filter spectrum FFT_M(b)/M, in the
// storage order of fft_fwd_m_ff.  Ends with a barrier.
__device__ inline void kernel_spectrum_ff(float4* x, int nseq, int es, int ss, const Dft1ff& D, bool seq_fast) {
  const int N = D.N, M = dft_len(D), P = M - N;
  const DivBy dv1_ = div_by(P);
  for (int it = threadIdx.x; it < nseq * P; it += blockDim.x) {
    int q, j;
    seq_item_ff(it, nseq, dv1_, seq_fast, q, j);
    float4* base = x + q * ss;
    const int m = N + j;  // targets m >= N; sources m - M + N < N
    base[m * es] = (m >= M - N + 1) ? base[(m - M + N) * es] : zzero();
  }
  __syncthreads();
  fft_fwd_m_ff(x, D, nseq, es, ss, seq_fast);
  const DivBy dv2_ = div_by(M);
  for (int it = threadIdx.x; it < nseq * M; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv2_, seq_fast, q, k);
    float4* p = x + q * ss + k * es;
    *p = zscale(*p, D.invM);
  }
  __syncthreads();
}

// The filtering pass on nseq sequences holding x at k < N: zero padding to
// M, forward sweep, product with the filter spectrum (element m of sequence
// q at ks[m * ksm + q * ksq], for the first nvalid sequences; the others
// hold zeros), inverse sweep; the filtered values are at k < N.  Ends with a
// barrier.
__device__ inline void filter_ff(float4* x, int nseq, int es, int ss, const Dft1ff& D, bool seq_fast,
                                 const float4* __restrict__ ks, int ksm, int ksq, int nvalid) {
  const int N = D.N, M = dft_len(D), P = M - N;
  const DivBy dv3_ = div_by(P);
  for (int it = threadIdx.x; it < nseq * P; it += blockDim.x) {
    int q, j;
    seq_item_ff(it, nseq, dv3_, seq_fast, q, j);
    x[q * ss + (N + j) * es] = zzero();
  }
  __syncthreads();
  fft_fwd_m_ff(x, D, nseq, es, ss, seq_fast);
  const DivBy dv4_ = div_by(M);
  for (int it = threadIdx.x; it < nseq * M; it += blockDim.x) {
    int q, k;
    seq_item_ff(it, nseq, dv4_, seq_fast, q, k);
    if (q >= nvalid) continue;
    float4* p = x + q * ss + k * es;
    *p = zmul(*p, __ldg(ks + (size_t)k * ksm + (size_t)q * ksq));
  }
  __syncthreads();
  fft_inv_m_ff(x, D, nseq, es, ss, seq_fast);
}

// The gain conj(S) / (|S|^2 + K) itself
__device__ __forceinline__ float4 wiener_gain1(float4 S, float K) {
  return wiener_gain(S, mkc(make_float2(1.f, 0.f), make_float2(0.f, 0.f)), K);
}

// Storage position of frequency k in a transformed sequence: bit-reversed
// for the power-of-two sweeps, natural for Bluestein's form.
__device__ __forceinline__ int spec_pos(const Dft1ff& D, int k) {
  if (D.c != nullptr || D.logM == 0) return k;
  return (int)(__brev((unsigned)k) >> (32 - D.logM));
}

// Real rows in pairs (ROW_*_R2C, ROW_INV_C2R): sequence q carries image rows
// 2q (real part) and 2q+1 (imaginary part).  A real row's spectrum is
// Hermitian, X(N-k) = conj X(k), so columns k = 0..N/2 hold all of it.
// From Z = X1 + i X2:  X1 = (Z(k) + conj Z(N-k))/2,  X2 = -i (Z(k) - conj Z(N-k))/2.
__device__ __forceinline__ void unpack_pair(float4 Zk, float4 Zm, float4& X1, float4& X2) {
  X1 = zhalf(mkc(ff_add(re_(Zk), re_(Zm)), ff_sub(im_(Zk), im_(Zm))));
  X2 = zhalf(mkc(ff_add(im_(Zk), im_(Zm)), ff_sub(re_(Zm), re_(Zk))));
}

// Row transforms: a CTA owns R consecutive sequences (capacity M each)
// starting at q0.  Global inputs are staged with asynchronous copies.
template <int MODE>
__device__ __forceinline__ void rows_body(float4* smem4, const FftArgs& a, int q0, int R) {
  const int N = a.D.N, M = dft_len(a.D);
  const DivBy dN = div_by(N), dM = div_by(M), dNh = div_by(N / 2 + 1);
  float4* x = smem4;
  float* stage = (float*)(x + R * M);  // real rows (x2 for row pairs)
  for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    int c;
    const int r = div_q(idx, dN, c);
    const int q = q0 + r;
    if (q >= a.nrows) continue;
    if (MODE == ROW_FWD_REAL) {
      cp_async4(stage + idx, a.fin + (size_t)q * a.ldf + c);
    } else if (MODE == ROW_INV_REAL || MODE == ROW_FWD_CPLX) {
      cp_async16(x + r * M + c, a.cbuf + (size_t)q * a.ldc + c);
    } else if (MODE == ROW_WIENER_1D || MODE == ROW_FWD_R2C || MODE == ROW_FILTER_1D) {
      cp_async4(stage + 2 * idx, a.fin + (size_t)(2 * q) * a.ldf + c);
      if (2 * q + 1 < a.img_rows) cp_async4(stage + 2 * idx + 1, a.fin + (size_t)(2 * q + 1) * a.ldf + c);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (MODE == ROW_INV_C2R) {
    // full Hermitian spectra of rows 2q, 2q+1 from their halves, packed as
    // Z = Y1 + i Y2, placed in transform order
    const int Nh = N / 2 + 1;
    for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
      int k;
      const int r = div_q(idx, dN, k);
      const int q = q0 + r;
      float4 Z = zzero();
      if (q < a.nrows) {
        const bool lo = k < Nh;
        const int kk = lo ? k : N - k;
        float4 Y1 = __ldg(a.cbuf + (size_t)(2 * q) * a.ldc + kk);
        float4 Y2 = (2 * q + 1 < a.img_rows) ? __ldg(a.cbuf + (size_t)(2 * q + 1) * a.ldc + kk) : zzero();
        if (!lo) { Y1 = zconj(Y1); Y2 = zconj(Y2); }
        Z = zadd(Y1, zmul_pi(Y2));
      }
      x[r * M + spec_pos(a.D, k)] = Z;
    }
  } else if (MODE != ROW_INV_REAL && MODE != ROW_FWD_CPLX) {
    for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    int c;
    const int r = div_q(idx, dN, c);
      const int q = q0 + r;
      float4 v = zzero();
      if (q < a.nrows) {
        if (MODE == ROW_PSF) {
          // wrapped PSF image of a.nrows rows: row q holds tap row (q + cy) mod nrows
          const int cy = a.kh >> 1, cx = a.kw >> 1;
          const int ta = (q + cy) % a.nrows, tb = (c + cx) % N;
          if (ta < a.kh && tb < a.kw) v.x = __ldg(a.taps + ta * a.kw + tb);
        } else if (MODE == ROW_PSF_R2C) {
          // rows 2q, 2q+1 of the wrapped PSF image of a.img_rows rows
          const int cy = a.kh >> 1, cx = a.kw >> 1;
          const int tb = (c + cx) % N;
          const int ta0 = (2 * q + cy) % a.img_rows, ta1 = (2 * q + 1 + cy) % a.img_rows;
          if (ta0 < a.kh && tb < a.kw) v.x = __ldg(a.taps + ta0 * a.kw + tb);
          if (2 * q + 1 < a.img_rows && ta1 < a.kh && tb < a.kw) v.z = __ldg(a.taps + ta1 * a.kw + tb);
        } else if (MODE == ROW_FWD_REAL) {
          v.x = fmaxf(stage[idx], a.floor_);
        } else if (MODE == ROW_KSPEC) {  // the gain; the spectrum is in natural order
          v = wiener_gain1(__ldg(&a.spec[c]), a.K);
        } else {  // ROW_WIENER_1D, ROW_FILTER_1D: sequence q packs image rows 2q and 2q+1
          v.x = fmaxf(stage[2 * idx], a.floor_);
          if (2 * q + 1 < a.img_rows) v.z = fmaxf(stage[2 * idx + 1], a.floor_);
        }
      }
      x[r * M + c] = v;
    }
  }
  __syncthreads();
  if (MODE == ROW_INV_REAL || MODE == ROW_INV_C2R) {
    dft_inv_ff(x, R, 1, M, a.D, false);
  } else if (MODE == ROW_FILTER_1D) {
    filter_ff(x, R, 1, M, a.D, false, a.kspec, 1, 0, R);
  } else if (MODE == ROW_KSPEC) {
    dft_inv_ff(x, R, 1, M, a.D, false);
    kernel_spectrum_ff(x, R, 1, M, a.D, false);
  } else {
    dft_fwd_ff(x, R, 1, M, a.D, false);
    if (MODE == ROW_WIENER_1D) {
      for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    int c;
    const int r = div_q(idx, dN, c);
        x[r * M + c] = wiener_gain(__ldg(&a.spec[c]), x[r * M + c], a.K);
      }
      __syncthreads();
      dft_inv_ff(x, R, 1, M, a.D, false);
    }
  }
  if constexpr (MODE == ROW_KSPEC) {  // all M elements of each filter spectrum
    for (int idx = threadIdx.x; idx < R * M; idx += blockDim.x) {
      int m;
      const int r = div_q(idx, dM, m);
      const int q = q0 + r;
      if (q < a.nrows) a.cbuf[(size_t)q * a.ldc + m] = x[r * M + m];
    }
  } else if constexpr (MODE == ROW_FWD_R2C || MODE == ROW_PSF_R2C) {
    const int Nh = N / 2 + 1;
    for (int idx = threadIdx.x; idx < R * Nh; idx += blockDim.x) {
      int k;
      const int r = div_q(idx, dNh, k);
      const int q = q0 + r;
      if (q >= a.nrows) continue;
      float4 X1, X2;
      unpack_pair(x[r * M + spec_pos(a.D, k)], x[r * M + spec_pos(a.D, k == 0 ? 0 : N - k)], X1, X2);
      a.cbuf[(size_t)(2 * q) * a.ldc + k] = X1;
      if (2 * q + 1 < a.img_rows) a.cbuf[(size_t)(2 * q + 1) * a.ldc + k] = X2;
    }
  } else {
    for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    int c;
    const int r = div_q(idx, dN, c);
      const int q = q0 + r;
      if (q >= a.nrows) continue;
      const float4 v = x[r * M + c];
      if (MODE == ROW_INV_C2R) {
        a.uout[(size_t)(2 * q) * a.ldu + c] = fmaxf(ff_round(ff_mul(re_(v), a.scale)), a.floor_);
        if (2 * q + 1 < a.img_rows)
          a.uout[(size_t)(2 * q + 1) * a.ldu + c] = fmaxf(ff_round(ff_mul(im_(v), a.scale)), a.floor_);
      } else if (MODE == ROW_PSF || MODE == ROW_FWD_REAL || MODE == ROW_FWD_CPLX) {
        a.cbuf[(size_t)q * a.ldc + c] = v;
      } else if (MODE == ROW_INV_REAL) {
        a.uout[(size_t)q * a.ldu + c] = fmaxf(ff_round(ff_mul(re_(v), a.scale)), a.floor_);
      } else {
        a.uout[(size_t)(2 * q) * a.ldu + c] = fmaxf(ff_round(ff_mul(re_(v), a.scale)), a.floor_);
        if (2 * q + 1 < a.img_rows)
          a.uout[(size_t)(2 * q + 1) * a.ldu + c] = fmaxf(ff_round(ff_mul(im_(v), a.scale)), a.floor_);
      }
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_fft_rows(FftArgs a, int R) {
  extern __shared__ float4 smem4[];
  rows_body<MODE>(smem4, a, blockIdx.x * R, R);
}

// Batched forms.  The batch's stages are launched back to back with
// programmatic dependent launch (wiener_batch_run): a stage's CTAs may start
// while the previous stage's last CTAs still run.  A stage that reads what an
// earlier stage of the run wrote (the 2D column passes read the forward row
// pass, the inverse row pass reads the column passes) waits for its
// predecessor first; the others work on images no earlier stage of the run
// touches and wait for their predecessor only before they exit.  Either way a
// stage completes after its predecessor, so each wait covers every earlier
// stage.  Job and item tables are written at plan time, before the run.
__device__ __host__ constexpr bool wb_reads_earlier_stage(int mode) {
  return mode == COL_WIENER || mode == COL_FILTER || mode == ROW_INV_C2R;
}

// CTA b transforms sequence items[b].y of job items[b].x.
template <int MODE>
__global__ void __launch_bounds__(256) k_fft_rows_batch(const FftArgs* __restrict__ jobs,
                                                        const int2* __restrict__ items) {
  extern __shared__ float4 smem4[];
  pdl_trigger();
  const int2 it = items[blockIdx.x];
  const FftArgs a = jobs[it.x];
  if (wb_reads_earlier_stage(MODE)) pdl_wait();
  rows_body<MODE>(smem4, a, it.y, a.seqs_per_cta);
  if (!wb_reads_earlier_stage(MODE)) pdl_wait();
}

// Column transforms: a CTA owns C adjacent sequences laid out across a row
// (element stride C in shared memory, capacity M each) starting at c0.  For
// COL_WIENER_1D_REAL, sequence c packs image columns 2c and 2c+1 and a.nrows
// counts the image columns.
template <int MODE, int C>
__device__ __forceinline__ void cols_body(float4* smem4, const FftArgs& a, int c0) {
  const int N = a.D.N, M = dft_len(a.D);
  float4* x = smem4;
  float* stage = (float*)(x + M * C);  // COL_WIENER_1D_REAL: 2*C real columns
  constexpr bool REAL1D = MODE == COL_WIENER_1D_REAL || MODE == COL_FILTER_1D_REAL;
  const int nseq_total = REAL1D ? (a.nrows + 1) / 2 : a.nrows;
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int k = idx / C, c = idx - k * C;
    const int q = c0 + c;
    if (q >= nseq_total) continue;
    if (MODE == COL_KSPEC) {
      x[idx] = wiener_gain1(__ldg(&a.spec[(size_t)k * a.ldspec + q]), a.K);
    } else if (REAL1D) {
      cp_async4(stage + 2 * idx, a.fin + (size_t)k * a.ldf + 2 * q);
      if (2 * q + 1 < a.nrows) cp_async4(stage + 2 * idx + 1, a.fin + (size_t)k * a.ldf + 2 * q + 1);
    } else {
      cp_async16(x + idx, a.cbuf + (size_t)k * a.ldc + q);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int c = idx - (idx / C) * C;
    const int q = c0 + c;
    if (q >= nseq_total) {
      x[idx] = zzero();
    } else if (REAL1D) {
      float4 v = zzero();
      v.x = fmaxf(stage[2 * idx], a.floor_);
      if (2 * q + 1 < a.nrows) v.z = fmaxf(stage[2 * idx + 1], a.floor_);
      x[idx] = v;
    }
  }
  __syncthreads();
  if (MODE == COL_KSPEC) {
    dft_inv_ff(x, C, C, 1, a.D, true);
    kernel_spectrum_ff(x, C, C, 1, a.D, true);
    for (int idx = threadIdx.x; idx < M * C; idx += blockDim.x) {
      const int m = idx / C, c = idx - m * C;
      if (c0 + c < nseq_total) a.cbuf[(size_t)m * a.ldc + c0 + c] = x[idx];
    }
    return;
  }
  if (MODE == COL_FILTER)
    filter_ff(x, C, C, 1, a.D, true, a.kspec + c0, a.ldk, 1, nseq_total - c0);
  else if (MODE == COL_FILTER_1D_REAL)
    filter_ff(x, C, C, 1, a.D, true, a.kspec, 1, 0, C);
  else
    dft_fwd_ff(x, C, C, 1, a.D, true);
  if (MODE == COL_WIENER || MODE == COL_WIENER_1D_REAL) {
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int k = idx / C, c = idx - k * C;
      const int q = c0 + c;
      if (q >= nseq_total) continue;
      const float4 S = (MODE == COL_WIENER) ? __ldg(&a.spec[(size_t)k * a.ldspec + q]) : __ldg(&a.spec[k]);
      x[idx] = wiener_gain(S, x[idx], a.K);
    }
    __syncthreads();
    dft_inv_ff(x, C, C, 1, a.D, true);
  }
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int k = idx / C, c = idx - k * C;
    const int q = c0 + c;
    if (q >= nseq_total) continue;
    const float4 v = x[idx];
    if (REAL1D) {
      a.uout[(size_t)k * a.ldu + 2 * q] = fmaxf(ff_round(ff_mul(re_(v), a.scale)), a.floor_);
      if (2 * q + 1 < a.nrows)
        a.uout[(size_t)k * a.ldu + 2 * q + 1] = fmaxf(ff_round(ff_mul(im_(v), a.scale)), a.floor_);
    } else {
      a.cbuf[(size_t)k * a.ldc + q] = v;
    }
  }
}

template <int MODE, int C>
__global__ void __launch_bounds__(256) k_fft_cols(FftArgs a) {
  extern __shared__ float4 smem4[];
  cols_body<MODE, C>(smem4, a, blockIdx.x * C);
}

template <int MODE, int C>
__global__ void __launch_bounds__(256) k_fft_cols_batch(const FftArgs* __restrict__ jobs,
                                                        const int2* __restrict__ items) {
  extern __shared__ float4 smem4[];
  pdl_trigger();
  const int2 it = items[blockIdx.x];
  const FftArgs a = jobs[it.x];
  if (wb_reads_earlier_stage(MODE)) pdl_wait();
  cols_body<MODE, C>(smem4, a, it.y);
  if (!wb_reads_earlier_stage(MODE)) pdl_wait();
}

static constexpr size_t kSmemLimit = 227 * 1024;

template <typename Kern>
static cudaError_t set_dyn_smem(Kern k, size_t smem) {
  if (smem > kSmemLimit) return cudaErrorInvalidValue;  // never reaches the runtime
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return e; }
  }
  return cudaSuccess;
}

template <int MODE>
static cudaError_t launch_rows(FftArgs a, cudaStream_t s) {
  const int M = dft_len(a.D);
  // up to 2048 / M sequences per CTA (a power of two), but at least two
  // CTAs per SM where the rows allow it
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  int R = 1;
  while (2 * R * M <= 2048) R *= 2;
  while (R > 1 && (a.nrows + R - 1) / R < 2 * sms) R >>= 1;
  const int grid = (a.nrows + R - 1) / R;
  const size_t smem = (size_t)R * M * sizeof(float4) + (size_t)2 * R * a.D.N * sizeof(float);
  cudaError_t e = set_dyn_smem(k_fft_rows<MODE>, smem);
  if (e != cudaSuccess) return e;
  k_fft_rows<MODE><<<grid, 256, smem, s>>>(a, R);
  count_launch();
  return cudaGetLastError();
}

template <int MODE, int C>
static cudaError_t launch_cols_c(FftArgs a, int nseq, cudaStream_t s) {
  const int M = dft_len(a.D);
  const size_t st = (MODE == COL_WIENER_1D_REAL || MODE == COL_FILTER_1D_REAL) ? 1 : 0;  // packed real columns
  const size_t smem = (size_t)C * M * sizeof(float4) + st * 2 * C * a.D.N * sizeof(float);
  cudaError_t e = set_dyn_smem(k_fft_cols<MODE, C>, smem);
  if (e != cudaSuccess) return e;
  k_fft_cols<MODE, C><<<(nseq + C - 1) / C, 256, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

// Columns per CTA: up to 4 (2 for M = 4096, shared-memory bound), but one
// when grouping would leave fewer than two CTAs per SM (the 513 half-spectrum
// columns of a 1024^2 image: 0.070 ms for the Wiener filter with one column
// per CTA against 0.082 ms with four).
template <int MODE>
static cudaError_t launch_cols(FftArgs a, int nseq, cudaStream_t s) {
  const int M = dft_len(a.D);
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  if ((nseq + 3) / 4 < 2 * sms || M > 4096) return launch_cols_c<MODE, 1>(a, nseq, s);
  if (M <= 2048) return launch_cols_c<MODE, 4>(a, nseq, s);
  return launch_cols_c<MODE, 2>(a, nseq, s);
}

static int dft_len_host(int N) {
  int logM, M3;
  dft_plan(N, &logM, &M3);
  int M = 1 << logM;
  while (M3-- > 0) M *= 3;
  return M;
}

size_t wiener_kspec_elems(int H, int W, int kh, int kw) {
  if (kh == 1) return is_pow2(W) ? 0 : (size_t)dft_len_host(W);
  if (kw == 1) return is_pow2(H) ? 0 : (size_t)dft_len_host(H);
  return is_pow2(H) ? 0 : (size_t)(W / 2 + 1) * dft_len_host(H);
}

// Filter spectra of a Wiener filter (kernel_spectrum_ff) from the PSF
// spectrum `spec` and K: one for a one-axis PSF along the axis of D, one per
// half-spectrum column (pitch W/2 + 1) for a 2D PSF.  Untimed set-up.
static cudaError_t prepare_kspec(const float4* spec, int H, int W, int kh, int kw, float K, const Dft1ff& D,
                                 float4* kspec, cudaStream_t s);

// Fill the tables of a length-N axis in `tab` (dft_table_elems(N) float4s).
// `ff` receives the float-float descriptor, `f32` (optional) the FP32
// twiddles for the power-of-two sweeps of fft.cuh.
cudaError_t prepare_dft(int N, float4* tab, Dft1ff* ff, Dft1* f32, cudaStream_t s) {
  Dft1ff D;
  D.N = N;
  dft_plan(N, &D.logM, &D.M3);
  const int M = dft_len(D);
  const double inv = 1.0 / (double)M;
  D.invM = make_float2((float)inv, (float)(inv - (double)(float)inv));
  D.tw = tab;
  D.c = nullptr;
  D.Bf = nullptr;
  float4* rest = tab + M;
  if (!is_pow2(N)) rest += (size_t)N + M;
  float2* tw32 = (float2*)rest;
  k_twiddles<<<(M + 255) / 256, 256, 0, s>>>(tab, tw32, M);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (!is_pow2(N)) {
    float4* c = tab + M;
    float4* Bf = c + N;
    k_chirp<<<(M + 255) / 256, 256, 0, s>>>(c, Bf, N, M);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Bf <- forward power-of-two transform of the circular chirp (in place)
    FftArgs a = {};
    Dft1ff P;
    P.N = M; P.logM = D.logM; P.M3 = D.M3; P.invM = D.invM; P.tw = tab; P.c = nullptr; P.Bf = nullptr;
    a.D = P; a.cbuf = Bf; a.ldc = M; a.nrows = 1;
    if ((e = launch_rows<ROW_FWD_CPLX>(a, s)) != cudaSuccess) return e;
    D.c = c;
    D.Bf = Bf;
  }
  if (ff) *ff = D;
  if (f32) {
    f32->N = N; f32->logM = D.logM; f32->tw = tw32; f32->c = nullptr; f32->Bf = nullptr;
  }
  return cudaSuccess;
}

cudaError_t run_psf_spectrum_2d(const float* taps, int kh, int kw, int H, int W, float4* spec,
                                const Dft1ff& DW, const Dft1ff& DH, cudaStream_t s) {
  FftArgs a = {};
  a.taps = taps; a.kh = kh; a.kw = kw; a.nrows = H; a.D = DW;
  a.cbuf = spec; a.ldc = W;
  cudaError_t e;
  if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
  FftArgs c = {};
  c.cbuf = spec; c.ldc = W; c.nrows = W; c.D = DH;
  return launch_cols<COL_FWD>(c, W, s);
}

// Half spectrum of a 2D PSF for the real-pair Wiener passes: H rows (column
// transform order) x (W/2 + 1) columns (natural order), pitch W/2 + 1.
cudaError_t run_psf_spectrum_half(const float* taps, int kh, int kw, int H, int W, float4* spec,
                                  const Dft1ff& DW, const Dft1ff& DH, cudaStream_t s) {
  const int Wh = W / 2 + 1;
  FftArgs a = {};
  a.taps = taps; a.kh = kh; a.kw = kw; a.nrows = (H + 1) / 2; a.img_rows = H; a.D = DW;
  a.cbuf = spec; a.ldc = Wh;
  cudaError_t e;
  if ((e = launch_rows<ROW_PSF_R2C>(a, s)) != cudaSuccess) return e;
  FftArgs c = {};
  c.cbuf = spec; c.ldc = Wh; c.nrows = Wh; c.D = DH;
  return launch_cols<COL_FWD>(c, Wh, s);
}

// Spectrum (storage order of D) of a one-row PSF of kw taps.
cudaError_t psf_row_spectrum(const float* taps, int kw, const Dft1ff& D, float4* out, cudaStream_t s) {
  FftArgs a = {};
  a.taps = taps; a.kh = 1; a.kw = kw; a.nrows = 1; a.D = D; a.cbuf = out; a.ldc = D.N;
  return launch_rows<ROW_PSF>(a, s);
}

// FP32 copy of an H x W float-float spectrum, stored column by column
// (out[c H + k] = in[k W + c]): the column passes that multiply with it then
// read each column as one contiguous run.
__global__ void k_round_spectrum(const float4* __restrict__ in, float2* __restrict__ out, int H, int W) {
  const size_t n = (size_t)H * W;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / W), c = (int)(e - (size_t)k * W);
    const float4 v = in[e];
    out[(size_t)c * H + k] = make_float2(v.x + v.y, v.z + v.w);
  }
}

cudaError_t round_spectrum(const float4* in, float2* out, int H, int W, cudaStream_t s) {
  k_round_spectrum<<<592, 256, 0, s>>>(in, out, H, W);
  count_launch();
  return cudaGetLastError();
}

static cudaError_t prepare_kspec(const float4* spec, int H, int W, int kh, int kw, float K, const Dft1ff& D,
                                 float4* kspec, cudaStream_t s) {
  FftArgs a = {};
  a.spec = spec; a.K = K; a.D = D; a.cbuf = kspec;
  if (kh == 1 || kw == 1) {
    a.nrows = 1; a.ldc = dft_len(D);
    return launch_rows<ROW_KSPEC>(a, s);
  }
  const int Wh = W / 2 + 1;
  a.ldspec = Wh; a.nrows = Wh; a.ldc = Wh;
  (void)H;
  return launch_cols<COL_KSPEC>(a, Wh, s);
}

static float2 ff_const(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// Set-up part of the Wiener filter: transform tables and the PSF spectrum
// (depends on the taps and the image size only).
cudaError_t wiener_prepare(int H, int W, const float* taps, int kh, int kw, float K, void* ws, const WsLayout& L,
                           WienerState* st, cudaStream_t s) {
  char* base = (char*)ws;
  float4* spec = (float4*)(base + L.spec);
  float4* tabW = (float4*)(base + L.tw);
  float4* tabH = tabW + dft_table_elems(W);
  cudaError_t e;
  WienerState S = {};
  S.H = H; S.W = W; S.kh = kh; S.kw = kw;
  if (kw > 1 || kh == 1) { if ((e = prepare_dft(W, tabW, &S.DW, nullptr, s)) != cudaSuccess) return e; }
  if (kh > 1) { if ((e = prepare_dft(H, tabH, &S.DH, nullptr, s)) != cudaSuccess) return e; }
  FftArgs a = {};
  if (kh == 1) {
    a.taps = taps; a.kh = 1; a.kw = kw; a.nrows = 1; a.D = S.DW; a.cbuf = spec; a.ldc = W;
    if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
  } else if (kw == 1) {
    // a kh x 1 tap array has the memory layout of a 1 x kh row
    a.taps = taps; a.kh = 1; a.kw = kh; a.nrows = 1; a.D = S.DH; a.cbuf = spec; a.ldc = H;
    if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
  } else {
    if ((e = run_psf_spectrum_half(taps, kh, kw, H, W, spec, S.DW, S.DH, s)) != cudaSuccess) return e;
  }
  // the filtering pass along a non-power-of-two axis as one circular
  // convolution (its filter spectra depend on K, fixed here)
  if (wiener_kspec_elems(H, W, kh, kw) > 0) {
    float4* kspec = (float4*)(base + L.kspec);
    if ((e = prepare_kspec(spec, H, W, kh, kw, K, kh == 1 ? S.DW : S.DH, kspec, s)) != cudaSuccess) return e;
    S.kspec = kspec;
  }
  *st = S;
  return cudaSuccess;
}

// Image part: the transforms of f, the gain and the inverse transforms.
cudaError_t wiener_apply(const float* f, float* u0, int ld, float K, float floor_, void* ws, const WsLayout& L,
                         const WienerState& S, cudaStream_t s) {
  char* base = (char*)ws;
  float4* spec = (float4*)(base + L.spec);
  float4* work = (float4*)(base + L.work);
  const int H = S.H, W = S.W;
  if (S.kh == 1) {
    FftArgs b = {};
    b.fin = f; b.ldf = ld; b.uout = u0; b.ldu = ld; b.spec = spec; b.kspec = S.kspec; b.D = S.DW;
    b.nrows = (H + 1) / 2; b.img_rows = H;
    b.K = K; b.floor_ = floor_; b.scale = ff_const(1.0 / W);
    return S.kspec ? launch_rows<ROW_FILTER_1D>(b, s) : launch_rows<ROW_WIENER_1D>(b, s);
  }
  if (S.kw == 1) {
    FftArgs b = {};
    b.fin = f; b.ldf = ld; b.uout = u0; b.ldu = ld; b.spec = spec; b.kspec = S.kspec; b.D = S.DH;
    b.nrows = W;
    b.K = K; b.floor_ = floor_; b.scale = ff_const(1.0 / H);
    return S.kspec ? launch_cols<COL_FILTER_1D_REAL>(b, (W + 1) / 2, s)
                   : launch_cols<COL_WIENER_1D_REAL>(b, (W + 1) / 2, s);
  }
  // real rows in pairs; only the W/2 + 1 columns of the Hermitian half
  // spectrum go through the column pass
  cudaError_t e;
  const int Wh = W / 2 + 1;
  FftArgs d = {};
  d.fin = f; d.ldf = ld; d.cbuf = work; d.ldc = Wh; d.nrows = (H + 1) / 2; d.img_rows = H; d.D = S.DW;
  d.floor_ = floor_;
  if ((e = launch_rows<ROW_FWD_R2C>(d, s)) != cudaSuccess) return e;
  FftArgs g = {};
  g.cbuf = work; g.ldc = Wh; g.spec = spec; g.ldspec = Wh; g.nrows = Wh; g.D = S.DH; g.K = K;
  g.kspec = S.kspec; g.ldk = Wh;
  if ((e = S.kspec ? launch_cols<COL_FILTER>(g, Wh, s) : launch_cols<COL_WIENER>(g, Wh, s)) != cudaSuccess)
    return e;
  FftArgs o = {};
  o.cbuf = work; o.ldc = Wh; o.uout = u0; o.ldu = ld; o.nrows = (H + 1) / 2; o.img_rows = H; o.D = S.DW;
  o.floor_ = floor_; o.scale = ff_const(1.0 / ((double)H * (double)W));
  return launch_rows<ROW_INV_C2R>(o, s);
}

cudaError_t run_wiener(const float* f, float* u0, int H, int W, int ld, const float* taps, int kh,
                       int kw, float K, float floor_, void* ws, const WsLayout& L, int* status,
                       cudaStream_t s) {
  (void)status;
  WienerState S;
  cudaError_t e = wiener_prepare(H, W, taps, kh, kw, K, ws, L, &S, s);
  if (e != cudaSuccess) return e;
  return wiener_apply(f, u0, ld, K, floor_, ws, L, S, s);
}

// ---------------------------------------------------------------------------
// batched Wiener filter: every image of a batch in five launches (one per
// transform stage), each CTA working on one row (pair) or column group of
// one image with that image's own transform lengths.
// ---------------------------------------------------------------------------
// The *_F stages are the filtering passes along non-power-of-two axes in
// their circular-convolution form (filter spectra prepared with the plan).
enum { WB_ROW_1D = 0, WB_ROW_FWD = 1, WB_COL_1D = 2, WB_COL_2D = 3, WB_ROW_INV = 4, WB_ROW_1D_F = 5,
       WB_COL_1D_F = 6, WB_COL_2D_F = 7, WB_STAGES = 8 };
// Column passes: columns per CTA by transform length, in classes launched
// separately: 2 (the longest transforms: 4 per CTA left one CTA per SM,
// 36.0 against 30.8 ms for batch512's Wiener), 4 or 8 while C x M <= 4096,
// so that short transforms still give the CTA's threads work.
constexpr int kColClasses = 3;
__host__ __device__ constexpr int col_class_c(int k) { return 2 << k; }
static int col_class(int M) {
  int k = 0;
  while (k + 1 < kColClasses && col_class_c(k + 1) * M <= 4096) ++k;
  return k;
}

struct WienerBatch {
  std::vector<FftArgs> jobs[WB_STAGES];
  std::vector<int2> items[WB_STAGES][kColClasses];  // row stages use class 0 only
  FftArgs* d_jobs[WB_STAGES] = {};
  int2* d_items[WB_STAGES][kColClasses] = {};
  size_t smem[WB_STAGES][kColClasses] = {};
};

// Sequences per CTA of a batched row job: as many as keep R x M <= 2048
// (a power of two, at most the job's rows), so that short transforms still
// give the CTA's 256 threads work in every stage.
static int batch_row_seqs(int M, int nrows) {
  int R = 1;
  while (2 * R * M <= 2048 && 2 * R <= nrows) R *= 2;
  return R;
}

// Append the items of a batched row job (one per group of seqs_per_cta rows)
// and grow the stage's shared memory to the job's need.
static void add_row_items(WienerBatch* b, int stage, int id, FftArgs& j, int N) {
  const int M = dft_len(j.D), R = batch_row_seqs(M, j.nrows);
  j.seqs_per_cta = R;
  for (int q = 0; q < j.nrows; q += R) b->items[stage][0].push_back(make_int2(id, q));
  const size_t sm = (size_t)R * M * sizeof(float4) + (size_t)2 * R * N * sizeof(float);
  if (sm > b->smem[stage][0]) b->smem[stage][0] = sm;
}

WienerBatch* wiener_batch_new() { return new WienerBatch(); }
size_t wiener_job_bytes() { return sizeof(FftArgs); }
void wiener_batch_delete(WienerBatch* b) { delete b; }

// Precompute the image's PSF spectrum and, for a filtering pass along a
// non-power-of-two axis, its filter spectra (untimed set-up), and append
// its jobs.
cudaError_t wiener_batch_add(WienerBatch* b, const WienerImage& im, cudaStream_t s) {
  cudaError_t e;
  const int H = im.H, W = im.W;
  if (im.kh == 1) {
    FftArgs a = {};
    a.taps = im.taps; a.kh = 1; a.kw = im.kw; a.nrows = 1; a.D = (*im.pDW); a.cbuf = im.spec; a.ldc = W;
    if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
    if (im.kspec && (e = prepare_kspec(im.spec, H, W, 1, im.kw, im.K, *im.pDW, im.kspec, s)) != cudaSuccess)
      return e;
    FftArgs j = {};
    j.fin = im.f; j.ldf = im.ld; j.uout = im.u0; j.ldu = im.ldu; j.spec = im.spec; j.kspec = im.kspec;
    j.D = (*im.pDW);
    j.nrows = (H + 1) / 2; j.img_rows = H; j.K = im.K; j.floor_ = im.floor_; j.scale = ff_const(1.0 / W);
    const int st = im.kspec ? WB_ROW_1D_F : WB_ROW_1D;
    const int id = (int)b->jobs[st].size();
    add_row_items(b, st, id, j, W);
    b->jobs[st].push_back(j);
    return cudaSuccess;
  }
  if (im.kw == 1) {
    FftArgs a = {};
    a.taps = im.taps; a.kh = 1; a.kw = im.kh; a.nrows = 1; a.D = (*im.pDH); a.cbuf = im.spec; a.ldc = H;
    if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
    if (im.kspec && (e = prepare_kspec(im.spec, H, W, im.kh, 1, im.K, *im.pDH, im.kspec, s)) != cudaSuccess)
      return e;
    FftArgs j = {};
    j.fin = im.f; j.ldf = im.ld; j.uout = im.u0; j.ldu = im.ldu; j.spec = im.spec; j.kspec = im.kspec;
    j.D = (*im.pDH);
    j.nrows = W; j.K = im.K; j.floor_ = im.floor_; j.scale = ff_const(1.0 / H);
    const int st = im.kspec ? WB_COL_1D_F : WB_COL_1D;
    const int id = (int)b->jobs[st].size();
    b->jobs[st].push_back(j);
    const int nseq = (W + 1) / 2, M = dft_len(*im.pDH), k = col_class(M), C = col_class_c(k);
    for (int c0 = 0; c0 < nseq; c0 += C) b->items[st][k].push_back(make_int2(id, c0));
    const size_t sm = (size_t)C * M * sizeof(float4) + (size_t)2 * C * H * sizeof(float);
    if (sm > b->smem[st][k]) b->smem[st][k] = sm;
    return cudaSuccess;
  }
  if ((e = run_psf_spectrum_half(im.taps, im.kh, im.kw, H, W, im.spec, (*im.pDW), (*im.pDH), s)) != cudaSuccess)
    return e;
  if (im.kspec && (e = prepare_kspec(im.spec, H, W, im.kh, im.kw, im.K, *im.pDH, im.kspec, s)) != cudaSuccess)
    return e;
  const int Wh = W / 2 + 1, Hp = (H + 1) / 2;
  FftArgs d = {};
  d.fin = im.f; d.ldf = im.ld; d.cbuf = im.work; d.ldc = Wh; d.nrows = Hp; d.img_rows = H; d.D = (*im.pDW);
  d.floor_ = im.floor_;
  FftArgs g = {};
  g.cbuf = im.work; g.ldc = Wh; g.spec = im.spec; g.ldspec = Wh; g.nrows = Wh; g.D = (*im.pDH); g.K = im.K;
  g.kspec = im.kspec; g.ldk = Wh;
  const int gst = im.kspec ? WB_COL_2D_F : WB_COL_2D;
  FftArgs o = {};
  o.cbuf = im.work; o.ldc = Wh; o.uout = im.u0; o.ldu = im.ldu; o.nrows = Hp; o.img_rows = H; o.D = (*im.pDW);
  o.floor_ = im.floor_; o.scale = ff_const(1.0 / ((double)H * (double)W));
  const int i1 = (int)b->jobs[WB_ROW_FWD].size(), i2 = (int)b->jobs[gst].size(),
            i3 = (int)b->jobs[WB_ROW_INV].size();
  add_row_items(b, WB_ROW_FWD, i1, d, W);
  add_row_items(b, WB_ROW_INV, i3, o, W);
  b->jobs[WB_ROW_FWD].push_back(d);
  b->jobs[gst].push_back(g);
  b->jobs[WB_ROW_INV].push_back(o);
  const int MH = dft_len(*im.pDH), kc = col_class(MH), CC = col_class_c(kc);
  for (int c0 = 0; c0 < Wh; c0 += CC) b->items[gst][kc].push_back(make_int2(i2, c0));
  const size_t smc = (size_t)CC * MH * sizeof(float4);
  if (smc > b->smem[gst][kc]) b->smem[gst][kc] = smc;
  return cudaSuccess;
}

size_t wiener_batch_table_bytes(const WienerBatch* b) {
  size_t n = 0;
  for (int k = 0; k < WB_STAGES; ++k) {
    n += align256(b->jobs[k].size() * sizeof(FftArgs));
    for (int c = 0; c < kColClasses; ++c) n += align256(b->items[k][c].size() * sizeof(int2));
  }
  return n;
}

// Upload the job tables into `dst` (wiener_batch_table_bytes bytes).
cudaError_t wiener_batch_upload(WienerBatch* b, void* dst, cudaStream_t s) {
  char* p = (char*)dst;
  for (int k = 0; k < WB_STAGES; ++k) {
    b->d_jobs[k] = (FftArgs*)p;
    if (!b->jobs[k].empty()) {
      cudaError_t e = cudaMemcpyAsync(p, b->jobs[k].data(), b->jobs[k].size() * sizeof(FftArgs),
                                      cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return e;
    }
    p += align256(b->jobs[k].size() * sizeof(FftArgs));
    for (int c = 0; c < kColClasses; ++c) {
      b->d_items[k][c] = (int2*)p;
      if (!b->items[k][c].empty()) {
        cudaError_t e = cudaMemcpyAsync(p, b->items[k][c].data(), b->items[k][c].size() * sizeof(int2),
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
      }
      p += align256(b->items[k][c].size() * sizeof(int2));
      if (b->smem[k][c] > kSmemLimit) return cudaErrorInvalidValue;
    }
  }
  return cudaSuccess;
}

// Launch a batched stage kernel; `pdl`: programmatic dependent launch on the
// previous launch of the run (every launch of the run but its first).
template <typename Kern>
static cudaError_t launch_wb(Kern kern, unsigned grid, size_t smem, bool pdl, const WienerBatch* b, int stage,
                             int cls, cudaStream_t s) {
  cudaError_t e = set_dyn_smem(kern, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if ((e = cudaLaunchKernelEx(&cfg, kern, (const FftArgs*)b->d_jobs[stage], (const int2*)b->d_items[stage][cls])) !=
      cudaSuccess) {
    (void)cudaGetLastError();
    return e;
  }
  count_launch();
  return cudaSuccess;
}

template <int MODE>
static cudaError_t launch_rows_batch(const WienerBatch* b, int stage, bool& pdl, cudaStream_t s) {
  if (b->items[stage][0].empty()) return cudaSuccess;
  const cudaError_t e = launch_wb(k_fft_rows_batch<MODE>, (unsigned)b->items[stage][0].size(), b->smem[stage][0],
                                  pdl, b, stage, 0, s);
  pdl = true;
  return e;
}

template <int MODE, int K>
static cudaError_t launch_cols_batch_c(const WienerBatch* b, int stage, bool& pdl, cudaStream_t s) {
  if (b->items[stage][K].empty()) return cudaSuccess;
  const cudaError_t e = launch_wb(k_fft_cols_batch<MODE, col_class_c(K)>, (unsigned)b->items[stage][K].size(),
                                  b->smem[stage][K], pdl, b, stage, K, s);
  pdl = true;
  return e;
}

template <int MODE>
static cudaError_t launch_cols_batch(const WienerBatch* b, int stage, bool& pdl, cudaStream_t s) {
  static_assert(kColClasses == 3, "one launch per column class");
  cudaError_t e;
  if ((e = launch_cols_batch_c<MODE, 0>(b, stage, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_cols_batch_c<MODE, 1>(b, stage, pdl, s)) != cudaSuccess) return e;
  return launch_cols_batch_c<MODE, 2>(b, stage, pdl, s);
}

// The stages in launch order.  The run's first launch depends on everything
// before it in the stream in full; each later one is a programmatic
// dependent of the launch before it (see k_fft_rows_batch).
cudaError_t wiener_batch_run(const WienerBatch* b, cudaStream_t s) {
  cudaError_t e;
  bool pdl = false;
  if ((e = launch_rows_batch<ROW_WIENER_1D>(b, WB_ROW_1D, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_rows_batch<ROW_FILTER_1D>(b, WB_ROW_1D_F, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_cols_batch<COL_WIENER_1D_REAL>(b, WB_COL_1D, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_cols_batch<COL_FILTER_1D_REAL>(b, WB_COL_1D_F, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_rows_batch<ROW_FWD_R2C>(b, WB_ROW_FWD, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_cols_batch<COL_WIENER>(b, WB_COL_2D, pdl, s)) != cudaSuccess) return e;
  if ((e = launch_cols_batch<COL_FILTER>(b, WB_COL_2D_F, pdl, s)) != cudaSuccess) return e;
  return launch_rows_batch<ROW_INV_C2R>(b, WB_ROW_INV, pdl, s);
}

}  // namespace db
