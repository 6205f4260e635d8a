// Wiener filter (Sec. 2.1, Eq. 2) with the positivity floor of Sec. 3.2.
//
//   u0 = max( Re IDFT( DFT(f0) * conj(h^) / (|h^|^2 + K) ), delta ),  f0 = max(f, delta)
//
// h^ is the DFT of the PSF wrapped periodically with its origin at (0,0).
// A PSF on one row (column) is filtered with 1D transforms along rows
// (columns), the paper's 1D variant (Sec. 4.3); the general case uses a
// row pass and a column pass of 1D transforms.  Two real rows (columns) are
// packed into one complex sequence wherever the operator is applied to each
// of them independently: multiplying by the spectrum of a real filter is
// real-linear, so real and imaginary parts stay separate.
#include <cuda_runtime.h>

#include "fft.cuh"
#include "internal.cuh"

namespace db {

// tw[k] = exp(-2 pi i k / N) for k < N, correctly rounded from double.
__global__ void k_twiddles(float2* __restrict__ tw, int N) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)N, &s, &c);
    tw[k] = make_float2((float)c, (float)s);
  }
}

cudaError_t launch_twiddles(float2* tw, int N, cudaStream_t s) {
  k_twiddles<<<(N + 255) / 256, 256, 0, s>>>(tw, N);
  count_launch();
  return cudaGetLastError();
}

enum RowMode { ROW_PSF = 0, ROW_FWD_REAL = 1, ROW_INV_REAL = 2, ROW_WIENER_1D = 3 };
enum ColMode { COL_FWD = 0, COL_WIENER = 1, COL_WIENER_1D_REAL = 2 };

struct FftArgs {
  const float* fin; int ldf;   // real input image
  float* uout; int ldu;        // real output image
  float2* cbuf; int ldc;       // complex rows (row pitch ldc elements)
  const float2* spec;          // spectrum (bit-reversed order)
  int ldspec;
  const float* taps; int kh, kw;
  const float2* twg;           // twiddle table for the transform length (global)
  int nrows;                   // rows (row kernels) or columns (column kernels) of data
  int img_rows;                // image rows (packed row-pair Wiener)
  int logN;                    // log2 of the transform length
  float K, floor_, scale;
};

// The filter is linear, so it is applied to f0 - c (c = mid-grey) and the
// exact response c * M(0) to the constant is added back: this keeps the
// transform's rounding error, which scales with the signal norm, smaller.
// M(0) = S0/(S0^2 + K) with S0 the zero-frequency PSF coefficient (element 0
// of the spectrum in bit-reversed order is frequency 0).
constexpr float kMidGrey = 128.0f;

__device__ __forceinline__ float dc_response(const float2* spec, float K) {
  const float2 S0 = __ldg(spec);
  return kMidGrey * (S0.x / fmaf(S0.x, S0.x, fmaf(S0.y, S0.y, K)));
}

__device__ __forceinline__ float2 wiener_gain(float2 S, float2 X, float K) {
  // X * conj(S) / (|S|^2 + K)
  const float den = fmaf(S.x, S.x, fmaf(S.y, S.y, K));
  const float2 t = cmulc(X, S);
  const float inv = 1.0f / den;
  return make_float2(t.x * inv, t.y * inv);
}

// Row transforms: each CTA owns R consecutive sequences of length N.  Global
// inputs are staged with asynchronous copies (real inputs into the upper
// half of each complex slot's memory first), so every load of the CTA is in
// flight at once.
template <int MODE>
__global__ void __launch_bounds__(256) k_fft_rows(FftArgs a, int R) {
  extern __shared__ float2 smem[];
  const int N = 1 << a.logN;
  float2* tw = smem;
  float2* x = smem + N;
  float* stage = (float*)(x + R * N);  // real rows staged here (R*N floats, x2 for row pairs)
  fft_load_twiddles(tw, a.twg, N);
  const int q0 = blockIdx.x * R;  // first sequence of this CTA
  // ---- load
  for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    const int r = idx >> a.logN, c = idx & (N - 1);
    const int q = q0 + r;
    if (q >= a.nrows) continue;
    if (MODE == ROW_FWD_REAL) {
      cp_async4(stage + idx, a.fin + (size_t)q * a.ldf + c);
    } else if (MODE == ROW_INV_REAL) {
      cp_async8(x + idx, a.cbuf + (size_t)q * a.ldc + c);
    } else if (MODE == ROW_WIENER_1D) {
      cp_async4(stage + 2 * idx, a.fin + (size_t)(2 * q) * a.ldf + c);
      if (2 * q + 1 < a.img_rows) cp_async4(stage + 2 * idx + 1, a.fin + (size_t)(2 * q + 1) * a.ldf + c);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    const int r = idx >> a.logN, c = idx & (N - 1);
    const int q = q0 + r;
    float2 v = make_float2(0.f, 0.f);
    if (q < a.nrows) {
      if (MODE == ROW_PSF) {
        // wrapped PSF image of a.nrows rows: row q holds tap row (q + cy) mod nrows
        const int cy = a.kh >> 1, cx = a.kw >> 1;
        const int ta = (q + cy) % a.nrows, tb = (c + cx) & (N - 1);
        if (ta < a.kh && tb < a.kw) v.x = __ldg(a.taps + ta * a.kw + tb);
      } else if (MODE == ROW_FWD_REAL) {
        v.x = fmaxf(stage[idx], a.floor_) - kMidGrey;
      } else if (MODE == ROW_INV_REAL) {
        v = x[idx];
      } else {  // ROW_WIENER_1D: sequence q packs image rows 2q and 2q+1
        v.x = fmaxf(stage[2 * idx], a.floor_) - kMidGrey;
        if (2 * q + 1 < a.img_rows) v.y = fmaxf(stage[2 * idx + 1], a.floor_) - kMidGrey;
      }
    }
    x[idx] = v;
  }
  __syncthreads();
  // ---- transform
  if (MODE == ROW_INV_REAL) {
    fft_dit_inv(x, a.logN, R, 1, N, tw, 0, false);
  } else {
    fft_dif(x, a.logN, R, 1, N, tw, 0, false);
    if (MODE == ROW_WIENER_1D) {
      for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
        const int c = idx & (N - 1);
        x[idx] = wiener_gain(__ldg(&a.spec[c]), x[idx], a.K);
      }
      __syncthreads();
      fft_dit_inv(x, a.logN, R, 1, N, tw, 0, false);
    }
  }
  // ---- store
  const float dc = (MODE == ROW_INV_REAL || MODE == ROW_WIENER_1D) ? dc_response(a.spec, a.K) : 0.f;
  for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    const int r = idx >> a.logN, c = idx & (N - 1);
    const int q = q0 + r;
    if (q >= a.nrows) continue;
    const float2 v = x[idx];
    if (MODE == ROW_PSF || MODE == ROW_FWD_REAL) {
      a.cbuf[(size_t)q * a.ldc + c] = v;
    } else if (MODE == ROW_INV_REAL) {
      a.uout[(size_t)q * a.ldu + c] = fmaxf(fmaf(v.x, a.scale, dc), a.floor_);
    } else {
      a.uout[(size_t)(2 * q) * a.ldu + c] = fmaxf(fmaf(v.x, a.scale, dc), a.floor_);
      if (2 * q + 1 < a.img_rows) a.uout[(size_t)(2 * q + 1) * a.ldu + c] = fmaxf(fmaf(v.y, a.scale, dc), a.floor_);
    }
  }
}

// Column transforms: each CTA owns C adjacent sequences laid out across a row
// (element stride C in shared memory).  For COL_WIENER_1D_REAL, sequence c
// packs image columns 2c and 2c+1 and a.nrows counts the image columns.
template <int MODE, int C>
__global__ void __launch_bounds__(256) k_fft_cols(FftArgs a) {
  extern __shared__ float2 smem[];
  const int N = 1 << a.logN;
  float2* tw = smem;
  float2* x = smem + N;
  float* stage = (float*)(x + N * C);  // COL_WIENER_1D_REAL: 2*C real columns
  fft_load_twiddles(tw, a.twg, N);
  const int c0 = blockIdx.x * C;  // first sequence
  const int nseq_total = (MODE == COL_WIENER_1D_REAL) ? (a.nrows + 1) / 2 : a.nrows;
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int k = idx / C, c = idx - (idx / C) * C;
    const int q = c0 + c;
    if (q >= nseq_total) continue;
    if (MODE == COL_WIENER_1D_REAL) {
      cp_async4(stage + 2 * idx, a.fin + (size_t)k * a.ldf + 2 * q);
      if (2 * q + 1 < a.nrows) cp_async4(stage + 2 * idx + 1, a.fin + (size_t)k * a.ldf + 2 * q + 1);
    } else {
      cp_async8(x + idx, a.cbuf + (size_t)k * a.ldc + q);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int c = idx - (idx / C) * C;
    const int q = c0 + c;
    if (q >= nseq_total) {
      x[idx] = make_float2(0.f, 0.f);
    } else if (MODE == COL_WIENER_1D_REAL) {
      float2 v;
      v.x = fmaxf(stage[2 * idx], a.floor_) - kMidGrey;
      v.y = (2 * q + 1 < a.nrows) ? fmaxf(stage[2 * idx + 1], a.floor_) - kMidGrey : 0.f;
      x[idx] = v;
    }
  }
  __syncthreads();
  fft_dif(x, a.logN, C, C, 1, tw, 0, true);
  if (MODE != COL_FWD) {
    for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
      const int k = idx / C, c = idx - (idx / C) * C;
      const int q = c0 + c;
      if (q >= nseq_total) continue;
      const float2 S = (MODE == COL_WIENER) ? __ldg(&a.spec[(size_t)k * a.ldspec + q]) : __ldg(&a.spec[k]);
      x[idx] = wiener_gain(S, x[idx], a.K);
    }
    __syncthreads();
    fft_dit_inv(x, a.logN, C, C, 1, tw, 0, true);
  }
  const float dc = (MODE == COL_WIENER_1D_REAL) ? dc_response(a.spec, a.K) : 0.f;
  for (int idx = threadIdx.x; idx < N * C; idx += blockDim.x) {
    const int k = idx / C, c = idx - (idx / C) * C;
    const int q = c0 + c;
    if (q >= nseq_total) continue;
    const float2 v = x[idx];
    if (MODE == COL_WIENER_1D_REAL) {
      a.uout[(size_t)k * a.ldu + 2 * q] = fmaxf(fmaf(v.x, a.scale, dc), a.floor_);
      if (2 * q + 1 < a.nrows) a.uout[(size_t)k * a.ldu + 2 * q + 1] = fmaxf(fmaf(v.y, a.scale, dc), a.floor_);
    } else {
      a.cbuf[(size_t)k * a.ldc + q] = v;
    }
  }
}

template <typename Kern>
static cudaError_t launch_smem(Kern k, dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                               const FftArgs& a) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_rows(FftArgs a, cudaStream_t s) {
  const int N = 1 << a.logN;
  const int R = N >= 2048 ? 1 : 2048 / N;
  const int grid = (a.nrows + R - 1) / R;
  const size_t smem = (size_t)(N + R * N) * sizeof(float2) + (size_t)2 * R * N * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_fft_rows<MODE><<<grid, 256, smem, s>>>(a, R);
  count_launch();
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_cols(FftArgs a, int nseq, cudaStream_t s) {
  const int N = 1 << a.logN;
  const size_t st = (MODE == COL_WIENER_1D_REAL) ? 1 : 0;  // real staging only for packed real columns
  if (N <= 1024) {
    constexpr int C = 8;
    const size_t smem = (size_t)(N + C * N) * sizeof(float2) + st * 2 * C * N * sizeof(float);
    return launch_smem(k_fft_cols<MODE, C>, dim3((nseq + C - 1) / C), dim3(256), smem, s, a);
  } else if (N <= 2048) {
    constexpr int C = 4;
    const size_t smem = (size_t)(N + C * N) * sizeof(float2) + st * 2 * C * N * sizeof(float);
    return launch_smem(k_fft_cols<MODE, C>, dim3((nseq + C - 1) / C), dim3(256), smem, s, a);
  } else {
    constexpr int C = 2;
    const size_t smem = (size_t)(N + C * N) * sizeof(float2) + st * 2 * C * N * sizeof(float);
    return launch_smem(k_fft_cols<MODE, C>, dim3((nseq + C - 1) / C), dim3(256), smem, s, a);
  }
}

cudaError_t run_psf_spectrum_2d(const float* taps, int kh, int kw, int H, int W, float2* spec,
                                const float2* twW, const float2* twH, cudaStream_t s) {
  FftArgs a = {};
  a.taps = taps; a.kh = kh; a.kw = kw; a.nrows = H; a.logN = ilog2(W);
  a.cbuf = spec; a.ldc = W; a.twg = twW;
  cudaError_t e;
  if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
  FftArgs c = {};
  c.cbuf = spec; c.ldc = W; c.nrows = W; c.logN = ilog2(H); c.twg = twH;
  return launch_cols<COL_FWD>(c, W, s);
}

cudaError_t run_wiener(const float* f, float* u0, int H, int W, int ld, const float* taps, int kh,
                       int kw, float K, float floor_, void* ws, const WsLayout& L, int* status,
                       cudaStream_t s) {
  (void)status;
  char* base = (char*)ws;
  float2* spec = (float2*)(base + L.spec);
  float2* work = (float2*)(base + L.work);
  float2* twW = (float2*)(base + L.tw);
  float2* twH = twW + W;
  cudaError_t e;
  if (kw > 1 || kh == 1) { if ((e = launch_twiddles(twW, W, s)) != cudaSuccess) return e; }
  if (kh > 1) { if ((e = launch_twiddles(twH, H, s)) != cudaSuccess) return e; }
  FftArgs a = {};
  a.K = K;
  a.floor_ = floor_;
  if (kh == 1) {
    // PSF along rows: 1D spectrum of length W, then packed row pairs.
    a.taps = taps; a.kh = 1; a.kw = kw; a.nrows = 1; a.logN = ilog2(W);
    a.cbuf = spec; a.ldc = W; a.twg = twW;
    if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
    FftArgs b = {};
    b.fin = f; b.ldf = ld; b.uout = u0; b.ldu = ld; b.spec = spec; b.twg = twW;
    b.nrows = (H + 1) / 2; b.img_rows = H; b.logN = ilog2(W);
    b.K = K; b.floor_ = floor_; b.scale = 1.0f / (float)W;
    return launch_rows<ROW_WIENER_1D>(b, s);
  }
  if (kw == 1) {
    // PSF along columns: 1D spectrum of length H (a kh x 1 tap array has the
    // memory layout of a 1 x kh row), then packed column pairs.
    a.taps = taps; a.kh = 1; a.kw = kh; a.nrows = 1; a.logN = ilog2(H);
    a.cbuf = spec; a.ldc = H; a.twg = twH;
    if ((e = launch_rows<ROW_PSF>(a, s)) != cudaSuccess) return e;
    FftArgs b = {};
    b.fin = f; b.ldf = ld; b.uout = u0; b.ldu = ld; b.spec = spec; b.twg = twH;
    b.nrows = W; b.logN = ilog2(H);
    b.K = K; b.floor_ = floor_; b.scale = 1.0f / (float)H;
    return launch_cols<COL_WIENER_1D_REAL>(b, (W + 1) / 2, s);
  }
  // General 2D PSF: spectrum (rows then columns), then the image.
  if ((e = run_psf_spectrum_2d(taps, kh, kw, H, W, spec, twW, twH, s)) != cudaSuccess) return e;
  FftArgs d = {};
  d.fin = f; d.ldf = ld; d.cbuf = work; d.ldc = W; d.nrows = H; d.logN = ilog2(W); d.floor_ = floor_;
  d.twg = twW;
  if ((e = launch_rows<ROW_FWD_REAL>(d, s)) != cudaSuccess) return e;
  FftArgs g = {};
  g.cbuf = work; g.ldc = W; g.spec = spec; g.ldspec = W; g.nrows = W; g.logN = ilog2(H); g.K = K;
  g.twg = twH;
  if ((e = launch_cols<COL_WIENER>(g, W, s)) != cudaSuccess) return e;
  FftArgs o = {};
  o.cbuf = work; o.ldc = W; o.uout = u0; o.ldu = ld; o.nrows = H; o.logN = ilog2(W); o.twg = twW;
  o.floor_ = floor_; o.scale = 1.0f / ((float)H * (float)W); o.spec = spec; o.K = K;
  return launch_rows<ROW_INV_REAL>(o, s);
}

}  // namespace db
