// FFT tiles: the spatial iteration's blur and correlations for larger 2D
// PSFs computed as circular convolutions of 64 x 64 windows (Sec. 4.2
// "Fourier transform": convolution by pointwise products of spectra; the
// paper's general 2D variant, Sec. 4.3, uses FFT convolution).
//
// The result is the constant-continuation sum of Eq. 9, not the periodic
// one: a window holds u (or q) at clamped image positions, and only the
// outputs whose whole PSF footprint lies inside the window are kept, where
// circular and linear convolution coincide.  A tile therefore covers
// (65 - kh) x (65 - kw) outputs of a 64 x 64 window.
//
//  - q phase, two horizontally adjacent tiles per CTA: the complex window
//    uA + i uB goes through one forward 2D transform, a product with the
//    PSF's spectrum and one inverse transform; the real part is uA*h, the
//    imaginary part uB*h (h is real).
//  - update phase, one tile per CTA: the window e + iW, multiplied by the
//    conjugate spectrum (correlation with h*), gives Delta (real part) and
//    B (imaginary part) together.
//
// Transforms are FP32, register-resident radix-8 (fft8.cuh): 64 = 8 x 8 per
// axis, so a 2D transform is four passes of 8-point DFTs, each over 512
// groups of 8 elements, with a shared-memory exchange between passes.  The
// forward chain (rows then columns, DIF: natural order in, bit-reversed
// out), the spectrum product and the first inverse pass run back to back on
// the same registers; the inverse chain (columns then rows, DIT) returns
// natural order, so no reordering pass exists.  The PSF spectrum comes out
// of the same forward chain (k_prepare_fft_spec) in the storage order of the
// data it multiplies, scaled by 1/4096 for the unnormalised inverse.
//
// Shared layout of the 64 x 64 complex window: element (r, c) at
// r * 68 + c + c / 16.  With the thread-to-group maps below, a bank model of
// every pass finds each warp access at the minimum of two wavefronts.
//
// The bodies run with 256 threads (two groups of every pass per thread, so
// that each thread has two independent chains in flight).  Every output is
// a fixed function of its window, independent of the launch, so the split
// kernels and the batched kernel give the same bits.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"
#include "fft8.cuh"
#include "internal.cuh"
#include "rrl_tiles.cuh"
#include "tma.cuh"

namespace db {
namespace ftile {

constexpr int kN = 64;              // window side
constexpr int kRS = 68;             // row stride of the complex window (float2)
constexpr int kPos = kN * kRS;      // float2 slots of the window
constexpr int kGroups = 512;        // groups of 8 elements per pass
constexpr int kUS = 72;             // row stride of the staged u (update phase)
constexpr int kThreads = 256;       // threads of a CTA running the bodies
constexpr int kSR = 4;              // rows of an update strip
constexpr int kTS = 10;             // row stride of the twiddle table (float2): the 16-byte
                                    // reads of the eight rows fall on distinct banks
constexpr int kTwSlots = 8 * kTS;   // float2 slots of the twiddle table

__device__ __forceinline__ int tid_flat() { return threadIdx.y * blockDim.x + threadIdx.x; }

// Twiddle table of the top passes: tw[kTS j + s] = w^(j bitrev3(s)),
// w = exp(-2 pi i / 64), the factor of output slot s of group j (slot s of
// dif8 holds DFT index bitrev3(s)); one CTA-wide table of 8 rows.
__device__ __forceinline__ void make_twiddles(float2* tw) {
  const int t = tid_flat();
  if (t < kN) {
    const int j = t >> 3, sl = t & 7;
    const int e = ((sl & 1) << 2) | (sl & 2) | (sl >> 2);
    float sn, cs;
    sincospif(-(float)(j * e) / 32.0f, &sn, &cs);
    tw[kTS * j + sl] = make_float2(cs, sn);
  }
}

__device__ __forceinline__ void group_twiddles(const float2* tw, int j, float2 (&w)[8]) {
  const float4* t4 = reinterpret_cast<const float4*>(tw + kTS * j);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = t4[k];
    w[2 * k] = make_float2(v.x, v.y);
    w[2 * k + 1] = make_float2(v.z, v.w);
  }
}

// Group maps.  Row passes: top groups (r, j) hold columns j + 8m, bottom
// groups (r, t) columns 8t + m; column passes: top groups (c, j) rows j + 8m,
// bottom groups (c, t) rows 8t + m (m = 0..7, the register index).
__device__ __forceinline__ void row_top_group(int g, int& r, int& j) {
  j = g & 7;
  const int rs = (g >> 3) & 3;  // rows r, r+2 share a half-warp
  r = ((g >> 5) << 2) + ((rs & 1) << 1) + (rs >> 1);
}
__device__ __forceinline__ int row_top_base(int r, int j) { return r * kRS + j; }
__device__ __forceinline__ constexpr int row_top_off(int m) { return 8 * m + (m >> 1); }
__device__ __forceinline__ int row_bot_base(int g) {
  const int t = g & 7, r = g >> 3;
  return r * kRS + 8 * t + (t >> 1);
}
__device__ __forceinline__ int col_top_base(int g) {
  const int c = g & 63, j = g >> 6;
  return j * kRS + c + (c >> 4);
}
__device__ __forceinline__ int col_bot_base(int g) {
  const int c = g & 63, t = g >> 6;
  return 8 * t * kRS + c + (c >> 4);
}

// Forward row top pass: elements from ld(r, c), DIF with twiddles, to A.
// Both groups' elements are loaded before either is transformed (sixteen
// loads in flight per thread).  SYNC: ld reads shared memory that A
// overlays, so every thread's loads finish (CTA barrier) before any writes.
template <bool SYNC = false, class Load>
__device__ __forceinline__ void rows_top_fwd(float2* A, const float2* tw, Load ld) {
  const int g0 = tid_flat();
  int r[2], j[2];
  row_top_group(g0, r[0], j[0]);
  row_top_group(g0 + kThreads, r[1], j[1]);
  float2 v[2][8];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int m = 0; m < 8; ++m) v[h][m] = ld(r[h], j[h] + 8 * m);
  if (SYNC) __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    f8::dif8(v[h]);
    float2 w[8];
    group_twiddles(tw, j[h], w);
#pragma unroll
    for (int s = 1; s < 8; ++s) v[h][s] = cmul(v[h][s], w[s]);
    float2* p = A + row_top_base(r[h], j[h]);
#pragma unroll
    for (int m = 0; m < 8; ++m) p[row_top_off(m)] = v[h][m];
  }
}

// Inverse row top pass over the rows r_lo <= r < r_hi: conjugate twiddles,
// DIT, natural-order elements to out(r, c, value).
template <class Out>
__device__ __forceinline__ void rows_top_inv(const float2* A, const float2* tw, int r_lo, int r_hi, Out out) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int g = tid_flat() + h * kThreads;
    int r, j;
    row_top_group(g, r, j);
    if (r < r_lo || r >= r_hi) continue;
    const float2* p = A + row_top_base(r, j);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = p[row_top_off(m)];
    float2 w[8];
    group_twiddles(tw, j, w);
#pragma unroll
    for (int s = 1; s < 8; ++s) v[s] = cmulc(v[s], w[s]);
    f8::dit8_inv(v);
#pragma unroll
    for (int m = 0; m < 8; ++m) out(r, j + 8 * m, v[m]);
  }
}

// Row bottom pass (no twiddles), forward or inverse, in place, over the
// rows r_lo <= r < r_hi.
template <bool INV>
__device__ __forceinline__ void rows_bot(float2* A, int r_lo = 0, int r_hi = kN) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int g = tid_flat() + h * kThreads;
    if ((g >> 3) < r_lo || (g >> 3) >= r_hi) continue;
    float2* p = A + row_bot_base(g);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = p[m];
    if (INV) f8::dit8_inv(v);
    else f8::dif8(v);
#pragma unroll
    for (int m = 0; m < 8; ++m) p[m] = v[m];
  }
}

// Column top pass, forward (DIF, then twiddles) or inverse (conjugate
// twiddles, then DIT), in place.
template <bool INV>
__device__ __forceinline__ void cols_top(float2* A, const float2* tw) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int g = tid_flat() + h * kThreads;
    float2* p = A + col_top_base(g);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = p[8 * kRS * m];
    float2 w[8];
    group_twiddles(tw, g >> 6, w);
    if (!INV) {
      f8::dif8(v);
#pragma unroll
      for (int s = 1; s < 8; ++s) v[s] = cmul(v[s], w[s]);
    } else {
#pragma unroll
      for (int s = 1; s < 8; ++s) v[s] = cmulc(v[s], w[s]);
      f8::dit8_inv(v);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) p[8 * kRS * m] = v[m];
  }
}

// Column bottom pass: forward DIF, product with the spectrum (conjugated
// for a correlation), inverse DIT, in place.  The spectrum is stored as
// spec[m * 512 + g] for register m of group g (coalesced reads).
template <bool CONJ>
__device__ __forceinline__ void cols_bot_product(float2* A, const float2* __restrict__ spec) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int g = tid_flat() + h * kThreads;
    float2* p = A + col_bot_base(g);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = p[kRS * m];
    f8::dif8(v);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float2 s = __ldg(spec + m * kGroups + g);
      v[m] = CONJ ? cmulc(v[m], s) : cmul(v[m], s);
    }
    f8::dit8_inv(v);
#pragma unroll
    for (int m = 0; m < 8; ++m) p[kRS * m] = v[m];
  }
}

// out(r, c, y) for y = IDFT(DFT(x) . S) (CONJ: . conj(S)) over the 64 x 64
// window x(r, c) = ld(r, c), S the prepared spectrum (1/4096 included), for
// the rows r_lo <= r < r_hi (the inverse row passes skip the others).
// tw must be ready and A free on entry (the caller's barrier); the
// barriers between passes are inside.
// The two row passes of a row exchange data within one warp (both group
// maps give warp w the rows 4w..4w+3 and 32+4w..32+4w+3), so a warp barrier
// separates them; the column passes span four warps and take CTA barriers.
template <bool CONJ, bool SYNC_LOAD = false, class Load, class Out>
__device__ __forceinline__ void conv64(float2* A, const float2* tw, const float2* __restrict__ spec, int r_lo,
                                       int r_hi, Load ld, Out out) {
  rows_top_fwd<SYNC_LOAD>(A, tw, ld);
  __syncwarp();
  rows_bot<false>(A);
  __syncthreads();
  cols_top<false>(A, tw);
  __syncthreads();
  cols_bot_product<CONJ>(A, spec);
  __syncthreads();
  cols_top<true>(A, tw);
  __syncthreads();
  rows_bot<true>(A, r_lo, r_hi);
  __syncwarp();
  rows_top_inv(A, tw, r_lo, r_hi, out);
}

// Spectrum of the PSF for conv64: the circular kernel k(r, c) = h(a, b) at
// r = (a - cy) mod 64, c = (b - cx) mod 64 (centre (kh/2, kw/2)), through the
// forward chain, times 1/4096.  One CTA; A: kPos float2 of shared memory.
__device__ __forceinline__ void psf_spectrum(float2* A, float2* tw, const float* __restrict__ taps, int kh, int kw,
                                             float2* __restrict__ spec) {
  make_twiddles(tw);
  __syncthreads();
  const int cy = kh >> 1, cx = kw >> 1;
  rows_top_fwd(A, tw, [&](int r, int c) {
    const int a = (r + cy) & (kN - 1), b = (c + cx) & (kN - 1);
    return make_float2(a < kh && b < kw ? __ldg(taps + a * kw + b) : 0.0f, 0.0f);
  });
  __syncwarp();
  rows_bot<false>(A);
  __syncthreads();
  cols_top<false>(A, tw);
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int g = tid_flat() + h * kThreads;
    const float2* p = A + col_bot_base(g);
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = p[kRS * m];
    f8::dif8(v);
    constexpr float sc = 1.0f / 4096.0f;
#pragma unroll
    for (int m = 0; m < 8; ++m) spec[m * kGroups + g] = make_float2(v[m].x * sc, v[m].y * sc);
  }
}

// Outputs of a tile: rows (65 - kh), columns (65 - kw).
__host__ __device__ inline int tile_oh(int kh) { return kN + 1 - kh; }
__host__ __device__ inline int tile_ow(int kw) { return kN + 1 - kw; }

// Shared memory of the bodies (bytes): twiddles, window, staged u.
__host__ __device__ inline int staged_u_rows(int kh) { return ((tile_oh(kh) + kSR - 1) / kSR) * kSR + 4; }
__host__ __device__ inline size_t smem_q() { return (size_t)(kTwSlots + kPos) * sizeof(float2); }
__host__ __device__ inline size_t smem_update(int kh) {
  return smem_q() + (size_t)staged_u_rows(kh) * kUS * sizeof(float);
}

// TMA staging of the q phase's u window (tma.cuh): both tiles' windows,
// columns xa .. xb + 63, as one box of kN rows x kBoxW columns whose x starts
// at xa rounded down to a multiple of 4.  The box overlays the transform
// buffer A exactly (kBoxW floats = kRS float2 per row): its row stride of
// 136 floats puts the four rows a warp's first pass reads on distinct banks.
constexpr int kBoxW = 2 * kRS;
static_assert(kBoxW % 4 == 0 && kBoxW >= 3 + 2 * kN + 2 && kN * kBoxW * 4 == kPos * 8, "box over A");
struct WinTma {
  const CUtensorMap* map;   // 3D map (W, H, images) of u with kBoxW x kN x 1 boxes
  int z;                    // the image's index in the map
  unsigned long long* bar;  // the CTA's mbarrier (count 1)
  unsigned parity;          // parity of the barrier phase this copy completes
  long long limit;          // bound of the wait (clock cycles)
  int* status;              // DB_FLAG_TIMEOUT if the wait runs out
};

// q = (e, W) on the tiles at (i0, j0) and (i0, j0 + OW) (the second one if it
// starts inside the image), planar: qe, qw (pitch ldqp).  The u window of a
// tile starts dy = kh-1-kh/2 rows and dx = kw-1-kw/2 columns before it: the
// blur b(i, j) = sum h(a, b) u(i - a + kh/2, j - b + kw/2) reaches that far
// up and left.  smem_raw: smem_q() bytes.  With `tma` (and A 128-byte
// aligned) the windows arrive by one TMA copy; elements outside the image
// then take their clamped neighbours' values in shared memory, so that both
// ways load the same values and give the same bits.
template <typename Dep = NoDep>
__device__ __forceinline__ void q_tile(unsigned char* smem_raw, const float* __restrict__ f, int ldf,
                                       const float* uin, int ldin, float* qe, float* qw, int ldqp, int H, int W,
                                       const float2* __restrict__ spec, int kh, int kw, const RrlParams& p, int i0,
                                       int j0, Dep dep = Dep(), const WinTma* tma = nullptr) {
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* A = tw + kTwSlots;
  make_twiddles(tw);
  const int dy = kh - 1 - (kh >> 1), dx = kw - 1 - (kw >> 1);
  const int OH = tile_oh(kh), OW = tile_ow(kw);
  const int ys = i0 - dy, xa = j0 - dx, xb = xa + OW;
  const bool has_b = j0 + OW < W;
  // both windows inside the image: no clamping
  const bool inside = ys >= 0 && ys + kN <= H && xa >= 0 && (has_b ? xb : xa) + kN <= W;
  dep();
  float* box = reinterpret_cast<float*>(A);
  const int x0 = xa & ~3, e = xa - x0;  // x0: a multiple of 4 at or left of xa
  const bool staged = tma != nullptr && (smem_u32(box) & 127u) == 0;
  if (staged) {
    if (tid_flat() == 0) {
      fence_proxy_async_smem();  // the CTA's earlier uses of A (barrier before the tile) come first
      mbar_arrive_expect_tx(tma->bar, kN * kBoxW * (unsigned)sizeof(float));
      tma_load_3d(box, tma->map, x0, ys, tma->z, tma->bar);
    }
    const bool late = !mbar_wait_bounded(tma->bar, tma->parity, tma->limit);
    if (__syncthreads_or(late)) {  // also publishes the twiddles
      if (tid_flat() == 0 && tma->status) atomicOr(tma->status, DB_FLAG_TIMEOUT);
      (void)mbar_wait_bounded(tma->bar, tma->parity, tma->limit);  // the copy in flight, bounded again
      return;
    }
    if (!inside) {  // constant continuation: outside elements copy their clamped neighbours
      for (int k = tid_flat(); k < kN * kBoxW; k += kThreads) {
        const int t = k / kBoxW, c = k - t * kBoxW;
        const int ty = min(max(ys + t, 0), H - 1) - ys, tx = min(max(x0 + c, 0), W - 1) - x0;
        if (ty != t || tx != c) box[k] = box[ty * kBoxW + tx];
      }
      __syncthreads();
    }
    conv64<false, true>(
        A, tw, spec, dy, dy + OH,
        [&](int r, int c) {
          const float* row = box + r * kBoxW + e + c;
          return make_float2(row[0], has_b ? row[OW] : 0.0f);
        },
        [&](int r, int c, float2 v) { A[r * kRS + c + (c >> 4)] = v; });
  } else {
    __syncthreads();  // twiddles
    conv64<false>(
        A, tw, spec, dy, dy + OH,
        [&](int r, int c) {
          if (inside) {
            const float* row = uin + (size_t)(ys + r) * ldin;
            return make_float2(row[xa + c], has_b ? row[xb + c] : 0.0f);
          }
          const float* row = uin + (size_t)min(max(ys + r, 0), H - 1) * ldin;
          const float a = row[min(max(xa + c, 0), W - 1)];
          const float b = has_b ? row[min(max(xb + c, 0), W - 1)] : 0.0f;
          return make_float2(a, b);
        },
        // each (bA, bB) back into the slot its group read it from
        [&](int r, int c, float2 v) { A[r * kRS + c + (c >> 4)] = v; });
  }
  __syncthreads();
  // (e, W) over both tiles' outputs as one row of 2 OW columns: consecutive
  // threads take consecutive image columns.  A thread's items go in groups of
  // kQB whose f loads are issued together.
  constexpr int kQB = 4;
  const int nr = min(OH, H - i0), nc = min(2 * OW, W - j0), n = nr * nc;
  // item = oi nc + oj2, advanced by kThreads = dq nc + dr without a division
  const int dq = kThreads / nc, dr = kThreads - dq * nc;
  int oi_n = tid_flat() / nc, oj_n = tid_flat() - oi_n * nc;
  for (int base = tid_flat(); base < n; base += kQB * kThreads) {
    float fv[kQB];
    int ois[kQB], ojs[kQB];
#pragma unroll
    for (int k = 0; k < kQB; ++k) {
      const int item = base + k * kThreads;
      fv[k] = 0.f;
      ois[k] = oi_n;
      ojs[k] = oj_n;
      if (item < n) fv[k] = __ldg(f + (size_t)(i0 + oi_n) * ldf + j0 + oj_n);
      oi_n += dq;
      oj_n += dr;
      if (oj_n >= nc) { oj_n -= nc; ++oi_n; }
    }
#pragma unroll
    for (int k = 0; k < kQB; ++k) {
      if (base + k * kThreads >= n) break;
      const int oi = ois[k], oj2 = ojs[k];
      const int second = oj2 >= OW, c = dx + oj2 - (second ? OW : 0);
      const float2 v = A[(dy + oi) * kRS + c + (c >> 4)];
      const int i = i0 + oi, j = j0 + oj2;
      const float2 q = weighted_residual(second ? v.y : v.x, fmaxf(fv[k], p.floor), p);
      qe[(size_t)i * ldqp + j] = q.x;
      qw[(size_t)i * ldqp + j] = q.y;
    }
  }
}

// Delta, B from planar q, the diffusion term and the update on the tile at
// (i0, j0).  The q window starts kh/2 rows and kw/2 columns before the tile
// (the correlation reaches that far up and left).  The transform leaves
// (Delta, B) in the window's shared-memory slots; the update then runs in
// vertical strips of kSR outputs (the diffusion term shares its stencil rows
// within a strip).  u is staged with two pixels of halo from the 4-column
// boundary at or left of j0 - 2.  smem_raw: smem_update(kh) bytes.
template <typename Dep = NoDep>
__device__ __forceinline__ void update_tile(unsigned char* smem_raw, const float* qe, const float* qw, int ldqp,
                                            const float* uin, int ldin, float* __restrict__ uout, int ldout, int H,
                                            int W, const float2* __restrict__ spec, int kh, int kw,
                                            const RrlParams& p, int* status, int i0, int j0, Dep dep = Dep()) {
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* A = tw + kTwSlots;
  float* us = reinterpret_cast<float*>(A + kPos);
  make_twiddles(tw);
  const int cy = kh >> 1, cx = kw >> 1;
  const int OH = tile_oh(kh), OW = tile_ow(kw);
  const int xu = (j0 - 2) & ~3;  // a multiple of 4 at or left of j0 - 2
  const int ncu = (j0 + OW + 2 - xu + 3) >> 2;
  stage_tile<float, kUS>(us, uin, ldin, H, W, i0 - 2, staged_u_rows(kh), xu, ncu, rows_aligned16(uin, ldin));
  dep();
  const int ys = i0 - cy, xs = j0 - cx;
  const bool inside = ys >= 0 && ys + kN <= H && xs >= 0 && xs + kN <= W;
  cp_async_wait_all();
  __syncthreads();  // twiddles, staged u
  conv64<true>(
      A, tw, spec, cy, cy + OH,
      [&](int r, int c) {
        const size_t o = inside ? (size_t)(ys + r) * ldqp + (xs + c)
                                : (size_t)min(max(ys + r, 0), H - 1) * ldqp + min(max(xs + c, 0), W - 1);
        return make_float2(qe[o], qw[o]);
      },
      // each (Delta, B) back into the slot its group read it from
      [&](int r, int c, float2 v) { A[r * kRS + c + (c >> 4)] = v; });
  __syncthreads();
  bool bad = false;
  const int nsr = (OH + kSR - 1) / kSR;
  // item = sr OW + oj, advanced by kThreads = dq OW + dr without a division
  const int dq = kThreads / OW, dr = kThreads - dq * OW;
  int sr = tid_flat() / OW, oj = tid_flat() - sr * OW;
  for (int item = tid_flat(); item < nsr * OW; item += kThreads, sr += dq, oj += dr) {
    if (oj >= OW) { oj -= OW; ++sr; }
    const int oi0 = sr * kSR, j = j0 + oj;
    if (j >= W) continue;
    float D[kSR], ctr[kSR];
    diffusion_strip<kSR, kUS>(us + (oi0 + 2) * kUS + (j - xu), p, D, ctr);
    const int c = cx + oj;
    const float2* a = A + (cy + oi0) * kRS + c + (c >> 4);
#pragma unroll
    for (int t = 0; t < kSR; ++t) {
      const int i = i0 + oi0 + t;
      if (oi0 + t >= OH || i >= H) break;
      const float2 v = a[t * kRS];
      const float un = rrl_update(ctr[t], v.x, v.y, D[t], p);
      bad |= !isfinite(un);
      uout[(size_t)i * ldout + j] = un;
    }
  }
  if (bad && status) atomicOr(status, DB_FLAG_NONFINITE);
}

}  // namespace ftile
}  // namespace db
