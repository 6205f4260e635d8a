// Internal declarations shared by the libdeblur translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "libdeblur.h"

namespace db {

// A run of up to kMaxGroupH vertically adjacent taps of one PSF column:
// weights w[k] at offsets (dy0 + k, dx) from the origin (weights beyond the
// group's height are 0).  Groups are stored sorted by height; the height
// classes are delimited by the class starts (group_class_starts).
constexpr int kMaxGroupH = 7;
struct TapGroup {
  float w[7];  // kMaxGroupH <= 7
  int16_t dy0, dx;
};
static_assert(sizeof(TapGroup) == 32, "TapGroup is 32 bytes");
// Shared-memory record of a group: (w0, w1, w2, offset bits), (w3 .. w6).
constexpr int kGroupRecordBytes = 32;
// Class starts written by k_prepare_taps next to the group count: starts[m-1]
// is the first group of height m, starts[kMaxGroupH] the group count.
__host__ __device__ inline const int* group_class_starts(const int* ngroups) { return ngroups + 264; }
__host__ __device__ inline int* group_class_starts(int* ngroups) { return ngroups + 264; }

// RRRL parameters as the kernels consume them.
struct RrlParams {
  float alpha, eps_phi, eps_psi, floor;
  int phi_robust, psi_tv;
  const float* rf_lut;  // table of r_1 (DB_RF_LUT), nullptr: log1p form
};

// Table of r_1 for DB_RF_LUT (rf_lut.cu): entries at s_j = j * 65/kRfLutN.
constexpr int kRfLutN = 8192;
constexpr float kRfLutSmax = 65.0f;
const float* rf_lut_device();  // this device's table, or nullptr in log1p mode
int rf_mode();

// r_f(b) = b - f - f ln(b/f) (Eq. 7).  log1p form: f (t - log1p t) with
// t = (b - f)/f, free of cancellation near b = f.  Table form (Sec. 4.1):
// f r_1(b/f), r_1 interpolated linearly between table entries, the closed
// form below the first entry, the tangent at 65 beyond the table.
__device__ __forceinline__ float rf_divergence(float b, float f, const RrlParams& p) {
  if (p.rf_lut) {
    const float x = __fdividef(b, f);
    const float k = x * ((float)kRfLutN / kRfLutSmax);
    float r1;
    if (k < 1.0f) {
      r1 = x - 1.0f - logf(x);
    } else if (x > kRfLutSmax) {
      r1 = fmaf(1.0f - 1.0f / kRfLutSmax, x - kRfLutSmax, __ldg(p.rf_lut + kRfLutN - 1));
    } else {
      const int j = min((int)k, kRfLutN - 1);
      const float fr = k - (float)j;
      const float a = __ldg(p.rf_lut + j - 1), c = __ldg(p.rf_lut + j);
      r1 = fmaf(fr, c - a, a);
    }
    return f * r1;
  }
  const float t = __fdividef(b - f, f);
  return f * (t - log1pf(t));
}

// A 1D DFT of length N along one axis: a power-of-two transform of length
// M = 2^logM (M == N), or Bluestein's form with chirp c (N values) and the
// forward transform Bf of the circular chirp (M values, M >= 2N-1).  tw is the
// twiddle table for length M.  All tables live in device memory.
struct Dft1 {
  int N, logM;
  const float2* tw;
  const float2* c;   // nullptr for power-of-two N
  const float2* Bf;
};

constexpr int kMaxSide = 4096;   // largest H or W
constexpr int kMaxTapSide = 255; // largest kh or kw

// Number of kernels this library has launched (host-side count).
void count_launch(int n = 1);

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Copy an H x W float image between buffers of row strides dst_ld and src_ld
// (bytes), as one linear copy when both are packed: row-wise copies of short
// rows between host and device ran at less than half the linear rate.
inline cudaError_t copy_image_async(void* dst, size_t dst_ld, const void* src, size_t src_ld, int H, int W,
                                    cudaMemcpyKind kind, cudaStream_t s) {
  const size_t row = (size_t)W * sizeof(float);
  if (dst_ld == row && src_ld == row) return cudaMemcpyAsync(dst, src, row * (size_t)H, kind, s);
  return cudaMemcpy2DAsync(dst, dst_ld, src, src_ld, row, (size_t)H, kind, s);
}
// Bytes k_prepare_taps writes next to the tap groups: the group count (int),
// at +4 the dense flag, at +16 the box weights (e0, w, e1, L), at +32 the taps of a one-axis PSF,
// at +1056 the group class starts (kMaxGroupH + 1 ints).
constexpr size_t kAuxBytes = 1280;
// Form of the split and flow tiles for a PSF: 0 tap groups, 1 box
// (sliding-window sums), 2 other one-axis PSF of length >= one_axis_min()
// (register-window tap sums).
int one_axis_min(bool row);
// Smallest share of non-zero taps (percent) for which k_prepare_taps selects
// the dense bodies of an eligible 2D PSF (db_set_dense_min; 101: never).
int dense_min_pct();
inline int axis_mode(int kind, int kh, int kw) {
  if (kind == DB_PSF_BOX) return 1;
  return (kh == 1 || kw == 1) && kh * kw >= one_axis_min(kh == 1) ? 2 : 0;
}
// Row pitches of workspace images: float rows padded to 16 bytes, float2
// (q) rows to an even count, so that tile staging can copy 16-byte chunks.
__host__ __device__ inline int upitch(int W) { return (W + 3) & ~3; }
__host__ __device__ inline int qpitch(int W) { return (W + 1) & ~1; }
inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// Workspace layout for one image (offsets in bytes from ws).
struct WsLayout {
  size_t taps;     // tap_region_bytes(kh, kw): TapGroup[max_tap_groups(kh, kw)], dense table
  size_t ntaps;    // kAuxBytes: group count, one-axis weights and taps
  size_t utmp;     // float[H*upitch(W)]  (RRRL ping-pong)
  size_t qbuf;     // float2[H*upitch(W)] (split schedule: q = (e, W) interleaved with pitch qpitch(W),
                   // or planar e, W planes of pitch upitch(W) for dense PSFs; Fourier mode: Z)
  size_t spec;     // float4[spec_elems]  (PSF spectrum, float-float)
  size_t work;     // float4[work_elems]  (Wiener rows, float-float; Fourier mode: X)
  size_t s32;      // float2[H*W]         (Fourier mode: FP32 PSF spectrum)
  size_t tw;       // float2[dft_table_elems(W) + dft_table_elems(H)]  (transform tables)
  size_t kspec;    // float4[wiener_kspec_elems]  (Wiener filter spectra, float-float)
  size_t flow;     // flow_ws_bytes(H, W): task counter and per-tile progress counters
  size_t total;
};
// n: images sharing it.  iterate_only: the regions db_rrl_iterate reads in
// spatial mode (taps, ping-pong, q, flow counters), without the Wiener
// spectrum, work rows and transform tables.
WsLayout ws_layout(int H, int W, int kh, int kw, int conv, int n = 1, bool iterate_only = false);
// Bytes of the iterate_only layout (0 for invalid arguments).
size_t rrl_iterate_ws_bytes(int H, int W, const db_psf* psf, const db_params* p);
// Copy n images of H x W: image z from src + z*zsrc (pitch lds) to dst + z*zdst (pitch ldd).
cudaError_t copy_images(const float* src, int lds, long long zsrc, float* dst, int ldd, long long zdst, int H, int W,
                        int n, cudaStream_t s);

// ---- tap tables ----------------------------------------------------------
// Upper bound of the tap-group count of a kh x kw PSF.
__host__ __device__ inline int max_tap_groups(int kh, int kw) { return kw * ((kh + 2) / 3); }
// Dense 2D PSFs (rrl_dense.cuh): odd sides from 3 to kDenseMaxSide.  For
// these shapes k_prepare_taps also writes the taps as a dense table (kh rows
// of dense_tap_stride(kw) floats, 16-byte aligned) after the tap groups, and
// sets the flag word dense_flag(ngroups) when at least half the taps are
// non-zero: the split and batched tile bodies then use the dense sums.
constexpr int kDenseMaxSide = 25;
__host__ __device__ inline bool dense_eligible(int kh, int kw) {
  return (kh & 1) && (kw & 1) && kh >= 3 && kw >= 3 && kh <= kDenseMaxSide && kw <= kDenseMaxSide;
}
__host__ __device__ inline int dense_tap_stride(int kw) { return (kw + 3) & ~3; }
__host__ __device__ inline size_t tap_groups_bytes(int kh, int kw) {
  return ((size_t)max_tap_groups(kh, kw) * sizeof(TapGroup) + 255) & ~size_t(255);
}
__host__ __device__ inline size_t dense_table_bytes(int kh, int kw) {
  return dense_eligible(kh, kw) ? (((size_t)kh * dense_tap_stride(kw) * 4 + 255) & ~size_t(255)) : 0;
}
// FFT tiles (rrl_fft_tile.cuh): 2D PSFs with sides 2..kFftMaxSide can run the
// split schedule's blur and correlations as 64 x 64 circular convolutions.
// Their tap region ends with the PSF's 64 x 64 spectrum (FP32 complex, in
// the transform's storage order), written when the taps are prepared.
constexpr int kFftMaxSide = 48;
constexpr size_t kFftSpecBytes = (size_t)64 * 64 * 8;
__host__ __device__ inline bool fft_tile_shape(int kh, int kw) {
  return kh >= 2 && kw >= 2 && kh <= kFftMaxSide && kw <= kFftMaxSide;
}
// Smallest kh * kw for which the split schedule and the batch use the FFT
// tiles for a PSF of fft_tile_shape (db_set_fft_tiles; above 48 * 48:
// never).  Every entry point decides from the shape alone, so that plans,
// batches and single calls run the same form.
int fft_tile_min();
constexpr int kFftTileMinDefault = 225;
inline bool fft_tile_form(int kh, int kw, int min_taps) { return fft_tile_shape(kh, kw) && kh * kw >= min_taps; }
inline bool fft_tile_form(int kh, int kw) { return fft_tile_form(kh, kw, fft_tile_min()); }
// Bytes of the tap region of a workspace: the groups, the dense table and
// the FFT-tile spectrum.
__host__ __device__ inline size_t tap_region_bytes(int kh, int kw) {
  return tap_groups_bytes(kh, kw) + dense_table_bytes(kh, kw) + (fft_tile_shape(kh, kw) ? kFftSpecBytes : 0);
}
__host__ __device__ inline const float2* fft_tile_spec(const TapGroup* groups, int kh, int kw) {
  return (const float2*)((const char*)groups + tap_groups_bytes(kh, kw) + dense_table_bytes(kh, kw));
}
__host__ __device__ inline const float* dense_taps(const TapGroup* groups, int kh, int kw) {
  return (const float*)((const char*)groups + tap_groups_bytes(kh, kw));
}
// Flag word next to the group count: 1 when the dense sums are used.
__host__ __device__ inline const int* dense_flag(const int* ngroups) { return ngroups + 1; }

// ---- launchers (return cudaError_t of the launch) --------------------------
cudaError_t launch_prepare_taps(const float* taps, int kh, int kw, int kind, TapGroup* groups,
                                int* ngroups, int* status, cudaStream_t s);
size_t rrl_spatial_smem(int kh, int kw);
size_t rrl_split_smem(int kh, int kw);  // larger of the two split kernels (direct sums)
size_t rrl_fft_tile_smem(int kh);       // larger of the two FFT-tile split kernels
// axis: 0 tap groups or dense sums, 1 box sums, 2 register windows (one-axis
// PSFs), 3 FFT tiles (2D PSFs of fft_tile_shape)
cudaError_t launch_rrl_split(const float* f, int ldf, const float* uin, int ldin, float* uout,
                             int ldout, float2* q, int H, int W, const TapGroup* groups,
                             const int* ngroups, int kh, int kw, const RrlParams& p, int* status,
                             int ng_bound, int axis, cudaStream_t s, int nz = 1, long long zf = 0,
                             long long zin = 0, long long zout = 0, long long zq = 0);
size_t rrl_box_smem(int kh, int kw);  // split kernels of a one-axis PSF (kh == 1 or kw == 1)

// all iterations in one persistent launch ordered by tile dependencies;
// flow_ws: flow_ws_bytes(H, W), 256-byte aligned
size_t flow_ws_bytes(int H, int W);
size_t flow_smem(int kh, int kw, int ng_max, int axis = 0);  // axis: axis_mode() form of the tiles

// Cluster-resident schedule (rrl_cluster.cu): the whole image in the shared
// memory of one cluster of kClusterCTAs CTAs, all iterations in one launch;
// one-row PSFs (axis 1 box, 2 register windows), H a multiple of
// 8 kClusterCTAs, W a multiple of 8, no checkpoints.
constexpr int kClusterCTAs = 8;

// Generation count of the process-wide settings (schedule, one-axis form, r_f
// evaluation, wait bound): every db_set_* call bumps it, so work captured
// under older settings is captured again.
void bump_settings();
unsigned settings_gen();
bool cluster_fits(int H, int W, int kh, int kw, int axis);
cudaError_t launch_rrl_cluster(const float* f, int ldf, float* u, int ldu, int H, int W, const int* ngroups, int kw,
                               int axis, const RrlParams& p, int iters, int* status, cudaStream_t s);
void set_flow_spin_limit(long long cycles);
cudaError_t launch_rrl_flow(const float* f, int ldf, float* u, int ldu, float* utmp, int ldt, float2* q, int H, int W,
                            const TapGroup* groups, const int* ngroups, int kh, int kw, int ng_bound,
                            const RrlParams& p, int iters, void* flow_ws, int* status, cudaStream_t s,
                            int axis = 0);

cudaError_t run_wiener(const float* f, float* u0, int H, int W, int ld, const float* taps,
                       int kh, int kw, float K, float floor_, void* ws, const WsLayout& L,
                       int* status, cudaStream_t s);

// PSF spectrum h^ on an H x W grid (bit-reversed order in both axes).
struct Dft1ff;
int dft_len_n(int N);  // transform length of an axis of N points (Bluestein: 2^a 3^b >= 2N-1)
size_t dft_table_elems(int N);  // float4 units
// float4 elements of the filter spectra of a Wiener filter whose filtering
// pass runs along a non-power-of-two axis (0 otherwise): one length-M
// spectrum for a one-axis PSF, one per half-spectrum column (W/2 + 1) for a
// 2D PSF.
size_t wiener_kspec_elems(int H, int W, int kh, int kw);
cudaError_t prepare_dft(int N, float4* tab, Dft1ff* ff, Dft1* f32, cudaStream_t s);
cudaError_t run_psf_spectrum_2d(const float* taps, int kh, int kw, int H, int W, float4* spec,
                                const Dft1ff& DW, const Dft1ff& DH, cudaStream_t s);
cudaError_t round_spectrum(const float4* in, float2* out, int H, int W, cudaStream_t s);  // column-major out
cudaError_t psf_row_spectrum(const float* taps, int kw, const Dft1ff& D, float4* out, cudaStream_t s);

// Wiener filter in two parts: set-up (tables, PSF spectrum) and image passes.
struct WienerState;
cudaError_t wiener_prepare(int H, int W, const float* taps, int kh, int kw, float K, void* ws, const WsLayout& L,
                           WienerState* st, cudaStream_t s);
cudaError_t wiener_apply(const float* f, float* u0, int ld, float K, float floor_, void* ws, const WsLayout& L,
                         const WienerState& S, cudaStream_t s);

// batched Wiener filter (host-side plan)
struct WienerImage {
  const float* f; int ld;        // observed image
  float* u0; int ldu;            // Wiener output (floored)
  int H, W;
  const float* taps; int kh, kw;
  float K, floor_;
  float4* spec;                  // PSF spectrum (1D: length of the axis; 2D: H x W)
  float4* work;                  // 2D only: H x W complex rows
  float4* kspec;                 // filter spectra (wiener_kspec_elems), or null
  const Dft1ff* pDW;             // transforms (tables already prepared)
  const Dft1ff* pDH;
};
struct WienerBatch;
WienerBatch* wiener_batch_new();
size_t wiener_job_bytes();
void wiener_batch_delete(WienerBatch* b);
cudaError_t wiener_batch_add(WienerBatch* b, const WienerImage& im, cudaStream_t s);
size_t wiener_batch_table_bytes(const WienerBatch* b);
cudaError_t wiener_batch_upload(WienerBatch* b, void* dst, cudaStream_t s);
cudaError_t wiener_batch_run(const WienerBatch* b, cudaStream_t s);

// Fourier-mode (periodic) RRRL iterations, in place on u.
cudaError_t run_rrl_fourier(const float* f, int ldf, float* u, int ld, float* utmp, int H, int W,
                            float2* X, float2* Z, const float2* S, const float2* twW,
                            const float2* twH, const RrlParams& p, int iters, float* ckpt,
                            int ckpt_every, int* status, cudaStream_t s);

cudaError_t launch_rrl_spatial(const float* f, int ldf, const float* uin, int ldin, float* uout,
                               int ldout, int H, int W, const TapGroup* groups, const int* ngroups,
                               int kh, int kw, const RrlParams& p, int* status, cudaStream_t s);

// Asynchronous global->shared copies (cp.async, sm_80+): each thread issues
// its copies without waiting on any of them; cp_async_wait_all() then blocks
// until this thread's copies have landed (a __syncthreads() must follow
// before other threads read them).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialization attribute may start while the previous kernel in
// the stream is still running.  pdl_trigger() lets the next kernel's CTAs be
// scheduled; pdl_wait() blocks until the previous kernel has completed and
// its writes are visible.  Every kernel below calls pdl_wait() before its
// first global-memory access.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace db
