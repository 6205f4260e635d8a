// C ABI of libdeblur: argument validation, workspace layout and dispatch.
// The operations themselves are documented in include/libdeblur.h.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_df.cuh"
#include "internal.cuh"

#include <atomic>

namespace db {

static std::atomic<long long> g_launches{0};
static std::atomic<int> g_schedule{0};
static std::atomic<unsigned> g_settings_gen{0};
void bump_settings() { g_settings_gen.fetch_add(1); }
unsigned settings_gen() { return g_settings_gen.load(); }
static std::atomic<int> g_one_axis_min{0};
static std::atomic<int> g_dense_min_pct{50};
int dense_min_pct() { return g_dense_min_pct.load(std::memory_order_relaxed); }
static std::atomic<int> g_fft_tile_min{kFftTileMinDefault};
int fft_tile_min() { return g_fft_tile_min.load(std::memory_order_relaxed); }
int one_axis_min(bool row) {
  const int v = g_one_axis_min.load(std::memory_order_relaxed);
  return v > 0 ? v : row ? 16 : 32;
}
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

WsLayout ws_layout(int H, int W, int kh, int kw, int conv, int n, bool iterate_only) {
  const bool spatial_only = iterate_only && conv != DB_CONV_PERIODIC;
  WsLayout L = {};
  size_t off = 0;
  L.taps = off;  off += tap_region_bytes(kh, kw);
  L.ntaps = off; off += kAuxBytes;
  L.utmp = off;  off += align256((size_t)n * H * upitch(W) * sizeof(float));
  L.qbuf = off;  off += align256((size_t)n * H * upitch(W) * sizeof(float2));
  size_t spec_elems, work_elems;
  if (conv == DB_CONV_PERIODIC) { spec_elems = (size_t)H * W; work_elems = (size_t)H * W; }
  else if (kh == 1) { spec_elems = (size_t)W; work_elems = 0; }
  else if (kw == 1) { spec_elems = (size_t)H; work_elems = 0; }
  else { spec_elems = (size_t)H * W; work_elems = (size_t)H * W; }
  if (spatial_only) { spec_elems = 0; work_elems = 0; }
  L.spec = off;  off += align256(spec_elems * sizeof(float4));
  L.work = off;  off += align256(work_elems * sizeof(float4));
  L.s32 = off;   off += (conv == DB_CONV_PERIODIC) ? align256((size_t)H * W * sizeof(float2)) : 0;
  L.tw = off;    off += spatial_only ? 0 : align256((dft_table_elems(W) + dft_table_elems(H)) * sizeof(float4));
  L.kspec = off; off += spatial_only ? 0 : align256(wiener_kspec_elems(H, W, kh, kw) * sizeof(float4));
  L.flow = off;  off += (conv == DB_CONV_PERIODIC) ? 0 : align256(flow_ws_bytes(H, W));
  L.total = off;
  return L;
}

static db_status check_image(const void* a, const void* b, int H, int W, int ld) {
  if (!a || !b) return DB_ERR_ARG;
  if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide || ld < W) return DB_ERR_SHAPE;
  return DB_OK;
}

static db_status check_psf(const db_psf* psf, int H, int W) {
  if (!psf || !psf->taps) return DB_ERR_ARG;
  if (psf->kh < 1 || psf->kw < 1 || psf->kh > kMaxTapSide || psf->kw > kMaxTapSide) return DB_ERR_PSF;
  if (psf->kh > H || psf->kw > W) return DB_ERR_PSF;
  if (psf->kind != DB_PSF_GENERAL && psf->kind != DB_PSF_BOX) return DB_ERR_ARG;
  if (psf->kind == DB_PSF_BOX && psf->kh != 1 && psf->kw != 1) return DB_ERR_PSF;
  return DB_OK;
}

static db_status check_params(const db_params* p) {
  if (!p) return DB_ERR_ARG;
  if (!(p->K > 0.f) || !(p->alpha >= 0.f) || !(p->eps_phi > 0.f) || !(p->eps_psi > 0.f) ||
      !(p->pos_floor > 0.f))
    return DB_ERR_ARG;
  if (p->conv != DB_CONV_CLAMP && p->conv != DB_CONV_PERIODIC) return DB_ERR_ARG;
  if ((p->phi_robust != 0 && p->phi_robust != 1) || (p->psi_tv != 0 && p->psi_tv != 1)) return DB_ERR_ARG;
  return DB_OK;
}

static db_status check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (!ws || ((uintptr_t)ws & 255u) != 0) return DB_ERR_WORKSPACE;
  if (ws_bytes < need) return DB_ERR_WORKSPACE;
  return DB_OK;
}

static bool wiener_supported(int H, int W, int kh, int kw) {
  (void)kh; (void)kw;
  return H <= kMaxSide && W <= kMaxSide;  // any size: Bluestein covers other lengths
}

static RrlParams to_rrl(const db_params* p) {
  RrlParams r;
  r.alpha = p->alpha; r.eps_phi = p->eps_phi; r.eps_psi = p->eps_psi; r.floor = p->pos_floor;
  r.phi_robust = p->phi_robust; r.psi_tv = p->psi_tv;
  r.rf_lut = rf_lut_device();
  return r;
}

// Spatial-mode iterations with tap groups already prepared in the workspace.
// ng_bound: the tap-group count when the caller knows it (0 otherwise).
// kind: one-axis PSFs (a box, or kh == 1 or kw == 1) run the one-axis form of
// the split schedule unless the flow or fused schedule is set explicitly.
// sched_in, axis_in (>= 0): a plan's tuned schedule and one-axis form
// (0 tap groups, 2 register windows), overriding the process-wide settings.
static db_status iterate_spatial(const float* f, float* u, int H, int W, int ld, int kh, int kw, int kind,
                                 const RrlParams& rp, int iters, float* ckpt, int ckpt_every, void* ws,
                                 const WsLayout& L, int* dev_status, cudaStream_t s, int ng_bound = 0,
                                 int sched_in = -1, int axis_in = -1) {
  char* base = (char*)ws;
  TapGroup* groups = (TapGroup*)(base + L.taps);
  int* ngroups = (int*)(base + L.ntaps);
  float* tmp = (float*)(base + L.utmp);
  float2* qbuf = (float2*)(base + L.qbuf);
  // schedule: split (q through a global buffer) by default; its flow form
  // (all iterations in one launch, no checkpoints) from 512K to 2M pixels,
  // where enough tiles keep every SM busy with overlapping phases while the
  // image stays resident in L2.  Measured on B300 (us per iteration, fused /
  // split / flow): 1024^2 line PSF 53 / 27 / 26; 1536^2 124 / 68 / 76; 4096^2
  // 752 / 348 / 425; the fused schedule's halo recompute costs more than q's
  // round trip at every size.
  int sched = sched_in >= 0 ? sched_in : g_schedule.load();
  // form: axis_mode's one-axis forms; 2D PSFs of fft_tile_shape take the FFT
  // tiles (3) by the size rule or by a plan's tuned form
  int axis = axis_mode(kind, kh, kw);
  if (axis_in >= 0 && axis != 1)
    axis = (axis_in == 2 && (kh == 1 || kw == 1)) ? 2 : (axis_in == 3 && fft_tile_shape(kh, kw)) ? 3 : 0;
  else if (axis == 0 && fft_tile_form(kh, kw))
    axis = 3;
  if (sched == DB_SCHED_AUTO) {
    const size_t px = (size_t)H * W;
    sched = (px >= (size_t)512 * 1024 && px <= (size_t)2 << 20) ? DB_SCHED_FLOW : DB_SCHED_SPLIT;
  }
  // the flow and cluster schedules write no checkpoints: the split schedule
  // (same tile bodies, bitwise equal result) stands in; a box keeps its
  // window sums; the cluster schedule runs one-row PSFs on images that fit
  if (sched == DB_SCHED_CLUSTER && kh == 1 && axis == 0) axis = 2;
  if (sched == DB_SCHED_CLUSTER && (ckpt || !cluster_fits(H, W, kh, kw, axis))) sched = DB_SCHED_SPLIT;
  // dense-eligible 2D PSFs run the split pair with the dense tile bodies
  if ((sched == DB_SCHED_FLOW && (ckpt || axis == 3 || (axis == 0 && dense_eligible(kh, kw)))) ||
      (sched == DB_SCHED_FUSED && axis == 1))
    sched = DB_SCHED_SPLIT;
  if (sched == DB_SCHED_FUSED) axis = 0;
  if (sched == DB_SCHED_CLUSTER) {
    const cudaError_t e = launch_rrl_cluster(f, ld, u, ld, H, W, ngroups, kw, axis, rp, iters, dev_status, s);
    if (e == cudaSuccess) return DB_OK;
    if (e != cudaErrorNotSupported) return DB_ERR_CUDA;
    sched = DB_SCHED_SPLIT;  // no cluster of this shape fits on the device
  }
  if (sched == DB_SCHED_FLOW) {
    if (flow_smem(kh, kw, ng_bound > 0 ? ng_bound : max_tap_groups(kh, kw), axis) > 227 * 1024)
      return DB_ERR_UNSUPPORTED;
    if (launch_rrl_flow(f, ld, u, ld, tmp, upitch(W), qbuf, H, W, groups, ngroups, kh, kw, ng_bound, rp, iters,
                        base + L.flow, dev_status, s, axis) != cudaSuccess)
      return DB_ERR_CUDA;
    if (iters % 2 == 1 &&
        cudaMemcpy2DAsync(u, (size_t)ld * sizeof(float), tmp, (size_t)upitch(W) * sizeof(float),
                          (size_t)W * sizeof(float), H, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return DB_ERR_CUDA;
    return DB_OK;
  }
  const size_t smem_need = axis == 3 ? rrl_fft_tile_smem(kh)
                           : axis    ? rrl_box_smem(kh, kw)
                           : sched == DB_SCHED_SPLIT ? rrl_split_smem(kh, kw) : rrl_spatial_smem(kh, kw);
  if (smem_need > 227 * 1024) return DB_ERR_UNSUPPORTED;
  const float* src = u;
  int ld_src = ld;
  for (int k = 0; k < iters; ++k) {
    if (ckpt && k % ckpt_every == 0) {
      float* dst = ckpt + (size_t)(k / ckpt_every) * H * W;
      if (cudaMemcpy2DAsync(dst, (size_t)W * sizeof(float), src, (size_t)ld_src * sizeof(float),
                            (size_t)W * sizeof(float), H, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return DB_ERR_CUDA;
    }
    float* dst = (k % 2 == 0) ? tmp : u;
    const int ld_dst = (k % 2 == 0) ? upitch(W) : ld;
    const cudaError_t e =
        sched == DB_SCHED_SPLIT
            ? launch_rrl_split(f, ld, src, ld_src, dst, ld_dst, qbuf, H, W, groups, ngroups, kh, kw, rp,
                               dev_status, ng_bound, axis, s)
            : launch_rrl_spatial(f, ld, src, ld_src, dst, ld_dst, H, W, groups, ngroups, kh, kw, rp,
                                 dev_status, s);
    if (e != cudaSuccess) return DB_ERR_CUDA;
    src = dst;
    ld_src = ld_dst;
  }
  if (src != u) {
    if (cudaMemcpy2DAsync(u, (size_t)ld * sizeof(float), src, (size_t)ld_src * sizeof(float),
                          (size_t)W * sizeof(float), H, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return DB_ERR_CUDA;
  }
  return DB_OK;
}

}  // namespace db

using namespace db;

extern "C" {

size_t db_workspace_bytes(int H, int W, const db_psf* psf, const db_params* p) {
  if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide || !psf) return 0;
  if (psf->kh < 1 || psf->kw < 1 || psf->kh > kMaxTapSide || psf->kw > kMaxTapSide) return 0;
  if (psf->kh > H || psf->kw > W || check_params(p) != DB_OK) return 0;
  return ws_layout(H, W, psf->kh, psf->kw, p->conv).total;
}

db_status db_wiener(const float* f, float* u0, int H, int W, int ld, const db_psf* psf,
                    const db_params* p, void* ws, size_t ws_bytes, int* dev_status, void* stream) {
  db_status st;
  if ((st = check_image(f, u0, H, W, ld)) != DB_OK) return st;
  if ((st = check_psf(psf, H, W)) != DB_OK) return st;
  if ((st = check_params(p)) != DB_OK) return st;
  if (f == u0) return DB_ERR_ARG;
  const WsLayout L = ws_layout(H, W, psf->kh, psf->kw, p->conv);
  if ((st = check_ws(ws, ws_bytes, L.total)) != DB_OK) return st;
  if (!wiener_supported(H, W, psf->kh, psf->kw)) return DB_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  if (launch_prepare_taps(psf->taps, psf->kh, psf->kw, psf->kind, (TapGroup*)(base + L.taps),
                          (int*)(base + L.ntaps), dev_status, s) != cudaSuccess)
    return DB_ERR_CUDA;
  if (run_wiener(f, u0, H, W, ld, psf->taps, psf->kh, psf->kw, p->K, p->pos_floor, ws, L,
                 dev_status, s) != cudaSuccess)
    return DB_ERR_CUDA;
  return DB_OK;
}

db_status db_rrl_iterate(const float* f, float* u, int H, int W, int ld, const db_psf* psf,
                         const db_params* p, int iters, float* ckpt, int ckpt_every, void* ws,
                         size_t ws_bytes, int* dev_status, void* stream) {
  db_status st;
  if ((st = check_image(f, u, H, W, ld)) != DB_OK) return st;
  if ((st = check_psf(psf, H, W)) != DB_OK) return st;
  if ((st = check_params(p)) != DB_OK) return st;
  if (iters < 0) return DB_ERR_ARG;
  if (ckpt && ckpt_every < 1) return DB_ERR_ARG;
  if (f == u) return DB_ERR_ARG;
  // spatial mode touches only the iteration regions (rrl_iterate_ws_bytes)
  const WsLayout L = ws_layout(H, W, psf->kh, psf->kw, p->conv, 1, true);
  if ((st = check_ws(ws, ws_bytes, L.total)) != DB_OK) return st;
  if (p->conv == DB_CONV_PERIODIC && !(is_pow2(H) && is_pow2(W))) return DB_ERR_UNSUPPORTED;
  if (iters == 0) return DB_OK;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  if (p->conv == DB_CONV_PERIODIC) {
    // blur and correlation through the Fourier domain (Sec. 4.3, general 2D)
    TapGroup* groups = (TapGroup*)(base + L.taps);
    if (launch_prepare_taps(psf->taps, psf->kh, psf->kw, psf->kind, groups, (int*)(base + L.ntaps),
                            dev_status, s) != cudaSuccess)
      return DB_ERR_CUDA;
    // PSF spectrum in float-float, rounded once to the FP32 copy the
    // iterations multiply with
    float4* Sff = (float4*)(base + L.spec);
    float2* S = (float2*)(base + L.s32);
    float4* tabW = (float4*)(base + L.tw);
    float4* tabH = tabW + dft_table_elems(W);
    Dft1ff FW, FH;
    Dft1 DW, DH;
    if (prepare_dft(W, tabW, &FW, &DW, s) != cudaSuccess || prepare_dft(H, tabH, &FH, &DH, s) != cudaSuccess)
      return DB_ERR_CUDA;
    if (run_psf_spectrum_2d(psf->taps, psf->kh, psf->kw, H, W, Sff, FW, FH, s) != cudaSuccess)
      return DB_ERR_CUDA;
    if (round_spectrum(Sff, S, H, W, s) != cudaSuccess) return DB_ERR_CUDA;
    if (run_rrl_fourier(f, ld, u, ld, (float*)(base + L.utmp), H, W, (float2*)(base + L.work),
                        (float2*)(base + L.qbuf), S, DW.tw, DH.tw, to_rrl(p), iters, ckpt, ckpt_every,
                        dev_status, s) != cudaSuccess)
      return DB_ERR_CUDA;
    return DB_OK;
  }
  if (launch_prepare_taps(psf->taps, psf->kh, psf->kw, psf->kind, (TapGroup*)(base + L.taps),
                          (int*)(base + L.ntaps), dev_status, s) != cudaSuccess)
    return DB_ERR_CUDA;
  return iterate_spatial(f, u, H, W, ld, psf->kh, psf->kw, psf->kind, to_rrl(p), iters, ckpt, ckpt_every, ws, L,
                         dev_status, s);
}

db_status db_deblur(const float* f, float* u, int H, int W, int ld, const db_psf* psf,
                    const db_params* p, int iters, void* ws, size_t ws_bytes, int* dev_status,
                    void* stream) {
  db_status st = db_wiener(f, u, H, W, ld, psf, p, ws, ws_bytes, dev_status, stream);
  if (st != DB_OK) return st;
  return db_rrl_iterate(f, u, H, W, ld, psf, p, iters, nullptr, 0, ws, ws_bytes, dev_status, stream);
}

// ---- N equally sized images ------------------------------------------------
size_t db_workspace_bytes_n(int H, int W, int n, const db_psf* psf, const db_params* p) {
  if (n < 1 || db_workspace_bytes(H, W, psf, p) == 0 || p->conv != DB_CONV_CLAMP) return 0;
  return ws_layout(H, W, psf->kh, psf->kw, p->conv, n).total;
}

db_status db_deblur_n(const float* f, float* u, int H, int W, int ld, int n, long long img_stride,
                      const db_psf* psf, const db_params* p, int iters, float* ckpt, int ckpt_every, void* ws,
                      size_t ws_bytes, int* dev_status, void* stream) {
  db_status st;
  if ((st = check_image(f, u, H, W, ld)) != DB_OK) return st;
  if (n < 1 || img_stride < (long long)H * ld) return DB_ERR_SHAPE;
  if ((st = check_psf(psf, H, W)) != DB_OK) return st;
  if ((st = check_params(p)) != DB_OK) return st;
  if (p->conv != DB_CONV_CLAMP) return DB_ERR_UNSUPPORTED;
  if (iters < 0 || (ckpt && ckpt_every < 1)) return DB_ERR_ARG;
  const WsLayout L = ws_layout(H, W, psf->kh, psf->kw, p->conv, n);
  if ((st = check_ws(ws, ws_bytes, L.total)) != DB_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  // Wiener: prepared once; a one-row PSF filters rows on their own, so the
  // images of a contiguous stack of even height go through as one image of
  // n*H rows (the row pairs of the packed transforms stay those of each image)
  WienerState S;
  if (wiener_prepare(H, W, psf->taps, psf->kh, psf->kw, p->K, ws, L, &S, s) != cudaSuccess) return DB_ERR_CUDA;
  if (psf->kh == 1 && img_stride == (long long)H * ld && H % 2 == 0) {  // same row pairs as one image
    WienerState Sn = S;
    Sn.H = n * H;
    if (wiener_apply(f, u, ld, p->K, p->pos_floor, ws, L, Sn, s) != cudaSuccess) return DB_ERR_CUDA;
  } else {
    for (int z = 0; z < n; ++z)
      if (wiener_apply(f + z * img_stride, u + z * img_stride, ld, p->K, p->pos_floor, ws, L, S, s) != cudaSuccess)
        return DB_ERR_CUDA;
  }
  if (launch_prepare_taps(psf->taps, psf->kh, psf->kw, psf->kind, (TapGroup*)(base + L.taps),
                          (int*)(base + L.ntaps), dev_status, s) != cudaSuccess)
    return DB_ERR_CUDA;
  if (iters == 0 && !ckpt) return DB_OK;
  int axis = axis_mode(psf->kind, psf->kh, psf->kw);
  if (axis == 0 && fft_tile_form(psf->kh, psf->kw)) axis = 3;
  const size_t smem_need = axis == 3 ? rrl_fft_tile_smem(psf->kh)
                           : axis    ? rrl_box_smem(psf->kh, psf->kw)
                                     : rrl_split_smem(psf->kh, psf->kw);
  if (smem_need > 227 * 1024) return DB_ERR_UNSUPPORTED;
  const RrlParams rp = to_rrl(p);
  float* tmp = (float*)(base + L.utmp);
  float2* qbuf = (float2*)(base + L.qbuf);
  const int ldt = upitch(W);
  const long long zt = (long long)H * ldt, zq = (long long)H * upitch(W), hw = (long long)H * W;
  const int nck = ckpt ? (iters > 0 ? (iters - 1) / ckpt_every + 1 : 1) : 0;
  const float* src = u;
  int ld_src = ld;
  long long z_src = img_stride;
  for (int k = 0; k < iters || (k == 0 && ckpt); ++k) {
    if (ckpt && k % ckpt_every == 0 && k / ckpt_every < nck) {
      // image z's checkpoint c goes to ckpt + (z * nck + c) * H * W
      if (copy_images(src, ld_src, z_src, ckpt + (size_t)(k / ckpt_every) * hw, W, nck * hw, H, W, n, s) !=
          cudaSuccess)
        return DB_ERR_CUDA;
    }
    if (k >= iters) break;
    float* dst = (k % 2 == 0) ? tmp : u;
    const int ld_dst = (k % 2 == 0) ? ldt : ld;
    const long long z_dst = (k % 2 == 0) ? zt : img_stride;
    if (launch_rrl_split(f, ld, src, ld_src, dst, ld_dst, qbuf, H, W, (TapGroup*)(base + L.taps),
                         (int*)(base + L.ntaps), psf->kh, psf->kw, rp, dev_status, 0, axis, s, n,
                         img_stride, z_src, z_dst, zq) != cudaSuccess)
      return DB_ERR_CUDA;
    src = dst;
    ld_src = ld_dst;
    z_src = z_dst;
  }
  if (src != u && copy_images(src, ld_src, z_src, u, ld, img_stride, H, W, n, s) != cudaSuccess) return DB_ERR_CUDA;
  return DB_OK;
}

}  // extern "C"

namespace db {
// Workspace db_rrl_iterate alone needs (no Wiener regions in spatial mode).
size_t rrl_iterate_ws_bytes(int H, int W, const db_psf* psf, const db_params* p) {
  if (db_workspace_bytes(H, W, psf, p) == 0) return 0;
  return ws_layout(H, W, psf->kh, psf->kw, p->conv, 1, true).total;
}
}  // namespace db


namespace db {
struct SinglePlan {
  int H, W, ld, kh, kw, kind, iters, conv;
  db_params p;
  void* ws;
  WsLayout L;
  WienerState wst;
  Dft1 DW32, DH32;  // periodic mode: FP32 twiddles of the iteration transforms
  int ng = 0;       // tap-group count (0: unknown)
  RrlParams rp;     // kernel parameters, r_f evaluation as selected at creation
  int sched = -1;   // tuned schedule (db_plan_autotune; -1: the process-wide setting)
  int axis = -1;    // tuned form (0 direct sums, 2 register windows, 3 FFT tiles; -1: settings)
  // db_plan_run_host: the run captured as a CUDA graph for one set of device
  // buffers, status word, settings generation and tuned form
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const float* g_f = nullptr;
  float* g_u = nullptr;
  int* g_status = nullptr;
  unsigned g_gen = 0;
  int g_sched = -2, g_axis = -2;
  ~SinglePlan() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};
}  // namespace db

extern "C" {

db_status db_plan_create(int H, int W, int ld, const db_psf* psf, const db_params* p, int iters, void* ws,
                         size_t ws_bytes, int* dev_status, void* stream, db_plan** out) {
  if (!out) return DB_ERR_ARG;
  *out = nullptr;
  db_status st;
  if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide || ld < W) return DB_ERR_SHAPE;
  if ((st = check_psf(psf, H, W)) != DB_OK) return st;
  if ((st = check_params(p)) != DB_OK) return st;
  if (iters < 0) return DB_ERR_ARG;
  const WsLayout L = ws_layout(H, W, psf->kh, psf->kw, p->conv);
  if ((st = check_ws(ws, ws_bytes, L.total)) != DB_OK) return st;
  if (p->conv == DB_CONV_PERIODIC && !(is_pow2(H) && is_pow2(W))) return DB_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)ws;
  SinglePlan* P = new SinglePlan();
  P->H = H; P->W = W; P->ld = ld; P->kh = psf->kh; P->kw = psf->kw; P->kind = psf->kind;
  P->iters = iters; P->conv = p->conv; P->p = *p; P->ws = ws; P->L = L; P->rp = to_rrl(p);
  if (launch_prepare_taps(psf->taps, psf->kh, psf->kw, psf->kind, (TapGroup*)(base + L.taps),
                          (int*)(base + L.ntaps), dev_status, s) != cudaSuccess) {
    delete P; return DB_ERR_CUDA;
  }
  // the group count sizes the tap table in shared memory of every launch
  if (cudaMemcpyAsync(&P->ng, base + L.ntaps, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    delete P; return DB_ERR_CUDA;
  }
  if (P->ng < 1 || P->ng > max_tap_groups(psf->kh, psf->kw)) P->ng = 0;
  if (p->conv == DB_CONV_PERIODIC) {
    // Wiener in float-float with its own spectrum region, iteration spectrum in FP32
    float4* Sff = (float4*)(base + L.spec);
    float4* tabW = (float4*)(base + L.tw);
    float4* tabH = tabW + dft_table_elems(W);
    Dft1ff FW, FH;
    if (prepare_dft(W, tabW, &FW, &P->DW32, s) != cudaSuccess || prepare_dft(H, tabH, &FH, &P->DH32, s) != cudaSuccess ||
        run_psf_spectrum_2d(psf->taps, psf->kh, psf->kw, H, W, Sff, FW, FH, s) != cudaSuccess ||
        round_spectrum(Sff, (float2*)(base + L.s32), H, W, s) != cudaSuccess) {
      delete P; return DB_ERR_CUDA;
    }
    // the Wiener filter's own spectrum (1D, or the 2D half spectrum of the
    // real-pair passes) replaces the full one, already rounded for the
    // iterations; the transform tables it rebuilds are the same
    if (wiener_prepare(H, W, psf->taps, psf->kh, psf->kw, p->K, ws, L, &P->wst, s) != cudaSuccess) {
      delete P; return DB_ERR_CUDA;
    }
  } else {
    if (wiener_prepare(H, W, psf->taps, psf->kh, psf->kw, p->K, ws, L, &P->wst, s) != cudaSuccess) {
      delete P; return DB_ERR_CUDA;
    }
  }
  *out = (db_plan*)P;
  return DB_OK;
}

db_status db_plan_run(db_plan* plan, const float* f, float* u, int* dev_status, void* stream) {
  SinglePlan* P = (SinglePlan*)plan;
  if (!P || !f || !u || f == u) return DB_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* base = (char*)P->ws;
  if (wiener_apply(f, u, P->ld, P->p.K, P->p.pos_floor, P->ws, P->L, P->wst, s) != cudaSuccess) return DB_ERR_CUDA;
  if (P->iters == 0) return DB_OK;
  if (P->conv == DB_CONV_PERIODIC) {
    if (run_rrl_fourier(f, P->ld, u, P->ld, (float*)(base + P->L.utmp), P->H, P->W, (float2*)(base + P->L.work),
                        (float2*)(base + P->L.qbuf), (const float2*)(base + P->L.s32), P->DW32.tw, P->DH32.tw,
                        P->rp, P->iters, nullptr, 0, dev_status, s) != cudaSuccess)
      return DB_ERR_CUDA;
    return DB_OK;
  }
  return iterate_spatial(f, u, P->H, P->W, P->ld, P->kh, P->kw, P->kind, P->rp, P->iters, nullptr, 0, P->ws,
                         P->L, dev_status, s, P->ng, P->sched, P->axis);
}

db_status db_plan_autotune(db_plan* plan, const float* f, float* u, int reps, int* dev_status, void* stream,
                           int* chosen_schedule, int* chosen_axis) {
  SinglePlan* P = (SinglePlan*)plan;
  if (!P || !f || !u || f == u || reps < 1) return DB_ERR_ARG;
  if (chosen_schedule) *chosen_schedule = -1;
  if (chosen_axis) *chosen_axis = -1;
  if (P->conv == DB_CONV_PERIODIC || P->iters == 0) return DB_OK;  // one form only
  cudaStream_t s = (cudaStream_t)stream;
  const bool one_axis = P->kind != DB_PSF_BOX && (P->kh == 1 || P->kw == 1);
  const int scheds[4] = {DB_SCHED_SPLIT, DB_SCHED_FLOW, DB_SCHED_FUSED, DB_SCHED_CLUSTER};
  const int axes[2] = {0, 2};
  // 2D PSFs of the FFT tiles' shape range: direct sums in every schedule,
  // and the FFT tiles (split schedule)
  const bool fft2d = !one_axis && P->kind != DB_PSF_BOX && fft_tile_shape(P->kh, P->kw);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DB_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return DB_ERR_CUDA; }
  float best = -1.f;
  int best_s = -1, best_a = -1;
  db_status st = DB_OK;
  for (int is = 0; is < 4 && st == DB_OK; ++is) {
    const bool fused = scheds[is] == DB_SCHED_FUSED;
    if (fused && P->kind == DB_PSF_BOX) continue;  // runs as split
    if (scheds[is] == DB_SCHED_CLUSTER) {  // one form (row PSFs on images that fit), else split
      if (!cluster_fits(P->H, P->W, P->kh, P->kw, P->kind == DB_PSF_BOX ? 1 : 2)) continue;
      P->sched = DB_SCHED_CLUSTER;
      P->axis = -1;
      if (db_plan_run(plan, f, u, dev_status, stream) != DB_OK) continue;
      if (cudaEventRecord(e0, s) != cudaSuccess) { st = DB_ERR_CUDA; break; }
      db_status r = DB_OK;
      for (int k = 0; k < reps && r == DB_OK; ++k) r = db_plan_run(plan, f, u, dev_status, stream);
      float ms = 0.f;
      if (r != DB_OK) continue;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { st = DB_ERR_CUDA; break; }
      if (best < 0.f || ms < best) { best = ms; best_s = P->sched; best_a = P->axis; }
      continue;
    }
    int forms[2] = {-1, -1}, nf = 1;
    if (one_axis && !fused) { forms[0] = axes[0]; forms[1] = axes[1]; nf = 2; }
    else if (fft2d) { forms[0] = 0; if (scheds[is] == DB_SCHED_SPLIT) forms[nf++] = 3; }
    for (int ia = 0; ia < nf; ++ia) {
      P->sched = scheds[is];
      P->axis = forms[ia];
      if (db_plan_run(plan, f, u, dev_status, stream) != DB_OK) continue;  // e.g. too large for this form
      if (cudaEventRecord(e0, s) != cudaSuccess) { st = DB_ERR_CUDA; break; }
      db_status r = DB_OK;
      for (int k = 0; k < reps && r == DB_OK; ++k) r = db_plan_run(plan, f, u, dev_status, stream);
      if (r != DB_OK) continue;
      float ms = 0.f;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { st = DB_ERR_CUDA; break; }
      if (best < 0.f || ms < best) { best = ms; best_s = P->sched; best_a = P->axis; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->sched = best_s;
  P->axis = best_a;
  if (st != DB_OK) return st;
  if (best_s < 0) return DB_ERR_UNSUPPORTED;
  if (chosen_schedule) *chosen_schedule = best_s;
  if (chosen_axis) *chosen_axis = best_a;
  return DB_OK;
}

// The plan's run as an instantiated CUDA graph for these buffers, captured
// on the plan's own stream on first use (and again after a settings change
// or a new tuned form).  false: capture not possible; the caller runs eagerly.
static bool plan_graph(SinglePlan* P, db_plan* plan, const float* f, float* u, int* status) {
  const unsigned gen = settings_gen();
  if (P->gexec && P->g_f == f && P->g_u == u && P->g_status == status && P->g_gen == gen &&
      P->g_sched == P->sched && P->g_axis == P->axis)
    return true;
  if (P->gexec) {
    cudaGraphExecDestroy(P->gexec);
    P->gexec = nullptr;
  }
  if (!P->cap_stream && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    P->cap_stream = nullptr;
    (void)cudaGetLastError();
    return false;
  }
  if (cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  const db_status rs = db_plan_run(plan, f, u, status, P->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(P->cap_stream, &g);
  cudaError_t ie = cudaErrorUnknown;
  if (rs == DB_OK && ee == cudaSuccess && g) ie = cudaGraphInstantiate(&P->gexec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    P->gexec = nullptr;
    (void)cudaGetLastError();
    return false;
  }
  P->g_f = f;
  P->g_u = u;
  P->g_status = status;
  P->g_gen = gen;
  P->g_sched = P->sched;
  P->g_axis = P->axis;
  return true;
}

db_status db_plan_run_host(db_plan* plan, const float* f_host, float* u_host, float* f_dev, float* u_dev,
                           int* dev_status, void* stream) {
  SinglePlan* P = (SinglePlan*)plan;
  if (!P || !f_host || !u_host || !f_dev || !u_dev || f_dev == u_dev) return DB_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t row = (size_t)P->W * sizeof(float), pitch = (size_t)P->ld * sizeof(float);
  if (copy_image_async(f_dev, pitch, f_host, row, P->H, P->W, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DB_ERR_CUDA;
  if (plan_graph(P, plan, f_dev, u_dev, dev_status)) {
    if (cudaGraphLaunch(P->gexec, s) != cudaSuccess) return DB_ERR_CUDA;
  } else {
    const db_status st = db_plan_run(plan, f_dev, u_dev, dev_status, stream);
    if (st != DB_OK) return st;
  }
  if (copy_image_async(u_host, row, u_dev, pitch, P->H, P->W, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return DB_ERR_CUDA;
  return DB_OK;
}

void db_plan_destroy(db_plan* plan) { delete (SinglePlan*)plan; }

db_status db_host_alloc(size_t bytes, void** out) {
  if (!out) return DB_ERR_ARG;
  *out = nullptr;
  if (bytes == 0) return DB_ERR_ARG;
  return cudaHostAlloc(out, bytes, cudaHostAllocDefault) == cudaSuccess ? DB_OK : DB_ERR_CUDA;
}

void db_host_free(void* p) {
  if (p) (void)cudaFreeHost(p);
}

const char* db_status_string(db_status s) {
  switch (s) {
    case DB_OK: return "ok";
    case DB_ERR_ARG: return "invalid argument";
    case DB_ERR_SHAPE: return "image shape out of range";
    case DB_ERR_PSF: return "invalid PSF extent";
    case DB_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case DB_ERR_UNSUPPORTED: return "unsupported configuration";
    case DB_ERR_CUDA: return "CUDA launch or copy failed";
    case DB_ERR_TIMEOUT: return "bounded device wait gave up";
    case DB_ERR_NONFINITE: return "non-finite value produced";
    case DB_ERR_TAPS: return "invalid PSF taps";
  }
  return "unknown status";
}

db_status db_status_from_flags(int flags) {
  if (flags == 0) return DB_OK;
  if (flags & DB_FLAG_TIMEOUT) return DB_ERR_TIMEOUT;
  if (flags & (DB_FLAG_TAPS | DB_FLAG_BOX)) return DB_ERR_TAPS;
  if (flags & DB_FLAG_NONFINITE) return DB_ERR_NONFINITE;
  return DB_ERR_ARG;
}

const char* db_version(void) { return "libdeblur 0.1 sm_103a"; }

long long db_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

db_status db_set_one_axis_min(int min_len) {
  if (min_len < 0 || min_len > kMaxTapSide + 1) return DB_ERR_ARG;
  g_one_axis_min.store(min_len);
  bump_settings();
  return DB_OK;
}

db_status db_set_dense_min(int percent) {
  if (percent < 0 || percent > 101) return DB_ERR_ARG;
  g_dense_min_pct.store(percent == 0 ? 50 : percent);
  bump_settings();
  return DB_OK;
}

db_status db_set_fft_tiles(int min_taps) {
  if (min_taps < 0) return DB_ERR_ARG;
  g_fft_tile_min.store(min_taps == 0 ? kFftTileMinDefault : min_taps);
  bump_settings();
  return DB_OK;
}

db_status db_set_schedule(int schedule) {
  if (schedule != DB_SCHED_AUTO && schedule != DB_SCHED_FUSED && schedule != DB_SCHED_SPLIT &&
      schedule != DB_SCHED_FLOW && schedule != DB_SCHED_CLUSTER)
    return DB_ERR_ARG;
  g_schedule.store(schedule);
  bump_settings();
  return DB_OK;
}

}  // extern "C"
