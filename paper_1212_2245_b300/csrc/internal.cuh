// Internal declarations shared by the libdeblur translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "libdeblur.h"

namespace db {

// One non-zero PSF tap: weight and offset (dy, dx) from the origin.
struct Tap {
  float w;
  int16_t dy, dx;
};
static_assert(sizeof(Tap) == 8, "Tap is 8 bytes");

// RRRL parameters as the kernels consume them.
struct RrlParams {
  float alpha, eps_phi, eps_psi, floor;
  int phi_robust, psi_tv;
};

constexpr int kMaxSide = 4096;   // largest H or W
constexpr int kMaxTapSide = 255; // largest kh or kw

// Number of kernels this library has launched (host-side count).
void count_launch(int n = 1);

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

// Workspace layout for one image (offsets in bytes from ws).
struct WsLayout {
  size_t taps;     // Tap[kh*kw]
  size_t ntaps;    // int
  size_t utmp;     // float[H*W]  (RRRL ping-pong)
  size_t spec;     // float2[spec_elems]  (PSF spectrum)
  size_t work;     // float2[work_elems]  (FFT data)
  size_t total;
};
WsLayout ws_layout(int H, int W, int kh, int kw, int conv);

// ---- launchers (return cudaError_t of the launch) --------------------------
cudaError_t launch_compact_taps(const float* taps, int kh, int kw, int kind, Tap* out,
                                int* nout, int* status, cudaStream_t s);

cudaError_t run_wiener(const float* f, float* u0, int H, int W, int ld, const float* taps,
                       int kh, int kw, float K, float floor_, void* ws, const WsLayout& L,
                       int* status, cudaStream_t s);

cudaError_t launch_rrl_spatial(const float* f, int ldf, const float* uin, int ldin, float* uout,
                               int ldout, int H, int W, const Tap* taps, const int* ntaps,
                               int kh, int kw, const RrlParams& p, int* status, cudaStream_t s);

}  // namespace db
