// Cluster-resident RRRL iterations for small images blurred along rows
// (Sec. 2.3, Eq. 9-12; one-row PSFs of Sec. 4.3: uniform or non-uniform
// linear motion along x).
//
// One thread-block cluster of 8 or 16 CTAs holds the whole image in shared
// memory for all iterations: CTA k owns the rows [k RB, (k+1) RB)
// with their f, u, q = (W f/b, W) and the correlation results.  A row PSF
// reaches along rows only, so the blur and both correlations never leave a
// CTA; only the TV term's central differences reach two rows into the
// neighbouring CTAs.  After each update a CTA pushes its two top rows of the
// new u into the upper neighbour's halo buffer and its two bottom rows into
// the lower one's (distributed shared memory, double-buffered by iteration
// parity), and one cluster barrier per iteration orders the pushes before
// the neighbours read them.  u leaves shared memory once, after the last
// iteration.
//
// Every pixel is computed by the device functions of the split schedule's
// one-axis tiles -- the same sliding-window or register-window runs along a
// row, the same weighted residual, diffusion strips and update -- so the
// result equals the split schedule's bit for bit.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "internal.cuh"
#include "rrl_box.cuh"
#include "rrl_tiles.cuh"

namespace db {

namespace cg = cooperative_groups;

constexpr int kClusterThreads = 512;
constexpr int kClusterR = 8;  // rows per diffusion strip

// Shared-memory geometry of one CTA (RB own rows of W pixels, PSF length L).
struct ClusterGeom {
  int RB, W, L;
  int before, c0;   // conv window: `before` pixels left of the output; corr window: c0 left
  int PL, US;       // u rows: PL clamped columns on the left, row stride US (odd)
  int QS;           // q rows: c0 clamped columns on the left, row stride QS (odd)
  int DS;           // result rows (b, then (Delta, B)): stride W + 1
  size_t o_taps, o_f, o_u, o_q, o_d, o_h, bytes;
  __host__ __device__ ClusterGeom(int RB_, int W_, int L_) : RB(RB_), W(W_), L(L_) {
    before = L - 1 - (L >> 1);
    c0 = L >> 1;
    PL = before > 2 ? before : 2;
    const int PR = c0 > 2 ? c0 : 2;
    US = (PL + W + PR) | 1;
    QS = (W + L - 1) | 1;
    DS = W + 1;
    size_t o = 0;
    o_taps = o; o += 2 * kAxisTapsSmem;                               // reversed (q) and forward (update) taps
    o_f = o;    o += round16((size_t)RB * W * 4);
    o_u = o;    o += round16((size_t)(RB + 4) * US * 4);              // rows -2 .. RB+1
    o_q = o;    o += round16((size_t)RB * QS * 8);
    o_d = o;    o += round16((size_t)RB * DS * 8);
    o_h = o;    o += (size_t)2 * 4 * W * 4;                            // halo rows by parity: 2 above, 2 below
    bytes = o;
  }
};

// Fill the clamped columns of u rows rr0 .. rr1-1 (shared row indices).
__device__ __forceinline__ void cluster_pad_rows(float* us, const ClusterGeom& g, int rr0, int rr1) {
  const int padr = g.US - g.PL - g.W;
  const int per = g.PL + padr;
  for (int k = threadIdx.x; k < (rr1 - rr0) * per; k += blockDim.x) {
    const int rr = rr0 + k / per, t = k % per;
    float* row = us + rr * g.US + g.PL;
    if (t < g.PL) row[-1 - t] = row[0];
    else row[g.W + (t - g.PL)] = row[g.W - 1];
  }
}

// Element loop over an n-row x W block without a division per element: the
// flat index k = tid + i nth advances (r, x) by (nth / W, nth % W).
struct RowWalk {
  int r, x, dr, dx, W;
  __device__ RowWalk(int W_, int tid, int nth) : W(W_) {
    r = tid / W; x = tid - r * W; dr = nth / W; dx = nth - dr * W;
  }
  __device__ __forceinline__ void next() {
    r += dr; x += dx;
    if (x >= W) { x -= W; ++r; }
  }
};

template <bool BOX>
__global__ void __launch_bounds__(kClusterThreads, 1)
    k_rrl_cluster(const float* __restrict__ f, int ldf, float* __restrict__ u, int ldu, int H, int W,
                  const int* __restrict__ ngroups, RrlParams p, int iters, int* status) {
  extern __shared__ __align__(16) unsigned char csm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank(), nc = (int)cluster.num_blocks();
  const int RB = H / nc, y0 = rank * RB;
  const float4 bw = load_box_weights(ngroups);
  const int L = __float_as_int(bw.w);
  const ClusterGeom g(RB, W, L);
  float* taps_q = (float*)(csm + g.o_taps);
  float* taps_u = taps_q + kAxisTapsSmem / 4;
  float* fs = (float*)(csm + g.o_f);
  float* us = (float*)(csm + g.o_u);
  float2* qs = (float2*)(csm + g.o_q);
  float2* ds = (float2*)(csm + g.o_d);
  float* bs = (float*)ds;  // b shares the result rows (stride DS floats)
  float* hb = (float*)(csm + g.o_h);
  const int tid = threadIdx.x, nth = blockDim.x;
  if (!BOX) {
    for (int k = tid; k < L; k += nth) {
      taps_q[k] = __ldg(axis_taps(ngroups) + L - 1 - k);
      taps_u[k] = __ldg(axis_taps(ngroups) + k);
    }
  }
  // f and u0 of the own rows, u0 of the two rows above and below (clamped)
  for (RowWalk w(W, tid, nth); w.r < RB; w.next()) fs[w.r * W + w.x] = f[(size_t)(y0 + w.r) * ldf + w.x];
  for (RowWalk w(W, tid, nth); w.r < RB + 4; w.next()) {
    const int y = min(max(y0 + w.r - 2, 0), H - 1);
    us[w.r * g.US + g.PL + w.x] = u[(size_t)y * ldu + w.x];
  }
  __syncthreads();
  cluster_pad_rows(us, g, 0, RB + 4);
  cluster.sync();  // every CTA of the cluster is running before any remote store
  float* up_nb = rank > 0 ? cluster.map_shared_rank(hb, rank - 1) : nullptr;
  float* dn_nb = rank + 1 < nc ? cluster.map_shared_rank(hb, rank + 1) : nullptr;
  bool bad = false;
  const int qpr = g.QS - g.c0 - W;  // continued columns right of a q row
  for (int it = 0; it < iters; ++it) {
    // here u holds the iterate on the own rows and the halo rows, each row
    // continued beyond its ends
    // blur b along rows into the result rows
    for (int item = tid; item < RB * W / kBoxSeg; item += nth) {
      const int r = item % RB, x0 = (item / RB) * kBoxSeg;
      const float* src = us + (r + 2) * g.US + g.PL - g.before + x0;
      if (BOX) box_run<float>(src, 1, L, bw.z, bw.y, bw.x, bs + r * g.DS + x0, 1);
      else axis_run<float>(src, 1, L, taps_q, bs + r * g.DS + x0, 1);
    }
    __syncthreads();
    // q = (W f/b, W), then q of the end pixels continued along the row
    for (RowWalk w(W, tid, nth); w.r < RB; w.next())
      qs[w.r * g.QS + g.c0 + w.x] = weighted_residual(bs[w.r * g.DS + w.x], fmaxf(fs[w.r * W + w.x], p.floor), p);
    __syncthreads();
    for (int k = tid; k < RB * (g.c0 + qpr); k += nth) {
      const int r = k / (g.c0 + qpr), t = k - r * (g.c0 + qpr);
      float2* row = qs + r * g.QS + g.c0;
      if (t < g.c0) row[-1 - t] = row[0];
      else row[W + (t - g.c0)] = row[W - 1];
    }
    __syncthreads();
    // Delta, B: correlation along rows into the result rows
    for (int item = tid; item < RB * W / kBoxSeg; item += nth) {
      const int r = item % RB, x0 = (item / RB) * kBoxSeg;
      const float2* src = qs + r * g.QS + x0;  // window of output x0 starts c0 left of it
      if (BOX) box_run<float2>(src, 1, L, bw.x, bw.y, bw.z, ds + r * g.DS + x0, 1);
      else axis_run<float2>(src, 1, L, taps_u, ds + r * g.DS + x0, 1);
    }
    __syncthreads();
    // D on vertical strips and the update; u' goes to the result rows first
    // (neighbouring strips still read u)
    for (RowWalk w(W, tid, nth); w.r < RB / kClusterR; w.next()) {
      const int s = w.r, x = w.x;
      float D[kClusterR], c[kClusterR];
      diffusion_strip<kClusterR, 0>(us + (s * kClusterR + 2) * g.US + g.PL + x, p, D, c, g.US);
#pragma unroll
      for (int r = 0; r < kClusterR; ++r) {
        float2* d = ds + (s * kClusterR + r) * g.DS + x;
        const float un = rrl_update(c[r], d->x, d->y, D[r], p);
        bad |= !isfinite(un);
        d->x = un;
      }
    }
    __syncthreads();
    // u' on the own rows
    for (RowWalk w(W, tid, nth); w.r < RB; w.next()) us[(w.r + 2) * g.US + g.PL + w.x] = ds[w.r * g.DS + w.x].x;
    if (it + 1 == iters) break;
    // halo rows of the next iteration: pushed to the neighbours (image rows
    // y0, y0+1 become the upper neighbour's rows below; y0+RB-2, y0+RB-1 the
    // lower neighbour's rows above), clamped at the image's top and bottom
    const int par = (it + 1) & 1;
    float* hpar = hb + par * 4 * W;
    for (int k = tid; k < 2 * W; k += nth) {
      const int r = k / W, x = k - r * W;
      const float top = ds[r * g.DS + x].x, bot = ds[(RB - 2 + r) * g.DS + x].x;
      if (up_nb) up_nb[par * 4 * W + (2 + r) * W + x] = top;
      else hpar[r * W + x] = ds[x].x;                            // rows -2, -1 -> row 0
      if (dn_nb) dn_nb[par * 4 * W + r * W + x] = bot;
      else hpar[(2 + r) * W + x] = ds[(RB - 1) * g.DS + x].x;    // rows RB, RB+1 -> row RB-1
    }
    cluster.sync();
    for (int k = tid; k < 4 * W; k += nth) {
      const int h = k / W, x = k - h * W;
      us[(h < 2 ? h : RB + h) * g.US + g.PL + x] = hpar[k];
    }
    __syncthreads();
    cluster_pad_rows(us, g, 0, RB + 4);  // every row continued beyond its ends
    __syncthreads();
  }
  __syncthreads();
  for (RowWalk w(W, tid, nth); w.r < RB; w.next()) u[(size_t)(y0 + w.r) * ldu + w.x] = us[(w.r + 2) * g.US + g.PL + w.x];
  if (bad && status) atomicOr(status, DB_FLAG_NONFINITE);
}

// CTAs per cluster: 16 (a non-portable size, twice the SMs) when the rows
// split into 16 bands of whole 8-row strips, else 8.
static int cluster_ctas(int H) { return H % (16 * kClusterR) == 0 ? 16 : kClusterCTAs; }

size_t cluster_smem(int H, int W, int L) {
  const ClusterGeom g(H / cluster_ctas(H), W, L);
  return g.bytes;
}

bool cluster_fits(int H, int W, int kh, int kw, int axis) {
  if (kh != 1 || (axis != 1 && axis != 2) || W < kBoxSeg || W % kBoxSeg != 0) return false;
  if (H % (kClusterCTAs * kClusterR) != 0) return false;
  if (kw > kAxisTapsSmem / 4) return false;
  return cluster_smem(H, W, kw) <= 227 * 1024;
}

cudaError_t launch_rrl_cluster(const float* f, int ldf, float* u, int ldu, int H, int W, const int* ngroups, int kw,
                               int axis, const RrlParams& p, int iters, int* status, cudaStream_t s) {
  auto k = axis == 1 ? k_rrl_cluster<true> : k_rrl_cluster<false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  // 16 CTAs where the rows allow it and the device can place such a cluster,
  // else 8; cudaErrorNotSupported when neither fits (the caller runs split)
  for (int nc = cluster_ctas(H); nc >= kClusterCTAs; nc /= 2) {
    const ClusterGeom g(H / nc, W, kw);
    if (g.bytes > 227 * 1024) continue;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.bytes)) != cudaSuccess)
      return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = nc;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = g.bytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg) != cudaSuccess || nclusters < 1) {
      (void)cudaGetLastError();  // clear a refused query
      continue;
    }
    if ((e = cudaLaunchKernelEx(&cfg, k, f, ldf, u, ldu, H, W, ngroups, p, iters, status)) != cudaSuccess) return e;
    count_launch();
    return cudaSuccess;
  }
  return cudaErrorNotSupported;
}

}  // namespace db
