/*
 * libdeblur -- Wiener + robust regularised Richardson-Lucy (WR3L) deblurring
 * on one NVIDIA B300 (sm_103a).  C ABI.
 *
 * Method: Welk, Raudaschl, Schwarzbauer, Erler, Laeuter, "Fast and Robust
 * Linear Motion Deblurring".  The observed grey image f is modelled as
 * f = g*h + n for a known space-invariant point-spread function h (Sec. 2,
 * Eq. 1).  The pipeline is a Wiener filter (Sec. 2.1, Eq. 2), a positivity
 * floor (Sec. 3.2) and a fixed number of RRRL iterations (Sec. 2.3,
 * Eq. 9-12).
 *
 * General conventions for every entry point:
 *   - Images are float32, row-major, H rows x W columns, with a row pitch of
 *     `ld` elements (ld >= W).  Pixel (i, j) is at ptr[i*ld + j].
 *   - All image, tap, workspace and status pointers are DEVICE pointers owned
 *     by the caller, except the host images of db_plan_run_host and
 *     db_batch_stream_run_host.  The library allocates no device memory of
 *     its own for data: scratch space is the caller's workspace `ws` of
 *     `ws_bytes` bytes (see db_workspace_bytes), which must be 256-byte
 *     aligned.  Exceptions: db_host_alloc hands out page-locked host memory
 *     on request; plans and batches keep small host-side records;
 *     db_plan_run_host creates a stream of the plan's own and instantiates a
 *     CUDA graph per set of device buffers (its first call for a buffer set
 *     must not happen inside a stream capture); db_batch_stream_create
 *     creates two streams and events; the allocation-free entry point holds
 *     a fixed array compiled into the library.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued asynchronously.  Run calls never synchronise; the set-up and
 *     tuning calls that say so (plan and batch creation, the autotuners,
 *     settings that fill device tables) synchronise their stream.
 *   - Argument errors are returned synchronously as a db_status and nothing is
 *     enqueued.  Errors found on the device (invalid taps, non-finite values,
 *     a bounded wait that ran out) are OR-ed as DB_FLAG_* bits into the int32
 *     word `*dev_status` (may be NULL to skip checking), which the caller
 *     zeroes before and reads after synchronising; db_status_from_flags maps
 *     it to a db_status.
 *   - A PSF tap (a, b) sits at offset (dy, dx) = (a - kh/2, b - kw/2) (integer
 *     division) from the origin.  Convolution is
 *       (u*h)(i,j)  = sum_ab h[a][b] u(i-dy, j-dx),
 *     correlation with the adjoint h*(x) = h(-x) (Sec. 2) is
 *       (v*h*)(i,j) = sum_ab h[a][b] v(i+dy, j+dx).
 *     Spatial-mode sums continue the image constantly across the boundary
 *     (clamped indices), Fourier-mode sums periodically (Sec. 4.2).
 */
#ifndef LIBDEBLUR_H
#define LIBDEBLUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DB_OK = 0,
  DB_ERR_ARG = 1,          /* NULL pointer, bad enum, non-positive size      */
  DB_ERR_SHAPE = 2,        /* H, W or ld out of the supported range          */
  DB_ERR_PSF = 3,          /* PSF extent invalid or larger than the image    */
  DB_ERR_WORKSPACE = 4,    /* ws NULL, misaligned or smaller than required   */
  DB_ERR_UNSUPPORTED = 5,  /* valid request this build does not implement    */
  DB_ERR_CUDA = 6,         /* a kernel launch or async copy failed           */
  DB_ERR_TIMEOUT = 7,      /* device flag: a bounded wait gave up            */
  DB_ERR_NONFINITE = 8,    /* device flag: NaN/Inf produced or consumed      */
  DB_ERR_TAPS = 9          /* device flag: negative/non-finite taps, sum<=0,
                              or a "box" PSF whose interior taps differ     */
} db_status;

/* Device status bits (OR-ed into *dev_status). */
#define DB_FLAG_TAPS      0x1
#define DB_FLAG_NONFINITE 0x2
#define DB_FLAG_TIMEOUT   0x4
#define DB_FLAG_BOX       0x8

typedef enum {
  DB_PSF_GENERAL = 0,  /* any non-negative kh x kw taps                      */
  DB_PSF_BOX = 1       /* uniform motion along a coordinate axis (Sec. 4.3,
                          "Uniform linear motion"): kh == 1 or kw == 1, all
                          taps equal except possibly the first and the last
                          (lighter end pixels of a non-integer blur length).
                          The spatial iterations then blur and correlate by
                          sliding-window sums (split and flow schedules; a
                          fused schedule request runs split).               */
} db_psf_kind;

typedef enum {
  DB_CONV_CLAMP = 0,    /* spatial sums, constant continuation (Sec. 4.2)   */
  DB_CONV_PERIODIC = 1  /* Fourier-domain sums, periodic continuation        */
} db_conv_mode;

typedef struct {
  int kh, kw;          /* PSF extent, 1..255 each, kh <= H and kw <= W       */
  int kind;            /* db_psf_kind                                        */
  const float* taps;   /* DEVICE, kh*kw floats row-major; used as given (the
                          caller normalises), must be >= 0 with a positive sum */
} db_psf;

typedef struct {
  float K;          /* Wiener noise weight, > 0 (Eq. 2)                      */
  float alpha;      /* regulariser weight, >= 0 (Eq. 9)                      */
  float eps_phi;    /* robust data penaliser: phi'(z) = eps/sqrt(z+eps^2)    */
  float eps_psi;    /* TV diffusivity: psi'(z) = 1/sqrt(z+eps^2)             */
  float pos_floor;  /* delta > 0: f and the Wiener output are floored at it  */
  int phi_robust;   /* 1: robust phi' above, 0: phi' == 1 (plain RL data term) */
  int psi_tv;       /* 1: TV psi' above, 0: psi' == 1 (linear diffusion)     */
  int conv;         /* db_conv_mode used by the RRRL blur/correlation        */
} db_params;

/* Bytes of workspace the calls below need for one image of H x W with this
 * PSF and parameters (the maximum over db_wiener, db_rrl_iterate and
 * db_deblur).  Returns 0 for invalid arguments. */
size_t db_workspace_bytes(int H, int W, const db_psf* psf, const db_params* p);

/* Wiener initialisation (Sec. 2.1, Eq. 2, and Sec. 3.2):
 *   f0 = max(f, delta);  u0 = max( Re IDFT( DFT(f0) conj(h^) / (|h^|^2 + K) ), delta )
 * with the DFT at the native image size and h^ the DFT of the PSF wrapped
 * with its origin at (0,0).  A PSF on one row (kh == 1) or one column
 * (kw == 1) is filtered with 1D transforms along that axis, which is the same
 * operator (Sec. 4.3, "Non-uniform linear motion").  f and u0 may not alias.
 * Supported sizes: H, W in 1..4096 (power-of-two extents use radix-2^k
 * transforms, other extents Bluestein's chirp-z form of the same DFT). */
db_status db_wiener(const float* f, float* u0, int H, int W, int ld,
                    const db_psf* psf, const db_params* p,
                    void* ws, size_t ws_bytes, int* dev_status, void* stream);

/* `iters` RRRL iterations in place on u (Sec. 2.3, Eq. 9-12):
 *   b = u*h;  W = phi'(r_f(b)) with r_f(s) = s - f - f ln(s/f)  (Eq. 7, 10)
 *   A = (W f/b)*h*;  B = W*h*;  D = div(psi'(|grad u|^2) grad u)  (Eq. 11)
 *   u <- u (A + alpha [D]+) / (B - alpha [D]-),   [z]+- = (z +- |z|)/2 (Eq. 12)
 * with f0 = max(f, delta) in place of f.  D uses central differences and zero
 * flux across the image boundary (Sec. 4.1).  p->conv selects spatial sums
 * with constant continuation (any size) or Fourier-domain sums with periodic
 * continuation (Sec. 4.3, general 2D variant; power-of-two H and W, else
 * DB_ERR_UNSUPPORTED).  u must be > 0 on entry (the
 * Wiener output of db_wiener is).  If `ckpt` is not NULL, u before iteration
 * k is also written to ckpt + (k/ckpt_every)*H*W (packed, pitch W) for every
 * k that is a multiple of ckpt_every (k = 0 included); ckpt holds
 * (iters-1)/ckpt_every + 1 images. */
db_status db_rrl_iterate(const float* f, float* u, int H, int W, int ld,
                         const db_psf* psf, const db_params* p, int iters,
                         float* ckpt, int ckpt_every,
                         void* ws, size_t ws_bytes, int* dev_status, void* stream);

/* db_wiener followed by db_rrl_iterate: the whole WR3L pipeline (Sec. 3.2). */
db_status db_deblur(const float* f, float* u, int H, int W, int ld,
                    const db_psf* psf, const db_params* p, int iters,
                    void* ws, size_t ws_bytes, int* dev_status, void* stream);

/* ---- reverse mode -------------------------------------------------------------
 * Gradients of a scalar loss through the whole WR3L chain (db_wiener
 * followed by db_rrl_iterate with checkpoints), for tuning the PSF taps, alpha
 * and K from data.  No counterpart in the paper: it differentiates the
 * operators of Sec. 2.1, Eq. 2 and Sec. 2.3, Eq. 7-12 as evaluated here, with
 * the exact transposes of the clamped convolution and correlation and the
 * conventions d[z]+/dz = 1[z>0], d[z]-/dz = 1[z<0], d max(z,delta)/dz =
 * 1[z>delta].  Supported: spatial mode (p->conv == DB_CONV_CLAMP), a PSF on
 * one row (kh == 1, the 1D motion case of Sec. 4.3), kw <= 1024.
 * A batch of `batch` images that share the PSF and parameters is handled in
 * one call; image n of f, grad_u and grad_f starts at n*H*ld.
 *   f       the forward's observed images (pitch ld)
 *   ckpt    the checkpoints the forward db_rrl_iterate wrote with the same
 *           iters and ckpt_every, image after image: image n's checkpoints
 *           start at n*nck*H*W, nck = (iters-1)/ckpt_every + 1 (u0 first;
 *           packed, pitch W)
 *   grad_u  dLoss/du_iters (pitch ld)
 * Outputs: grad_f = dLoss/df (written, pitch ld); grad_taps (kh*kw doubles),
 * grad_alpha and grad_K (one double each) are ACCUMULATED (+=) over the
 * batch; the caller zeroes them.  The iterates inside a checkpoint segment
 * are recomputed once, with their intermediates (b, q, A, B, g) kept for the
 * segment's reverse steps: the workspace holds about (64 + 28 ckpt_every)
 * bytes per pixel of the batch plus fixed terms (db_backward_workspace_bytes);
 * all reductions are deterministic. */
size_t db_backward_workspace_bytes(int H, int W, int batch, const db_psf* psf, int ckpt_every);
db_status db_rrl_backward(const float* f, const float* ckpt, const float* grad_u, int H, int W, int ld,
                          int batch, const db_psf* psf, const db_params* p, int iters, int ckpt_every,
                          float* grad_f, double* grad_taps, double* grad_alpha, double* grad_K,
                          void* ws, size_t ws_bytes, int* dev_status, void* stream);

/* ---- batches of images ----------------------------------------------------
 * Many images of uneven sizes, each with its own PSF and parameters (spatial
 * mode only), deblurred by the whole WR3L pipeline of db_deblur: one image's
 * result is the same as db_deblur's for that image.  No counterpart in the
 * paper (its closest relative is the persistent worker threads of Sec. 4.5).
 * A plan (db_batch_create) precomputes every transform table, PSF spectrum
 * and tap list and uploads the work tables into the workspace; running it
 * (db_batch_run) enqueues only launches and memsets, so it can be captured
 * in a CUDA graph and replayed.  The run is the batched Wiener launches (one
 * per transform stage and column class) and one cooperative persistent
 * launch for all RRRL iterations of all images.  By default its phases are
 * separated by grid barriers; db_set_batch_order selects a dependency order
 * instead (a tile waits only for the previous phase of its own image).
 * Every wait is bounded (db_set_spin_limit) and raises DB_FLAG_TIMEOUT
 * instead of hanging.  The plan holds pointers into the
 * workspace and to the images: keep them alive and unchanged in shape while
 * the plan is used; pixel values may change between runs. */
typedef struct {
  const float* f;    /* DEVICE, H x W, pitch ld */
  float* u;          /* DEVICE, result, same layout; may not alias f */
  int H, W, ld;
  db_psf psf;
  db_params p;       /* p.conv must be DB_CONV_CLAMP */
} db_image_desc;

typedef struct db_batch db_batch;  /* opaque host-side plan */

/* Workspace bytes for the batch (descs: HOST array of n descriptors); 0 if a
 * descriptor is invalid. */
size_t db_batch_workspace_bytes(const db_image_desc* descs, int n, int iters);

/* Build the plan (enqueues set-up work and host-to-device copies on stream;
 * not capturable).  On success *out owns a host object: db_batch_destroy. */
db_status db_batch_create(const db_image_desc* descs, int n, int iters, void* ws, size_t ws_bytes,
                          int* dev_status, void* stream, db_batch** out);

/* Run the planned batch on stream (capturable). */
db_status db_batch_run(db_batch* b, int* dev_status, void* stream);

void db_batch_destroy(db_batch* b);

/* Choose the batch's tile forms by measurement (the batched counterpart of
 * db_plan_autotune): runs the whole batch `reps` times after one warm-up per
 * candidate, timed with CUDA events on `stream`, and keeps the fastest
 * combination for every later db_batch_run.  A coordinate search from the
 * process-wide size rules: the form of non-box one-axis PSFs (the size rule
 * of db_set_one_axis_min's default, register windows for all, tap groups
 * for all), then the dense sums on and off (dense-eligible 2D PSFs, odd
 * sides 3..25), then the FFT-tile threshold (FFT tiles for the 2D PSFs with
 * kh * kw at or above it: each distinct kh * kw of the batch, and none).
 * Classes absent from the batch are not tried.  The runs overwrite the
 * images' outputs; synchronises `stream` (call it before capturing the run
 * in a graph; a graph captured earlier keeps working and picks up the
 * choice).  *dense_out (nullable) receives 1 when the dense sums were
 * chosen, *windows_out (nullable) 2 for the size rule, 1 for register
 * windows, 0 for tap groups, *fft_out (nullable) the FFT-tile threshold (0:
 * none).  The result of each image equals db_deblur's under the
 * corresponding process-wide settings (db_set_fft_tiles at that threshold,
 * 2305 for none; db_set_dense_min 50 or 101; db_set_one_axis_min 0, 1 or
 * 256).  DB_ERR_ARG for a null batch or reps < 1. */
db_status db_batch_autotune(db_batch* b, int reps, int* dev_status, void* stream, int* dense_out,
                            int* windows_out, int* fft_out);

/* db_batch_create + db_batch_run + db_batch_destroy. */
db_status db_deblur_batch(const db_image_desc* descs, int n, int iters, void* ws, size_t ws_bytes,
                          int* dev_status, void* stream);

/* ---- batches from host memory ------------------------------------------------
 * The batch above, fed from and returned to HOST memory, with the transfers
 * overlapped with the work (the paper reports its host-device transfers
 * separately, Sec. 5.3; this form hides most of them).  The images are split
 * into `parts` sub-batches (fewer when n < parts) whose pixel counts follow
 * the shares 1, 4, 16, ..., 16, 4, 1 in streaming order (largest images
 * first, each to the sub-batch least loaded for its share), each an ordinary
 * batch plan over its share of the workspace.  The small first and last
 * sub-batches shorten the first upload and the last download, which no run
 * overlaps; each run hides the next sub-batch's upload while runs take at
 * least four times as long as the uploads of the same pixels, and each
 * further sub-batch adds some run time (5 to 7 suit a 0.7 GB batch of 512
 * images).  db_batch_stream_run_host enqueues, per
 * sub-batch k: the copies of its host images into the descriptors' DEVICE
 * buffers f on an internal upload stream, its run on `stream` once those
 * copies have landed, and the copies of its results (the descriptors'
 * DEVICE buffers u) to the host on an internal download stream.  So the
 * uploads of later sub-batches and the downloads of earlier ones overlap the
 * runs.  The uploads start after all work enqueued on `stream` before the
 * call; `stream` itself waits for every download before anything enqueued
 * after the call, so synchronising `stream` makes u_host valid.  Each
 * image's result equals db_deblur's for it, whatever `parts` is.
 *   descs: HOST array of n descriptors (as for db_batch_create); the device
 *     buffers f and u serve as staging and must stay allocated.
 *   f_host[i], u_host[i]: HOST pointers to H x W floats (rows packed, no
 *     pitch), preferably page-locked (db_host_alloc); pageable memory works
 *     but its copies do not overlap.
 *   Errors: DB_ERR_ARG (null pointers, parts < 1), DB_ERR_WORKSPACE, and the
 *   codes of db_batch_create; the object owns two streams and a few events,
 *   released by db_batch_stream_destroy (which does not synchronise: finish
 *   the runs first).  Not capturable (it waits on events across streams). */
typedef struct db_batch_stream db_batch_stream;
size_t db_batch_stream_workspace_bytes(const db_image_desc* descs, int n, int iters, int parts);
db_status db_batch_stream_create(const db_image_desc* descs, int n, int iters, int parts, void* ws,
                                 size_t ws_bytes, int* dev_status, void* stream, db_batch_stream** out);
db_status db_batch_stream_run_host(db_batch_stream* b, const float* const* f_host, float* const* u_host,
                                   int* dev_status, void* stream);
/* Number of sub-batches actually planned. */
int db_batch_stream_parts(const db_batch_stream* b);
void db_batch_stream_destroy(db_batch_stream* b);

/* Clock-cycle budget of every bounded device wait (the batch kernel's
 * dependency waits and grid barriers, the flow schedule's tile waits);
 * default 4e9 (about two seconds). */
db_status db_set_spin_limit(long long cycles);

/* Order of the batch kernel's tiles (no counterpart in the paper): 0 one
 * task list over all iterations, each tile waiting only until the previous
 * phase of its own image is complete (per-image counters), so the phases of
 * different images overlap; 1 (the default) every phase of every image
 * before a grid barrier, then the next phase.  Both give the same bits.  On
 * B300 the barrier form is faster for batches of many small tiles: each
 * dependency costs a barrier, a release and an acquire per tile.
 * Process-wide; batches take it when they are created.  DB_ERR_ARG for other
 * values. */
db_status db_set_batch_order(int order);

/* TMA staging (no counterpart in the paper): 1 (the default) lets the
 * q phase of FFT tiles fetch each tile pair's 64 x 136 window of u with one
 * tensor copy (cp.async.bulk.tensor) into shared memory, where the elements
 * outside the image then take their clamped neighbours' values; 0 loads the
 * windows element by element with clamped indices.  Both load the same
 * values and give the same bits.  The copy needs u 16-byte aligned with a
 * row stride (and image stride) that is a multiple of 4 floats; other
 * buffers take the element-wise loads.  Process-wide; plans and batches take
 * it when their runs are enqueued or created.  DB_ERR_ARG for other values. */
db_status db_set_tma(int on);

/* Allocation-free RRRL iterations (no counterpart in the paper; an interface
 * convenience).  Some callers cannot allocate device memory at run time:
 * a deblurring step embedded in a fixed-latency frame loop (an inspection
 * line that must finish every frame within its budget) cannot risk a
 * cudaMalloc, which may synchronise the device and take unbounded time, and
 * a plugin running inside a host framework that owns all GPU memory may have
 * no allocator at all.  This call computes exactly what db_rrl_iterate
 * computes (same arguments without checkpoints and workspace) but takes its
 * scratch from a fixed array of DB_NOALLOC_SCRATCH_BYTES bytes compiled into
 * the library, which every GPU that loads the library keeps until the
 * process exits.
 *   - The scratch holds what db_rrl_iterate itself uses: the tap records,
 *     one ping-pong image (H x W floats, rows padded to 4), the q buffer of
 *     the split schedule (H x W float pairs, rows padded to 2) and the flow
 *     schedule's counters -- about 12 bytes per pixel, so images up to
 *     about 2.7 Mpx fit (1024 x 1024 with a 2D PSF takes 12.1 MiB; in
 *     periodic mode the spectra count too, 44 MiB at 1024 x 1024).  Larger
 *     requests are rejected with DB_ERR_WORKSPACE before anything is
 *     enqueued.
 *   - The first call on a device looks up the array's device address (with
 *     that device current), which may load the library's module: make that
 *     first call before any CUDA stream capture.  The address is kept for
 *     the life of the device's context; after cudaDeviceReset this entry
 *     point must not be called again in the process.
 *   - All calls on a device share the one array.  Calls whose work overlaps
 *     on the GPU (different streams, different host threads) race on it and
 *     give undefined results; serialise them.  The array keeps the last
 *     call's contents; every call writes the scratch it reads before
 *     reading it, so no state carries over between calls.
 *   - No cudaMalloc, cudaFree or allocating library routine is called. */
#define DB_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
db_status db_rrl_iterate_noalloc(const float* f, float* u, int H, int W, int ld,
                                 const db_psf* psf, const db_params* p, int iters,
                                 int* dev_status, void* stream);

/* ---- N equally sized images --------------------------------------------------
 * n images of H x W (pitch ld) sharing one PSF and one parameter set, image k
 * at f + k*img_stride (u likewise; img_stride >= H*ld elements): the Wiener
 * filter (Eq. 2) and `iters` RRRL iterations (Eq. 9-12) on all of them, the
 * iterations as launches over all images at once (spatial mode, constant
 * continuation; DB_CONV_PERIODIC gives DB_ERR_UNSUPPORTED).  The result of
 * each image equals db_deblur's on that image alone under the split
 * schedule.  ckpt (nullable, device, n x ((iters-1)/ckpt_every+1) x H x W
 * packed): image k's iterate at iteration c*ckpt_every is stored at
 * ckpt + (k*nck + c)*H*W -- the layout db_rrl_backward reads.  Workspace:
 * db_workspace_bytes_n.  The same ownership and error behaviour as
 * db_deblur. */
size_t db_workspace_bytes_n(int H, int W, int n, const db_psf* psf, const db_params* p);
db_status db_deblur_n(const float* f, float* u, int H, int W, int ld, int n, long long img_stride,
                      const db_psf* psf, const db_params* p, int iters, float* ckpt, int ckpt_every,
                      void* ws, size_t ws_bytes, int* dev_status, void* stream);

/* ---- prepared single-image pipeline ----------------------------------------
 * The paper computes the PSF transform once and reuses it for every image of
 * a given size (Sec. 5, the set-up excluded from its timings).  A plan does
 * that set-up once -- transform tables, PSF spectrum, tap groups -- for one
 * image size, PSF and parameter set; db_plan_run then applies the whole
 * pipeline of db_deblur to an image: the Wiener image passes and `iters`
 * RRRL iterations, enqueuing launches and async copies only (capturable in a
 * CUDA graph).  The plan keeps pointers into ws and the PSF values taken at
 * creation: re-create it when the taps change.  The result equals
 * db_deblur's bit for bit.  db_plan_create synchronises `stream` once: it
 * reads back the number of tap groups, which sizes the tap table that every
 * RRRL launch of the plan keeps in shared memory. */
typedef struct db_plan db_plan;
db_status db_plan_create(int H, int W, int ld, const db_psf* psf, const db_params* p, int iters, void* ws,
                         size_t ws_bytes, int* dev_status, void* stream, db_plan** out);
db_status db_plan_run(db_plan* plan, const float* f, float* u, int* dev_status, void* stream);
/* The plan's pipeline on an image in host memory: enqueues the copy of f_host
 * (H x W, packed) into f_dev (device, pitch ld), db_plan_run(f_dev -> u_dev),
 * and the copy of u_dev into u_host (H x W, packed), all on `stream`.  The
 * copies overlap other work only when the host buffers are page-locked
 * (db_host_alloc); the caller synchronises `stream` before reading u_host.
 * The run between the copies is one CUDA graph launch: the first call for a
 * given (f_dev, u_dev, dev_status) captures the plan's run on a stream of
 * the plan's own (host-side set-up, once), later calls replay it; a change
 * of any process-wide setting (db_set_*) or of the plan's tuned form
 * captures again.  If capture is not possible the run is launched directly.
 * The call itself is not capturable.  The buffers stay the caller's.
 * DB_ERR_ARG for null pointers or f_dev == u_dev, DB_ERR_CUDA when a copy or
 * launch fails. */
db_status db_plan_run_host(db_plan* plan, const float* f_host, float* u_host, float* f_dev, float* u_dev,
                           int* dev_status, void* stream);
void db_plan_destroy(db_plan* plan);

/* Choose the plan's kernel schedule by measurement: runs the plan on (f -> u)
 * once per candidate -- the split, flow, fused and (where it applies)
 * cluster schedules; for a non-box one-axis PSF both the tap-group and the
 * register-window form; for a 2D PSF with sides 2..48 the direct sums in
 * every schedule and the FFT tiles (split schedule) -- `reps` times after
 * one warm-up, timed with CUDA events on `stream`, and keeps the fastest
 * for every later db_plan_run of this plan (instead of the process-wide
 * db_set_schedule / db_set_one_axis_min / db_set_fft_tiles settings).
 * Synchronises `stream`; not capturable.  Results of all forms agree to
 * FP32 rounding.  *chosen_schedule (DB_SCHED_*) and *chosen_axis (0 direct
 * sums: tap groups or dense, 2 register windows, 3 FFT tiles, -1 not
 * applicable) report the choice (both nullable; -1 for a periodic plan,
 * which has one form).  DB_ERR_ARG for null pointers, f == u
 * or reps < 1; DB_ERR_UNSUPPORTED if no form runs. */
db_status db_plan_autotune(db_plan* plan, const float* f, float* u, int reps, int* dev_status, void* stream,
                           int* chosen_schedule, int* chosen_axis);

/* Page-locked host memory for db_plan_run_host (cudaHostAlloc): *out = a
 * buffer of `bytes` bytes, released with db_host_free.  DB_ERR_ARG for a null
 * out or zero bytes, DB_ERR_CUDA when the allocation fails (*out = NULL). */
db_status db_host_alloc(size_t bytes, void** out);
void db_host_free(void* p);

/* Human-readable name of a status code (static storage). */
const char* db_status_string(db_status s);

/* Map an OR of DB_FLAG_* bits to the most specific db_status (DB_OK if 0). */
db_status db_status_from_flags(int flags);

/* Library version string, e.g. "libdeblur 0.1 sm_103a". */
const char* db_version(void);

/* Kernel schedule of the spatial RRRL iteration (process-wide setting; the
 * arithmetic is the same in every schedule):
 *   DB_SCHED_AUTO  - flow from 512K to 2M pixels, split otherwise (default;
 *                    the choice measured fastest on B300)
 *   DB_SCHED_FUSED - one launch per iteration; each tile recomputes the
 *                    weighted ratio q on its halo (fewest HBM round trips)
 *   DB_SCHED_SPLIT - two launches per iteration; q = (W f/b, W) goes through
 *                    a global buffer in the workspace (no halo recompute)
 *   DB_SCHED_FLOW  - the split tiles, all iterations in one cooperative
 *                    persistent launch; tiles wait (bounded, DB_FLAG_TIMEOUT
 *                    on expiry; db_set_spin_limit) only for the neighbouring
 *                    tiles whose output they read, so the phases of
 *                    successive iterations overlap.  Calls that request
 *                    checkpoints run the split schedule.
 *   DB_SCHED_CLUSTER - for one-row PSFs (kh == 1) on images with H a
 *                    multiple of 64 and W a multiple of 8 that fit: the
 *                    whole image stays in the shared memory of one cluster
 *                    of 8 CTAs for all iterations (one launch; rows split
 *                    across the CTAs, TV halo rows exchanged through
 *                    distributed shared memory).  Same result as the split
 *                    schedule bit for bit (a short non-box row PSF is summed
 *                    with register windows here).  Other calls run split. */
#define DB_SCHED_AUTO 0
#define DB_SCHED_FUSED 1
#define DB_SCHED_SPLIT 2
#define DB_SCHED_FLOW 3
#define DB_SCHED_CLUSTER 4
db_status db_set_schedule(int schedule);

/* One-axis PSFs (kh == 1 or kw == 1) in the split and flow schedules: a box
 * (DB_PSF_BOX) is always summed by sliding windows; another one-axis PSF of
 * length L = kh * kw is summed with register windows (one shared-memory load
 * and 8 FMAs per tap for 8 outputs) when L >= min_len, with tap groups
 * otherwise.  Process-wide; min_len in 1..256 (256: never).  0 restores the
 * default: register windows for one-row PSFs from 16 taps and one-column
 * PSFs from 32 taps (shorter ones are faster as tap groups on B300).  The
 * result differs between the two forms by FP32 rounding only.  DB_ERR_ARG
 * for other values. */
db_status db_set_one_axis_min(int min_len);

/* Dense 2D PSFs (odd sides 3..25): the tap sums run as register-blocked
 * dense sums (2 x 4 outputs per thread, every tap of the kh x kw window)
 * when at least `percent` percent of the taps are non-zero, as tap groups
 * otherwise.  The choice is made on the device when the taps are prepared
 * (db_wiener, db_rrl_iterate, plans and batches: it applies to taps
 * prepared after the call).  Process-wide; percent in 1..101 (101: never),
 * 0 restores the default of 50.  The two forms differ by FP32 rounding
 * only.  DB_ERR_ARG for other values. */
db_status db_set_dense_min(int percent);

/* FFT tiles for 2D PSFs (sides 2..48; Sec. 4.2 "Fourier transform": the
 * blur and both correlations as pointwise products of spectra).  The split
 * schedule (and a batch image) computes them on 64 x 64 windows of u and q
 * taken with constant continuation, keeping the (65 - kh) x (65 - kw)
 * outputs whose PSF footprint lies inside the window, so the result is the
 * same constant-continuation iteration as the direct sums, up to FP32
 * rounding (FP32 transforms).  Their cost does not depend on the taps, the
 * direct sums' grows with the non-zero taps: the FFT tiles are used for a
 * PSF with kh * kw >= min_taps (the default suits dense PSFs such as
 * Gaussians; a sparse PSF of large support, such as a thin oblique line,
 * is often faster with the direct sums: db_plan_autotune measures both).
 * The flow schedule falls back to split for such PSFs.  Process-wide; min_taps >= 1 (above 2304:
 * never), 0 restores the default of 225.  Applies to runs started, and
 * plans and batches created, after the call.  DB_ERR_ARG for negative
 * values. */
db_status db_set_fft_tiles(int min_taps);

/* Evaluation of the information divergence r_f in the robust weight
 * (process-wide setting, all devices):
 *   DB_RF_LOG1P - r_f(b) = f (t - log1p t), t = (b - f)/f (default; exact up
 *                 to FP32 rounding, no cancellation near b = f)
 *   DB_RF_LUT   - r_f(b) = f r_1(b/f) with r_1(s) = s - 1 - ln s read from a
 *                 table on (0, 65] (Sec. 4.1, "Function evaluations"): 8192
 *                 entries at s_j = j * 65/8192, linear interpolation, the
 *                 closed form below the first entry and the tangent line at
 *                 65 beyond it.  Interpolation error <= h^2/(8 s^2), h = 65/8192.
 * Selecting DB_RF_LUT fills the table on every visible device (synchronous
 * copies; call it outside stream capture).  Plans and batches take the
 * setting at creation.  db_rrl_backward returns DB_ERR_UNSUPPORTED while
 * DB_RF_LUT is selected.  Returns DB_ERR_ARG for other modes. */
#define DB_RF_LOG1P 0
#define DB_RF_LUT 1
db_status db_set_rf_eval(int mode);

/* Number of CUDA kernels this library has enqueued in this process so far
 * (host-side counter; a CUDA-graph replay of captured calls adds nothing). */
long long db_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBDEBLUR_H */
