/*
 * ocgs.h — C ABI of the GB300-native object-centric 2D Gaussian Splatting rasterizer.
 *
 * The library implements the data-parallel hot path of "Object-Centric 2D
 * Gaussian Splatting" (Rogge & Stricker, arXiv 2501.08174): the differentiable
 * tile-based 2DGS rasterizer it extends (Sec. 3.2, Sec. 5.1), the background
 * loss on accumulated opacity (Sec. 4.2, Eq. 1) and the occlusion-aware
 * pruning that records which Gaussians take part in alpha blending
 * (Sec. 4.3).  One process drives one GPU; every call is asynchronous on the
 * context's CUDA stream unless stated otherwise.
 *
 * Conventions shared by every call
 *  - Pointers named "device" are CUDA device pointers owned by the caller; the
 *    library never frees them and never writes outside the stated extents.
 *    Pointers named "host" are ordinary host memory read during the call.
 *  - Parameter arrays are float32, one array per attribute, row-major:
 *      xyz [n,3], quat [n,4] = (w,x,y,z) (any non-zero norm; normalised inside),
 *      scale [n,2] = (s_u, s_v) > 0, opacity [n] in (0,1], sh [n,(deg+1)^2,3].
 *    These are the activated values; exp/sigmoid activations are the caller's.
 *  - Images of several views are concatenated: view v occupies pixels
 *    [off_v, off_v + W_v*H_v) with off_v = sum_{u<v} W_u*H_u, row-major inside
 *    a view.  rgb and normal are [P,3], alpha and depth are [P].
 *  - Cameras are pinhole, world->camera, OpenCV axes (+z forward, +y down);
 *    pixel (i,j) has its centre at (i+0.5, j+0.5).
 *  - Return value: OCGS_OK or an error code; on error ocgs_last_error() gives
 *    a one-line reason.  Argument errors are detected before any launch.
 *    Errors found on the device (non-finite parameters, a capacity overflow)
 *    are reported by the next call that synchronises (ocgs_render, ocgs_prune,
 *    ocgs_sync).  There is no CPU fallback: without a CUDA device every call
 *    returns OCGS_ERR_CUDA.
 */
#ifndef OCGS_H
#define OCGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OCGS_ABI_VERSION 4

typedef enum {
  OCGS_OK = 0,
  OCGS_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad degree) */
  OCGS_ERR_OOM = 2,        /* device allocation failed */
  OCGS_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  OCGS_ERR_TIMEOUT = 4,    /* a bounded device wait gave up */
  OCGS_ERR_NONFINITE = 5,  /* a parameter was NaN/Inf; that Gaussian was not rendered */
  OCGS_ERR_CAPACITY = 6,   /* more (tile, Gaussian) pairs than 2^31-1 in one call */
  OCGS_ERR_STATE = 7       /* forward state missing, released or from another context */
} ocgs_status;

typedef struct ocgs_ctx ocgs_ctx;
typedef struct ocgs_fwd_state ocgs_fwd_state;

/* Read-only Gaussian parameters (device, caller-owned). n may be 0. */
typedef struct {
  const float* xyz;
  const float* quat;
  const float* scale;
  const float* opacity;
  const float* sh;
  int64_t n;
  int32_t sh_degree; /* 0..3 */
  int32_t reserved;
} ocgs_gaussians;

/* Read-only 3D Gaussians for the 3DGS variant of the pruning record (Appendix
 * B): the layout of ocgs_gaussians with three scales per Gaussian, scale [n,3]
 * (any 4-byte alignment); quat [n,4] 16-byte aligned. */
typedef struct {
  const float* xyz;
  const float* quat;
  const float* scale;
  const float* opacity;
  const float* sh;
  int64_t n;
  int32_t sh_degree; /* 0..3 */
  int32_t reserved;
} ocgs_gaussians3d;

/* Writable arrays in the parameter layout (device, caller-owned): gradients
 * (accumulated with +=) or the destination of a pruning compaction. */
typedef struct {
  float* xyz;
  float* quat;
  float* scale;
  float* opacity;
  float* sh;
} ocgs_gaussians_out;

/* Pinhole camera (host). viewmat is row-major world->camera [R t; 0 0 0 1]. */
typedef struct {
  float viewmat[16];
  float fx, fy, cx, cy;
  int32_t width, height;  /* 1..16384 each */
  float near_plane;       /* > 0; a Gaussian whose 3-sigma square reaches it is culled */
  int32_t reserved;
} ocgs_camera;

/* Per-pixel images (device, caller-owned). As render output rgb, alpha, depth
 * and normal must be non-null; depth2 may be NULL (not computed).  As backward
 * cotangents any pointer may be NULL (zero). */
typedef struct {
  float* rgb;     /* [P,3] C = sum w rgb */
  float* alpha;   /* [P]   A = sum w, the accumulated opacity of Eq. 1 */
  float* depth;   /* [P]   D = sum w z  (not normalised by A) */
  float* normal;  /* [P,3] N = sum w n  (camera frame, not normalised) */
  float* depth2;  /* [P]   Q = sum w z^2, for the depth distortion of Eq. 3 */
} ocgs_image;

/* Launch options.  None of them changes a result: the support test is exact
 * and the screen bounds are conservative, so tiles only reshape the work, and
 * the two-pass binning below renders every tile from the same list as one pass.
 *
 * front_fraction (persistent renders and sweeps; 0 = one pass; the captured
 * sweep graph always bins in one pass): the
 * front-to-back walk of Sec. 4.3 stops a pixel once T falls below its bound,
 * so most (tile, Gaussian) pairs behind an opaque surface are never read.  In
 * two passes the renderer first bins and renders only the first
 * ceil(front_fraction * n * n_views) records of the depth order; each tile
 * with a pixel still running at the end of that prefix is then binned with
 * the records behind it and continues from where its pixels stopped.  The
 * tile's list is the one-pass list in two segments, and the backward walks
 * both. */
typedef struct {
  int32_t tile_w;             /* 8, 16 or 32 */
  int32_t tile_h;             /* 8 or 16: 16x16, 16x8, 8x8 or 32x8 */
  int32_t persistent;         /* 1: persistent CTAs draining a global tile queue, heaviest tiles first */
  int32_t pixels_per_thread;  /* vertically adjacent pixels per thread: 1, 2 (0 = 2), or 4 for 16x16 and 16x8 */
  float front_fraction;       /* in [0, 1]: share of the depth order binned in the first pass (0 = one pass) */
  int32_t batch;              /* Gaussians per batch: records a warp stages in shared memory at a time:
                                 32 (0 = 32), or 16 or 64 with 16x16 tiles and 2 or 4 pixels per
                                 thread or 16x8 tiles and 4 */
} ocgs_options;

/* Counters of the last ocgs_render / ocgs_accumulate_contribution. */
typedef struct {
  int64_t n_gaussians;    /* N */
  int64_t n_views;        /* V */
  int64_t n_pixels;       /* P, all views */
  int64_t n_visible;      /* (view, Gaussian) records with at least one tile */
  int64_t n_pairs;        /* K, (tile, Gaussian) pairs over all views */
  int64_t n_tiles;        /* tiles over all views */
  int32_t tile_w, tile_h;
} ocgs_stats;

/* Stages timed by the built-in profiler (CUDA events recorded on the context
 * stream around each stage's launches). */
typedef enum {
  OCGS_STAGE_PREPROCESS = 0,      /* projection, bounds, SH colour (per Gaussian) */
  OCGS_STAGE_DEPTH_SORT = 1,      /* radix sort of the records by centre depth */
  OCGS_STAGE_BINNING = 2,         /* tile counts scan, duplication, tile ranges */
  OCGS_STAGE_TILE_SORT = 3,       /* stable radix sort of the pairs by tile */
  OCGS_STAGE_RASTER_FWD = 4,      /* front-to-back compositing (+ contribution record) */
  OCGS_STAGE_LOSS = 5,            /* background loss and masked L1, with their adjoints */
  OCGS_STAGE_RASTER_BWD = 6,      /* back-to-front adjoint of the compositing */
  OCGS_STAGE_PREPROCESS_BWD = 7,  /* chain rule to the parameters */
  OCGS_STAGE_PRUNE = 8,           /* keep-set and compaction */
  OCGS_STAGE_ADAM = 9,            /* optimiser update of the parameters */
  OCGS_STAGE_COUNT = 10
} ocgs_stage;

typedef struct {
  double ms[16];        /* summed device time per stage, milliseconds */
  int64_t launches[16]; /* number of timed stage instances */
} ocgs_profile;

const char* ocgs_status_str(ocgs_status s);
const char* ocgs_last_error(const ocgs_ctx* ctx);
int32_t ocgs_abi_version(void);

/* Create a context on `device` that issues work on `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  The context owns its scratch memory
 * (stream-ordered pool allocations) and frees it in ocgs_destroy. */
ocgs_status ocgs_create(ocgs_ctx** ctx, int32_t device, void* stream);
ocgs_status ocgs_destroy(ocgs_ctx* ctx);
ocgs_status ocgs_set_stream(ocgs_ctx* ctx, void* stream);
ocgs_status ocgs_set_options(ocgs_ctx* ctx, const ocgs_options* opts);
ocgs_status ocgs_get_options(const ocgs_ctx* ctx, ocgs_options* opts);
/* Tile coverage of the binning (Sec. 4.3 front-to-back order over each tile's
 * list).  rect = 0 (the default): a (tile, Gaussian) pair is kept only where
 * the Gaussian's support {rho <= r_b}, bounded by a conic with FP32 margins,
 * reaches a pixel centre of the tile, and a warp stages only the records whose
 * support rows meet its band.  rect = 1: every tile of each record's
 * conservative screen rectangle and every band, with no support test; slower
 * (213 M instead of 101 M pairs on 500k surfels x 16 views in one pass), and
 * meant to check that the support test drops only pairs that blend no pixel,
 * so that both settings render the same bits.  Applies to the renders,
 * sweeps and graphs created after the call.  OCGS_ERR_ARG for another value. */
ocgs_status ocgs_set_coverage(ocgs_ctx* ctx, int32_t rect);
ocgs_status ocgs_get_stats(const ocgs_ctx* ctx, ocgs_stats* stats);
/* Wait for the context stream and report device-side errors. */
ocgs_status ocgs_sync(ocgs_ctx* ctx);

/*
 * ocgs_render — forward rasterization of n_views views in one batched pass
 * (surfel projection, tile binning with a key sort, front-to-back alpha
 * compositing that ends a pixel once it is nearly opaque; Sec. 3.2 and
 * Sec. 4.3).
 *   gaussians  device parameters (see above)
 *   cams       host [n_views] cameras, n_views >= 1
 *   out        device images, P = sum W*H pixels; fully overwritten
 *   score      device [n] or NULL. When given, score[i] = max(score[i], w) over
 *              every pixel where Gaussian i was blended with weight w (the
 *              visibility record kept during colour accumulation, Sec. 4.3
 *              and Sec. 5.1). The caller zeroes it before the first view.
 *   state      NULL, or receives an opaque forward state for
 *              ocgs_render_backward; release it with ocgs_state_release.
 * Synchronises with the host to size the pair buffers: once in one-pass
 * binning, twice in two-pass binning (the persistent default with images or a
 * score: the second pass's pair count is known only after the first pass).
 */
ocgs_status ocgs_render(ocgs_ctx* ctx, const ocgs_gaussians* gaussians, const ocgs_camera* cams,
                        int32_t n_views, const ocgs_image* out, float* score,
                        ocgs_fwd_state** state);

/*
 * ocgs_render_backward — gradients of a scalar loss through ocgs_render
 * (the backpropagation step of Sec. 3.2).  d_out holds dL/d(rgb, alpha, depth,
 * normal) per pixel (NULL planes are zero).  The gradients with respect to
 * xyz, quat (through the normalisation), scale, opacity and sh are ADDED to
 * d_params (device, caller-zeroed).  The parameters in `gaussians` must be the
 * ones the forward used.  The state stays valid for further backward calls.
 */
ocgs_status ocgs_render_backward(ocgs_ctx* ctx, const ocgs_fwd_state* state,
                                 const ocgs_gaussians* gaussians, const ocgs_image* d_out,
                                 const ocgs_gaussians_out* d_params);

ocgs_status ocgs_state_release(ocgs_ctx* ctx, ocgs_fwd_state* state);

/*
 * ocgs_background_loss — L_b = (1/(h*w)) * sum A*(1-M) per view (Eq. 1).
 *   alpha   device [P] accumulated opacity (render output)
 *   mask    device [P] uint8, 1 on the object, 0 on the background
 *   cams    host [n_views] (only width/height are read)
 *   loss    device [n_views] float64, overwritten with the unweighted L_b
 *   d_alpha device [P] or NULL: d_alpha += gamma*(1-M)/(h*w), the gradient of
 *           gamma*L_b (gamma = 0.5 in Sec. 5.1, weight of Eq. 3)
 * Deterministic (fixed-order FP64 reduction).
 */
ocgs_status ocgs_background_loss(ocgs_ctx* ctx, const float* alpha, const uint8_t* mask,
                                 const ocgs_camera* cams, int32_t n_views, float gamma,
                                 double* loss, float* d_alpha);

/*
 * ocgs_background_loss_noalloc — the same background loss and adjoint as
 * ocgs_background_loss, for callers that must not allocate device memory:
 * code whose device memory is all held by another allocator (a framework's
 * caching pool that reserves the GPU up front), or a loop with a latency
 * budget that cannot afford cudaMalloc/cudaFree, which may synchronise the
 * device and take unbounded time.  The paper has no counterpart; it is an
 * interface convenience of this library.
 *   alpha, mask, cams, n_views, gamma, loss, d_alpha  as in ocgs_background_loss
 *   stream   the cudaStream_t to run on (NULL = legacy default stream); the
 *            current device is used
 * It needs no context and allocates nothing: its scratch (per-block partial
 * sums, view table, block prefix) is one fixed static device array of
 * 643,076 bytes that every GPU loading this library holds until the process exits.
 * Limits: at most 1024 views and 65536 blocks of 4096 pixels
 * (268,435,456 pixels) per call; larger requests return OCGS_ERR_CAPACITY,
 * other bad arguments OCGS_ERR_ARG, before any device work.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture.  The address is kept
 * for the life of the process: do not call this entry point on a device
 * after cudaDeviceReset on it.  The view sizes reach the device as a kernel
 * argument, and the host memory of cams is not read after the call returns.
 * Every call shares the one array and leaves its contents behind; each call
 * overwrites all it reads, so nothing needs clearing, but calls whose work
 * overlaps on the GPU (different streams) race on it.  Errors are returned
 * only (there is no context for ocgs_last_error).
 */
ocgs_status ocgs_background_loss_noalloc(const float* alpha, const uint8_t* mask, const ocgs_camera* cams,
                                         int32_t n_views, float gamma, double* loss, float* d_alpha,
                                         void* stream);

/*
 * ocgs_accumulate_contribution — the occlusion-aware pruning sweep (Sec. 4.3,
 * Sec. 5.1): a forward pass over n_views views that only records, for every
 * Gaussian, score[i] = max(score[i], max blending weight over all pixels).
 * A Gaussian that is never blended (outside every frustum, or behind pixels
 * that reached the termination opacity first) keeps score 0.
 *   score  device [n], max-accumulated; the caller zeroes it once per sweep.
 */
ocgs_status ocgs_accumulate_contribution(ocgs_ctx* ctx, const ocgs_gaussians* gaussians,
                                         const ocgs_camera* cams, int32_t n_views, float* score);

/*
 * ocgs_contribution_graph_create — the pruning sweep of
 * ocgs_accumulate_contribution (score zeroed, then max-accumulated over all
 * n_views views, 16 views per chunk) captured once as one CUDA graph, so
 * that a periodic sweep (every 100 or 600 iterations in Sec. 5.1) costs one
 * graph launch and no host synchronisation.  The graph reads the parameter
 * arrays and writes score through the pointers given here: keep them alive
 * and in place; their contents may change between launches.  Creation runs
 * the sweep once to measure the largest chunk's (tile, Gaussian) pair count
 * and sizes the pair buffers to headroom (>= 1) times it.  A launch whose
 * pairs exceed that capacity leaves score incomplete and makes the next
 * ocgs_sync return OCGS_ERR_CAPACITY: re-create the graph then.  The graph
 * uses the context's options at creation.  Synchronises.
 */
typedef struct ocgs_graph ocgs_graph;
ocgs_status ocgs_contribution_graph_create(ocgs_ctx* ctx, const ocgs_gaussians* gaussians,
                                           const ocgs_camera* cams, int32_t n_views, float* score,
                                           float headroom, ocgs_graph** graph);
/* Launch the captured sweep on the context stream (asynchronous). */
ocgs_status ocgs_graph_launch(ocgs_ctx* ctx, ocgs_graph* graph);
ocgs_status ocgs_graph_destroy(ocgs_ctx* ctx, ocgs_graph* graph);

/*
 * ocgs_render_3d / ocgs_accumulate_contribution_3d — the pruning record of Sec.
 * 4.3 in 3DGS, as Appendix B runs it: 3D Gaussians splatted by the EWA
 * projection of their covariance, image covariance J W Sigma W^T J^T + 0.3 I
 * (Sigma = R diag(s^2) R^T, J the Jacobian of the pinhole projection at the
 * camera-frame mean), rho the Mahalanobis distance under it, and the same
 * skip (rho > 9, alpha < 1/255), 0.99 clamp, stop rule, depth order (centre
 * depth) and score (max blending weight) as the surfel path.  render_3d writes
 * rgb, alpha and depth (sum w z_c); normal is written as 0 and depth2 must be
 * NULL; score as for ocgs_render (may be NULL).  Forward only (no state).
 */
ocgs_status ocgs_render_3d(ocgs_ctx* ctx, const ocgs_gaussians3d* gaussians, const ocgs_camera* cams,
                           int32_t n_views, const ocgs_image* out, float* score);
ocgs_status ocgs_accumulate_contribution_3d(ocgs_ctx* ctx, const ocgs_gaussians3d* gaussians,
                                            const ocgs_camera* cams, int32_t n_views, float* score);

/*
 * ocgs_prune — keep-set {i : score[i] > threshold} (threshold 0 reproduces
 * the rule of Sec. 4.3: drop what no pixel ever blended) and stream
 * compaction of the parameters in their original order.
 *   in          device parameters, n Gaussians
 *   out         device arrays with room for n Gaussians (must not alias in)
 *   n_kept      host, receives the number kept
 *   borderline  device [borderline_cap] int64 or NULL: indices i with
 *               |score[i] - threshold| <= 1e-6, ascending
 *   n_borderline host, receives how many such indices exist (may exceed cap)
 * Synchronises.
 */
ocgs_status ocgs_prune(ocgs_ctx* ctx, const float* score, float threshold,
                       const ocgs_gaussians* in, const ocgs_gaussians_out* out, int64_t* n_kept,
                       int64_t* borderline, int64_t borderline_cap, int64_t* n_borderline);

/*
 * ocgs_adam_step — one Adam update of every parameter array, in one launch.
 *
 * The method trains its surfels with the optimiser of the 2DGS / 3DGS training
 * it extends (Sec. 5.1 keeps their schedule and coefficients); that optimiser is
 * Adam (Kingma & Ba, 2015, Algorithm 1), applied elementwise to each array with
 * its own learning rate:
 *     m <- beta1 m + (1 - beta1) g          v <- beta2 v + (1 - beta2) g^2
 *     p <- p - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)
 * The update acts on the arrays as given (the API's activated parameters: the
 * caller owns any re-parameterisation).
 *   grads   device gradients, read only; grads->n and grads->sh_degree give
 *           the sizes (n may be 0): xyz [n,3], quat [n,4], scale [n,2],
 *           opacity [n], sh [n,(deg+1)^2,3]
 *   params  device, same layout, updated in place
 *   m, v    device, same layout, first and second moments, updated in place
 *           (zero before the first step)
 *   cfg     host: lr[5] per array in the order xyz, quat, scale, opacity, sh;
 *           beta1, beta2 in [0,1); eps > 0; step t >= 1 (the step being taken).
 *           Double precision: 1 - beta and the bias corrections are formed in
 *           double and rounded once to the single-precision factors the
 *           kernel uses (a float beta2 = 0.999 alone would be 1.3e-5 off in
 *           1 - beta2).
 * Arrays of one parameter must not overlap each other.  Any 4-byte alignment is
 * accepted (16-byte aligned arrays take the vector path).  Non-finite gradients
 * propagate as in the formula and set the context's status word, which
 * ocgs_sync reports as OCGS_ERR_NONFINITE (ocgs_render clears it when it
 * starts).  Asynchronous on the context stream.
 */
typedef struct {
  double lr[5];
  double beta1;
  double beta2;
  double eps;
  int64_t step;
} ocgs_adam_config;

ocgs_status ocgs_adam_step(ocgs_ctx* ctx, const ocgs_gaussians* grads, const ocgs_gaussians_out* params,
                           const ocgs_gaussians_out* m, const ocgs_gaussians_out* v,
                           const ocgs_adam_config* cfg);

/*
 * ocgs_masked_l1 — the L1 part of the masked photometric loss of Eq. 2,
 * L_c^M = mean |I*M - R*M| over the 3*h*w colour values of each view.
 *   rgb     device [P,3] rendered colour R
 *   target  device [P,3] reference image I
 *   mask    device [P] uint8 object mask M
 *   loss    device [n_views] float64, overwritten
 *   d_rgb   device [P,3] or NULL: d_rgb += weight * dL_c^M/dR
 *           = weight * sign(R - I) * M / (3*h*w)
 * Deterministic (fixed-order FP64 reduction).
 */
ocgs_status ocgs_masked_l1(ocgs_ctx* ctx, const float* rgb, const float* target, const uint8_t* mask,
                           const ocgs_camera* cams, int32_t n_views, float weight, double* loss,
                           float* d_rgb);

/*
 * ocgs_ssim — SSIM of masked images, per view: both images are multiplied by
 * the mask first (Eq. 2 masks the inputs of the photometric loss; Sec. 5 masks
 * the inputs of the evaluation SSIM), then SSIM is taken with windowed
 * statistics under an 11x11 Gaussian window of sigma 1.5 (zero outside the
 * image) and C1 = 0.01^2, C2 = 0.03^2, as the 3DGS photometric loss the method
 * keeps defines it.
 *   rgb, target  device [P,3] rendered R and reference I; mask device [P] uint8
 *   ssim         device [n_views] float64, overwritten: mean of the SSIM map
 *                over all 3*h*w values (the D-SSIM term of L_c is 1 - ssim)
 *   ssim_masked  device [n_views] float64 or NULL: mean over the values of the
 *                mask pixels (the masked SSIM of Sec. 5; NaN without any)
 *   d_rgb        device [P,3] or NULL: d_rgb += weight * d(1 - ssim)/dR
 * Deterministic (fixed-order FP64 sums).  Allocates 36 bytes per pixel of
 * scratch when d_rgb is given.  Asynchronous on the context stream.
 */
ocgs_status ocgs_ssim(ocgs_ctx* ctx, const float* rgb, const float* target, const uint8_t* mask,
                      const ocgs_camera* cams, int32_t n_views, float weight, double* ssim, double* ssim_masked,
                      float* d_rgb);

/*
 * ocgs_masked_psnr — PSNR = 20 log10(max_i / sqrt(MSE)) per view, with the
 * masked MSE of Sec. 5: squared differences of the mask pixels summed over
 * pixels and channels, divided by the number of those values (3 per mask
 * pixel).  psnr device [n_views] float64, overwritten (+inf when the masked
 * images agree, NaN without mask pixels).  max_i > 0.
 */
ocgs_status ocgs_masked_psnr(ocgs_ctx* ctx, const float* rgb, const float* target, const uint8_t* mask,
                             const ocgs_camera* cams, int32_t n_views, float max_i, double* psnr);

/*
 * ocgs_depth_distortion — the 2DGS depth distortion that Eq. 3 adds (weight
 * alpha there), per view: the mean over pixels of sum_{i,j} w_i w_j (z_i - z_j)^2
 * over the pixel's blended entries, which equals 2 (A Q - D^2) with the planes
 * A = alpha, D = depth and Q = depth2 of ocgs_render (squared distances: the
 * form that the front-to-back accumulation gives exactly).
 *   alpha, depth, depth2  device [P]
 *   loss     device [n_views] float64, overwritten
 *   d_alpha, d_depth, d_depth2  device [P] or all NULL: += weight * d loss / d plane
 * Asynchronous on the context stream.
 */
ocgs_status ocgs_depth_distortion(ocgs_ctx* ctx, const float* alpha, const float* depth, const float* depth2,
                                  const ocgs_camera* cams, int32_t n_views, float weight, double* loss, float* d_alpha,
                                  float* d_depth, float* d_depth2);

/*
 * ocgs_normal_consistency — the 2DGS normal consistency that Eq. 3 adds (weight
 * beta there), per view: sum over counted pixels of sum_i w_i (1 - n_i . N) =
 * A - N . N_r, divided by h*w.  N_r is the normal plane of ocgs_render; N is the
 * unit normal of the expected-depth surface: camera-frame points
 * P = (D / A) ((x + 1/2 - cx) / fx, (y + 1/2 - cy) / fy, 1) at pixel centres,
 * N = normalize((P[x+1] - P[x-1]) x (P[y+1] - P[y-1])) turned towards the camera.
 * A pixel counts when it and its four neighbours lie inside the image and have
 * A > a_min (the expected depth needs coverage).
 *   alpha, depth  device [P];  normal device [P,3]
 *   loss     device [n_views] float64, overwritten
 *   d_alpha, d_depth, d_normal  device or all NULL: += weight * d loss / d plane
 *            (through N as well; allocates 24 bytes per pixel of scratch)
 * Asynchronous on the context stream.
 */
ocgs_status ocgs_normal_consistency(ocgs_ctx* ctx, const float* alpha, const float* depth, const float* normal,
                                    const ocgs_camera* cams, int32_t n_views, float weight, float a_min, double* loss,
                                    float* d_alpha, float* d_depth, float* d_normal);

/* Sizes of one forward state: K pairs, P pixels, and E = sum over pixels of
 * the length of the blended prefix of the pixel's tile list (the (pixel,
 * Gaussian) pairs that both the forward and the backward must evaluate).
 * Synchronises. */
typedef struct {
  int64_t n_pairs;
  int64_t n_pixels;
  int64_t n_tiles;
  int64_t n_views;
  int64_t n_evals;
} ocgs_state_info;
ocgs_status ocgs_state_query(ocgs_ctx* ctx, const ocgs_fwd_state* state, ocgs_state_info* info);

/* Number of CUDA kernels this library has launched in this process. */
int64_t ocgs_kernel_launches(void);

/* Result of ocgs_autotune. */
typedef struct {
  ocgs_options best;     /* chosen options (also set on the context) */
  double best_ms;        /* forward + backward time of the chosen options, ms */
  int32_t n_tried;       /* candidates timed (0 when taken from the cache) */
  int32_t from_cache;    /* 1: read from the cache file */
} ocgs_tune_result;

/*
 * ocgs_autotune — pick the launch options that make this workload's training
 * render and backward fastest on this GPU, and set them on the context.
 * Options never change a result (see ocgs_options), only the time.  The timed
 * pass is what a training step runs: a render with images and a contribution
 * score, then the backward of a colour and opacity loss (dL/dC = dL/dA = 1).
 * The search is staged: (1) tile shape, pixels per thread and persistence at
 * the context's front_fraction and 32 Gaussians per batch; (2) for a
 * persistent choice, front_fraction in {0, 0.05, 0.1, 0.2}; (3) 16 or 64
 * Gaussians per batch where the chosen shape offers them.  Each candidate runs
 * once untimed and twice timed (CUDA events on the context stream); one whose
 * pair count exceeds a render's capacity (OCGS_ERR_CAPACITY) is skipped.
 * cache_path (host string or NULL) names a text file of earlier choices keyed
 * by GPU, SM count, SH degree, views and power-of-two buckets of Gaussians and
 * pixels; a hit skips the timing, a miss appends a line.  Synchronises;
 * allocates its buffers from the context pool for the duration of the call.
 */
ocgs_status ocgs_autotune(ocgs_ctx* ctx, const ocgs_gaussians* gaussians, const ocgs_camera* cams,
                          int32_t n_views, const char* cache_path, ocgs_tune_result* result);

/* Built-in stage profiler: enable (1) resets the accumulators and starts
 * recording; read synchronises the stream and returns the sums so far. */
ocgs_status ocgs_profile_enable(ocgs_ctx* ctx, int32_t enable);
ocgs_status ocgs_profile_read(ocgs_ctx* ctx, ocgs_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* OCGS_H */
