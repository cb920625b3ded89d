/*
 * degraf.h - C ABI of the GB300 (sm_103a) DeGraF detection + RLOF tracking library.
 *
 * Implements the sparse-matching stage of DeGraF-Flow (Stephenson, Breckon,
 * Katramados, arXiv 1901.09971, Section 2): DeGraF key-points on an even grid of
 * frame 1 (Eq. 1-2 and the selection rule after them), tracked into frame 2 by
 * robust local optical flow (RLOF) over an image pyramid.
 *
 * Conventions for every entry point:
 *   - Array pointers marked "device" are CUDA device pointers owned by the caller.
 *     The library never allocates memory in these calls and keeps no pointer after
 *     returning.
 *   - Work is enqueued asynchronously on `stream` (0 = legacy default stream). The
 *     return value reports argument checks and launch errors only; errors raised
 *     while kernels run surface at the caller's next synchronisation.
 *   - Return value: DGF_OK (0) or a negative DGF_ERR_* code; dgf_strerror() names it.
 *   - Image coordinates: x = column, y = row, pixel centres at integers.
 *   - Floating-point work follows IEEE round-to-nearest (no fast-math).
 */
#ifndef DEGRAF_H
#define DEGRAF_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define DGF_OK 0
#define DGF_ERR_ARG (-1)       /* null pointer, bad size, pitch, window, radius or level count */
#define DGF_ERR_WORKSPACE (-2) /* a caller buffer is smaller than the size query asks for */
#define DGF_ERR_LEVELS (-3)    /* the coarsest pyramid level is smaller than the support */
#define DGF_ERR_CUDA (-4)      /* a CUDA launch or runtime call failed */
#define DGF_ERR_TIMEOUT (-5)   /* a bounded wait expired */
#define DGF_ERR_DEVICE (-6)    /* a kernel reported an error through its status word */

/* per-point tracking status (rlof_track `status` output) */
#define DGF_TRACKED 0   /* converged at level 0 */
#define DGF_OOB 1       /* the point centre left the level image */
#define DGF_SMALL_EIG 2 /* gradient matrix too weak: lambda_min / (2r+1)^2 < min_eig */
#define DGF_SINGULAR 3  /* non-positive Cholesky pivot in the Gauss-Newton solve */
#define DGF_MAXITER 4   /* tracked, but level 0 hit max_iter before converging */

/* pyramid storage types */
#define DGF_F32 0
#define DGF_F16 1

#define DGF_MAX_LEVELS 6
#define DGF_MAX_RADIUS 7
#define DGF_MAX_WINDOW 64
#define DGF_RLOF_PARAMS_VERSION 2

/* Human-readable name of a DGF_* status code (static string, never NULL). */
const char* dgf_strerror(int code);

/* Library ABI version (major * 100 + minor). */
int dgf_version(void);

/* device-side failures (dgf_device_status bits) */
#define DGF_DEV_STAGE_WAIT 1u     /* a detection or pyramid block gave up waiting for its staging copies */
#define DGF_DEV_EPIC_PASSES 2u    /* epic_interpolate: the labelling did not settle (pass limit or barrier) */
#define DGF_DEV_EPIC_CAPACITY 4u  /* epic_interpolate: a neighbourhood search outgrew its largest layout */

/*
 * Device-side failures on the current device since the last reset, as a set of
 * DGF_DEV_* bits in *bits (0: every launch ran to the end). Kernels report what the
 * host cannot check before launching here instead of synchronising the caller's
 * stream: detection and the pyramid stage frame rows with bulk asynchronous copies
 * when the frame's base, pitch and width are multiples of 16, and a block whose
 * copies never complete gives up after a bounded wait and leaves its outputs
 * unwritten; epic_interpolate reports a labelling that did not settle and a search
 * that outgrew its layout (its dense field is then incomplete). reset = 1 also
 * clears the word. Synchronous: waits for the device's pending work. The first
 * call on a device, or the first launch of those kernels, looks the word's address
 * up; make it before any stream capture.
 * Returns DGF_ERR_ARG for a null bits, DGF_ERR_CUDA if the word cannot be read.
 */
int dgf_device_status(unsigned* bits, int reset);

/* ---- DeGraF detection (Section 2, Eq. 1-2) ------------------------------- */

/*
 * Number of DeGraF key-points on a W x H frame: one per window position of the
 * sliding grid with step `step` (Section 2, "Point detection"), counting only
 * windows that lie fully inside the frame:
 *   N = (floor((W - win_w) / step) + 1) * (floor((H - win_h) / step) + 1),
 * or 0 when the window does not fit. Returns -1 on invalid arguments.
 */
long long dgf_degraf_count(int W, int H, int win_w, int win_h, int step);

/*
 * DeGraF key-point detection (Section 2, Eq. 1 and Eq. 2, selection rule after
 * Eq. 2). For window (u, v) with top-left pixel (u*step, v*step), i = row and
 * j = column inside the window:
 *   S_pos = sum I, C_pos = (sum j I, sum i I) / S_pos;  m = max I in the window;
 *   S_neg = sum (1 + m - I), C_neg = (sum j (1+m-I), sum i (1+m-I)) / S_neg;
 *   key-point = window origin + (S_neg > S_pos ? C_neg : C_pos).
 *   img      device, uint8 frame, row r at img + r * pitch (bytes), pitch >= W.
 *   win_w, win_h in [1, DGF_MAX_WINDOW]; step >= 1.
 *   pts      device, float [N][2] (x, y), N = dgf_degraf_count(); row-major over
 *            window positions (v outer, u inner).
 *   sums     device, nullable, int32 [N][4]: S_pos, sum j I, sum i I, m (exact).
 * N = 0 is not an error (nothing is launched).
 */
int degraf_detect(const uint8_t* img, int W, int H, int pitch, int win_w, int win_h, int step,
                  float* pts, int32_t* sums, cudaStream_t stream);

/* ---- image pyramid -------------------------------------------------------- */

/*
 * Layout of a pyramid buffer. RLOF tracks through an image pyramid (Section 2,
 * "Sparse point tracking"); the paper does not define it, and this library uses:
 * level 0 = the frame; level l+1 is floor(W_l / 2) x floor(H_l / 2) with each pixel
 * the mean of its 2x2 block of level l; gradients Ix, Iy are the Sobel kernels / 8
 * with the border clamped. All values are exact dyadic rationals, so FP32 storage
 * is exact; FP16 storage rounds each exact value once (round to nearest even).
 * Planes are stored I_0 .. I_{L-1}, then (with_grad) Ix_0 .. Ix_{L-1},
 * Iy_0 .. Iy_{L-1}; every plane starts on a 256-byte boundary and its rows are
 * `pitch` elements apart (a multiple of 128 bytes). The intensity planes sit at the
 * same offsets with or without gradients. off_I/off_Ix/off_Iy locate pixel (0, 0);
 * around it each plane carries a border of DGF_PYR_APRON pixels on every side that
 * repeats the plane's edge (pixel (x, y) outside the level holds the value at the
 * clamped position), so readers of bilinear taps near the border need no clamping.
 */
#define DGF_PYR_APRON 12

typedef struct {
    int levels, storage, with_grad;
    int W[DGF_MAX_LEVELS], H[DGF_MAX_LEVELS], pitch[DGF_MAX_LEVELS]; /* pitch in elements */
    size_t off_I[DGF_MAX_LEVELS], off_Ix[DGF_MAX_LEVELS], off_Iy[DGF_MAX_LEVELS]; /* bytes */
    size_t bytes;
} dgf_pyramid_layout;

/* Fills *out for a W x H frame; off_Ix/off_Iy are 0 when with_grad = 0. Returns
 * DGF_ERR_ARG for levels outside [1, DGF_MAX_LEVELS] or an empty coarsest level. */
int dgf_pyramid_layout_get(int W, int H, int levels, int storage, int with_grad,
                           dgf_pyramid_layout* out);

/* Bytes a pyramid buffer needs (0 on invalid arguments). */
size_t dgf_pyramid_bytes(int W, int H, int levels, int storage, int with_grad);

/*
 * Builds the pyramid of one uint8 frame into `pyr` (device, pyr_bytes >=
 * dgf_pyramid_bytes(), 256-byte aligned). img/pitch as in degraf_detect.
 * storage: DGF_F32 or DGF_F16. with_grad: 1 to also write Ix and Iy (frame 1 of a
 * pair needs them, frame 2 does not).
 */
int pyramid_build(const uint8_t* img, int W, int H, int pitch, int levels, int storage,
                  int with_grad, void* pyr, size_t pyr_bytes, cudaStream_t stream);

/* ---- RLOF tracking (Section 2 "Sparse point tracking"; Section 3 "Parameters") */

/*
 * Tracking parameters. The paper names RLOF with its illumination model but gives
 * no formulas; the reading implemented (identical in the FP64 test oracle):
 *   for each level l = levels-1 .. 0 (coarse to fine):
 *     p_l = (p + 1/2) / 2^l - 1/2; template T, Tx, Ty = bilinear samples of frame 1's
 *     level at p_l + k, k in [-radius, radius]^2 (border taps clamped);
 *     SMALL_EIG if lambda_min(sum [Tx Ty]^T [Tx Ty]) / (2 radius + 1)^2 < min_eig;
 *     d = 0; up to max_iter Gauss-Newton steps: q = p_l + g + d (OOB if q leaves
 *     [0, W_l-1] x [0, H_l-1]); J = bilinear frame-2 samples at q + k;
 *       model 4: r = J - (1+m) T - c, a = (Tx, Ty, -T, -1)
 *       model 2: r = J - T,           a = (Tx, Ty)
 *     Hampel IRLS weights w = psi(r)/r with knots (hampel_a, hampel_b, hampel_c):
 *       psi = r (|r|<=a), a sgn r (a<|r|<=b), a sgn r (c-|r|)/(c-b) (b<|r|<=c), 0 beyond;
 *     solve (sum w a a^T) delta = -(sum w a r) by Cholesky (SINGULAR on a
 *     non-positive pivot); d += delta[0:2], (m, c) += delta[2:4]; stop when
 *     |delta[0:2]| < eps. Then g = 2 (g + d) for the next finer level.
 *   flow = g + d at level 0.
 */
typedef struct {
    int version;  /* DGF_RLOF_PARAMS_VERSION */
    int levels;   /* pyramid levels, 1..DGF_MAX_LEVELS, as both pyramids were built */
    int radius;   /* support radius r, 1..DGF_MAX_RADIUS; (2r+1)^2 samples */
    int max_iter; /* Gauss-Newton iterations per level, 1..255 */
    int model;    /* 2 = translation, 4 = translation + gain/offset illumination */
    int storage;  /* DGF_F32 or DGF_F16, as both pyramids were built */
    float eps;    /* convergence threshold on |delta d| in pixels */
    float hampel_a, hampel_b, hampel_c; /* 0 < a <= b < c */
    float min_eig;
    /* Adaptive cross-based support (Section 3 "Parameters"; no formula in the paper):
     * 0 keeps the square (2r+1)^2 support. tau > 0: per level, around the point's
     * centre pixel (p_l rounded half up, clamped into the level) of frame 1's
     * intensity plane, a vertical arm runs up and down (at most r pixels each way)
     * while centre-column pixels differ from the centre by at most tau, and each
     * arm row runs left and right (at most r) while its pixels differ from the row's
     * centre-column pixel by at most tau; support samples outside this cross get
     * weight 0, and the minimum-eigenvalue test sums over the kept samples and
     * divides by their number. Pixels outside the level are read clamped. */
    float cross_tau;
} dgf_rlof_params;

/* Fills *p with the defaults: levels 3, radius 4, max_iter 30, model 4, F32,
 * eps 1e-3, Hampel (8, 16, 32), min_eig 1e-3, cross_tau 0 (square support). */
void dgf_rlof_params_default(dgf_rlof_params* p);

/* Tuning hook: lanes per tracked point, 8, 16 or 32 (0 = automatic choice, the
 * default). Applies to later rlof_track calls from any thread. Returns the previous
 * setting, or DGF_ERR_ARG for another value. Only radius 4 and 5 honour 8 or 16;
 * every other radius uses 32 lanes. */
int dgf_rlof_set_lanes(int lanes);

/*
 * Tracks n points from frame 1 into frame 2.
 *   pyr1   device, pyramid of frame 1 built with with_grad = 1.
 *   pyr2   device, pyramid of frame 2 (gradients optional).
 *   W, H   level-0 size of both frames.
 *   pts    device, float [n][2] start points in frame 1 (e.g. degraf_detect output).
 *   flow   device, float [n][2] output: displacement into frame 2; 0 for lost points.
 *   status device, uint8 [n] output: DGF_TRACKED .. DGF_MAXITER.
 *   iters  device, nullable, uint8 [n]: Gauss-Newton updates over all levels
 *          (saturates at 255).
 *   illum  device, nullable, float [n][2]: gain m and offset c (model 4; else 0).
 * Returns DGF_ERR_LEVELS when the coarsest level is narrower or lower than
 * 2 radius + 2 pixels. n = 0 is not an error.
 */
int rlof_track(const void* pyr1, const void* pyr2, int W, int H, const float* pts, int n,
               const dgf_rlof_params* p, float* flow, uint8_t* status, uint8_t* iters,
               float* illum, cudaStream_t stream);

/* ---- global-motion prior (Section 3 "Parameters": RLOF(IM-GM)) ------------ */

#define DGF_GM_PARAMS_VERSION 1

/* The paper runs RLOF with a global motion model and prints no formula. The model
 * used: a global affine motion q = A p + t (a[6]: q_x = a0 x + a1 y + a2,
 * q_y = a3 x + a4 y + a5), fitted to a sparse first pass and used as every point's
 * initial flow (A p + t - p, divided by 2^(levels - 1) at the coarsest level). */
typedef struct {
    int version;       /* DGF_GM_PARAMS_VERSION */
    int stride;        /* first pass tracks points 0, stride, 2 stride, ... (>= 1) */
    int extra_levels;  /* first pass uses levels + extra_levels pyramid levels (>= 0) */
    int iters;         /* IRLS iterations of the fit (1 .. 64; 1 = least squares) */
    double c0, c_min;  /* Tukey threshold c_k = max(c_min, c0 / 2^(k-1)) in pixels, 0 < c_min */
} dgf_gm_params;

/* Defaults: stride 4, extra_levels 2, iters 8, c0 32, c_min 2. */
void dgf_gm_params_default(dgf_gm_params* g);

/* Workspace bytes of rlof_track_gm for n points (0 for invalid arguments). Its first
 * 64 bytes hold, after the call, the fitted affine a[6] (doubles) and an int flag at
 * byte 48 (1 = fitted; 0 = fewer than 3 converged first-pass points or a singular
 * fit, a = identity motion). */
size_t dgf_gm_workspace(int n, const dgf_gm_params* g);

/*
 * Tracking with the global-motion prior, all on `stream`:
 *   1. first pass: points k * stride tracked with levels + extra_levels levels;
 *   2. fit: iteratively reweighted least squares over the first-pass points with
 *      status DGF_TRACKED: iteration 0 least squares, then Tukey biweights
 *      (1 - (e / c_k)^2)^2 of the residual distance e (0 beyond c_k); each step
 *      solves the 3 x 3 normal equations shared by the x and y rows in FP64 (a
 *      pivot below 1e-10 of its diagonal entry, or fewer than 3 weighted points,
 *      keeps the previous estimate and ends the fit);
 *   3. main pass: every point tracked with p->levels levels from the prior's flow.
 *   pyr1, pyr2  device pyramids built with pyr_levels >= p->levels + extra_levels
 *               levels (frame 1 with gradients).
 *   pts, n, flow, status, iters, illum: as for rlof_track (main-pass results).
 *   workspace   device, >= dgf_gm_workspace(n, g) bytes, 256-byte aligned.
 * Returns DGF_ERR_ARG for bad parameters or pyr_levels, DGF_ERR_LEVELS when the
 * first pass's coarsest level is smaller than 2 radius + 2 pixels,
 * DGF_ERR_WORKSPACE for a short workspace, else the rlof_track codes.
 */
int rlof_track_gm(const void* pyr1, const void* pyr2, int W, int H, int pyr_levels, const float* pts, int n,
                  const dgf_rlof_params* p, const dgf_gm_params* g, float* flow, uint8_t* status,
                  uint8_t* iters, float* illum, void* workspace, size_t ws_bytes, cudaStream_t stream);

/* ---- forward-backward consistency (not in the paper's text) ---------------- */

/* Status of a forward-tracked point that failed the forward-backward check. */
#define DGF_FB_REJECTED 5

/* Workspace bytes of rlof_track_fb for n points (0 for n < 0). */
size_t dgf_fb_workspace(int n);

/*
 * Forward-backward consistency filter, a common check on sparse tracks before
 * interpolation (the paper does not describe one): points are tracked from frame 1
 * to frame 2 (flow f), their end points p + f back from frame 2 to frame 1 (flow b)
 * with the same parameters, and the round-trip error is |f + b| where both passes
 * tracked the point (DGF_TRACKED or DGF_MAXITER), else +inf.
 *   pyr1, pyr2  device pyramids of both frames, BOTH built with gradients (the
 *               backward pass uses frame 2 as its template); pyr_bytes is the size
 *               of each buffer and must be at least dgf_pyramid_bytes(W, H,
 *               p->levels, p->storage, 1).
 *   fb_max      > 0: forward-tracked points with an error above fb_max get status
 *               DGF_FB_REJECTED (their flow is kept); 0: no status changes.
 *   flow, status  as for rlof_track (forward pass).
 *   fb_err      device, nullable, float [n]: the round-trip error.
 *   workspace   device, >= dgf_fb_workspace(n) bytes, 256-byte aligned.
 * Returns DGF_ERR_ARG for short pyramid buffers or bad arguments,
 * DGF_ERR_WORKSPACE for a short workspace, else the rlof_track codes.
 */
int rlof_track_fb(const void* pyr1, const void* pyr2, size_t pyr_bytes, int W, int H, const float* pts, int n,
                  const dgf_rlof_params* p, float fb_max, float* flow, uint8_t* status, float* fb_err,
                  void* workspace, size_t ws_bytes, cudaStream_t stream);

/* ---- EPIC interpolation (Section 2 "Interpolation"; k from Section 3) ---- */

#define DGF_EPIC_PARAMS_VERSION 1
#define DGF_EPIC_MAX_K 256
#define DGF_EPIC_MAX_W_PLUS_H 8192
#define DGF_EPIC_MAX_POINTS 16777215

/* Parameters of the interpolation (the paper fixes k = 128 and gradient-based
 * edges; the costs, the kernel and the fallback are this library's reading). */
typedef struct {
    int version;       /* DGF_EPIC_PARAMS_VERSION */
    int k;             /* nearest seeds per fit, 1 .. DGF_EPIC_MAX_K (128) */
    int model;         /* 1: locally affine fit (default), 0: weighted mean */
    int cost_base;     /* edge cost of a flat pixel, 1 .. 4096 (4) */
    int cost_gain;     /* multiplier of |Gx| + |Gy|, 0 .. 32 (1) */
    double a;          /* kernel decay per flat pixel of geodesic travel, >= 0 (0.1) */
    double min_spread; /* px; smallest weighted spread of the neighbours for an affine fit (1) */
} dgf_epic_params;

/* Fills *p with the defaults above. */
int dgf_epic_params_default(dgf_epic_params* p);

/* Optional device outputs of epic_interpolate, each nullable (for inspection and
 * tests; knn_idx and knn_dist go together). */
typedef struct {
    int32_t* labels;    /* [H][W]: seed of each pixel, -1 where no seed exists */
    int64_t* dist;      /* [H][W]: geodesic distance to that seed, -1 where none */
    int32_t* knn_idx;   /* [n][k]: the seed's neighbourhood, nearest first (first knn_count entries) */
    int64_t* knn_dist;  /* [n][k]: their seed-graph distances */
    int32_t* knn_count; /* [n]: neighbourhood size, 0 for matches that are not seeds */
    double* models;     /* [n][6]: (A00, A01, A10, A11, b0, b1), zeros for non-seeds */
    uint8_t* fit_kind;  /* [n]: 0 not a seed, 1 affine, 2 weighted mean */
    int32_t* retried;   /* [1]: searches redone with the large frontier (more than 128 entries) */
} dgf_epic_debug;

/* Workspace bytes of epic_interpolate (0 for sizes outside the limits). */
size_t dgf_epic_workspace(int W, int H, int n);

/*
 * Dense flow from sparse matches by edge-preserving interpolation (Section 2,
 * "Interpolation": an affine model fitted to the k nearest sparse vectors under a
 * geodesic distance that penalises crossing image edges, edges from image
 * gradients). Reading, every distance an exact integer:
 *   1. edge cost C(x) = cost_base + cost_gain (|Gx| + |Gy|), Gx, Gy the integer
 *      Sobel responses of frame 1 ([-1 0 1; -2 0 2; -1 0 1] and its transpose,
 *      clamped borders);
 *   2. seeds: matches with status DGF_TRACKED or DGF_MAXITER, at pixel
 *      (floor(x + 1/2), floor(y + 1/2)) clamped into the image; a seed whose pixel
 *      holds a lower-index seed is not used;
 *   3. geodesic distance on the 4-connected grid, a step between x and y costing
 *      C(x) + C(y); every pixel takes the lexicographically smallest (distance,
 *      seed index) over the seeds: distance D(x), label s(x);
 *   4. seed graph: 4-adjacent pixels x, y in different cells link s(x) and s(y)
 *      with weight D(x) + C(x) + C(y) + D(y), the smallest such weight per pair;
 *   5. neighbourhood of seed s: the k seeds with the smallest (graph distance,
 *      index), s first;
 *   6. fit, weights w = exp(-a d / (2 cost_base)): model 1 minimises
 *      sum w |A (p_t - p_s) + b - f_t|^2 when there are 3+ neighbours and the
 *      smallest eigenvalue of their weighted position covariance is at least
 *      min_spread^2, else (and always for model 0) A = 0 and b = the weighted mean;
 *   7. dense flow of pixel x: A_s(x) (x - p_s(x)) + b_s(x); 0 where no seed exists.
 *   img         device, uint8 frame 1, row pitch `pitch` bytes (>= W).
 *   pts, flow   device, float [n][2], 8-byte aligned: match positions and flows.
 *   status      device, uint8 [n]: the tracking statuses.
 *   dense       device, float [H][W][2] (contiguous rows of W), 8-byte aligned.
 *   dbg         host struct of nullable device outputs, or NULL.
 *   workspace   device, >= dgf_epic_workspace(W, H, n) bytes, 256-byte aligned.
 * Limits: W + H <= DGF_EPIC_MAX_W_PLUS_H, n <= DGF_EPIC_MAX_POINTS.
 * Asynchronous on `stream` like every entry point: the labelling's passes run in
 * one cooperative launch that stops at the first pass that changes nothing (at
 * most 4096), with no host round trip, so the call can follow tracking back to
 * back and be captured into a CUDA graph (after the first call on the device,
 * which looks up the status word). A labelling that did not settle and a
 * neighbourhood search that outgrew its largest shared-memory layout (more than
 * 8192 discovered or settled seeds) are reported through dgf_device_status
 * (DGF_DEV_EPIC_PASSES, DGF_DEV_EPIC_CAPACITY).
 * Returns DGF_ERR_ARG for bad arguments or parameters, DGF_ERR_WORKSPACE for a
 * short workspace, DGF_ERR_CUDA for a failed launch, else DGF_OK.
 */
int epic_interpolate(const uint8_t* img, int W, int H, int pitch, const float* pts, const float* flow,
                     const uint8_t* status, int n, const dgf_epic_params* p, float* dense, const dgf_epic_debug* dbg,
                     void* workspace, size_t ws_bytes, cudaStream_t stream);

/* ---- adjoints (gradients with respect to the frames; the paper has none) ---- */

/* Workspace bytes of degraf_detect_backward (one record per key-point). */
size_t dgf_degraf_backward_workspace(int W, int H, int win_w, int win_h, int step);

/*
 * Vector-Jacobian product of degraf_detect (Eq. 1-2 differentiated):
 * grad_img += sum_k grad_pts[k] . d(point_k)/d(img), treating the frame as real
 * valued. For C_pos: d(x)/dI_ij = (j - x_local) / S_pos (y likewise with i). For
 * C_neg: -(j - x_local) / S_neg, plus sum_ij (j - x_local) / S_neg on the window's
 * first maximum pixel in row-major order (m moves with it). Valid wherever the
 * selection and the maximum do not change.
 *   img, W, H, pitch, win_w, win_h, step: as given to degraf_detect.
 *   grad_pts   device, float [N][2].
 *   workspace  device, 256-byte aligned, ws_bytes >= dgf_degraf_backward_workspace().
 *   grad_img   device, float, row y at grad_img + y * grad_pitch (elements,
 *              >= W); accumulated into. Deterministic (gathered, no atomics).
 * DGF_ERR_ARG also for a float array that is not 4-byte aligned.
 */
int degraf_detect_backward(const uint8_t* img, int W, int H, int pitch, int win_w, int win_h, int step,
                           const float* grad_pts, void* workspace, size_t ws_bytes, float* grad_img,
                           int grad_pitch, cudaStream_t stream);

/* Workspace bytes of rlof_track_backward (three W x H float planes). */
size_t dgf_rlof_backward_workspace(int W, int H);

/*
 * Vector-Jacobian product of rlof_track by implicit differentiation at the
 * converged level-0 state theta = (d, m, c): there F = sum_k psi(r_k) a_k = 0, so
 * d(theta)/dI = -A^-1 dF/dI with A = sum_k psi'(r_k) a_k s_k^T, s_k = dr_k/dtheta
 * (exact derivatives of the bilinear interpolant of frame 2). With A^T lambda =
 * (grad_flow, grad_illum): grad_I2 += -sum_k psi'(r_k) (lambda . a_k) dJ_k/dI2, and
 * grad_I1 collects the template terms through the bilinear weights and the
 * transposed Sobel / 8 stencil. Coarser levels only select the basin and carry no
 * gradient; points whose status is not DGF_TRACKED contribute nothing. The key-
 * points are constants.
 *   pyr1, pyr2, W, H, pts, n, p: as given to rlof_track; flow, illum, status: its
 *   outputs (illum required for model 4).
 *   grad_flow   device, float [n][2]; grad_illum: nullable float [n][2] (model 4).
 *   workspace   device, 256-byte aligned, >= dgf_rlof_backward_workspace(W, H).
 *   grad_I1, grad_I2  device, float, row pitch grad_pitch elements; accumulated
 *               into with atomics (the summation order, and so the last bits, may
 *               vary between runs).
 * DGF_ERR_ARG also for a float array that is not 4-byte aligned.
 */
int rlof_track_backward(const void* pyr1, const void* pyr2, int W, int H, const float* pts, int n,
                        const dgf_rlof_params* p, const float* flow, const float* illum, const uint8_t* status,
                        const float* grad_flow, const float* grad_illum, void* workspace, size_t ws_bytes,
                        float* grad_I1, float* grad_I2, int grad_pitch, cudaStream_t stream);

/* ---- batched pipeline (Section 2 over many frame pairs) ------------------- */

/*
 * One frame pair of a batch: both frames, the DeGraF grid and the caller's output
 * buffers (device). N = dgf_degraf_count(W, H, win, win, step) key-points.
 */
typedef struct {
    const uint8_t* frame1; /* device, uint8 W x H, rows `pitch` bytes apart */
    const uint8_t* frame2; /* device, same size and pitch */
    int W, H, pitch;
    int win, step;         /* square DeGraF window and grid step */
    float* pts;            /* device out, float [N][2] key-points of frame 1 */
    float* flow;           /* device out, float [N][2] */
    uint8_t* status;       /* device out, uint8 [N] */
    uint8_t* iters;        /* device out, nullable, uint8 [N] */
} dgf_pair;

/*
 * Workspace bytes rlof_track_many needs for this batch (both pyramids of every
 * pair), or 0 when an argument is invalid.
 */
size_t dgf_track_many_workspace(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p);

/* stages of rlof_track_many */
#define DGF_STAGE_DETECT 1
#define DGF_STAGE_PYRAMID 2
#define DGF_STAGE_TRACK 4
#define DGF_STAGE_ALL 7

/*
 * DeGraF detection, both pyramids and RLOF tracking of every pair (the same
 * definitions as degraf_detect, pyramid_build and rlof_track, one parameter set
 * for all pairs). Per chunk of 64 pairs: one detection launch per distinct window
 * size, one pyramid launch for all frames and one tracking launch over every
 * point of the chunk. pairs: host array of n_pairs descriptors (read during the
 * call only). stages: DGF_STAGE_ALL, or a subset (tracking reads the points and
 * pyramids an earlier call left in the same outputs and workspace).
 * workspace: device, 256-byte aligned, ws_bytes >= dgf_track_many_workspace();
 * owned by the caller and in use until the work completes on `stream`.
 * use_graph = 1: the launch sequence is captured into a CUDA graph on first use
 * of a given argument set (descriptors, parameters, workspace, device, lanes
 * setting, stages) and the instantiated graph is replayed on later calls with the same
 * set; while `stream` is already being captured by the caller, plain launches are
 * enqueued instead. Returns DGF_ERR_WORKSPACE for a short workspace and the
 * rlof_track codes otherwise.
 */
int rlof_track_many(const dgf_pair* pairs, int n_pairs, const dgf_rlof_params* p, void* workspace,
                    size_t ws_bytes, int stages, int use_graph, cudaStream_t stream);

/* ---- one pair without allocation (no counterpart in the paper) ------------ */

/* Size of the scratch array rlof_track_pair_noalloc uses (24 MiB). */
#define DGF_NOALLOC_SCRATCH_BYTES (24u << 20)

/*
 * For callers that cannot allocate device memory while they track (a real-time
 * loop that must not risk an allocation stall, a plug-in inside an application
 * that owns the GPU's memory, code that forbids allocation after start-up): the
 * same detection + pyramids + tracking as rlof_track_many for ONE pair, with the
 * two pyramids placed in a fixed scratch array compiled into the library instead
 * of a caller workspace. The caller still provides the frames and every output
 * buffer of *pair. Nothing is allocated: no cudaMalloc, no cudaFree, no graph.
 *   - The scratch array (DGF_NOALLOC_SCRATCH_BYTES) occupies device memory on
 *     every GPU that loads the library until the process exits.
 *   - A pair whose two pyramids need more (dgf_track_many_workspace(pair, 1, p) >
 *     DGF_NOALLOC_SCRATCH_BYTES; e.g. beyond about 1280x720 at 5 FP32 levels) is
 *     rejected with DGF_ERR_WORKSPACE before anything is enqueued.
 *   - The first call on each device looks up the array's device address (the
 *     device must be current); make that first call before any stream capture.
 *   - All calls share the one array and it keeps the last call's pyramids. Calls
 *     whose work overlaps on the GPU (different streams without ordering between
 *     them, or several host threads) race on it: order them on one stream.
 * Returns the rlof_track_many codes.
 */
int rlof_track_pair_noalloc(const dgf_pair* pair, const dgf_rlof_params* p, cudaStream_t stream);

/* ---- measurement and accuracy probes (no counterpart in the paper) -------- */

/*
 * FP32 throughput probe, the measured ceiling of the tracking kernel's roofline
 * (tracking is bound by FP32 issue, not memory). Launches `blocks` x `threads`
 * threads (threads a multiple of 32, at most 256), each running 64 steps of eight
 * independent fused multiply-add chains per trip for `iters` trips; packed = 1 uses
 * the packed FP32x2 FMA (two FMAs per lane and instruction, the form the tracking
 * kernel issues), packed = 0 scalar FFMA. out: device float [blocks * threads],
 * written once per thread (a value of no interest that keeps the work alive).
 * The caller times the launch on `stream`; dgf_fp32_probe_flops() gives its FLOPs
 * (2 per FMA). Returns DGF_ERR_ARG for bad sizes.
 */
int dgf_fp32_probe(float* out, int blocks, int threads, int iters, int packed, cudaStream_t stream);
double dgf_fp32_probe_flops(int blocks, int threads, int iters, int packed);

/*
 * exp(-y) as the EPIC fit weights compute it (Tang's table-driven method, ACM TOMS
 * 15(2), 1989; FP64), for y >= 0, so that its error can be measured against a
 * reference exponential. y, out: device double [n]. Returns DGF_ERR_ARG for n < 0
 * or null pointers with n > 0.
 */
int dgf_epic_exp_neg(const double* y, double* out, int n, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* DEGRAF_H */
