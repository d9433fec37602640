/*
 * libpothole: GB300 (sm_103a) CUDA implementation of the stereo road pothole-detection path of
 * Fan, Ozgunalp, Wang, Liu, Pitas, "Rethinking Road Surface 3D Reconstruction and Pothole Detection:
 * From Perspective Transformation to Disparity Map Segmentation" (arXiv 2012.10802).
 *
 * The calls follow the paper's pipeline (Fig. 1 and Sec. II):
 *   warp (Sec. II-A) -> cost -> aggregate -> disparity (Sec. II-B) -> transform (Sec. II-C)
 *   -> superpixels (Sec. II-D) -> pothole mask (Sec. II-E).
 *
 * Conventions for every call:
 *   - All image/volume pointers are DEVICE pointers owned by the caller unless a parameter says
 *     "host".  Images are row-major; `pitch` is the row stride in bytes of a uint8 image (>= W).
 *     Every other array is dense with no row padding.  Volumes are [H][W][D], disparity innermost.
 *   - Work is enqueued on the context's stream and is asynchronous: outputs are valid once that
 *     stream has reached the call (e.g. after cudaStreamSynchronize).  Host outputs are written
 *     before the call returns.
 *   - Arguments are validated before anything is launched; a bad argument returns
 *     PD_ERR_INVALID_ARG and launches nothing.  A CUDA failure returns PD_ERR_CUDA.  In both cases
 *     pd_last_error() gives a one-line reason.  The context stays usable after an error.
 *   - The context owns its scratch memory.  It grows on demand (cudaMalloc, which synchronises the
 *     device); failure returns PD_ERR_OOM and leaves the context valid.  Call a stage once outside
 *     any CUDA-graph capture before capturing it, so the scratch already has its size.
 *   - A context is not thread-safe: use one per host thread / stream.
 *   - A disparity map value < 0 marks an invalid pixel.
 */
#ifndef POTHOLE_H
#define POTHOLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pd_ctx pd_ctx;

typedef enum {
  PD_OK = 0,
  PD_ERR_INVALID_ARG = 1,
  PD_ERR_OOM = 2,
  PD_ERR_CUDA = 3,
  PD_ERR_TIMEOUT = 4,
  PD_ERR_UNSUPPORTED = 5
} pd_status;

/* Road disparity model of Sec. II-A, Eq. (3), with the roll applied about the image centre:
 *   v' = (v - vc) cos(roll) - (u - uc) sin(roll) + vc,   uc = (W-1)/2, vc = (H-1)/2,
 *   f(u, v) = a[0] + a[1] v' + a[2] v'^2   (a[2] is used only when order == 2).
 * order 1 is the paper's linear model; order 2 adds the quadratic term. roll is in radians. */
typedef struct {
  int order;
  double a[3];
  double roll;
} pd_road_model;

/* Method parameters.  pd_default_params() fills the defaults given in brackets. */
typedef struct {
  int D;              /* disparity range searched after the warp [128]: 32, 64, 128 or 256 */
  int paths;          /* aggregation directions, 4 or 8 [8] */
  int P1, P2;         /* Eq. (7)-(8) penalties lambda1 < lambda2 [4, 32]; 24 + P2 <= 255 */
  int lr_tol;         /* left-right consistency tolerance in pixels [1] */
  float delta_pt;     /* Eq. (6) margin delta_PT [10] */
  float delta_dt;     /* Eq. (13) offset delta_DT [16] */
  float delta_pd;     /* Eq. (14) tolerance delta_PD [2.36, the paper's value] */
  int slic_K;         /* SLIC superpixel count [1000] */
  float slic_m;       /* SLIC compactness [10] */
  int slic_iters;     /* SLIC iterations [10] */
  int model_order;    /* road model fitted by the transform, 1 or 2 [2] */
  int threshold_mode; /* 0: t_s = road mean - delta_pd [0]; 1: t_s = t_r - delta_pd */
  int fit_iters;      /* robust refits of the road model on the inliers of the previous fit [0] */
  float fit_tau;      /* inlier band |D1 - f| <= fit_tau of those refits, pixels [1] */
} pd_params;

/* One connected component of the pothole mask (56 bytes). */
typedef struct {
  int32_t label;        /* the component's smallest raster index v * W + u */
  int32_t count;        /* pixels */
  int32_t umin, vmin, umax, vmax;
  int64_t sum_u, sum_v; /* centroid = sum / count */
  int32_t superpixels;  /* 1, or 2 meaning two or more */
  int32_t corner;       /* centroid in a corner cell of the image split 8 x 8 */
  int32_t single;       /* all pixels in one superpixel */
  int32_t fake;         /* corner or single (Sec. III-B) */
} pd_component;

/* Device-side outputs of pd_run_pipeline (all caller-owned device buffers; any may be NULL
 * except where noted). */
typedef struct {
  int32_t* kappa;          /* [H] row shifts */
  int16_t* d_int;          /* [H][W] integer disparity in the warped pair (required) */
  float* D1;               /* [H][W] disparity w.r.t. the original pair, -1 = invalid (required) */
  pd_road_model* fitted;   /* one fitted model (device) */
  float* D2;               /* [H][W] transformed disparity (required) */
  int32_t* labels;         /* [H][W] superpixel labels (required) */
  float* D3;               /* [H][W] superpixel-clustered transformed disparity (required) */
  double* thresholds;      /* [2]: t_r, t_s (device) */
  uint8_t* mask;           /* [H][W] pothole mask (required) */
  /* Connected components of the mask (pd_components); components == NULL skips that step. */
  int32_t* components;     /* [H][W] component numbers, -1 outside the mask */
  pd_component* comps;     /* up to max_comps records */
  int32_t max_comps;
  int32_t connectivity;    /* 8 or 4; 0 means 8 */
  int32_t* n_comps;        /* one int: the number of components, or -1 (see pd_components) */
} pd_outputs;

/* Per-stage device times of the last pd_run_pipeline call, in milliseconds (host struct). */
typedef struct {
  float sgm_ms, transform_ms, superpixel_ms, mask_ms, total_ms;
} pd_stage_times;

/* Device times summed over the calls made while profiling was on (host struct, milliseconds).
 * Stages a call does not run stay 0. */
typedef struct {
  int calls;            /* pd_sgm / pd_run_pipeline calls profiled */
  int pad;
  long long launches;   /* kernels those calls launched */
  double prep_ms;       /* row shifts, census and matching cost */
  double aggregate_ms;  /* Eq. (8) aggregation kernel */
  double disparity_ms;  /* winner-take-all, right view, left-right check */
  double transform_ms;  /* Sec. II-C */
  double superpixel_ms; /* Sec. II-D and D3 */
  double mask_ms;       /* Sec. II-E threshold and mask */
  double total_ms;      /* first to last event of each call */
} pd_profile;

/* ------------------------------------------------------------------------------ context */

/* Creates a context on CUDA device `device` that enqueues on `stream` (a cudaStream_t; NULL means
 * the legacy default stream).  The caller owns the stream. */
pd_status pd_create(pd_ctx** ctx, int device, void* stream);
/* Frees the context's scratch memory and the context.  NULL is accepted. */
pd_status pd_destroy(pd_ctx* ctx);
/* Changes the stream later calls enqueue on. */
pd_status pd_set_stream(pd_ctx* ctx, void* stream);
/* One-line description of the last error on this context ("" if none).  Valid until the next
 * call on the context. */
const char* pd_last_error(const pd_ctx* ctx);
/* Fills *p with the defaults listed in pd_params. */
pd_status pd_default_params(pd_params* p);
/* Bytes of scratch the context currently holds. */
size_t pd_workspace_bytes(const pd_ctx* ctx);

/* ------------------------------------------------------------------- Sec. II-A: the warp */

/* Eq. (6): kappa[v] = floor(min over x = 0..W-1 of f(x, v) - delta_pt), then the perspective
 * transformation of the right image: right_warped(u, v) = right(clamp(u - kappa[v], 0, W-1), v),
 * which makes the disparity w.r.t. (left, right_warped) equal to D1 - kappa (Eq. (10)).
 * model: host pointer.  right, right_warped: uint8 [H] rows of `pitch` bytes (right_warped may be
 * NULL to compute kappa only).  kappa: int32 [H]. */
pd_status pd_warp(pd_ctx* ctx, const uint8_t* right, int W, int H, size_t pitch,
                  const pd_road_model* model, float delta_pt, uint8_t* right_warped,
                  int32_t* kappa);

/* ------------------------------------------------------- Sec. II-B: matching cost c(p, d) */

/* Eq. (7)'s matching cost c, which the paper does not define: a 5x5 census transform (24 bits;
 * bit k, in raster order of the window without its centre, is set when that neighbour is darker
 * than the centre; neighbours outside the image are clamped to the edge).
 * img: uint8 rows of `pitch` bytes.  codes: uint32 [H][W]. */
pd_status pd_census(pd_ctx* ctx, const uint8_t* img, int W, int H, size_t pitch, uint32_t* codes);

/* c(p, d) = Hamming distance of the census codes of left(u, v) and right_warped(u - d, v), or 24
 * when u - d < 0.  Inputs are uint8 images (rows of `pitch` bytes); cost: uint8 [H][W][D],
 * 1 <= D <= 256. */
pd_status pd_cost(pd_ctx* ctx, const uint8_t* left, const uint8_t* right_warped, int W, int H,
                  size_t pitch, int D, uint8_t* cost);

/* ------------------------------------------------------ Sec. II-B: aggregation, Eq. (8) */

/* Eq. (8) along one direction r = (dx, dy), dx, dy in {-1, 0, 1}, not both 0:
 *   L(p, d) = c(p, d) + min(L(p-r, d), L(p-r, d-1) + P1, L(p-r, d+1) + P1, m + P2) - m,
 *   m = min_i L(p-r, i), and L = c where p - r is outside the image.
 * Subtracting m (the printed equation omits it) changes every d of a pixel by the same amount.
 * cost: uint8 [H][W][D]; L: uint8 [H][W][D].  D in {32, 64, 128, 256}; cost and L 16-byte
 * aligned. */
pd_status pd_aggregate_dir(pd_ctx* ctx, const uint8_t* cost, int W, int H, int D, int dx, int dy,
                           int P1, int P2, uint8_t* L);

/* S(p, d) = sum of L over 4 directions {(1,0), (-1,0), (0,1), (0,-1)} or those plus the four
 * diagonals.  cost: uint8 [H][W][D]; S: uint16 [H][W][D]. */
pd_status pd_aggregate(pd_ctx* ctx, const uint8_t* cost, int W, int H, int D, int paths, int P1,
                       int P2, uint16_t* S);

/* ------------------------------------------------- Sec. II-B: disparity, Eqs. (9) and (10) */

/* Eq. (9) winner-take-all d* = argmin_d S(p, d) (smallest d on ties); a parabola through
 * S(d*-1), S(d*), S(d*+1) for 0 < d* < D-1 (one IEEE float division); the right-view
 * disparity d_R(x) = argmin_{d : x+d < W} S(x+d, d); the pixel is valid when u >= D-1 (its
 * whole search range lies in the image), u - d* >= 0 and |d* - d_R(u - d*)| <= lr_tol.  Then Eq. (10): D1 = d_sub + kappa[v] for valid pixels with a
 * non-negative result, -1 otherwise.
 * S: uint16 [H][W][D]; kappa: int32 [H]; d_int: int16 [H][W] (d*); D1: float [H][W]. */
pd_status pd_disparity(pd_ctx* ctx, const uint16_t* S, int W, int H, int D, const int32_t* kappa,
                       int lr_tol, int16_t* d_int, float* D1);

/* The whole of Sec. II-A and II-B in one call (warp, census, cost, aggregation, disparity),
 * without materialising S: the same results as the staged calls above.
 * left, right: uint8 rows of `pitch` bytes; model, params: host pointers (params->D, paths, P1,
 * P2, lr_tol, delta_pt are used); kappa (may be NULL): int32 [H]; d_int: int16 [H][W];
 * D1: float [H][W]. */
pd_status pd_sgm(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                 size_t pitch, const pd_road_model* model, const pd_params* params,
                 int32_t* kappa, int16_t* d_int, float* D1);

/* ----------------------------------------------------- Sec. II-C: disparity transformation */

/* pd_transform with `iters` refits of the road model, each on the pixels within tau of the
 * previous fit (|D1 - f| <= tau, f in single precision as in Eq. (13)): potholes deeper than tau
 * stop pulling the fitted road towards them.  iters = 0 is pd_transform.  iters in 0..16. */
pd_status pd_transform_robust(pd_ctx* ctx, const float* D1, int W, int H, int order,
                              float delta_dt, int iters, float tau, pd_road_model* fitted,
                              float* D2);

/* Exact sums the road fit needs over the pixels with D1 >= 0, with q = rint(1024 D1) and doubled
 * centred coordinates u~ = 2u - (W-1), v~ = 2v - (H-1): count, sum u~^i v~^j (i + j <= 4),
 * sum q u~^i v~^j (i + j <= 2) and sum q^2, in that order (i outer, j inner), each a signed
 * 128-bit integer written as (low 64 bits, high 64 bits): sums is int64 [46] (device).
 * W, H <= 4096. */
pd_status pd_moments(pd_ctx* ctx, const float* D1, int W, int H, int64_t* sums);

/* Eqs. (11)-(13): fits the road model of the given order (roll by minimising Eq. (12): closed form
 * for order 1, 0.01-degree grid over +-15 degrees refined by golden-section search for order 2;
 * coefficients by Eq. (11)), then D2 = max(0, D1 - f + delta_dt) in single precision, with
 * delta_dt at invalid pixels.  The fit stays on the device (no host round trip).
 * fitted: one pd_road_model (device, 8-byte aligned, may be NULL; written whole, padding zero);
 * D2: float [H][W].  W, H <= 4096. */
pd_status pd_transform(pd_ctx* ctx, const float* D1, int W, int H, int order, float delta_dt,
                       pd_road_model* fitted, float* D2);

/* Allocation-free form of pd_transform, with no counterpart in the paper.  It is for callers
 * that may not allocate device memory: code running while a stream is captured into a CUDA graph
 * (allocation is not capturable), real-time loops that cannot afford cudaMalloc / cudaFree (the
 * latter synchronises the whole device), and processes whose device memory is owned by another
 * allocator.  It needs no pd_ctx and calls no cudaMalloc, cudaFree or other allocating routine:
 * its scratch is one fixed 512 KiB array in the library's device image, which every GPU that
 * loads the library holds until the process exits.
 *  - Same arguments and results as pd_transform, enqueued on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream) of the caller's current device.
 *  - Limits: W, H <= 4096 and W * H <= 4194304 (4 Mpixel); larger images return
 *    PD_ERR_INVALID_ARG without launching anything.  So do NULL D1/D2, an order other than 1 or 2
 *    and a non-finite delta_dt.  Launch failures return PD_ERR_CUDA.
 *  - The first call on a device looks up the array's device address on that device (the current
 *    one); make that first call before any stream capture.  After a device reset
 *    (cudaDeviceReset) the next call on that device looks the address up again, so make it
 *    outside a capture too.
 *  - All calls share the one array: calls that may overlap on the GPU (different streams, or
 *    different host threads on one device) race and must be serialised by the caller.  Each call
 *    overwrites what the previous one left there before reading it. */
pd_status pd_transform_noalloc(const float* D1, int W, int H, int order, float delta_dt,
                               pd_road_model* fitted, float* D2, void* stream);

/* ---------------------------------------------------------------- Sec. II-D: superpixels */

/* SLIC on D2: grid interval S = sqrt(W H / K), nx = round(W / S), ny = round(H / S) seeds moved
 * to the lowest-gradient pixel of their 3x3 neighbourhood; `iters` rounds of assignment (each
 * pixel to the nearest centre whose 2S x 2S window covers it, distance
 * (D2 - value)^2 + ((x - cx)^2 + (y - cy)^2) (m / S)^2, lower index on ties) and mean update.
 * Then D3 (Sec. II-E): every pixel gets the mean D2 of its superpixel.
 * labels: int32 [H][W]; D3: float [H][W]; centres (may be NULL): float [nx*ny][3].
 * Returns the centre count in *n_centres (host, may be NULL).
 * Centre means use exact integer sums of rint(1024 D2); they are exact for |D2| < 2^27 px. */
pd_status pd_superpixels(pd_ctx* ctx, const float* D2, int W, int H, int K, float m, int iters,
                         int32_t* labels, float* D3, float* centres, int* n_centres);

/* ---------------------------------------------------------- Sec. II-E: pothole detection */

/* Eqs. (14)-(17): the vectors g = [D2(p), sum of D2 over the 8 neighbours] of interior pixels
 * whose 3x3 window is valid in D1 are split at thresholds t = k/8 px (k = 1..255) along the
 * histogram diagonal; t_r minimises E2 (Eq. (17)); t_s = (mean D2 of the road cluster) - delta_pd
 * (mode 0) or t_r - delta_pd (mode 1); mask = D3 < t_s.
 * D2, D1, D3: float [H][W]; mask: uint8 [H][W]; thresholds (may be NULL): double [2] = t_r, t_s
 * (device); E2 (may be NULL): double [256] (device, NaN where a cluster is empty). */
pd_status pd_pothole_mask(pd_ctx* ctx, const float* D2, const float* D1, const float* D3, int W,
                          int H, float delta_pd, int mode, uint8_t* mask, double* thresholds,
                          double* E2);

/* --------------------------------------------------------------------------- profiling */

/* on != 0: later pd_sgm and pd_run_pipeline calls record CUDA events on the context's stream
 * around their stages (no synchronisation; at most 4096 calls are recorded between reads).
 * on == 2 records only the two events around the aggregation (aggregate_ms and total_ms are then
 * the aggregation's time): every event in the stream drains the GPU between two stages, so this
 * mode disturbs a timed run least.  on == 0 stops recording and discards what was recorded. */
pd_status pd_profile_enable(pd_ctx* ctx, int on);
/* Waits for the recorded events, writes the summed stage times to *out (host) and starts a new
 * recording. */
pd_status pd_profile_read(pd_ctx* ctx, pd_profile* out);

/* Measured integer peak for the roofline of Eq. (8) (a measurement aid; the paper has no
 * counterpart).  Runs a kernel of independent packed u16x2 DPX instructions (three-input minimum
 * and fused add-minimum, the instructions of the aggregation's recurrence) at 64 warps per SM,
 * `reps` rounds of 16 instructions per thread (reps in [1, 2^20]; 4096 takes about 1 ms), once
 * to warm up and once timed with CUDA events on the context's stream; synchronises the stream.
 * lane_ops_per_s (host, may be NULL): u16 lane-operations per second (2 per thread instruction);
 * instr_per_clk_sm (host, may be NULL): thread instructions per SM clock, averaged over the SMs
 * from each SM's own clock counter, so independent of the clock it ran at.  Uses the context's
 * scratch. */
pd_status pd_int_rate(pd_ctx* ctx, int reps, double* lane_ops_per_s, double* instr_per_clk_sm);

/* ------------------------------------------------- batched form (an extension of the paper) */

/* One stereo pair of a batch (host struct; the pointers are device pointers). */
typedef struct {
  const uint8_t* left;
  const uint8_t* right;
  int W, H;
  size_t pitch;
  int D;                /* 32, 64, 128 or 256, chosen per pair */
  int pad;
  pd_road_model model;  /* the pair's road model for the warp, by value */
  int32_t* kappa;       /* [H] row shifts, may be NULL */
  int16_t* d_int;       /* [H][W] */
  float* D1;            /* [H][W] */
} pd_pair;

/* Options of pd_sgm_batch on this context:
 *  - scratch_budget_bytes: device scratch the batch may use; pairs are processed in consecutive
 *    waves that fit it (0 keeps the default, 32 GiB).  A pair larger than the budget runs alone.
 *  - use_graph != 0: the launch sequence of a batch is captured into a CUDA graph the first time a
 *    batch of the same shape (sizes, D, parameters) is run on a non-default stream and replayed on
 *    later calls with any buffers.
 *  - autotune != 0 (default): on the first batch of a shape, the persistent aggregation kernel is
 *    timed with 2, 4 and 8 warps per block and the fastest is kept for that shape.  Every choice
 *    gives identical results. */
pd_status pd_batch_config(pd_ctx* ctx, size_t scratch_budget_bytes, int use_graph, int autotune);

/* Sec. II-A and II-B for n pairs of any sizes and disparity ranges with one launch per stage and
 * wave (Eq. (9): one launch per pair); the aggregation is one persistent launch whose warps take
 * line groups from a shared counter over a task list ordered pair by pair, the largest pair
 * first.  Results are identical to n pd_sgm calls.
 * pairs: host array of n descriptors; params: host (paths, P1, P2, lr_tol, delta_pt are used; D
 * is per pair).  The call returns after enqueueing; it waits for the previous batch on this
 * context to pass its table upload before reusing the host staging buffer. */
pd_status pd_sgm_batch(pd_ctx* ctx, const pd_pair* pairs, int n, const pd_params* params);

/* ------------------------------------------- Sec. II-E: connected components of the mask */


/* Sec. II-E "different potholes are labeled using connect component labeling", and Sec. III-B's
 * rule that detections at a corner of the image or made of one superpixel are fake.  Components
 * of the mask pixels (mask != 0) with 8- or 4-connectivity, numbered 0, 1, ... in the raster
 * order of their first pixel.  labels: int32 [H][W], the component number or -1; comps: up to
 * max_comps records (device); n_comps: one int (device), the number of components (possibly
 * more than max_comps, whose records are then not written), or -1 if the union-find exceeded its
 * iteration limit.  mask: uint8 [H][W]; sp_labels: int32 [H][W] superpixel labels (as written
 * by pd_superpixels). */
pd_status pd_components(pd_ctx* ctx, const uint8_t* mask, const int32_t* sp_labels, int W, int H,
                        int connectivity, int32_t* labels, pd_component* comps, int max_comps,
                        int* n_comps);

/* ------------------------------------------------ Sec. III: accuracy against a ground truth */

/* Sec. III-A: over the q pixels with D1 >= 0 and a finite ground-truth disparity D4, the
 * percentage of error pixels e_p = 100 #{|D1 - D4| > eps_k} / q for the three tolerances eps
 * (host float [3]) and the RMSE e_r = sqrt(sum (D1 - D4)^2 / q); Sec. III-B: pixel precision,
 * recall, accuracy and F-score of the pothole mask against a ground-truth mask (non-zero =
 * pothole).  out (device, double [13]): q, e_p1, e_p2, e_p3, e_r, tp, fp, fn, tn, precision,
 * recall, accuracy, F-score (NaN where a denominator is 0).  Counts are exact; the squared-error
 * sum is accumulated in double precision in no fixed order. */
pd_status pd_accuracy(pd_ctx* ctx, const float* D1, const float* D4, const uint8_t* mask,
                      const uint8_t* gt_mask, int W, int H, const float* eps, double* out);

/* -------------------------------------- learned disparity band (an extension of the paper) */

/* Sec. II-A and II-B with the disparity search of each 16x16 tile restricted to a window:
 * tile (tx, ty) = (u / 16, v / 16) searches [lo, min(lo + band_width, D)) with
 * lo = min(tile_lo[ty][tx], D - 1), or the full range [0, D) where tile_lo[ty][tx] < 0.  Eq. (8)
 * runs over the windows with L = infinity outside them (its minima use only the previous pixel's
 * window); d* is the argmin over the window (smallest d on ties); the parabola needs d* - 1 and
 * d* + 1 inside the window; the right view of column x takes the candidates d inside the window
 * of pixel x + d; a pixel is valid when u >= hi - 1, u - d* >= 0 and |d* - d_R(u - d*)| <=
 * lr_tol.  With every tile_lo negative the results equal pd_sgm's.
 * tile_lo: int16 [ceil(H/16)][ceil(W/16)] (device); band_width in 1..D; other arguments as in
 * pd_sgm (D in {32, 64, 128, 256}). */
pd_status pd_sgm_band(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                      size_t pitch, const pd_road_model* model, const pd_params* params,
                      const int16_t* tile_lo, int band_width, int32_t* kappa, int16_t* d_int,
                      float* D1);

/* The band network: per 16x16 tile of the row-shifted pair, a disparity centre and a confidence
 * (an extension beyond the paper; it restates no passage of it).  Input x: bf16 [B][Hd][Wd][2],
 * Hd = ceil(H/4), Wd = ceil(W/4), as written by pd_band_input.  Four 3x3 convolutions with zero
 * padding 1, strides 1, 2, 2, 1 and channels 2 -> 32 -> 32 -> 32 -> 2, ReLU after the first three;
 * bf16 operands, fp32 accumulation, bf16 activations (each forward convolution an implicit GEMM on
 * the tensor cores with the accumulator in tensor memory).  Output out: float [B][Ho][Wo][2] with
 * Ho = ceil(Hd/4) = ceil(H/16) (likewise Wo): channel 0 = centre / 16 (pixels of the shifted
 * pair), channel 1 = logit of the confidence that the tile's disparities lie within +-7 of it.
 * Parameters: 19682 floats, per layer the weights [Cout][3][3][Cin] then the Cout biases. */
typedef struct pd_cnn pd_cnn;

/* Allocates a network (zero parameters) whose calls accept up to max_batch images of at most
 * max_hd x max_wd input cells on `device`.  PD_ERR_OOM if the buffers do not fit. */
pd_status pd_cnn_create(pd_cnn** net, int device, int max_batch, int max_hd, int max_wd);
pd_status pd_cnn_destroy(pd_cnn* net);
int pd_cnn_num_params(void);

/* Copies n = pd_cnn_num_params() parameters from / to host memory (synchronous on ctx's stream);
 * set_params also clears the Adam state and its step count. */
pd_status pd_cnn_set_params(pd_ctx* ctx, pd_cnn* net, const float* host_params, int n);
pd_status pd_cnn_get_params(pd_ctx* ctx, pd_cnn* net, float* host_params, int n);

/* Forward pass; x and out are device pointers (layouts above). */
pd_status pd_cnn_forward(pd_ctx* ctx, pd_cnn* net, const void* x, int B, int Hd, int Wd,
                         float* out);

/* The convolutions run on the fifth-generation tensor cores: one thread per CTA issues the MMAs
 * into tensor memory and every thread waits for their completion on an mbarrier, for about a
 * second at most.  A wait that runs out sets a flag in the network instead of hanging the device.
 * pd_cnn_check synchronises ctx's stream and returns PD_ERR_TIMEOUT (and clears the flag) if any
 * call since the last check saw a wait run out, else PD_OK.  pd_cnn_probe_timeout enqueues one
 * convolution CTA that issues no MMA, so that its wait runs out after limit_cycles SM clock cycles
 * (0 .. 2^31): the timeout path itself, for tests. */
pd_status pd_cnn_check(pd_ctx* ctx, pd_cnn* net);
pd_status pd_cnn_probe_timeout(pd_ctx* ctx, pd_cnn* net, long long limit_cycles);

/* Loss and its gradient with respect to the parameters.  targets: float [B][Ho][Wo][4] = (centre
 * in pixels, confidence label 0/1, centre weight, confidence weight).  Loss = sum of centre
 * weight * Huber_1(out0 - centre / 16) / max(1, total centre weight) + sum of confidence weight *
 * logistic loss(out1, label) / max(1, total confidence weight).  loss: one float, grad: float
 * [19682], both device. */
pd_status pd_cnn_loss_grad(pd_ctx* ctx, pd_cnn* net, const void* x, const float* targets, int B,
                           int Hd, int Wd, float* loss, float* grad);

/* pd_cnn_loss_grad followed by one Adam step (beta 0.9 / 0.999, eps 1e-8) of size lr on the fp32
 * master parameters.  loss (device, may be NULL) receives the loss before the step. */
pd_status pd_cnn_train_step(pd_ctx* ctx, pd_cnn* net, const void* x, const float* targets, int B,
                            int Hd, int Wd, float lr, float* loss);

/* Training checkpoints of the band network (a file format of this library; the paper trains no
 * network).  Layout, all little-endian: the magic "PDCNNCK" and a NUL byte, u32 format version
 * (1), u32 parameter count n, u64 Adam step count, u64 caller-state byte count r, f32[n] master
 * parameters, f32[n] Adam first moments, f32[n] Adam second moments, the r caller-state bytes,
 * and a u32 CRC-32 (IEEE 802.3 / zlib) of every byte before it.  The caller state is opaque to
 * the library (for instance the state of the training loop's random generator), r <= 1 MiB.
 * Training is bit-reproducible (the gradient sums run in a fixed order), so training N steps,
 * saving, loading into a fresh network and training M more gives the bits of N + M steps.
 *  - pd_cnn_save downloads the state (synchronising ctx's stream) and writes `path` through a
 *    temporary file "<path>.tmp" renamed over it.  PD_ERR_INVALID_ARG if it cannot be written.
 *  - pd_cnn_load checks the file (magic, version, n equal to pd_cnn_num_params(), size, CRC)
 *    before touching the network; a failed check returns PD_ERR_INVALID_ARG and leaves it
 *    unchanged.  Then it restores parameters, moments and step, refreshes the bf16 weights and
 *    synchronises ctx's stream.  state (may be NULL) receives min(state_cap, r) caller-state bytes,
 *    *state_bytes (may be NULL) is set to r.
 *  - pd_cnn_checkpoint_info runs the same checks on the host alone (no device or context) and
 *    reports n, the step and r; PD_ERR_INVALID_ARG for a missing or damaged file. */
pd_status pd_cnn_save(pd_ctx* ctx, pd_cnn* net, const char* path, const void* state,
                      size_t state_bytes);
pd_status pd_cnn_load(pd_ctx* ctx, pd_cnn* net, const char* path, void* state, size_t state_cap,
                      size_t* state_bytes);
pd_status pd_cnn_checkpoint_info(const char* path, int* n_params, long long* step,
                                 size_t* state_bytes);

/* The network input of one pair: the right image shifted row by row as in Sec. II-A
 * (right(clamp(u - kappa(v)))), both images summed over 4x4 blocks (edge rows and columns
 * repeated), mapped to (sum - 2048) / 1024 and rounded to bf16.  x: bf16 [Hd][Wd][2] (device). */
pd_status pd_band_input(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                        size_t pitch, const int32_t* kappa, void* x);

/* Training targets from a full-range result: per 16x16 tile, with n valid pixels (D1 >= 0), the
 * lower median c of their d*, confidence label 1 iff n >= 64 and at least 99.5 % lie in
 * [c - 7, c + 7], centre weight 1 iff n >= 64, confidence weight 1.  targets: float
 * [ceil(H/16)][ceil(W/16)][4] (device). */
pd_status pd_band_labels(pd_ctx* ctx, const int16_t* d_int, const float* D1, int W, int H, int D,
                         float* targets);

/* Windows from the network output: tiles with out1 >= ln 9 (confidence >= 0.9) start at
 * rint(16 out0) - band_width / 2 moved into [0, D - band_width]; the others get -1 (full range),
 * except that an unconfident tile of the left border columns tx < t0 = ceil((D - 1) / 16), where
 * the full-range search has no valid pixel, takes the window of tile (ty, t0).
 * cnn_out: float [tiles_h][tiles_w][2]; tile_lo: int16 [tiles_h][tiles_w] (device). */
pd_status pd_band_tiles(pd_ctx* ctx, const float* cnn_out, int tiles_h, int tiles_w, int D,
                        int band_width, int16_t* tile_lo);

/* The learned band path of one pair: row shifts, pd_band_input, the network, pd_band_tiles and
 * pd_sgm_band.  tile_lo (device, may be NULL) receives the windows used; the network must accept
 * one image of ceil(H/4) x ceil(W/4). */
pd_status pd_sgm_learned(pd_ctx* ctx, pd_cnn* net, const uint8_t* left, const uint8_t* right,
                         int W, int H, size_t pitch, const pd_road_model* model,
                         const pd_params* params, int band_width, int16_t* tile_lo,
                         int32_t* kappa, int16_t* d_int, float* D1);

/* -------------------------------------------------------------------------- whole path */

/* pd_sgm, pd_transform, pd_superpixels, pd_pothole_mask and (when out->components is set)
 * pd_components in sequence on one stream.  times (host, may be NULL) receives per-stage device
 * times (this synchronises the stream); mask_ms covers the threshold, the mask and the
 * components. */
pd_status pd_run_pipeline(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                          size_t pitch, const pd_road_model* model, const pd_params* params,
                          const pd_outputs* out, pd_stage_times* times);

/* Closed-loop form of pd_run_pipeline (Sec. II-A's perspective transformation driven by the road
 * model fitted in Sec. II-C on the previous frame): the same steps, with the model for the row
 * shifts read from device memory, so a stream of frames runs with no host round trip.  model_dev
 * may be out->fitted itself (the fit of this frame then replaces it once the shifts are taken).
 * A device model with an order other than 1 or 2 or a non-finite value gives zero shifts. */
pd_status pd_run_pipeline_dev(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W,
                              int H, size_t pitch, const pd_road_model* model_dev,
                              const pd_params* params, const pd_outputs* out,
                              pd_stage_times* times);

/* CUDA-graph replay of the whole path (pd_run_pipeline and pd_run_pipeline_dev).
 *  - use_graph != 0: a call without stage times (times == NULL) captures its enqueued sequence
 *    once into a CUDA graph (on a private capture stream) and replays it on the context's stream
 *    while the inputs, outputs, parameters, road model (its value for pd_run_pipeline, its
 *    address for pd_run_pipeline_dev), scratch and profiling state are those of the capture;
 *    any change captures again.  Results are identical to direct enqueueing.  Profiled calls keep
 *    their per-stage times: the graph's stage marks are retargeted to each call's events.
 *  - use_graph == 0 (default): every call enqueues its kernels directly; a held graph is freed.
 * Returns PD_OK, or PD_ERR_INVALID_ARG for a NULL context. */
pd_status pd_pipeline_config(pd_ctx* ctx, int use_graph);

#ifdef __cplusplus
}
#endif
#endif
