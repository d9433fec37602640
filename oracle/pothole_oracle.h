/*
 * Reference oracle for the stereo pothole-detection path of Fan, Ozgunalp, Wang, Liu, Pitas,
 * "Rethinking Road Surface 3D Reconstruction and Pothole Detection: From Perspective Transformation
 * to Disparity Map Segmentation" (arXiv 2012.10802).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded CPU restatement of the paper's
 * steps, used to check the CUDA library.  It shares no code with the CUDA path.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it; the product path
 * never calls it and has no CPU fallback.
 *
 * Conventions (shared by every function below):
 *   images are row-major, u = column 0..W-1, v = row 0..H-1 (v points down), no row padding;
 *   volumes are [H][W][D] with the disparity innermost;
 *   a disparity map value < 0 marks an invalid pixel.
 *
 * Parity status: every function here is pinned by tests under tests/ (brute force, closed forms,
 * invariants or textbook special cases); none is "parity unpinned".
 */
#ifndef POTHOLE_ORACLE_H
#define POTHOLE_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Road disparity model, Sec. II-A Eq. (3) with the roll applied about the image centre:
 *   v' = (v - vc) cos(roll) - (u - uc) sin(roll) + vc,  uc = (W-1)/2, vc = (H-1)/2,
 *   f  = a0 + a1 v' + a2 v'^2          (a2 used only when order == 2). */
typedef struct {
  int order;
  double a[3];
  double roll;
} or_road_model;

/* Exact moment sums for the road fit (Sec. II-C, Eqs. (11)-(12)); see or_moments(). */
typedef struct {
  int64_t count;
  __int128 m[5][5];  /* m[i][j] = sum u~^i v~^j, i + j <= 4 */
  __int128 q[3][3];  /* q[i][j] = sum q u~^i v~^j, i + j <= 2 */
  __int128 qq;       /* sum q^2 */
} or_moment_sums;

/* Sec. II-A, Eq. (6): kappa(v) = floor(min_{x=0..W-1} f(a,(x,v),phi) - delta_pt). */
void or_kappa(const or_road_model* model, int W, int H, double delta_pt, int32_t* kappa);
double or_road_f(const or_road_model* model, int W, int H, double u, double v);

/* Sec. II-A: the row-shifted right image right'(u,v) = right(clamp(u - kappa(v)), v). */
void or_warp(const uint8_t* right, int W, int H, const int32_t* kappa, uint8_t* warped);

/* Matching cost c of Eq. (7): 5x5 census (24 bits) and Hamming distance. */
void or_census(const uint8_t* img, int W, int H, uint32_t* codes);
void or_cost(const uint32_t* census_left, const uint32_t* census_right, int W, int H, int D,
             uint8_t* cost);

/* Eq. (8) along one direction (dx, dy), normalised by the previous pixel's minimum. */
void or_aggregate_dir(const uint8_t* cost, int W, int H, int D, int dx, int dy, int P1, int P2,
                      uint8_t* L);
/* Eq. (8) exactly as printed (no normalisation), in 64-bit integers. */
void or_aggregate_dir_raw(const uint8_t* cost, int W, int H, int D, int dx, int dy, int P1, int P2,
                          int64_t* L);
/* Sum of Eq. (8) over 4 or 8 directions. */
void or_aggregate(const uint8_t* cost, int W, int H, int D, int paths, int P1, int P2, uint16_t* S);

/* Eq. (9) winner-take-all, sub-pixel parabola, left-right check and Eq. (10) D1 = D0 + kappa. */
void or_disparity(const uint16_t* S, int W, int H, int D, const int32_t* kappa, int lr_tol,
                  int16_t* d_int, float* D1);

/* Sec. II-C: exact sums of the moments that Eqs. (11)-(12) need, over pixels with D1 >= 0. */
void or_moments(const float* D1, int W, int H, or_moment_sums* out);
/* Eq. (12) E0min(phi) for a model order, with the Eq. (11) coefficients returned in beta
 * (model in the scaled rotated coordinate w_s, see the .c file). */
double or_e0min(const or_moment_sums* mom, int order, int W, int H, double phi, double beta[3]);
/* Roll and model fit: order 1 closed form, order 2 grid + golden-section search. */
void or_fit_road(const or_moment_sums* mom, int order, int W, int H, or_road_model* fitted);

/* Eq. (13): D2 = D1 - f + delta_dt, clamped at 0; invalid pixels get delta_dt. */
void or_transform(const float* D1, int W, int H, const or_road_model* fitted, float delta_dt,
                  float* D2);

/* Sec. II-D SLIC.  Returns the number of centres (nx * ny) and fills labels [H][W]. */
int or_slic_grid(int W, int H, int K, int* nx, int* ny);
int or_slic(const float* D2, int W, int H, int K, float m, int iters, int32_t* labels,
            float* centres /* [n][3]: x, y, value, may be NULL */);
/* Sec. II-E: D3 = mean of D2 over each superpixel. */
void or_superpixel_mean(const float* D2, const int32_t* labels, int W, int H, int nlabels,
                        float* D3);

/* Sec. II-E, Eqs. (14)-(17): the adaptive threshold.  E2 (length 256, index k = threshold k/8 px)
 * gets NaN where a region is empty.  mode 0: t_s = (road-region mean of D2) - delta_pd,
 * mode 1: t_s = t_r - delta_pd.  Returns 0, or -1 if no threshold splits the pixels. */
int or_threshold(const float* D2, const float* D1, int W, int H, float delta_pd, int mode,
                 double* t_r, double* t_s, double* E2);
/* Sec. II-E: pothole mask = D3 < t_s. */
void or_mask(const float* D3, int W, int H, double t_s, uint8_t* mask);

/* Learned-band SGM (an extension beyond the paper): per-tile windows, aggregation restricted to
 * the windows (S = 0xFFFF outside), and the disparity step over the windows. */
void or_band_windows(const int16_t* tile_lo, int W, int H, int D, int band, int16_t* lo,
                     int16_t* hi);
void or_aggregate_band(const uint8_t* cost, const int16_t* lo, const int16_t* hi, int W, int H,
                       int D, int paths, int P1, int P2, uint16_t* S);
void or_disparity_band(const uint16_t* S, const int16_t* lo, const int16_t* hi, int W, int H, int D,
                       const int32_t* kappa, int lr_tol, int16_t* d_int, float* D1);

/* Sec. II-E connected components of the mask (readings R14, R15): labels = smallest raster index
 * of the component or -1; returns the component count.  or_components writes 12 int64 per
 * component (label, count, u/v min, u/v max, sum u, sum v, superpixels, corner, single, fake). */
int or_ccl(const uint8_t* mask, int W, int H, int conn, int32_t* labels);
void or_components(const int32_t* labels, const int32_t* sp, int W, int H, int ncomp,
                   int64_t* out);

/* Robust road fit (reading R17): moments over the inliers of a previous fit, and the fit
 * iterated on them. */
void or_moments_inliers(const float* D1, int W, int H, const or_road_model* fit, float tau,
                        or_moment_sums* out);
void or_fit_road_robust(const float* D1, int W, int H, int order, int iters, float tau,
                        or_road_model* fitted);

/* Test-harness helpers: the size of or_moment_sums, and its 23 sums as (low, high) 64-bit pairs. */
size_t or_moment_sums_size(void);
void or_moments_export(const or_moment_sums* mom, int64_t* out);

#ifdef __cplusplus
}
#endif
#endif
