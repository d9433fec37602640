/*
 * Reference oracle for arXiv 2012.10802 (stereo road pothole detection).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded restatement of the paper's steps in
 * the paper's order, used by the test suite, the smoke check and the benchmark's CPU-baseline leg.
 * It shares no code with the CUDA library and the CUDA library never calls it.
 *
 * Build with -ffp-contract=off: every floating-point expression below is evaluated exactly as
 * written (no fused multiply-add), which the parity tests rely on.
 *
 * Where the paper is silent or ambiguous this file follows one fixed reading; each is named at the
 * function that uses it:
 *   R1 roll about the image centre (Sec. II-A "rotated by phi around the image center");
 *   R2 integer row shift kappa = floor(min f - delta_pt) and right'(u) = right(clamp(u - kappa));
 *   R3 matching cost = 5x5 census + Hamming distance (Eq. (7) names c but does not define it);
 *   R4 Eq. (8) normalised by the previous pixel's minimum (argmin-preserving);
 *   R5 parabola sub-pixel step, a 1-px left-right check, invalid left border band u < D-1;
 *   R6 road pixels = all left-right-consistent pixels, fixed-point moments;
 *   R7 roll: closed form for the linear model, grid + golden section for the quadratic one;
 *   R8 SLIC grid/tie rules, fixed iteration count;
 *   R9 threshold regions on the diagonal with exact (fixed-point) g; t_s from the road mean;
 *   R14 connected components of the mask: 8- or 4-connectivity, labelled by their smallest
 *       raster index (Sec. II-E names CCL only);
 *   R15 fake potholes (Sec. III-B): centroid in a corner cell of an 8 x 8 split, or one superpixel;
 *   R17 robust road fit (beyond Sec. II-C): refits on the inliers |D1 - f| <= tau of the previous fit;
 *   R10 (band SGM, beyond the paper) per-16x16-tile windows [lo, lo + band) clipped to [0, D),
 *       L = +infinity outside the window, minima of Eq. (8) over the previous pixel's window,
 *       winners and right views over in-window candidates, valid pixels need u >= hi - 1.
 */
#include "pothole_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define CENSUS_BITS 24

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* ---------------------------------------------------------------- Sec. II-A, Eqs. (3) and (6) */

/* Eq. (3) with reading R1: the inverse roll rotates pixel coordinates about the image centre. */
double or_road_f(const or_road_model* model, int W, int H, double u, double v) {
  double uc = (double)(W - 1) * 0.5;
  double vc = (double)(H - 1) * 0.5;
  double c = cos(model->roll);
  double s = sin(model->roll);
  double t1 = (v - vc) * c;
  double t2 = (u - uc) * s;
  double vp = (t1 - t2) + vc;
  double f = model->a[0] + model->a[1] * vp;
  if (model->order == 2) f = f + model->a[2] * (vp * vp);
  return f;
}

/* Eq. (6): kappa is the minimum over x = 0..W-1 of f - delta_pt; reading R2 takes its floor. */
void or_kappa(const or_road_model* model, int W, int H, double delta_pt, int32_t* kappa) {
  for (int v = 0; v < H; ++v) {
    double best = 0.0;
    for (int x = 0; x < W; ++x) {
      double f = or_road_f(model, W, H, (double)x, (double)v) - delta_pt;
      if (x == 0 || f < best) best = f;
    }
    kappa[v] = (int32_t)floor(best);
  }
}

/* Sec. II-A: each row v of the right image is shifted by kappa(v) (reading R2 for the direction,
 * chosen so that D1 = D0 + kappa of Eq. (10) holds; columns are clamped to the image). */
void or_warp(const uint8_t* right, int W, int H, const int32_t* kappa, uint8_t* warped) {
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u)
      warped[(size_t)v * W + u] = right[(size_t)v * W + clampi(u - kappa[v], 0, W - 1)];
}

/* ------------------------------------------------------------- Sec. II-B, Eq. (7) cost c(p,d) */

/* Reading R3: bit k (k = 0..23, raster order of the 5x5 window without its centre) is set when
 * that neighbour is darker than the centre; neighbours outside the image are clamped. */
void or_census(const uint8_t* img, int W, int H, uint32_t* codes) {
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      uint8_t centre = img[(size_t)v * W + u];
      uint32_t code = 0;
      int k = 0;
      for (int dy = -2; dy <= 2; ++dy) {
        for (int dx = -2; dx <= 2; ++dx) {
          if (dx == 0 && dy == 0) continue;
          int x = clampi(u + dx, 0, W - 1);
          int y = clampi(v + dy, 0, H - 1);
          if (img[(size_t)y * W + x] < centre) code |= 1u << k;
          ++k;
        }
      }
      codes[(size_t)v * W + u] = code;
    }
  }
}

static int popcount32(uint32_t x) {
  int n = 0;
  while (x) {
    n += (int)(x & 1u);
    x >>= 1;
  }
  return n;
}

/* c(p,d) = Hamming distance between the left code at (u,v) and the warped right code at (u-d,v);
 * a candidate that falls off the left edge costs the maximum, 24. */
void or_cost(const uint32_t* census_left, const uint32_t* census_right, int W, int H, int D,
             uint8_t* cost) {
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u)
      for (int d = 0; d < D; ++d) {
        uint8_t c = CENSUS_BITS;
        if (u - d >= 0)
          c = (uint8_t)popcount32(census_left[(size_t)v * W + u] ^
                                  census_right[(size_t)v * W + (u - d)]);
        cost[((size_t)v * W + u) * D + d] = c;
      }
}

/* ------------------------------------------------------------------ Sec. II-B, Eq. (8) */

/* Visit order so that p - r is always visited before p. */
static void path_order(int n, int step, int* start, int* inc) {
  *start = step >= 0 ? 0 : n - 1;
  *inc = step >= 0 ? 1 : -1;
}

/* Eq. (8) along r = (dx, dy).  Reading R4: the term min_i c_agg(p - r, i) is subtracted after the
 * update so values stay below Cmax + P2; this shifts every d of a pixel by the same amount and so
 * leaves Eq. (9)'s argmin unchanged.  A pixel whose predecessor p - r lies outside the image
 * starts the path: c_agg = c. */
void or_aggregate_dir(const uint8_t* cost, int W, int H, int D, int dx, int dy, int P1, int P2,
                      uint8_t* L) {
  int v0, vi, u0, ui;
  path_order(H, dy, &v0, &vi);
  path_order(W, dx, &u0, &ui);
  for (int iv = 0, v = v0; iv < H; ++iv, v += vi) {
    for (int iu = 0, u = u0; iu < W; ++iu, u += ui) {
      const uint8_t* c = cost + ((size_t)v * W + u) * D;
      uint8_t* out = L + ((size_t)v * W + u) * D;
      int pu = u - dx, pv = v - dy;
      if (pu < 0 || pu >= W || pv < 0 || pv >= H) {
        memcpy(out, c, (size_t)D);
        continue;
      }
      const uint8_t* prev = L + ((size_t)pv * W + pu) * D;
      int m = prev[0];
      for (int d = 1; d < D; ++d)
        if (prev[d] < m) m = prev[d];
      for (int d = 0; d < D; ++d) {
        int best = prev[d];
        if (d > 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
        if (d < D - 1 && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
        if (m + P2 < best) best = m + P2;
        out[d] = (uint8_t)(c[d] + best - m);
      }
    }
  }
}

/* Eq. (8) exactly as printed: no normalisation, 64-bit values. */
void or_aggregate_dir_raw(const uint8_t* cost, int W, int H, int D, int dx, int dy, int P1, int P2,
                          int64_t* L) {
  int v0, vi, u0, ui;
  path_order(H, dy, &v0, &vi);
  path_order(W, dx, &u0, &ui);
  for (int iv = 0, v = v0; iv < H; ++iv, v += vi) {
    for (int iu = 0, u = u0; iu < W; ++iu, u += ui) {
      const uint8_t* c = cost + ((size_t)v * W + u) * D;
      int64_t* out = L + ((size_t)v * W + u) * D;
      int pu = u - dx, pv = v - dy;
      if (pu < 0 || pu >= W || pv < 0 || pv >= H) {
        for (int d = 0; d < D; ++d) out[d] = c[d];
        continue;
      }
      const int64_t* prev = L + ((size_t)pv * W + pu) * D;
      int64_t m = prev[0];
      for (int d = 1; d < D; ++d)
        if (prev[d] < m) m = prev[d];
      for (int d = 0; d < D; ++d) {
        int64_t best = prev[d];
        if (d > 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
        if (d < D - 1 && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
        if (m + P2 < best) best = m + P2;
        out[d] = c[d] + best;
      }
    }
  }
}

/* The paper aggregates "along all directions"; 4 paths = the axis directions, 8 adds diagonals. */
static const int kDirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};

void or_aggregate(const uint8_t* cost, int W, int H, int D, int paths, int P1, int P2, uint16_t* S) {
  size_t n = (size_t)W * H * D;
  uint8_t* L = (uint8_t*)malloc(n);
  memset(S, 0, n * sizeof(uint16_t));
  for (int r = 0; r < paths; ++r) {
    or_aggregate_dir(cost, W, H, D, kDirs[r][0], kDirs[r][1], P1, P2, L);
    for (size_t i = 0; i < n; ++i) S[i] = (uint16_t)(S[i] + L[i]);
  }
  free(L);
}

/* ---------------------------------------------------------- Sec. II-B, Eqs. (9)-(10) */

/* Eq. (9) (the printed "min" is an argmin; the smallest d wins ties), reading R5 for the sub-pixel
 * parabola and the left-right check, then Eq. (10): D1 = D0 + kappa.  Invalid pixels get -1.
 * Reading R5 also marks invalid the left border band u < D-1, where the search range d < D runs
 * past the image edge and left pixels without a true match agree with a wrong right view. */
void or_disparity(const uint16_t* S, int W, int H, int D, const int32_t* kappa, int lr_tol,
                  int16_t* d_int, float* D1) {
  int* dright = (int*)malloc(sizeof(int) * (size_t)W);
  int* dleft = (int*)malloc(sizeof(int) * (size_t)W);
  for (int v = 0; v < H; ++v) {
    const uint16_t* row = S + (size_t)v * W * D;
    for (int u = 0; u < W; ++u) {
      const uint16_t* s = row + (size_t)u * D;
      int best = 0;
      for (int d = 1; d < D; ++d)
        if (s[d] < s[best]) best = d;
      dleft[u] = best;
    }
    /* right view: the best d for right-image column x pairs it with left column x + d */
    for (int x = 0; x < W; ++x) {
      int best = 0;
      unsigned bestv = row[(size_t)x * D + 0];
      for (int d = 1; d < D && x + d < W; ++d) {
        unsigned val = row[(size_t)(x + d) * D + d];
        if (val < bestv) {
          bestv = val;
          best = d;
        }
      }
      dright[x] = best;
    }
    for (int u = 0; u < W; ++u) {
      const uint16_t* s = row + (size_t)u * D;
      int ds = dleft[u];
      float dsub = (float)ds;
      if (ds > 0 && ds < D - 1) {
        int num = (int)s[ds - 1] - (int)s[ds + 1];
        int den = 2 * ((int)s[ds - 1] + (int)s[ds + 1] - 2 * (int)s[ds]);
        if (den > 0) dsub = (float)ds + (float)num / (float)den;
      }
      d_int[(size_t)v * W + u] = (int16_t)ds;
      int xr = u - ds;
      int valid = u >= D - 1 && xr >= 0 && abs(ds - dright[xr]) <= lr_tol;
      float d1 = dsub + (float)kappa[v];
      D1[(size_t)v * W + u] = (valid && d1 >= 0.0f) ? d1 : -1.0f;
    }
  }
  free(dright);
  free(dleft);
}

/* --------------------------------------------------------- Sec. II-C, Eqs. (11)-(12) */

/* Reading R6: the road disparities d of Eqs. (11)-(12) are every pixel with D1 >= 0.  Each value
 * is held as q = rint(1024 D1) and each pixel position as doubled centred integers
 * u~ = 2u - (W-1), v~ = 2v - (H-1), so that all sums are exact integers. */
void or_moments(const float* D1, int W, int H, or_moment_sums* out) {
  memset(out, 0, sizeof(*out));
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      float d = D1[(size_t)v * W + u];
      if (!(d >= 0.0f)) continue;
      __int128 q = (__int128)(int64_t)rint((double)d * 1024.0);
      __int128 ut = 2 * u - (W - 1), vt = 2 * v - (H - 1);
      __int128 up[5], vp[5];
      up[0] = 1;
      vp[0] = 1;
      for (int i = 1; i < 5; ++i) {
        up[i] = up[i - 1] * ut;
        vp[i] = vp[i - 1] * vt;
      }
      out->count += 1;
      for (int i = 0; i <= 4; ++i)
        for (int j = 0; i + j <= 4; ++j) out->m[i][j] += up[i] * vp[j];
      for (int i = 0; i <= 2; ++i)
        for (int j = 0; i + j <= 2; ++j) out->q[i][j] += q * up[i] * vp[j];
      out->qq += q * q;
    }
  }
}

/* Scale for the rotated coordinate: the smallest power of two >= max(W, H). */
static double coord_scale(int W, int H) {
  int m = W > H ? W : H;
  double s = 1.0;
  while (s < (double)m) s *= 2.0;
  return s;
}

static const double kBinom[5][5] = {
    {1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};

/* Solve the symmetric positive-definite system A x = b (n <= 3) by Cholesky factorisation. */
static int spd_solve(int n, const double A[3][3], const double b[3], double x[3]) {
  double Lm[3][3] = {{0}};
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= Lm[i][k] * Lm[j][k];
      if (i == j) {
        if (!(s > 0.0)) return -1;
        Lm[i][i] = sqrt(s);
      } else {
        Lm[i][j] = s / Lm[j][j];
      }
    }
  }
  double y[3];
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= Lm[i][k] * y[k];
    y[i] = s / Lm[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= Lm[k][i] * x[k];
    x[i] = s / Lm[i][i];
  }
  return 0;
}

/* Eq. (12) at one phi.  With w = v~ cos(phi) - u~ sin(phi) = 2 (v' - vc) and w_s = w / scale, the
 * columns of T(phi) (Eq. (5), extended by w_s^2 for the quadratic model) are 1, w_s, w_s^2, so
 * T'T and T'd follow from the moment sums by the binomial expansion of w_s^k.  beta receives the
 * Eq. (11) solution in that basis. */
double or_e0min(const or_moment_sums* mom, int order, int W, int H, double phi, double beta[3]) {
  int n = order + 1;
  double sc = coord_scale(W, H);
  double cs = cos(phi) / sc;
  double ss = -sin(phi) / sc;
  double pc[5], ps[5];
  pc[0] = 1.0;
  ps[0] = 1.0;
  for (int i = 1; i < 5; ++i) {
    pc[i] = pc[i - 1] * cs;
    ps[i] = ps[i - 1] * ss;
  }
  double sw[5], sqw[3];
  for (int k = 0; k <= 2 * order; ++k) {
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += kBinom[k][j] * pc[j] * ps[k - j] * (double)mom->m[k - j][j];
    sw[k] = acc;
  }
  for (int k = 0; k <= order; ++k) {
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += kBinom[k][j] * pc[j] * ps[k - j] * (double)mom->q[k - j][j];
    sqw[k] = acc / 1024.0;
  }
  double A[3][3] = {{0}}, b[3] = {0}, x[3] = {0};
  for (int i = 0; i < n; ++i) {
    b[i] = sqw[i];
    for (int k = 0; k < n; ++k) A[i][k] = sw[i + k];
  }
  if (spd_solve(n, A, b, x) != 0) {
    for (int i = 0; i < 3; ++i) beta[i] = 0.0;
    return INFINITY;
  }
  double dd = (double)mom->qq / 1048576.0;
  double fit = 0.0;
  for (int i = 0; i < n; ++i) fit += b[i] * x[i];
  for (int i = 0; i < 3; ++i) beta[i] = i < n ? x[i] : 0.0;
  return dd - fit;
}

/* Convert the w_s-basis coefficients to the (a0, a1, a2) of Eq. (3) in v'. */
static void beta_to_model(const double beta[3], int order, int W, int H, double phi,
                          or_road_model* out) {
  double k = 2.0 / coord_scale(W, H);
  double vc = (double)(H - 1) * 0.5;
  double b0 = beta[0], b1 = beta[1], b2 = order == 2 ? beta[2] : 0.0;
  out->order = order;
  out->roll = phi;
  out->a[2] = b2 * k * k;
  out->a[1] = b1 * k - 2.0 * b2 * k * k * vc;
  out->a[0] = b0 - b1 * k * vc + b2 * k * k * vc * vc;
}

#define ROLL_GRID_N 3001
#define ROLL_GRID_STEP 1.7453292519943295e-04 /* 0.01 degree in radians */

/* Reading R7.  Eq. (12) is minimised over phi; the paper defers the solver to a citation.
 * Linear model: the minimum over (a, phi) is the least-squares plane d = k0 + kv v~ + ku u~
 * (kv = a1 cos(phi)/2, ku = -a1 sin(phi)/2), so phi = atan(-ku / kv) on the |phi| < 90 deg branch.
 * Quadratic model: E0min is evaluated on a grid of 0.01 deg over +-15 deg, and the best grid
 * point's bracket is refined by golden-section search to a width below 1e-12 rad.
 * In both cases a(phi) then comes from Eq. (11). */
void or_fit_road(const or_moment_sums* mom, int order, int W, int H, or_road_model* fitted) {
  double beta[3];
  double phi = 0.0;
  if (order == 1) {
    double sc = coord_scale(W, H);
    double s1 = sc, s2 = sc * sc;
    double A[3][3] = {
        {(double)mom->m[0][0], (double)mom->m[0][1] / s1, (double)mom->m[1][0] / s1},
        {(double)mom->m[0][1] / s1, (double)mom->m[0][2] / s2, (double)mom->m[1][1] / s2},
        {(double)mom->m[1][0] / s1, (double)mom->m[1][1] / s2, (double)mom->m[2][0] / s2}};
    double b[3] = {(double)mom->q[0][0] / 1024.0, (double)mom->q[0][1] / s1 / 1024.0,
                   (double)mom->q[1][0] / s1 / 1024.0};
    double x[3] = {0, 0, 0};
    if (spd_solve(3, A, b, x) == 0 && x[1] != 0.0) phi = atan(-x[2] / x[1]);
  } else {
    int best = 0;
    double bestE = INFINITY;
    for (int k = 0; k < ROLL_GRID_N; ++k) {
      double e = or_e0min(mom, order, W, H, (double)(k - ROLL_GRID_N / 2) * ROLL_GRID_STEP, beta);
      if (e < bestE) {
        bestE = e;
        best = k;
      }
    }
    int klo = best > 0 ? best - 1 : 0;
    int khi = best < ROLL_GRID_N - 1 ? best + 1 : ROLL_GRID_N - 1;
    double a = (double)(klo - ROLL_GRID_N / 2) * ROLL_GRID_STEP;
    double b = (double)(khi - ROLL_GRID_N / 2) * ROLL_GRID_STEP;
    const double g = 0.6180339887498949;
    double x1 = b - g * (b - a), x2 = a + g * (b - a);
    double f1 = or_e0min(mom, order, W, H, x1, beta);
    double f2 = or_e0min(mom, order, W, H, x2, beta);
    for (int it = 0; it < 200 && (b - a) > 1e-12; ++it) {
      if (f1 <= f2) {
        b = x2;
        x2 = x1;
        f2 = f1;
        x1 = b - g * (b - a);
        f1 = or_e0min(mom, order, W, H, x1, beta);
      } else {
        a = x1;
        x1 = x2;
        f1 = f2;
        x2 = a + g * (b - a);
        f2 = or_e0min(mom, order, W, H, x2, beta);
      }
    }
    phi = 0.5 * (a + b);
  }
  or_e0min(mom, order, W, H, phi, beta);
  beta_to_model(beta, order, W, H, phi, fitted);
}

/* Eq. (13) in single precision with the fitted coefficients rounded to float:
 * D2 = max(0, (D1 - f) + delta_dt); pixels with D1 < 0 get delta_dt (road level). */
void or_transform(const float* D1, int W, int H, const or_road_model* fitted, float delta_dt,
                  float* D2) {
  float c = (float)cos(fitted->roll), s = (float)sin(fitted->roll);
  float a0 = (float)fitted->a[0], a1 = (float)fitted->a[1];
  float a2 = fitted->order == 2 ? (float)fitted->a[2] : 0.0f;
  float uc = (float)((double)(W - 1) * 0.5), vc = (float)((double)(H - 1) * 0.5);
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      float d1 = D1[(size_t)v * W + u];
      float out = delta_dt;
      if (d1 >= 0.0f) {
        float t1 = ((float)v - vc) * c;
        float t2 = ((float)u - uc) * s;
        float vp = (t1 - t2) + vc;
        float f = (a0 + a1 * vp) + a2 * (vp * vp);
        out = (d1 - f) + delta_dt;
        if (out < 0.0f) out = 0.0f;
      }
      D2[(size_t)v * W + u] = out;
    }
  }
}

/* ------------------------------------------------------------------- Sec. II-D SLIC */

/* Reading R8 of the grid sentence of Sec. II-D: grid interval S = sqrt(W H / K), nx = round(W/S),
 * ny = round(H/S), each at least 1 and at most the image size. */
int or_slic_grid(int W, int H, int K, int* nx, int* ny) {
  double S = sqrt((double)W * (double)H / (double)K);
  int a = (int)floor((double)W / S + 0.5);
  int b = (int)floor((double)H / S + 0.5);
  a = clampi(a, 1, W);
  b = clampi(b, 1, H);
  *nx = a;
  *ny = b;
  return a * b;
}

static float slic_gradient(const float* D2, int W, int H, int x, int y) {
  float gx = D2[(size_t)y * W + clampi(x + 1, 0, W - 1)] - D2[(size_t)y * W + clampi(x - 1, 0, W - 1)];
  float gy = D2[(size_t)clampi(y + 1, 0, H - 1) * W + x] - D2[(size_t)clampi(y - 1, 0, H - 1) * W + x];
  return gx * gx + gy * gy;
}

/* Sec. II-D.  Seeds on a regular grid move to the lowest-gradient pixel of their 3x3 neighbourhood
 * (the seed itself wins ties, then raster order).  Each iteration assigns every pixel to the
 * nearest centre whose 2S x 2S search window covers it, with
 *   dist = (D2 - value)^2 + ((x - cx)^2 + (y - cy)^2) (m/S)^2    (float, this operation order),
 * the lower centre index winning ties and uncovered pixels keeping their label; then every centre
 * becomes the mean of its members (exact integer sums of x, y and rint(1024 D2)).  Initial labels
 * are the grid cells.  Exactly `iters` iterations are run. */
int or_slic(const float* D2, int W, int H, int K, float m, int iters, int32_t* labels,
            float* centres) {
  int nx, ny;
  int n = or_slic_grid(W, H, K, &nx, &ny);
  float Sf = (float)sqrt((double)W * (double)H / (double)K);
  float coef = (float)((double)m * (double)m * (double)K / ((double)W * (double)H));
  float* cx = (float*)malloc(sizeof(float) * (size_t)n);
  float* cy = (float*)malloc(sizeof(float) * (size_t)n);
  float* cv = (float*)malloc(sizeof(float) * (size_t)n);
  float* dist = (float*)malloc(sizeof(float) * (size_t)W * H);
  int64_t* acc = (int64_t*)malloc(sizeof(int64_t) * 4 * (size_t)n);

  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      int sx = (int)(((int64_t)(2 * i + 1) * W) / (2 * nx));
      int sy = (int)(((int64_t)(2 * j + 1) * H) / (2 * ny));
      int bx = sx, by = sy;
      float bg = slic_gradient(D2, W, H, sx, sy);
      for (int dy = -1; dy <= 1; ++dy) {
        for (int dx = -1; dx <= 1; ++dx) {
          int x = sx + dx, y = sy + dy;
          if (x < 0 || x >= W || y < 0 || y >= H) continue;
          float g = slic_gradient(D2, W, H, x, y);
          if (g < bg) {
            bg = g;
            bx = x;
            by = y;
          }
        }
      }
      int k = j * nx + i;
      cx[k] = (float)bx;
      cy[k] = (float)by;
      cv[k] = D2[(size_t)by * W + bx];
    }
  }
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x)
      labels[(size_t)y * W + x] = (int32_t)(((int64_t)y * ny / H) * nx + ((int64_t)x * nx / W));

  for (int it = 0; it < iters; ++it) {
    for (size_t p = 0; p < (size_t)W * H; ++p) dist[p] = INFINITY;
    for (int k = 0; k < n; ++k) {
      int xlo = clampi((int)floor((double)cx[k] - (double)Sf) - 1, 0, W - 1);
      int xhi = clampi((int)ceil((double)cx[k] + (double)Sf) + 1, 0, W - 1);
      int ylo = clampi((int)floor((double)cy[k] - (double)Sf) - 1, 0, H - 1);
      int yhi = clampi((int)ceil((double)cy[k] + (double)Sf) + 1, 0, H - 1);
      for (int y = ylo; y <= yhi; ++y) {
        for (int x = xlo; x <= xhi; ++x) {
          float fx = (float)x - cx[k];
          float fy = (float)y - cy[k];
          if (!(fabsf(fx) <= Sf && fabsf(fy) <= Sf)) continue;
          size_t p = (size_t)y * W + x;
          float dv = D2[p] - cv[k];
          float dd = dv * dv + (fx * fx + fy * fy) * coef;
          if (dd < dist[p]) {
            dist[p] = dd;
            labels[p] = k;
          }
        }
      }
    }
    memset(acc, 0, sizeof(int64_t) * 4 * (size_t)n);
    for (int y = 0; y < H; ++y) {
      for (int x = 0; x < W; ++x) {
        size_t p = (size_t)y * W + x;
        int64_t* a = acc + 4 * (size_t)labels[p];
        a[0] += 1;
        a[1] += x;
        a[2] += y;
        a[3] += (int64_t)rint((double)D2[p] * 1024.0);
      }
    }
    for (int k = 0; k < n; ++k) {
      int64_t* a = acc + 4 * (size_t)k;
      if (a[0] == 0) continue;
      cx[k] = (float)((double)a[1] / (double)a[0]);
      cy[k] = (float)((double)a[2] / (double)a[0]);
      cv[k] = (float)(((double)a[3] / (double)a[0]) / 1024.0);
    }
  }
  if (centres)
    for (int k = 0; k < n; ++k) {
      centres[3 * k + 0] = cx[k];
      centres[3 * k + 1] = cy[k];
      centres[3 * k + 2] = cv[k];
    }
  free(cx);
  free(cy);
  free(cv);
  free(dist);
  free(acc);
  return n;
}

/* Sec. II-E: each superpixel's value is the mean of its transformed disparities (exact sums of
 * rint(1024 D2), one double division), written to every pixel of the superpixel. */
void or_superpixel_mean(const float* D2, const int32_t* labels, int W, int H, int nlabels,
                        float* D3) {
  int64_t* cnt = (int64_t*)calloc((size_t)nlabels, sizeof(int64_t));
  int64_t* sum = (int64_t*)calloc((size_t)nlabels, sizeof(int64_t));
  float* val = (float*)calloc((size_t)nlabels, sizeof(float));
  for (size_t p = 0; p < (size_t)W * H; ++p) {
    cnt[labels[p]] += 1;
    sum[labels[p]] += (int64_t)rint((double)D2[p] * 1024.0);
  }
  for (int k = 0; k < nlabels; ++k)
    if (cnt[k] > 0) val[k] = (float)(((double)sum[k] / (double)cnt[k]) / 1024.0);
  for (size_t p = 0; p < (size_t)W * H; ++p) D3[p] = val[labels[p]];
  free(cnt);
  free(sum);
  free(val);
}

/* ------------------------------------------------------- Sec. II-E, Eqs. (14)-(17) */

/* Reading R9.  g = [D2(p), sum of D2 over the 8 neighbours] (Eq. (15)), held exactly as
 * a = rint(1024 D2(p)) and b = sum of rint(1024 D2(q)).  Only interior pixels whose 3x3 window is
 * all valid (D1 >= 0) take part.  For a threshold t = k/8 px (k = 1..255) on the histogram
 * diagonal, region 1 (pothole) is {D2 < t and b/8 < t} and region 2 (road) is {D2 >= t and
 * b/8 >= t}; the off-diagonal regions 3 and 4 are left out.  E2(t) is Eq. (17) evaluated brute
 * force, over every pixel for every t.  t_r is the smallest t that minimises E2 among the t with
 * both regions non-empty.  mode 0 (default): t_s = (mean D2 of region 2 at t_r) - delta_pd, using
 * the road-mean sentence of Sec. II-E; mode 1: t_s = t_r - delta_pd as Eq. (14) is printed. */
int or_threshold(const float* D2, const float* D1, int W, int H, float delta_pd, int mode,
                 double* t_r, double* t_s, double* E2) {
  size_t N = (size_t)W * H;
  int64_t* qa = (int64_t*)malloc(sizeof(int64_t) * N);
  int64_t* qb = (int64_t*)malloc(sizeof(int64_t) * N);
  uint8_t* use = (uint8_t*)calloc(N, 1);
  for (size_t p = 0; p < N; ++p) qa[p] = (int64_t)rint((double)D2[p] * 1024.0);
  for (int v = 1; v < H - 1; ++v) {
    for (int u = 1; u < W - 1; ++u) {
      int ok = 1;
      int64_t b = 0;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          size_t q = (size_t)(v + dy) * W + (u + dx);
          if (!(D1[q] >= 0.0f)) ok = 0;
          if (dx != 0 || dy != 0) b += qa[q];
        }
      size_t p = (size_t)v * W + u;
      use[p] = (uint8_t)ok;
      qb[p] = b;
    }
  }
  int best = -1;
  double bestE = 0.0, bestMean = 0.0;
  for (int k = 0; k < 256; ++k) E2[k] = NAN;
  for (int k = 1; k < 256; ++k) {
    int64_t n1 = 0, n2 = 0, a1 = 0, a2 = 0, b1 = 0, b2 = 0;
    __int128 s1 = 0, s2 = 0;
    for (size_t p = 0; p < N; ++p) {
      if (!use[p]) continue;
      int64_t a = qa[p], b = qb[p];
      if (a < 128 * (int64_t)k && b < 1024 * (int64_t)k) {
        n1 += 1;
        a1 += a;
        b1 += b;
        s1 += (__int128)a * a + (__int128)b * b;
      } else if (a >= 128 * (int64_t)k && b >= 1024 * (int64_t)k) {
        n2 += 1;
        a2 += a;
        b2 += b;
        s2 += (__int128)a * a + (__int128)b * b;
      }
    }
    if (n1 == 0 || n2 == 0) continue;
    double e1 = (double)s1 - ((double)a1 * (double)a1 + (double)b1 * (double)b1) / (double)n1;
    double e2 = (double)s2 - ((double)a2 * (double)a2 + (double)b2 * (double)b2) / (double)n2;
    double e = e1 + e2;
    E2[k] = e;
    if (best < 0 || e < bestE) {
      best = k;
      bestE = e;
      bestMean = ((double)a2 / (double)n2) / 1024.0;
    }
  }
  free(qa);
  free(qb);
  free(use);
  if (best < 0) {
    *t_r = NAN;
    *t_s = -INFINITY;
    return -1;
  }
  *t_r = (double)best * 0.125;
  *t_s = (mode == 0 ? bestMean : *t_r) - (double)delta_pd;
  return 0;
}

/* Sec. II-E: a pixel belongs to a pothole when its superpixel value D3 is below t_s. */
void or_mask(const float* D3, int W, int H, double t_s, uint8_t* mask) {
  for (size_t p = 0; p < (size_t)W * H; ++p) mask[p] = (double)D3[p] < t_s ? 1 : 0;
}

/* ------------------------------------------------------------ helpers for the test harness */

size_t or_moment_sums_size(void) { return sizeof(or_moment_sums); }

/* Writes count, m[i][j] (i + j <= 4; i outer, j inner), q[i][j] (i + j <= 2) and qq as 23 signed
 * 128-bit integers, each as (low 64 bits, high 64 bits). */
void or_moments_export(const or_moment_sums* mom, int64_t* out) {
  int k = 0;
  __int128 vals[23];
  vals[k++] = mom->count;
  for (int i = 0; i <= 4; ++i)
    for (int j = 0; i + j <= 4; ++j) vals[k++] = mom->m[i][j];
  for (int i = 0; i <= 2; ++i)
    for (int j = 0; i + j <= 2; ++j) vals[k++] = mom->q[i][j];
  vals[k++] = mom->qq;
  for (int i = 0; i < 23; ++i) {
    out[2 * i] = (int64_t)(uint64_t)vals[i];
    out[2 * i + 1] = (int64_t)(vals[i] >> 64);
  }
}

/* ------------------------------------------------ learned-band SGM (an extension of the paper) */

/* Reading R10.  Each 16x16 tile (tile (u/16, v/16)) searches the window [lo, lo + band) clipped to
 * [0, D), or the full range [0, D) when its entry of tile_lo is negative.  Writes each pixel's
 * window as [lo[p], hi[p]). */
void or_band_windows(const int16_t* tile_lo, int W, int H, int D, int band, int16_t* lo,
                     int16_t* hi) {
  int tw = (W + 15) / 16;
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      int t = tile_lo[(v / 16) * tw + (u / 16)];
      int a = 0, b = D;
      if (t >= 0) {
        a = clampi(t, 0, D - 1);
        b = a + band < D ? a + band : D;
      }
      lo[(size_t)v * W + u] = (int16_t)a;
      hi[(size_t)v * W + u] = (int16_t)b;
    }
}

/* Eq. (8) restricted to the windows: L_r(p, d) exists for d in [lo(p), hi(p)); the terms of the
 * minimum use only d' inside the predecessor's window, and m is the minimum over that window.
 * S is 0xFFFF outside the window. */
void or_aggregate_band(const uint8_t* cost, const int16_t* lo, const int16_t* hi, int W, int H,
                       int D, int paths, int P1, int P2, uint16_t* S) {
  const int64_t INF = (int64_t)1 << 40;
  size_t n = (size_t)W * H * D;
  int64_t* L = (int64_t*)malloc(sizeof(int64_t) * n);
  int64_t* acc = (int64_t*)calloc(n, sizeof(int64_t));
  for (int r = 0; r < paths; ++r) {
    int dx = kDirs[r][0], dy = kDirs[r][1];
    int v0, vi, u0, ui;
    path_order(H, dy, &v0, &vi);
    path_order(W, dx, &u0, &ui);
    for (int iv = 0, v = v0; iv < H; ++iv, v += vi) {
      for (int iu = 0, u = u0; iu < W; ++iu, u += ui) {
        size_t p = (size_t)v * W + u;
        const uint8_t* c = cost + p * D;
        int64_t* out = L + p * D;
        for (int d = 0; d < D; ++d) out[d] = INF;
        int pu = u - dx, pv = v - dy;
        if (pu < 0 || pu >= W || pv < 0 || pv >= H) {
          for (int d = lo[p]; d < hi[p]; ++d) out[d] = c[d];
          continue;
        }
        size_t q = (size_t)pv * W + pu;
        const int64_t* prev = L + q * D;
        int plo = lo[q], phi = hi[q];
        int64_t m = INF;
        for (int d = plo; d < phi; ++d)
          if (prev[d] < m) m = prev[d];
        for (int d = lo[p]; d < hi[p]; ++d) {
          int64_t best = m + P2;
          if (d >= plo && d < phi && prev[d] < best) best = prev[d];
          if (d - 1 >= plo && d - 1 < phi && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
          if (d + 1 >= plo && d + 1 < phi && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
          out[d] = c[d] + best - m;
        }
      }
    }
    for (size_t i = 0; i < n; ++i)
      if (L[i] < INF) acc[i] += L[i];
  }
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      size_t p = (size_t)v * W + u;
      for (int d = 0; d < D; ++d)
        S[p * D + d] = (d >= lo[p] && d < hi[p]) ? (uint16_t)acc[p * D + d] : (uint16_t)0xFFFF;
    }
  free(L);
  free(acc);
}

/* Eqs. (9)-(10) over the windows: d* = argmin over [lo, hi); the parabola needs d* - 1 and
 * d* + 1 inside the window; the right view of column x takes the d with x + d inside the image
 * and d inside the window of pixel x + d; valid pixels need u >= hi - 1, a right view at u - d*
 * and |d* - d_R| <= lr_tol. */
void or_disparity_band(const uint16_t* S, const int16_t* lo, const int16_t* hi, int W, int H, int D,
                       const int32_t* kappa, int lr_tol, int16_t* d_int, float* D1) {
  int* dright = (int*)malloc(sizeof(int) * (size_t)W);
  for (int v = 0; v < H; ++v) {
    const uint16_t* row = S + (size_t)v * W * D;
    for (int x = 0; x < W; ++x) {
      int best = -1;
      unsigned bestv = 0;
      for (int d = 0; d < D && x + d < W; ++d) {
        size_t p = (size_t)v * W + x + d;
        if (d < lo[p] || d >= hi[p]) continue;
        unsigned val = row[(size_t)(x + d) * D + d];
        if (best < 0 || val < bestv) {
          bestv = val;
          best = d;
        }
      }
      dright[x] = best;
    }
    for (int u = 0; u < W; ++u) {
      size_t p = (size_t)v * W + u;
      const uint16_t* s = row + (size_t)u * D;
      int a = lo[p], b = hi[p];
      int ds = a;
      for (int d = a + 1; d < b; ++d)
        if (s[d] < s[ds]) ds = d;
      float dsub = (float)ds;
      if (ds - 1 >= a && ds + 1 < b) {
        int num = (int)s[ds - 1] - (int)s[ds + 1];
        int den = 2 * ((int)s[ds - 1] + (int)s[ds + 1] - 2 * (int)s[ds]);
        if (den > 0) dsub = (float)ds + (float)num / (float)den;
      }
      d_int[p] = (int16_t)ds;
      int xr = u - ds;
      int valid = u >= b - 1 && xr >= 0 && dright[xr] >= 0 && abs(ds - dright[xr]) <= lr_tol;
      float d1 = dsub + (float)kappa[v];
      D1[p] = (valid && d1 >= 0.0f) ? d1 : -1.0f;
    }
  }
  free(dright);
}

/* --------------------------------------------------- Sec. II-E: connected component labelling */

/* Reading R14: the pothole mask's connected components, with 8- or 4-connectivity (the paper
 * names CCL without fixing it), each labelled by the smallest raster index p = v W + u among its
 * pixels; breadth-first search from every unlabelled mask pixel in raster order.  Pixels outside
 * the mask get -1.  Returns the number of components. */
int or_ccl(const uint8_t* mask, int W, int H, int conn, int32_t* labels) {
  size_t n = (size_t)W * H;
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
  int count = 0;
  for (size_t p = 0; p < n; ++p) labels[p] = -1;
  for (size_t p = 0; p < n; ++p) {
    if (!mask[p] || labels[p] >= 0) continue;
    ++count;
    size_t head = 0, tail = 0;
    labels[p] = (int32_t)p;
    queue[tail++] = (int32_t)p;
    while (head < tail) {
      int q = queue[head++];
      int u = q % W, v = q / W;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0) continue;
          if (conn == 4 && dx != 0 && dy != 0) continue;
          int x = u + dx, y = v + dy;
          if (x < 0 || x >= W || y < 0 || y >= H) continue;
          size_t r = (size_t)y * W + x;
          if (mask[r] && labels[r] < 0) {
            labels[r] = (int32_t)p;
            queue[tail++] = (int32_t)r;
          }
        }
    }
  }
  free(queue);
  return count;
}

/* Per-component statistics in the order of the components' labels, and the fake-pothole rule
 * (Sec. III-B: detections at a corner of the image or made of a single superpixel are fake).
 * Reading R15: a component lies at a corner when its centroid falls in one of the four corner
 * cells of the image split 8 x 8 (u < W/8 or u >= 7W/8, and v < H/8 or v >= 7H/8, compared
 * exactly as 8 sum_u < W n, ...); it is made of one superpixel when all its pixels carry the same
 * SLIC label.  out: per component 12 int64 values: label, pixel count, u min, v min, u max, v max,
 * sum u, sum v, superpixels (1, or 2 meaning two or more), corner, single, fake. */
void or_components(const int32_t* labels, const int32_t* sp, int W, int H, int ncomp,
                   int64_t* out) {
  size_t n = (size_t)W * H;
  int k = 0;
  for (size_t p = 0; p < n && k < ncomp; ++p) {
    if (labels[p] != (int32_t)p) continue;
    int64_t* o = out + (size_t)k * 12;
    int64_t cnt = 0, su = 0, sv = 0;
    int umin = W, vmin = H, umax = -1, vmax = -1;
    int32_t first_sp = 0;
    int multi = 0;
    for (size_t q = p; q < n; ++q) {
      if (labels[q] != (int32_t)p) continue;
      int u = (int)(q % W), v = (int)(q / W);
      if (cnt == 0)
        first_sp = sp[q];
      else if (sp[q] != first_sp)
        multi = 1;
      ++cnt;
      su += u;
      sv += v;
      if (u < umin) umin = u;
      if (u > umax) umax = u;
      if (v < vmin) vmin = v;
      if (v > vmax) vmax = v;
    }
    int left = 8 * su < (int64_t)W * cnt, right = 8 * su >= (int64_t)7 * W * cnt;
    int top = 8 * sv < (int64_t)H * cnt, bottom = 8 * sv >= (int64_t)7 * H * cnt;
    int corner = (left || right) && (top || bottom);
    o[0] = (int64_t)p;
    o[1] = cnt;
    o[2] = umin;
    o[3] = vmin;
    o[4] = umax;
    o[5] = vmax;
    o[6] = su;
    o[7] = sv;
    o[8] = multi ? 2 : 1;
    o[9] = corner;
    o[10] = !multi;
    o[11] = corner || !multi;
    ++k;
  }
}

/* ------------------------------------------------------- robust road fit (beyond Sec. II-C) */

/* Reading R17: the moments of Sec. II-C over the inliers of a previous fit only: pixels with
 * D1 >= 0 and |D1 - f(p)| <= tau, f evaluated in single precision exactly as in the transform. */
void or_moments_inliers(const float* D1, int W, int H, const or_road_model* fit, float tau,
                        or_moment_sums* out) {
  float c = (float)cos(fit->roll), s = (float)sin(fit->roll);
  float a0 = (float)fit->a[0], a1 = (float)fit->a[1];
  float a2 = fit->order == 2 ? (float)fit->a[2] : 0.0f;
  float uc = (float)((double)(W - 1) * 0.5), vc = (float)((double)(H - 1) * 0.5);
  size_t n = (size_t)W * H;
  float* masked = (float*)malloc(sizeof(float) * n);
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      size_t p = (size_t)v * W + u;
      float d1 = D1[p];
      masked[p] = -1.0f;
      if (!(d1 >= 0.0f)) continue;
      float t1 = ((float)v - vc) * c;
      float t2 = ((float)u - uc) * s;
      float vp = (t1 - t2) + vc;
      float f = (a0 + a1 * vp) + a2 * (vp * vp);
      if (fabsf(d1 - f) <= tau) masked[p] = d1;
    }
  or_moments(masked, W, H, out);
  free(masked);
}

/* The fit of Sec. II-C followed by `iters` refits on the inliers (within tau) of the previous
 * fit. */
void or_fit_road_robust(const float* D1, int W, int H, int order, int iters, float tau,
                        or_road_model* fitted) {
  or_moment_sums m;
  or_moments(D1, W, H, &m);
  or_fit_road(&m, order, W, H, fitted);
  for (int k = 0; k < iters; ++k) {
    or_road_model prev = *fitted;
    or_moments_inliers(D1, W, H, &prev, tau, &m);
    or_fit_road(&m, order, W, H, fitted);
  }
}
