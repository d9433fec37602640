// Sec. II-C on the GPU: exact moment sums of the road disparities, the roll / road-model fit of
// Eqs. (11)-(12) on the device (a grid of angles over many SMs, then one refining block; no host
// round trip), and the Eq. (13) transformation.
#include <math.h>

#include <mutex>

#include "common.cuh"

// Fixed scratch of the allocation-free transform entry point (pd_transform_noalloc): every GPU
// that loads the library holds it until the process exits.
static constexpr size_t kNoAllocScratchBytes = 512 * 1024;
static constexpr long long kNoAllocMaxPixels = 4194304;  // W * H limit that fits the scratch
static __device__ __align__(256) unsigned char g_transform_scratch[kNoAllocScratchBytes];

namespace pd {

namespace {

constexpr int kMomThreads = 256;
constexpr int kMomPixPerBlock = 2048;  // keeps every per-block int64 partial exact (W, H <= 4096)
static_assert(kMomPixPerBlock % kMomThreads == 0, "whole pixels per thread");
constexpr int kNumSums = 23;

__device__ __forceinline__ long long warp_sum_ll(long long x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// The road model of a fit at pixel (u, v), in single precision in the operation order of the
// model definition (no FMA): the value the transform subtracts.
__device__ __forceinline__ float road_f32(const RoadCoefF& c, int u, int v) {
  const float t1 = ((float)v - c.vc) * c.c;
  const float t2 = ((float)u - c.uc) * c.s;
  const float vp = (t1 - t2) + c.vc;
  return (c.a0 + c.a1 * vp) + c.a2 * (vp * vp);
}

// Per-block int64 partial sums: count, sum u~^i v~^j (i + j <= 4), sum q u~^i v~^j (i + j <= 2),
// sum q^2 with q = rint(1024 D1), u~ = 2u - (W-1), v~ = 2v - (H-1), over pixels with D1 >= 0 and,
// when fit is given, |D1 - f(p)| <= tau (the inliers of that fit).
__global__ void __launch_bounds__(kMomThreads) k_moments_partial(const float* __restrict__ D1,
                                                                 int W, int H,
                                                                 long long* __restrict__ partial,
                                                                 const RoadCoefF* __restrict__ fit,
                                                                 float tau) {
  RoadCoefF cf;
  if (fit) cf = *fit;
  long long acc[kNumSums];
#pragma unroll
  for (int i = 0; i < kNumSums; ++i) acc[i] = 0;
  const size_t N = (size_t)W * H;
  const size_t start = (size_t)blockIdx.x * kMomPixPerBlock;
  const size_t end = min(start + (size_t)kMomPixPerBlock, N);
  // the thread's kMomPixPerBlock / kMomThreads disparities are loaded together first, so their
  // memory latencies overlap instead of adding up
  constexpr int kPer = kMomPixPerBlock / kMomThreads;
  float dv[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const size_t p = start + threadIdx.x + (size_t)j * kMomThreads;
    dv[j] = p < end ? D1[p] : -1.0f;
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const size_t p = start + threadIdx.x + (size_t)j * kMomThreads;
    const float d = dv[j];
    if (!(d >= 0.0f)) continue;  // also every p >= end
    const int pi = (int)p;  // W * H <= 2^24: a 32-bit division
    int u = pi % W, v = pi / W;
    if (fit && !(fabsf(d - road_f32(cf, u, v)) <= tau)) continue;
    long long q = rint_to_ll(d * 1024.0f);  // exact scaling; rounds half to even like rint
    long long ut = 2LL * u - (W - 1), vt = 2LL * v - (H - 1);
    long long up[5], vp[5];
    up[0] = vp[0] = 1;
#pragma unroll
    for (int i = 1; i < 5; ++i) {
      up[i] = up[i - 1] * ut;
      vp[i] = vp[i - 1] * vt;
    }
    int k = 0;
    acc[k++] += 1;
#pragma unroll
    for (int i = 0; i <= 4; ++i)
#pragma unroll
      for (int j = 0; i + j <= 4; ++j) acc[k++] += up[i] * vp[j];
#pragma unroll
    for (int i = 0; i <= 2; ++i)
#pragma unroll
      for (int j = 0; i + j <= 2; ++j) acc[k++] += q * up[i] * vp[j];
    acc[k++] += q * q;
  }
  __shared__ long long red[kMomThreads / 32][kNumSums];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < kNumSums; ++i) {
    long long s = warp_sum_ll(acc[i]);
    if (lane == 0) red[warp][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < kNumSums) {
    long long s = 0;
    for (int w = 0; w < kMomThreads / 32; ++w) s += red[w][threadIdx.x];
    partial[(size_t)blockIdx.x * kNumSums + threadIdx.x] = s;
  }
}

// Sums the block partials exactly in 128 bits; writes (low, high) 64-bit pairs.  One warp per sum.
__global__ void k_moments_final(const long long* __restrict__ partial, int nblocks,
                                int64_t* __restrict__ sums) {
  __shared__ __int128 red[kNumSums][32];
  const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __int128 s = 0;
  for (int b = lane; b < nblocks; b += 32) s += (__int128)partial[(size_t)b * kNumSums + i];
  red[i][lane] = s;
  __syncwarp();
  if (lane == 0) {
    __int128 t = 0;
    for (int l = 0; l < 32; ++l) t += red[i][l];
    sums[2 * i] = (int64_t)(unsigned long long)t;
    sums[2 * i + 1] = (int64_t)(t >> 64);
  }
}

// Correctly rounded conversion of a signed 128-bit integer (lo, hi) to double: the top 64
// significant bits with a sticky bit for everything below, converted once, then scaled exactly.
__device__ double i128_to_double(unsigned long long lo, long long hi) {
  bool neg = hi < 0;
  unsigned long long mlo = lo, mhi = (unsigned long long)hi;
  if (neg) {
    mlo = ~mlo + 1ULL;
    mhi = ~mhi + (mlo == 0ULL ? 1ULL : 0ULL);
  }
  double r;
  if (mhi == 0ULL) {
    r = __ull2double_rn(mlo);
  } else {
    int lz = __clzll((long long)mhi);
    unsigned long long top = lz ? ((mhi << lz) | (mlo >> (64 - lz))) : mhi;
    unsigned long long rest = lz ? (mlo << lz) : mlo;
    if (rest) top |= 1ULL;
    r = ldexp(__ull2double_rn(top), 64 - lz);
  }
  return neg ? -r : r;
}

struct MomD {
  double m[5][5];
  double q[3][3];
  double qq;
};

__device__ const double kBinomD[5][5] = {
    {1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};

// Cholesky solve of a symmetric positive-definite n x n system (n <= 3).
__device__ int spd_solve_d(int n, const double A[3][3], const double b[3], double x[3]) {
  double Lm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
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

// Eq. (12) for given cos(phi), sin(phi), by an LDL' factorisation of T'T (no square roots, three
// divisions: FP64 runs at about one operation per clock per SM on this part, so the evaluation
// is kept short).  E0min = d'd - sum_i y_i^2 / D_i with L y = T'd; beta = the Eq. (11) solution.
__device__ double e0min_cs(const MomD& M, int order, double sc, double cphi, double sphi,
                           double beta[3]) {
  const int n = order + 1;
  const double cs = cphi / sc, ss = -sphi / sc;
  double pc[5], ps[5];
  pc[0] = 1.0;
  ps[0] = 1.0;
#pragma unroll
  for (int i = 1; i < 5; ++i) {
    pc[i] = pc[i - 1] * cs;
    ps[i] = ps[i - 1] * ss;
  }
  double sw[5] = {0, 0, 0, 0, 0}, b[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (k > 2 * order) break;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j <= k; ++j) acc += kBinomD[k][j] * pc[j] * ps[k - j] * M.m[k - j][j];
    sw[k] = acc;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k > order) break;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j <= k; ++j) acc += kBinomD[k][j] * pc[j] * ps[k - j] * M.q[k - j][j];
    b[k] = acc / 1024.0;
  }
  const double dd = M.qq / 1048576.0;
  beta[0] = beta[1] = beta[2] = 0.0;
  // A = [[sw0, sw1, sw2], [sw1, sw2, sw3], [sw2, sw3, sw4]] (top-left n x n block)
  const double d0 = sw[0];
  if (!(d0 > 0.0)) return INFINITY;
  const double i0 = 1.0 / d0;
  const double l10 = sw[1] * i0;
  const double d1 = sw[2] - l10 * sw[1];
  if (!(d1 > 0.0)) return INFINITY;
  const double i1 = 1.0 / d1;
  const double y0 = b[0], y1 = b[1] - l10 * y0;
  if (n == 2) {
    const double x1 = y1 * i1;
    beta[1] = x1;
    beta[0] = y0 * i0 - l10 * x1;
    return dd - (y0 * y0 * i0 + y1 * y1 * i1);
  }
  const double l20 = sw[2] * i0;
  const double l21 = (sw[3] - l20 * sw[1]) * i1;
  const double d2 = sw[4] - l20 * sw[2] - l21 * l21 * d1;
  if (!(d2 > 0.0)) return INFINITY;
  const double i2 = 1.0 / d2;
  const double y2 = b[2] - l20 * y0 - l21 * y1;
  const double x2 = y2 * i2;
  const double x1 = y1 * i1 - l21 * x2;
  beta[2] = x2;
  beta[1] = x1;
  beta[0] = y0 * i0 - l10 * x1 - l20 * x2;
  return dd - (y0 * y0 * i0 + y1 * y1 * i1 + y2 * y2 * i2);
}

constexpr int kGridN = 3001;
constexpr double kGridStep = 1.7453292519943295e-04;  // 0.01 degree
constexpr int kRollWarp = 32;
constexpr int kGridBlocks = (kGridN + kRollWarp - 1) / kRollWarp;
constexpr int kRoundBlocks = 152;
constexpr int kRoundPoints = kRoundBlocks * kRollWarp;  // shrinks the bracket ~2400x per round
constexpr int kRefineRounds = 2;                        // 0.02 degree -> below 1e-10 rad

// (energy, index) candidates are compared through an order-preserving int64 key of the energy:
// FP64 compares cost about 63 cycles each on this GPU, integer compares a few.
struct RollBest {
  long long key;
  int k;
  int pad;
};

// cos, sin and the Eq. (11) coefficients at a refinement block's best angle: the final stage
// takes the winner's instead of evaluating the angle again (a double sincos and fit cost ~20k
// cycles of the FP64 pipe).
struct RollFit {
  double c, s, beta[3];
};


// Converts the 22 sums (after the count) to doubles, one per lane of the calling warp; the caller
// synchronises before reading M.
__device__ void load_moments(const int64_t* __restrict__ sums, MomD& M) {
  const int t = threadIdx.x;
  if (t >= 22) return;
  const int k = t + 1;  // skip the count; m[0][0] is the same number
  const double x = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
  if (t < 15) {  // m[i][j], i + j <= 4, i outer
    int i = 0, r = t;
    while (r >= 5 - i) {
      r -= 5 - i;
      ++i;
    }
    M.m[i][r] = x;
  } else if (t < 21) {  // q[i][j], i + j <= 2
    int i = 0, r = t - 15;
    while (r >= 3 - i) {
      r -= 3 - i;
      ++i;
    }
    M.q[i][r] = x;
  } else {
    M.qq = x;
  }
}

__device__ double coord_scale_d(int W, int H) {
  int mmax = W > H ? W : H;
  double sc = 1.0;
  while (sc < (double)mmax) sc *= 2.0;
  return sc;
}

__device__ __forceinline__ bool better(long long e, int k, long long eo, int ko) {
  return eo < e || (eo == e && ko < k);
}

// Warp-wide (key, k) minimum, smallest k on ties; every lane gets the result.
__device__ void warp_argmin(long long& e, int& k) {
  for (int o = 16; o > 0; o >>= 1) {
    long long eo = __shfl_xor_sync(0xffffffffu, e, o);
    int ko = __shfl_xor_sync(0xffffffffu, k, o);
    if (better(e, k, eo, ko)) {
      e = eo;
      k = ko;
    }
  }
}

// Minimum over n per-block results, by one warp.
__device__ void reduce_best(const RollBest* __restrict__ res, int n, long long& e, int& k) {
  e = 0x7fffffffffffffffLL;
  k = 0x7fffffff;
  for (int i = threadIdx.x & 31; i < n; i += 32)
    if (better(e, k, res[i].key, res[i].k)) {
      e = res[i].key;
      k = res[i].k;
    }
  warp_argmin(e, k);
}

// Bracket [a, b] searched by refinement round `round` (1..kRefineRounds), or the final bracket
// and winning angle after the last round: the best grid angle's neighbours, then for each round
// the neighbours of its best interior point.
__device__ void bracket_chain(const RollBest* __restrict__ res, int round, double& a, double& b,
                              double& phi, int* last_w = nullptr) {
  long long e;
  int w;
  reduce_best(res, kGridBlocks, e, w);
  int best = w < kGridN ? w : 0;
  int klo = best > 0 ? best - 1 : 0;
  int khi = best < kGridN - 1 ? best + 1 : kGridN - 1;
  a = (double)(klo - kGridN / 2) * kGridStep;
  b = (double)(khi - kGridN / 2) * kGridStep;
  phi = (double)(best - kGridN / 2) * kGridStep;
  for (int q = 1; q < round; ++q) {
    reduce_best(res + kGridBlocks + (q - 1) * kRoundBlocks, kRoundBlocks, e, w);
    if (w >= kRoundPoints) w = kRoundPoints / 2;
    const double h = (b - a) / (double)(kRoundPoints + 1);
    phi = a + h * (double)(w + 1);
    const double na = a + h * (double)w;
    const double nb = a + h * (double)(w + 2);
    a = na;
    b = nb;
    if (last_w) *last_w = w;
  }
}

// Grid stage: E0min at the 0.01-degree angles over +-15 degrees, one angle per thread, one warp
// per block so the FP64 work spreads over many SMs; each block writes its best (E, index).
__global__ void __launch_bounds__(kRollWarp) k_roll_grid(const int64_t* __restrict__ sums,
                                                         int order, int W, int H,
                                                         RollBest* __restrict__ res) {
  __shared__ MomD M;
  load_moments(sums, M);
  __syncthreads();
  int k = blockIdx.x * kRollWarp + threadIdx.x;
  double e = INFINITY, beta[3];
  if (k < kGridN) {
    double sp, cp;
    sincos((double)(k - kGridN / 2) * kGridStep, &sp, &cp);
    e = e0min_cs(M, order, coord_scale_d(W, H), cp, sp, beta);
  }
  int kk = k < kGridN ? k : 0x7fffffff;
  long long key = f64_order_key(e);
  warp_argmin(key, kk);
  if (threadIdx.x == 0) res[blockIdx.x] = RollBest{key, kk, 0};
}

// Refinement round: kRoundPoints interior points of the current bracket.
__global__ void __launch_bounds__(kRollWarp) k_roll_round(const int64_t* __restrict__ sums,
                                                          int order, int W, int H, int round,
                                                          RollBest* __restrict__ res,
                                                          RollFit* __restrict__ fits) {
  __shared__ MomD M;
  load_moments(sums, M);
  __syncthreads();
  __shared__ double sa, ca;
  double a, b, phi;
  bracket_chain(res, round, a, b, phi);
  if (threadIdx.x == 0) sincos(a, &sa, &ca);
  __syncwarp();
  const double h = (b - a) / (double)(kRoundPoints + 1);
  const int i = blockIdx.x * kRollWarp + threadIdx.x;
  // cos / sin of a + t by angle addition; |t| < 4e-4 rad, so the Taylor series below are exact to
  // far below double rounding
  const double t = h * (double)(i + 1), t2 = t * t;
  const double ct = 1.0 - t2 * (0.5 - t2 * (1.0 / 24.0 - t2 * (1.0 / 720.0)));
  const double st = t * (1.0 - t2 * (1.0 / 6.0 - t2 * (1.0 / 120.0 - t2 * (1.0 / 5040.0))));
  double beta[3];
  const double cphi = ca * ct - sa * st, sphi = sa * ct + ca * st;
  double e = e0min_cs(M, order, coord_scale_d(W, H), cphi, sphi, beta);
  int k = i;
  long long key = f64_order_key(e);
  warp_argmin(key, k);
  if (threadIdx.x == 0)
    res[kGridBlocks + (round - 1) * kRoundBlocks + blockIdx.x] = RollBest{key, k, 0};
  if (i == k) fits[(round - 1) * kRoundBlocks + blockIdx.x] = RollFit{cphi, sphi, {beta[0], beta[1], beta[2]}};
}

// Final stage (one warp): the roll (order 2: the winner of the last round; order 1: the
// least-squares plane in closed form), Eq. (11) for the coefficients, the model and its float
// form for the transform kernel.
__global__ void __launch_bounds__(kRollWarp) k_roll_final(const int64_t* __restrict__ sums,
                                                          const RollBest* __restrict__ res,
                                                          const RollFit* __restrict__ fits,
                                                          int order, int W, int H,
                                                          pd_road_model* fitted,
                                                          RoadCoefF* coef) {
  __shared__ MomD M;
  load_moments(sums, M);
  __syncthreads();
  const double sc = coord_scale_d(W, H);
  double phi = 0.0;
  int w = 0;
  if (order == 2) {
    double a, b;
    bracket_chain(res, kRefineRounds + 1, a, b, phi, &w);
  }
  if (threadIdx.x != 0) return;
  if (order == 1) {
    double s1 = sc, s2 = sc * sc;
    double A[3][3] = {{M.m[0][0], M.m[0][1] / s1, M.m[1][0] / s1},
                      {M.m[0][1] / s1, M.m[0][2] / s2, M.m[1][1] / s2},
                      {M.m[1][0] / s1, M.m[1][1] / s2, M.m[2][0] / s2}};
    double b[3] = {M.q[0][0] / 1024.0, M.q[0][1] / s1 / 1024.0, M.q[1][0] / s1 / 1024.0};
    double x[3] = {0, 0, 0};
    if (spd_solve_d(3, A, b, x) == 0 && x[1] != 0.0) phi = atan(-x[2] / x[1]);
  }
  double beta[3];
  double sp, cp;
  if (order == 2) {  // the last round evaluated this angle already: its block kept the fit
    const RollFit f = fits[(kRefineRounds - 1) * kRoundBlocks + w / kRollWarp];
    cp = f.c;
    sp = f.s;
    beta[0] = f.beta[0];
    beta[1] = f.beta[1];
    beta[2] = f.beta[2];
  } else {
    sincos(phi, &sp, &cp);
    e0min_cs(M, order, sc, cp, sp, beta);
  }
  double k = 2.0 / sc;
  double vc = (double)(H - 1) * 0.5;
  double b0 = beta[0], b1 = beta[1], b2 = order == 2 ? beta[2] : 0.0;
  pd_road_model out{};  // zero-initialised: the padding after `order` is written as zeros
  out.order = order;
  out.roll = phi;
  out.a[2] = b2 * k * k;
  out.a[1] = b1 * k - 2.0 * b2 * k * k * vc;
  out.a[0] = b0 - b1 * k * vc + b2 * k * k * vc * vc;
  if (fitted) {  // written as whole words, so the padding after `order` is defined (zero)
    static_assert(sizeof(pd_road_model) == 40, "pd_road_model layout");
    unsigned long long* w = reinterpret_cast<unsigned long long*>(fitted);
    w[0] = (unsigned long long)(unsigned int)out.order;
    w[1] = (unsigned long long)__double_as_longlong(out.a[0]);
    w[2] = (unsigned long long)__double_as_longlong(out.a[1]);
    w[3] = (unsigned long long)__double_as_longlong(out.a[2]);
    w[4] = (unsigned long long)__double_as_longlong(out.roll);
  }
  RoadCoefF cf;
  cf.c = (float)cp;
  cf.s = (float)sp;
  cf.a0 = (float)out.a[0];
  cf.a1 = (float)out.a[1];
  cf.a2 = order == 2 ? (float)out.a[2] : 0.0f;
  cf.uc = (float)((double)(W - 1) * 0.5);
  cf.vc = (float)vc;
  cf.pad = 0.0f;
  *coef = cf;
}

// Eq. (13) in single precision, the operation order of the model definition (no FMA).
__global__ void k_d2(const float* __restrict__ D1, int W, int H, const RoadCoefF* __restrict__ cf,
                     float delta_dt, float* __restrict__ D2) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  int v = blockIdx.y;
  if (u >= W) return;
  RoadCoefF c = *cf;
  size_t p = (size_t)v * W + u;
  float d1 = D1[p];
  float out = delta_dt;
  if (d1 >= 0.0f) {
    const float f = road_f32(c, u, v);
    out = (d1 - f) + delta_dt;
    if (out < 0.0f) out = 0.0f;
  }
  D2[p] = out;
}

}  // namespace

size_t moments_scratch_bytes(int W, int H) {
  size_t n = ((size_t)W * H + kMomPixPerBlock - 1) / kMomPixPerBlock;
  return n * kNumSums * sizeof(long long);
}

constexpr size_t kRollFitsOffset = (size_t)(kGridBlocks + kRefineRounds * kRoundBlocks) * sizeof(RollBest);
static_assert(kRollFitsOffset % alignof(RollFit) == 0, "RollFit alignment");

size_t roll_scratch_bytes() {
  return kRollFitsOffset + (size_t)kRefineRounds * kRoundBlocks * sizeof(RollFit);
}

void launch_moments(cudaStream_t s, const float* D1, int W, int H, void* scratch, int64_t* sums,
                    const RoadCoefF* fit, float tau) {
  int nblocks = (int)(((size_t)W * H + kMomPixPerBlock - 1) / kMomPixPerBlock);
  long long* partial = static_cast<long long*>(scratch);
  k_moments_partial<<<nblocks, kMomThreads, 0, s>>>(D1, W, H, partial, fit, tau);
  k_moments_final<<<1, kNumSums * 32, 0, s>>>(partial, nblocks, sums);
}

int launch_roll_solve(cudaStream_t s, const int64_t* sums, int order, int W, int H,
                      pd_road_model* fitted, RoadCoefF* coef, double* grid_scratch) {
  RollBest* res = reinterpret_cast<RollBest*>(grid_scratch);
  RollFit* fits = reinterpret_cast<RollFit*>(reinterpret_cast<char*>(grid_scratch) + kRollFitsOffset);
  int n = 1;
  if (order == 2) {
    k_roll_grid<<<kGridBlocks, kRollWarp, 0, s>>>(sums, order, W, H, res);
    for (int r = 1; r <= kRefineRounds; ++r)
      k_roll_round<<<kRoundBlocks, kRollWarp, 0, s>>>(sums, order, W, H, r, res, fits);
    n += 1 + kRefineRounds;
  }
  k_roll_final<<<1, kRollWarp, 0, s>>>(sums, res, fits, order, W, H, fitted, coef);
  return n;
}

void launch_d2(cudaStream_t s, const float* D1, int W, int H, const RoadCoefF* coef,
               float delta_dt, float* D2) {
  dim3 grid((W + 255) / 256, H);
  k_d2<<<grid, 256, 0, s>>>(D1, W, H, coef, delta_dt, D2);
}

}  // namespace pd

// ---------------------------------------------------------------- allocation-free transform

namespace pd {
namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Per device: the unique id of the context the address was looked up in, and the address.  A
// device reset (cudaDeviceReset) destroys the context and unloads the module, so the address is
// looked up again whenever the current context's id differs from the cached one.
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {0};
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};

// cuCtxGetCurrent and cuCtxGetId, reached through the runtime's driver entry points so that the
// library does not link the driver library itself.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// The unique id of the calling thread's current context, or 0 if it cannot be had.  Called with
// g_noalloc_mu held.
unsigned long long current_context_id() {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) !=
            cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b) {
      cudaGetLastError();
      return 0;
    }
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != 0 || !ctx || g_ctx_get_id(ctx, &id) != 0) return 0;
  return id;
}
}  // namespace

}  // namespace pd

extern "C" pd_status pd_transform_noalloc(const float* D1, int W, int H, int order,
                                          float delta_dt, pd_road_model* fitted, float* D2,
                                          void* stream) {
  using namespace pd;
  if (!D1 || !D2) return PD_ERR_INVALID_ARG;
  if (W < 1 || H < 1 || W > kMaxImage || H > kMaxImage) return PD_ERR_INVALID_ARG;
  if ((long long)W * (long long)H > kNoAllocMaxPixels) return PD_ERR_INVALID_ARG;
  if (order != 1 && order != 2) return PD_ERR_INVALID_ARG;
  if (!isfinite(delta_dt)) return PD_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(fitted) & 7u) return PD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return PD_ERR_UNSUPPORTED;
  void* base = nullptr;
  {
    // set-up once per device (and again after a device reset), on the caller's current device:
    // the device address of the fixed scratch (the array's name in host code is not a device
    // address)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long id = current_context_id();
    if (!g_noalloc_ptr[dev] || id == 0 || id != g_noalloc_ctx[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_transform_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        g_noalloc_ptr[dev] = nullptr;
        return PD_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = p;
      g_noalloc_ctx[dev] = id;
    }
    base = g_noalloc_ptr[dev];
  }
  size_t need = 0;
  carve_size<uint8_t>(need, moments_scratch_bytes(W, H));
  carve_size<int64_t>(need, 46);
  carve_size<pd_road_model>(need, 1);
  carve_size<RoadCoefF>(need, 1);
  carve_size<uint8_t>(need, roll_scratch_bytes());
  if (need > kNoAllocScratchBytes) return PD_ERR_INVALID_ARG;
  Carve c(base);
  void* part = c.take<uint8_t>(moments_scratch_bytes(W, H));
  int64_t* sums = c.take<int64_t>(46);
  pd_road_model* fit = c.take<pd_road_model>(1);
  RoadCoefF* coef = c.take<RoadCoefF>(1);
  double* grid = reinterpret_cast<double*>(c.take<uint8_t>(roll_scratch_bytes()));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // every piece is fully written before it is read, so nothing needs clearing between calls
  launch_moments(s, D1, W, H, part, sums);
  launch_roll_solve(s, sums, order, W, H, fitted ? fitted : fit, coef, grid);
  launch_d2(s, D1, W, H, coef, delta_dt, D2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PD_OK : PD_ERR_CUDA;
}
