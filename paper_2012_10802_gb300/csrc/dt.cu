// Sec. II-C on the GPU: exact moment sums of the road disparities, the roll / road-model fit of
// Eqs. (11)-(12) in one thread block (no host round trip), and the Eq. (13) transformation.
#include "common.cuh"

namespace pd {

namespace {

constexpr int kMomThreads = 256;
constexpr int kMomPixPerBlock = 16384;  // keeps every per-block int64 partial exact (W, H <= 4096)
constexpr int kNumSums = 23;

__device__ __forceinline__ long long warp_sum_ll(long long x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Per-block int64 partial sums: count, sum u~^i v~^j (i + j <= 4), sum q u~^i v~^j (i + j <= 2),
// sum q^2 with q = rint(1024 D1), u~ = 2u - (W-1), v~ = 2v - (H-1), over pixels with D1 >= 0.
__global__ void __launch_bounds__(kMomThreads) k_moments_partial(const float* __restrict__ D1,
                                                                 int W, int H,
                                                                 long long* __restrict__ partial) {
  long long acc[kNumSums];
#pragma unroll
  for (int i = 0; i < kNumSums; ++i) acc[i] = 0;
  const size_t N = (size_t)W * H;
  const size_t start = (size_t)blockIdx.x * kMomPixPerBlock;
  const size_t end = min(start + (size_t)kMomPixPerBlock, N);
  for (size_t p = start + threadIdx.x; p < end; p += kMomThreads) {
    float d = D1[p];
    if (!(d >= 0.0f)) continue;
    long long q = __double2ll_rn((double)d * 1024.0);
    int u = (int)(p % W), v = (int)(p / W);
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

// Sums the block partials exactly in 128 bits; writes (low, high) 64-bit pairs.
__global__ void k_moments_final(const long long* __restrict__ partial, int nblocks,
                                int64_t* __restrict__ sums) {
  int i = threadIdx.x;
  if (i >= kNumSums) return;
  __int128 s = 0;
  for (int b = 0; b < nblocks; ++b) s += (__int128)partial[(size_t)b * kNumSums + i];
  sums[2 * i] = (int64_t)(unsigned long long)s;
  sums[2 * i + 1] = (int64_t)(s >> 64);
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

// Eq. (12) at one roll angle for a model of the given order; beta gets the Eq. (11) solution in
// the basis 1, w_s, w_s^2 with w_s = (v~ cos(phi) - u~ sin(phi)) / sc.
__device__ double e0min_d(const MomD& M, int order, double sc, double phi, double beta[3]) {
  int n = order + 1;
  double cs = cos(phi) / sc;
  double ss = -sin(phi) / sc;
  double pc[5], ps[5];
  pc[0] = 1.0;
  ps[0] = 1.0;
  for (int i = 1; i < 5; ++i) {
    pc[i] = pc[i - 1] * cs;
    ps[i] = ps[i - 1] * ss;
  }
  double sw[5] = {0, 0, 0, 0, 0}, sqw[3] = {0, 0, 0};
  for (int k = 0; k <= 2 * order; ++k) {
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += kBinomD[k][j] * pc[j] * ps[k - j] * M.m[k - j][j];
    sw[k] = acc;
  }
  for (int k = 0; k <= order; ++k) {
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += kBinomD[k][j] * pc[j] * ps[k - j] * M.q[k - j][j];
    sqw[k] = acc / 1024.0;
  }
  double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, b[3] = {0, 0, 0}, x[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    b[i] = sqw[i];
    for (int k = 0; k < n; ++k) A[i][k] = sw[i + k];
  }
  if (spd_solve_d(n, A, b, x) != 0) {
    beta[0] = beta[1] = beta[2] = 0.0;
    return INFINITY;
  }
  double dd = M.qq / 1048576.0;
  double fit = 0.0;
  for (int i = 0; i < n; ++i) fit += b[i] * x[i];
  for (int i = 0; i < 3; ++i) beta[i] = i < n ? x[i] : 0.0;
  return dd - fit;
}

constexpr int kRollThreads = 256;
constexpr int kGridN = 3001;
constexpr double kGridStep = 1.7453292519943295e-04;  // 0.01 degree

// One block: reads the exact sums, finds phi (closed form for order 1; 0.01-degree grid over
// +-15 degrees and golden-section refinement for order 2), solves Eq. (11) for the coefficients,
// and writes the model plus its float coefficients for the transform kernel.
__global__ void __launch_bounds__(kRollThreads) k_roll_solve(const int64_t* __restrict__ sums,
                                                             int order, int W, int H,
                                                             pd_road_model* fitted,
                                                             RoadCoefF* coef) {
  __shared__ MomD M;
  __shared__ double sE[kRollThreads];
  __shared__ int sK[kRollThreads];
  if (threadIdx.x == 0) {
    int k = 1;  // skip the count; m[0][0] is the same number
    for (int i = 0; i <= 4; ++i)
      for (int j = 0; i + j <= 4; ++j, ++k)
        M.m[i][j] = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
    for (int i = 0; i <= 2; ++i)
      for (int j = 0; i + j <= 2; ++j, ++k)
        M.q[i][j] = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
    M.qq = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
  }
  __syncthreads();
  int mmax = W > H ? W : H;
  double sc = 1.0;
  while (sc < (double)mmax) sc *= 2.0;
  double beta[3];
  double phi = 0.0;
  if (order == 1) {
    if (threadIdx.x == 0) {
      double s1 = sc, s2 = sc * sc;
      double A[3][3] = {{M.m[0][0], M.m[0][1] / s1, M.m[1][0] / s1},
                        {M.m[0][1] / s1, M.m[0][2] / s2, M.m[1][1] / s2},
                        {M.m[1][0] / s1, M.m[1][1] / s2, M.m[2][0] / s2}};
      double b[3] = {M.q[0][0] / 1024.0, M.q[0][1] / s1 / 1024.0, M.q[1][0] / s1 / 1024.0};
      double x[3] = {0, 0, 0};
      if (spd_solve_d(3, A, b, x) == 0 && x[1] != 0.0) phi = atan(-x[2] / x[1]);
    }
  } else {
    double bestE = INFINITY;
    int bestK = kGridN;
    for (int k = threadIdx.x; k < kGridN; k += kRollThreads) {
      double e = e0min_d(M, order, sc, (double)(k - kGridN / 2) * kGridStep, beta);
      if (e < bestE) {
        bestE = e;
        bestK = k;
      }
    }
    sE[threadIdx.x] = bestE;
    sK[threadIdx.x] = bestK;
    __syncthreads();
    for (int s = kRollThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double eo = sE[threadIdx.x + s];
        int ko = sK[threadIdx.x + s];
        if (eo < sE[threadIdx.x] || (eo == sE[threadIdx.x] && ko < sK[threadIdx.x])) {
          sE[threadIdx.x] = eo;
          sK[threadIdx.x] = ko;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      int best = sK[0] < kGridN ? sK[0] : 0;
      int klo = best > 0 ? best - 1 : 0;
      int khi = best < kGridN - 1 ? best + 1 : kGridN - 1;
      double a = (double)(klo - kGridN / 2) * kGridStep;
      double b = (double)(khi - kGridN / 2) * kGridStep;
      const double g = 0.6180339887498949;
      double x1 = b - g * (b - a), x2 = a + g * (b - a);
      double f1 = e0min_d(M, order, sc, x1, beta);
      double f2 = e0min_d(M, order, sc, x2, beta);
      for (int it = 0; it < 200 && (b - a) > 1e-12; ++it) {
        if (f1 <= f2) {
          b = x2;
          x2 = x1;
          f2 = f1;
          x1 = b - g * (b - a);
          f1 = e0min_d(M, order, sc, x1, beta);
        } else {
          a = x1;
          x1 = x2;
          f1 = f2;
          x2 = a + g * (b - a);
          f2 = e0min_d(M, order, sc, x2, beta);
        }
      }
      phi = 0.5 * (a + b);
    }
  }
  if (threadIdx.x != 0) return;
  e0min_d(M, order, sc, phi, beta);
  double k = 2.0 / sc;
  double vc = (double)(H - 1) * 0.5;
  double b0 = beta[0], b1 = beta[1], b2 = order == 2 ? beta[2] : 0.0;
  pd_road_model out;
  out.order = order;
  out.roll = phi;
  out.a[2] = b2 * k * k;
  out.a[1] = b1 * k - 2.0 * b2 * k * k * vc;
  out.a[0] = b0 - b1 * k * vc + b2 * k * k * vc * vc;
  if (fitted) *fitted = out;
  RoadCoefF cf;
  cf.c = (float)cos(phi);
  cf.s = (float)sin(phi);
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
    float t1 = ((float)v - c.vc) * c.c;
    float t2 = ((float)u - c.uc) * c.s;
    float vp = (t1 - t2) + c.vc;
    float f = (c.a0 + c.a1 * vp) + c.a2 * (vp * vp);
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

void launch_moments(cudaStream_t s, const float* D1, int W, int H, void* scratch, int64_t* sums) {
  int nblocks = (int)(((size_t)W * H + kMomPixPerBlock - 1) / kMomPixPerBlock);
  long long* partial = static_cast<long long*>(scratch);
  k_moments_partial<<<nblocks, kMomThreads, 0, s>>>(D1, W, H, partial);
  k_moments_final<<<1, 32, 0, s>>>(partial, nblocks, sums);
}

void launch_roll_solve(cudaStream_t s, const int64_t* sums, int order, int W, int H,
                       pd_road_model* fitted, RoadCoefF* coef) {
  k_roll_solve<<<1, kRollThreads, 0, s>>>(sums, order, W, H, fitted, coef);
}

void launch_d2(cudaStream_t s, const float* D1, int W, int H, const RoadCoefF* coef,
               float delta_dt, float* D2) {
  dim3 grid((W + 255) / 256, H);
  k_d2<<<grid, 256, 0, s>>>(D1, W, H, coef, delta_dt, D2);
}

}  // namespace pd
