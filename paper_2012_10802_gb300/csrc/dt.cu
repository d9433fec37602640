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

constexpr int kGridN = 3001;
constexpr double kGridStep = 1.7453292519943295e-04;  // 0.01 degree
constexpr int kGridThreads = 128;
constexpr int kRefineThreads = 128;

__device__ void load_moments(const int64_t* __restrict__ sums, MomD& M) {
  int k = 1;  // skip the count; m[0][0] is the same number
  for (int i = 0; i <= 4; ++i)
    for (int j = 0; i + j <= 4; ++j, ++k)
      M.m[i][j] = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
  for (int i = 0; i <= 2; ++i)
    for (int j = 0; i + j <= 2; ++j, ++k)
      M.q[i][j] = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
  M.qq = i128_to_double((unsigned long long)sums[2 * k], (long long)sums[2 * k + 1]);
}

__device__ double coord_scale_d(int W, int H) {
  int mmax = W > H ? W : H;
  double sc = 1.0;
  while (sc < (double)mmax) sc *= 2.0;
  return sc;
}

// E0min on the 0.01-degree grid over +-15 degrees, one angle per thread across many SMs.
__global__ void __launch_bounds__(kGridThreads) k_roll_grid(const int64_t* __restrict__ sums,
                                                            int order, int W, int H,
                                                            double* __restrict__ E) {
  __shared__ MomD M;
  if (threadIdx.x == 0) load_moments(sums, M);
  __syncthreads();
  int k = blockIdx.x * kGridThreads + threadIdx.x;
  if (k >= kGridN) return;
  double beta[3];
  E[k] = e0min_d(M, order, coord_scale_d(W, H), (double)(k - kGridN / 2) * kGridStep, beta);
}

// Block argmin of (value, index), smallest index on ties.  Returns the winner to every thread.
__device__ void block_argmin(double e, int k, double* sE, int* sK, double& be, int& bk) {
  sE[threadIdx.x] = e;
  sK[threadIdx.x] = k;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
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
  be = sE[0];
  bk = sK[0];
  __syncthreads();
}

// Refines the roll (order 2: around the best grid angle, by rounds of kRefineThreads angles that
// shrink the bracket about 64x each, to below 1e-12 rad; order 1: the least-squares plane in
// closed form), solves Eq. (11) for the coefficients and writes the model and its float form.
__global__ void __launch_bounds__(kRefineThreads) k_roll_refine(const int64_t* __restrict__ sums,
                                                                const double* __restrict__ E,
                                                                int order, int W, int H,
                                                                pd_road_model* fitted,
                                                                RoadCoefF* coef) {
  __shared__ MomD M;
  __shared__ double sE[kRefineThreads];
  __shared__ int sK[kRefineThreads];
  __shared__ double sPhi;
  if (threadIdx.x == 0) load_moments(sums, M);
  __syncthreads();
  const double sc = coord_scale_d(W, H);
  double beta[3];
  if (order == 1) {
    if (threadIdx.x == 0) {
      double phi = 0.0;
      double s1 = sc, s2 = sc * sc;
      double A[3][3] = {{M.m[0][0], M.m[0][1] / s1, M.m[1][0] / s1},
                        {M.m[0][1] / s1, M.m[0][2] / s2, M.m[1][1] / s2},
                        {M.m[1][0] / s1, M.m[1][1] / s2, M.m[2][0] / s2}};
      double b[3] = {M.q[0][0] / 1024.0, M.q[0][1] / s1 / 1024.0, M.q[1][0] / s1 / 1024.0};
      double x[3] = {0, 0, 0};
      if (spd_solve_d(3, A, b, x) == 0 && x[1] != 0.0) phi = atan(-x[2] / x[1]);
      sPhi = phi;
    }
  } else {
    double be = INFINITY;
    int bk = kGridN;
    for (int k = threadIdx.x; k < kGridN; k += kRefineThreads) {
      double e = E[k];
      if (e < be) {
        be = e;
        bk = k;
      }
    }
    block_argmin(be, bk, sE, sK, be, bk);
    int best = bk < kGridN ? bk : 0;
    int klo = best > 0 ? best - 1 : 0;
    int khi = best < kGridN - 1 ? best + 1 : kGridN - 1;
    double a = (double)(klo - kGridN / 2) * kGridStep;
    double b = (double)(khi - kGridN / 2) * kGridStep;
    double phi = 0.5 * (a + b);
    for (int round = 0; round < 12 && (b - a) > 1e-12; ++round) {
      const double h = (b - a) / (double)(kRefineThreads + 1);
      double x = a + h * (double)(threadIdx.x + 1);
      double e = e0min_d(M, order, sc, x, beta);
      int t;
      block_argmin(e, threadIdx.x, sE, sK, e, t);
      phi = a + h * (double)(t + 1);
      double na = a + h * (double)t;
      double nb = a + h * (double)(t + 2);
      a = na;
      b = nb;
    }
    if (threadIdx.x == 0) sPhi = phi;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double phi = sPhi;
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

size_t roll_scratch_bytes() { return kGridN * sizeof(double); }

void launch_moments(cudaStream_t s, const float* D1, int W, int H, void* scratch, int64_t* sums) {
  int nblocks = (int)(((size_t)W * H + kMomPixPerBlock - 1) / kMomPixPerBlock);
  long long* partial = static_cast<long long*>(scratch);
  k_moments_partial<<<nblocks, kMomThreads, 0, s>>>(D1, W, H, partial);
  k_moments_final<<<1, kNumSums * 32, 0, s>>>(partial, nblocks, sums);
}

int launch_roll_solve(cudaStream_t s, const int64_t* sums, int order, int W, int H,
                      pd_road_model* fitted, RoadCoefF* coef, double* grid_scratch) {
  int n = 1;
  if (order == 2) {
    k_roll_grid<<<(kGridN + kGridThreads - 1) / kGridThreads, kGridThreads, 0, s>>>(
        sums, order, W, H, grid_scratch);
    ++n;
  }
  k_roll_refine<<<1, kRefineThreads, 0, s>>>(sums, grid_scratch, order, W, H, fitted, coef);
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
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) return PD_ERR_UNSUPPORTED;
  void* base = nullptr;
  {
    // one-time set-up per device, on the caller's current device: the device address of the
    // fixed scratch (the array's name in host code is not a device address)
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_transform_scratch);
      if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return PD_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = p;
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
