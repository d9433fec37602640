// Band-restricted SGM: the matching cost, Eq. (8) aggregation, Eq. (9) winner and the left-right
// check of Sec. II-B, each limited to a per-16x16-tile disparity window (an extension beyond the
// paper: the windows come from the band network in cnn.cu, or from the caller).  Outside its
// window a pixel's L is infinite; the volumes keep the full-range [H][W][D] interleaved layout, and
// only the 16-disparity groups that meet a pixel's window are computed, read and written.
#include "common.cuh"
#include "sgm_body.cuh"

namespace pd {

namespace {

using namespace body;

// Interleaved cost of the in-window groups of P = kCostThreads / (D/16) pixels of row v.
__global__ void __launch_bounds__(kCostThreads) k_cost_band(const uint32_t* __restrict__ cl,
                                                            const uint32_t* __restrict__ cr, int W,
                                                            int D, BandArgs band,
                                                            uint8_t* __restrict__ cost) {
  __shared__ uint32_t sR[kCostThreads + kMaxD];
  const int groups = D >> 4;
  const int P = kCostThreads / groups;
  const int v = blockIdx.y;
  const int u0 = blockIdx.x * P;
  const int base = u0 - D + 1;
  for (int i = threadIdx.x; i < P + D - 1; i += kCostThreads) {
    int x = base + i;
    sR[i] = (x >= 0 && x < W) ? cr[(size_t)v * W + x] : 0u;
  }
  __syncthreads();
  const int u = u0 + threadIdx.x / groups;
  const int g = threadIdx.x % groups;
  if (u >= W) return;
  int lo, hi;
  band_window(band, u, v, D, lo, hi);
  if (group_in_mask(g, lo, hi) == 0) return;
  const uint32_t c0 = cl[(size_t)v * W + u];
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t packed = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int p = 4 * i + b;
      int d = 16 * g + (p >> 1) + ((p & 1) << 3);
      int x = u - d;
      uint32_t c = x >= 0 ? (uint32_t)__popc(c0 ^ sR[x - base]) : (uint32_t)kCensusBits;
      packed |= c << (8 * b);
    }
    w[i] = packed;
  }
  *reinterpret_cast<uint4*>(cost + ((size_t)v * W + u) * D + 16 * g) = make_uint4(w[0], w[1], w[2], w[3]);
}

template <int G>
__global__ void __launch_bounds__(kAggWarps * 32, 6) k_aggregate_band(
    const uint8_t* __restrict__ cost, uint8_t* __restrict__ out, int W, int H, int D, uint32_t dirs,
    uint32_t P1x2, uint32_t K21x2, size_t vol_bytes, BandArgs band) {
  const int r = blockIdx.y;
  const uint32_t code = (dirs >> (4 * r)) & 0xfu;
  const int dx = (int)(code & 3u) - 1, dy = (int)(code >> 2) - 1;
  const int warp = threadIdx.x >> 5;
  agg_warp<G, true>(cost, out + (size_t)r * vol_bytes, W, H, D, dx, dy, P1x2, K21x2,
                    (blockIdx.x * kAggWarps + warp) * (32 / G), warp, band);
}

// 0xFFFF in every u16 half of word j whose disparity lies outside the window.
__device__ __forceinline__ uint32_t out_fill(uint32_t in16, int j) {
  const uint32_t out = ~in16;
  return (((out >> j) & 1u) * 0xffffu) | (((out >> (8 + j)) & 1u) * 0xffff0000u);
}

// Eq. (9) over the windows: P = 128 / G pixels of row v per block, G = D/16 threads per pixel.
// S is marked 0xFFFF outside a pixel's window (in-window sums stay below 8 * (24 + 255)).  The
// parabola needs d* - 1 and d* + 1 inside the window; the right view of column x takes only
// candidates d inside the window of pixel x + d.
__global__ void __launch_bounds__(kWtaThreads) k_wta_band(const uint8_t* __restrict__ vols,
                                                          int ndirs, size_t vol_bytes, int W,
                                                          int D, BandArgs band,
                                                          int16_t* __restrict__ d_int,
                                                          float* __restrict__ dsub,
                                                          uint32_t* __restrict__ rkeys) {
  extern __shared__ uint16_t sS[];  // [P][D]
  const int G = D >> 4;
  const int P = kWtaThreads / G;
  const int v = blockIdx.y;
  const int u0 = blockIdx.x * P;
  const int Peff = min(P, W - u0);
  const int pix = threadIdx.x / G, g = threadIdx.x % G;
  const int u = u0 + pix;
  uint32_t key = 0xffffffffu;
  int lo = 0, hi = D;
  if (pix < Peff) {
    band_window(band, u, v, D, lo, hi);
    const uint32_t in16 = group_in_mask(g, lo, hi);
    uint32_t sw[8], o[8];
    if (in16) {
      load_S_il(vols, ndirs, vol_bytes, ((size_t)v * W + u) * D + 16 * g, sw);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) sw[j] = 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sw[j] |= out_fill(in16, j);
    planar_to_natural(sw, o);
    uint4* row = reinterpret_cast<uint4*>(sS + pix * D + 16 * g);
    row[0] = make_uint4(o[0], o[1], o[2], o[3]);
    row[1] = make_uint4(o[4], o[5], o[6], o[7]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t klo = ((sw[j] & 0xffffu) << 8) | (uint32_t)(16 * g + j);
      uint32_t khi = ((sw[j] >> 16) << 8) | (uint32_t)(16 * g + 8 + j);
      key = min(key, min(klo, khi));
    }
  }
  for (int o = 1; o < G; o <<= 1) key = min(key, __shfl_xor_sync(kFull, key, o, G));
  __syncthreads();
  if (pix < Peff && g == 0) {
    int ds = (int)(key & 0xffu);
    float sub = (float)ds;
    if (ds - 1 >= lo && ds + 1 < hi) {
      int a = sS[pix * D + ds - 1], b = sS[pix * D + ds], c = sS[pix * D + ds + 1];
      int num = a - c;
      int den = 2 * (a + c - 2 * b);
      if (den > 0) sub = (float)ds + (float)num / (float)den;
    }
    d_int[(size_t)v * W + u] = (int16_t)ds;
    dsub[(size_t)v * W + u] = sub;
  }
  for (int i = threadIdx.x; i < Peff + D - 1; i += kWtaThreads) {
    int x = u0 - D + 1 + i;
    if (x < 0) continue;
    int dlo = max(0, u0 - x);
    int dhi = min(D - 1, u0 + Peff - 1 - x);
    uint32_t best = 0xffffffffu;
    for (int d = dlo; d <= dhi; ++d) {
      uint32_t sv = sS[(x + d - u0) * D + d];
      uint32_t k = (sv << 8) | (uint32_t)d;
      best = (sv != 0xffffu && k < best) ? k : best;
    }
    if (best != 0xffffffffu) atomicMin(rkeys + (size_t)v * W + x, best);
  }
}

// Validity over the windows: u >= hi - 1, a right view at u - d*, |d* - d_R| <= lr_tol.
__global__ void k_lr_band(const int16_t* __restrict__ d_int, const float* __restrict__ dsub,
                          const uint32_t* __restrict__ rkeys, const int32_t* __restrict__ kappa,
                          int W, int D, BandArgs band, int lr_tol, float* __restrict__ D1) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y;
  if (u >= W) return;
  const size_t p = (size_t)v * W + u;
  int lo, hi;
  band_window(band, u, v, D, lo, hi);
  const int ds = d_int[p];
  const int xr = u - ds;
  bool valid = u >= hi - 1 && xr >= 0;
  if (valid) {
    const uint32_t rk = rkeys[(size_t)v * W + xr];
    valid = rk != 0xffffffffu && abs(ds - (int)(rk & 0xffu)) <= lr_tol;
  }
  const float d1 = dsub[p] + (float)kappa[v];
  D1[p] = (valid && d1 >= 0.0f) ? d1 : -1.0f;
}

}  // namespace

void launch_cost_band(cudaStream_t s, const uint32_t* cl, const uint32_t* cr, int W, int H, int D,
                      const BandArgs& band, uint8_t* cost) {
  const int P = kCostThreads / (D / 16);
  k_cost_band<<<dim3((W + P - 1) / P, H), kCostThreads, 0, s>>>(cl, cr, W, D, band, cost);
}

void launch_aggregate_band(cudaStream_t s, const uint8_t* cost_il, int W, int H, int D,
                           const DirSet& dirs, int P1, int P2, uint8_t* out, size_t vol_bytes,
                           const BandArgs& band) {
  const int G = D / 16;
  int maxlines = 0;
  for (int r = 0; r < dirs.n; ++r) {
    int n = dirs.dy[r] == 0 ? H : (dirs.dx[r] == 0 ? W : W + H - 1);
    maxlines = n > maxlines ? n : maxlines;
  }
  const int lines_per_block = kAggWarps * (32 / G);
  dim3 grid((maxlines + lines_per_block - 1) / lines_per_block, dirs.n);
  const size_t smem = (size_t)kAggWarps * kStages * 32 * sizeof(uint4);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_aggregate_band<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_aggregate_band<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_aggregate_band<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_aggregate_band<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_set = true;
  }
  const uint32_t P1x2 = (uint32_t)P1 * 0x10001u;
  const uint32_t K21x2 = (uint32_t)(P2 - P1) * 0x10001u;
  uint32_t packed = 0;
  for (int r = 0; r < dirs.n; ++r)
    packed |= ((uint32_t)(dirs.dx[r] + 1) | ((uint32_t)(dirs.dy[r] + 1) << 2)) << (4 * r);
  switch (G) {
    case 2: k_aggregate_band<2><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    case 4: k_aggregate_band<4><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    case 8: k_aggregate_band<8><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    case 16: k_aggregate_band<16><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    default: break;  // the API admits D in {32, 64, 128, 256} only
  }
}

void launch_wta_band(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes, int W,
                     int H, int D, const BandArgs& band, int16_t* d_int, float* dsub,
                     uint32_t* rkeys) {
  const int P = kWtaThreads / (D / 16);
  k_wta_band<<<dim3((W + P - 1) / P, H), kWtaThreads, (size_t)P * D * sizeof(uint16_t), s>>>(
      vols, ndirs, vol_bytes, W, D, band, d_int, dsub, rkeys);
}

void launch_lr_band(cudaStream_t s, const int16_t* d_int, const float* dsub, const uint32_t* rkeys,
                    const int32_t* kappa, int W, int H, int D, const BandArgs& band, int lr_tol,
                    float* D1) {
  k_lr_band<<<dim3((W + 255) / 256, H), 256, 0, s>>>(d_int, dsub, rkeys, kappa, W, D, band, lr_tol,
                                                    D1);
}

}  // namespace pd
