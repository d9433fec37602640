// Sec. II-A and II-B on the GPU: row shifts (Eq. (6)), the perspective warp, census cost,
// Eq. (8) aggregation, Eq. (9) winner-take-all with sub-pixel step and left-right check, Eq. (10).
//
// Aggregation design: every path of every direction is an independent dynamic-programming line.
// A line is owned by G = D/16 lanes of a warp; each lane keeps 16 disparities as 8 packed u16x2
// words, word j holding (d = 16g + j, d = 16g + 8 + j).  With that pairing the d-1 / d+1
// neighbours of word j are words j-1 / j+1, so the recurrence needs no byte shuffling: per word it
// is one 3-input min and one fused add-min (Hopper/Blackwell DPX instructions) and one three-input
// add that adds the cost and subtracts the previous minimum, and only the two ends of a lane's
// range cross lanes.  The matching cost is computed once per (p, d) into
// a uint8 volume (popcount is a quarter-rate instruction) and every direction reads it with one
// 16-byte asynchronous copy per lane and step into a shared-memory ring, kStages - 1 steps ahead.
#include <cstdio>

#include "common.cuh"
#include "sgm_body.cuh"

namespace pd {

namespace {

using namespace body;

__global__ void k_kappa(int W, int H, int order, double a0, double a1, double a2, double cs,
                        double sn, double delta_pt, int32_t* __restrict__ kappa) {
  int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= H) return;
  kappa_row(W, H, order, a0, a1, a2, cs, sn, delta_pt, kappa, v, threadIdx.x & 31);
}

// Eq. (6) with the road model read from device memory (for instance the previous frame's fit):
// cos and sin of the roll are evaluated on the device.  A model with an order other than 1 or 2
// or a non-finite coefficient gives kappa = 0 (no shift).
__global__ void k_kappa_dev(int W, int H, const pd_road_model* __restrict__ m, double delta_pt,
                            int32_t* __restrict__ kappa) {
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= H) return;
  const pd_road_model mm = *m;
  const bool ok = (mm.order == 1 || mm.order == 2) && isfinite(mm.a[0]) && isfinite(mm.a[1]) &&
                  isfinite(mm.a[2]) && isfinite(mm.roll);
  if (!ok) {
    if ((threadIdx.x & 31) == 0) kappa[v] = 0;
    return;
  }
  double sn, cs;
  sincos(mm.roll, &sn, &cs);
  kappa_row(W, H, mm.order, mm.a[0], mm.a[1], mm.order == 2 ? mm.a[2] : 0.0, cs, sn, delta_pt,
            kappa, v, threadIdx.x & 31);
}

__global__ void k_census(const uint8_t* __restrict__ img, int W, int H, size_t pitch,
                         const int32_t* __restrict__ kappa, uint32_t* __restrict__ codes) {
  census_tile(img, W, H, pitch, kappa, codes, blockIdx.x, blockIdx.y);
}

// Both images of a pair in one launch: blockIdx.z = 0 is the left image, 1 the right image read
// through the row shifts kappa.
__global__ void k_census_pair(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right,
                              int W, int H, size_t pitch, const int32_t* __restrict__ kappa,
                              uint32_t* __restrict__ cl, uint32_t* __restrict__ cr) {
  if (blockIdx.z == 0)
    census_tile(left, W, H, pitch, nullptr, cl, blockIdx.x, blockIdx.y);
  else
    census_tile(right, W, H, pitch, kappa, cr, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(kCostThreads) k_cost_il(const uint32_t* __restrict__ cl,
                                                          const uint32_t* __restrict__ cr, int W,
                                                          int D, uint8_t* __restrict__ cost) {
  cost_il_block(cl, cr, W, D, cost, blockIdx.x, blockIdx.y);
}

// Directions are packed 4 bits each into `dirs` (bits 4r..4r+3 of direction r): dx + 1 in the
// low two bits, dy + 1 in the high two.
template <int G>
__global__ void __launch_bounds__(kAggWarps * 32, 6) k_aggregate(const uint8_t* __restrict__ cost,
                                                                 uint8_t* __restrict__ out, int W,
                                                                 int H, int D, uint32_t dirs,
                                                                 uint32_t P1x2, uint32_t K21x2,
                                                                 size_t vol_bytes) {
  const int r = blockIdx.y;
  const uint32_t code = (dirs >> (4 * r)) & 0xfu;
  const int dx = (int)(code & 3u) - 1, dy = (int)(code >> 2) - 1;
  const int warp = threadIdx.x >> 5;
  agg_warp<G>(cost, out + (size_t)r * vol_bytes, W, H, D, dx, dy, P1x2, K21x2,
              (blockIdx.x * kAggWarps + warp) * (32 / G), warp);
}

__global__ void __launch_bounds__(kWtaThreads) k_wta(const uint8_t* __restrict__ vols, int ndirs,
                                                     size_t vol_bytes,
                                                     const uint16_t* __restrict__ S, int W, int D,
                                                     int16_t* __restrict__ d_int,
                                                     float* __restrict__ dsub,
                                                     uint32_t* __restrict__ rkeys) {
  wta_block(vols, ndirs, vol_bytes, S, W, D, d_int, dsub, rkeys, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(kWtaThreads) k_sum_volumes(const uint8_t* __restrict__ vols,
                                                             int ndirs, size_t vol_bytes,
                                                             size_t n_groups,
                                                             uint16_t* __restrict__ S) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_groups) return;
  uint32_t sw[8], o[8];
  load_S_il(vols, ndirs, vol_bytes, 16 * t, sw);
  planar_to_natural(sw, o);
  uint4* d = reinterpret_cast<uint4*>(S + 16 * t);
  d[0] = make_uint4(o[0], o[1], o[2], o[3]);
  d[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

__global__ void k_lr(const int16_t* __restrict__ d_int, const float* __restrict__ dsub,
                     const uint32_t* __restrict__ rkeys, const int32_t* __restrict__ kappa, int W,
                     int H, int D, int lr_tol, float* __restrict__ D1) {
  lr_block(d_int, dsub, rkeys, kappa, W, D, lr_tol, D1, blockIdx.x, blockIdx.y);
}

__global__ void k_warp(const uint8_t* __restrict__ right, int W, int H, size_t pitch,
                       const int32_t* __restrict__ kappa, uint8_t* __restrict__ out) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  int v = blockIdx.y;
  if (u >= W) return;
  out[(size_t)v * pitch + u] = right[(size_t)v * pitch + clampi(u - kappa[v], 0, W - 1)];
}

// ----------------------------------------------------------------------------- census
// ----------------------------------------------------------------------------- cost
// Natural layout, any 1 <= D <= 256: one thread per (pixel, d).
__global__ void __launch_bounds__(kCostThreads) k_cost_nat(const uint32_t* __restrict__ cl,
                                                           const uint32_t* __restrict__ cr, int W,
                                                           int D, uint8_t* __restrict__ cost) {
  __shared__ uint32_t sR[kCostThreads + kMaxD];
  __shared__ uint32_t sL[kCostThreads];
  const int v = blockIdx.y;
  const size_t row0 = (size_t)v * W * D;
  const size_t first = (size_t)blockIdx.x * kCostThreads;  // first (u, d) index in the row
  const int u0 = (int)(first / D);
  const int ulast = (int)min((first + kCostThreads - 1) / D, (size_t)W - 1);
  const int base = u0 - D + 1;
  for (int i = threadIdx.x; i < ulast - base + 1; i += kCostThreads) {
    int x = base + i;
    sR[i] = (x >= 0 && x < W) ? cr[(size_t)v * W + x] : 0u;
  }
  for (int i = threadIdx.x; i < ulast - u0 + 1; i += kCostThreads) sL[i] = cl[(size_t)v * W + u0 + i];
  __syncthreads();
  size_t idx = first + threadIdx.x;
  if (idx >= (size_t)W * D) return;
  int u = (int)(idx / D), d = (int)(idx % D);
  int x = u - d;
  uint8_t c = x >= 0 ? (uint8_t)__popc(sL[u - u0] ^ sR[x - base]) : (uint8_t)kCensusBits;
  cost[row0 + idx] = c;
}

// Natural <-> interleaved byte order within each 16-disparity group.
__global__ void k_to_interleaved(const uint8_t* __restrict__ in, size_t n_groups,
                                 uint8_t* __restrict__ out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_groups) return;
  uint4 a = reinterpret_cast<const uint4*>(in)[t];
  uint32_t n[4] = {a.x, a.y, a.z, a.w};
  uint32_t o[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    o[i] = __byte_perm(n[i >> 1], n[2 + (i >> 1)], (i & 1) ? 0x7362 : 0x5140);
  reinterpret_cast<uint4*>(out)[t] = make_uint4(o[0], o[1], o[2], o[3]);
}

__global__ void k_to_natural(const uint8_t* __restrict__ in, size_t n_groups,
                             uint8_t* __restrict__ out) {
  size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_groups) return;
  uint4 a = reinterpret_cast<const uint4*>(in)[t];
  uint32_t r[4] = {a.x, a.y, a.z, a.w};
  uint32_t o[4];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    o[i] = __byte_perm(r[2 * i], r[2 * i + 1], 0x6420);
    o[2 + i] = __byte_perm(r[2 * i], r[2 * i + 1], 0x7531);
  }
  reinterpret_cast<uint4*>(out)[t] = make_uint4(o[0], o[1], o[2], o[3]);
}

// ----------------------------------------------------------------------------- Eq. (8)
// ------------------------------------------------------------- volume sums and Eq. (9)
}  // namespace

// ------------------------------------------------------------------------------ launchers

DirSet dir_set(int paths) {
  static const int8_t dx[8] = {1, -1, 0, 0, 1, -1, 1, -1};
  static const int8_t dy[8] = {0, 0, 1, -1, 1, -1, -1, 1};
  DirSet d;
  d.n = paths;
  for (int i = 0; i < 8; ++i) {
    d.dx[i] = dx[i];
    d.dy[i] = dy[i];
  }
  return d;
}

DirSet one_dir(int dx, int dy) {
  DirSet d = dir_set(1);
  d.dx[0] = (int8_t)dx;
  d.dy[0] = (int8_t)dy;
  return d;
}

void launch_kappa(cudaStream_t s, int W, int H, int order, const double a[3], double cs,
                  double sn, double delta_pt, int32_t* kappa) {
  k_kappa<<<(H + 3) / 4, 128, 0, s>>>(W, H, order, a[0], a[1], a[2], cs, sn, delta_pt, kappa);
}

void launch_kappa_dev(cudaStream_t s, int W, int H, const pd_road_model* model, double delta_pt,
                      int32_t* kappa) {
  k_kappa_dev<<<(H + 3) / 4, 128, 0, s>>>(W, H, model, delta_pt, kappa);
}

void launch_warp(cudaStream_t s, const uint8_t* right, int W, int H, size_t pitch,
                 const int32_t* kappa, uint8_t* out) {
  dim3 grid((W + 255) / 256, H);
  k_warp<<<grid, 256, 0, s>>>(right, W, H, pitch, kappa, out);
}

void launch_census(cudaStream_t s, const uint8_t* img, int W, int H, size_t pitch,
                   const int32_t* kappa, uint32_t* codes) {
  dim3 grid((W + kCT_W - 1) / kCT_W, (H + kCT_H - 1) / kCT_H);
  k_census<<<grid, dim3(kCT_W, kCT_TY), 0, s>>>(img, W, H, pitch, kappa, codes);
}

void launch_census_pair(cudaStream_t s, const uint8_t* left, const uint8_t* right, int W, int H,
                        size_t pitch, const int32_t* kappa, uint32_t* cl, uint32_t* cr) {
  dim3 grid((W + kCT_W - 1) / kCT_W, (H + kCT_H - 1) / kCT_H, 2);
  k_census_pair<<<grid, dim3(kCT_W, kCT_TY), 0, s>>>(left, right, W, H, pitch, kappa, cl, cr);
}

void launch_cost(cudaStream_t s, const uint32_t* cl, const uint32_t* cr, int W, int H, int D,
                 int layout, uint8_t* cost) {
  if (layout == 1) {
    dim3 grid(cost_blocks_per_row(W, D), H);
    k_cost_il<<<grid, kCostThreads, 0, s>>>(cl, cr, W, D, cost);
  } else {
    size_t per_row = (size_t)W * D;
    dim3 grid((unsigned)((per_row + kCostThreads - 1) / kCostThreads), H);
    k_cost_nat<<<grid, kCostThreads, 0, s>>>(cl, cr, W, D, cost);
  }
}

void launch_to_interleaved(cudaStream_t s, const uint8_t* natural, size_t n_pix, int D,
                           uint8_t* out) {
  size_t n = n_pix * (size_t)(D / 16);
  k_to_interleaved<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(natural, n, out);
}

void launch_to_natural(cudaStream_t s, const uint8_t* inter, size_t n_pix, int D, uint8_t* out) {
  size_t n = n_pix * (size_t)(D / 16);
  k_to_natural<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(inter, n, out);
}

void launch_aggregate(cudaStream_t s, const uint8_t* cost_il, int W, int H, int D,
                      const DirSet& dirs, int P1, int P2, uint8_t* out, size_t vol_bytes) {
  int G = D / 16;
  int maxlines = 0;
  for (int r = 0; r < dirs.n; ++r) {
    int n = dirs.dy[r] == 0 ? H : (dirs.dx[r] == 0 ? W : W + H - 1);
    maxlines = n > maxlines ? n : maxlines;
  }
  int lines_per_block = kAggWarps * (32 / G);
  dim3 grid((maxlines + lines_per_block - 1) / lines_per_block, dirs.n);
  const size_t smem = (size_t)kAggWarps * kStages * 32 * sizeof(uint4);
  raise_smem_limit((const void*)k_aggregate<2>, smem);
  raise_smem_limit((const void*)k_aggregate<4>, smem);
  raise_smem_limit((const void*)k_aggregate<8>, smem);
  raise_smem_limit((const void*)k_aggregate<16>, smem);
  uint32_t P1x2 = (uint32_t)P1 * 0x10001u;
  uint32_t K21x2 = (uint32_t)(P2 - P1) * 0x10001u;
  uint32_t packed = 0;
  for (int r = 0; r < dirs.n; ++r)
    packed |= ((uint32_t)(dirs.dx[r] + 1) | ((uint32_t)(dirs.dy[r] + 1) << 2)) << (4 * r);
  switch (G) {
    case 2: k_aggregate<2><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes); break;
    case 4: k_aggregate<4><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes); break;
    case 8: k_aggregate<8><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes); break;
    case 16: k_aggregate<16><<<grid, kAggWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes); break;
    default: break;  // the API admits D in {32, 64, 128, 256} only
  }
}

void launch_sum_volumes(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes, int W,
                        int H, int D, uint16_t* S) {
  size_t n = (size_t)W * H * (D / 16);
  k_sum_volumes<<<(unsigned)((n + kWtaThreads - 1) / kWtaThreads), kWtaThreads, 0, s>>>(
      vols, ndirs, vol_bytes, n, S);
}

void launch_wta(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes,
                const uint16_t* S, int W, int H, int D, int16_t* d_int, float* dsub,
                uint32_t* rkeys) {
  int G = D / 16;
  int P = kWtaThreads / G;
  dim3 grid((W + P - 1) / P, H);
  size_t smem = (size_t)P * D * sizeof(uint16_t);
  k_wta<<<grid, kWtaThreads, smem, s>>>(vols, ndirs, vol_bytes, S, W, D, d_int, dsub, rkeys);
}

void launch_lr(cudaStream_t s, const int16_t* d_int, const float* dsub, const uint32_t* rkeys,
               const int32_t* kappa, int W, int H, int D, int lr_tol, float* D1) {
  dim3 grid((W + 255) / 256, H);
  k_lr<<<grid, 256, 0, s>>>(d_int, dsub, rkeys, kappa, W, H, D, lr_tol, D1);
}

}  // namespace pd
