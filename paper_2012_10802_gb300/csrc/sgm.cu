// Sec. II-A and II-B on the GPU: row shifts (Eq. (6)), the perspective warp, census cost,
// Eq. (8) aggregation, Eq. (9) winner-take-all with sub-pixel step and left-right check, Eq. (10).
//
// Aggregation design: every path of every direction is an independent dynamic-programming line,
// walked by a group of lanes of one warp.  Each lane keeps 16 disparities of a line per
// 16-disparity group it owns as 8 packed u16x2 words, word j holding (d = 16g + j,
// d = 16g + 8 + j).  With that pairing the d-1 / d+1 neighbours of word j are words j-1 / j+1, so
// the recurrence needs no byte shuffling: per word it is one 3-input min and one fused add-min
// (DPX instructions) and one three-input add that adds the cost and subtracts the previous
// minimum; only the ends of a group cross to the lane's other group or to the neighbouring lane.
// Rows take one group per lane (D/16 lanes a row, the shortest step for the longest lines),
// columns and diagonals two groups per lane (D/32 lanes a line, fewer shuffles per disparity).
// One persistent launch covers all directions; its warps take line groups from a counter,
// longest first.  The matching cost is computed once per (p, d) into a uint8 volume (popcount is
// a quarter-rate instruction) and every direction reads it through a per-warp shared-memory ring
// of asynchronous copies, several steps ahead.
#include <cstdio>
#include <cstring>

#include <algorithm>
#include <map>
#include <mutex>

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

// Task plan of the persistent aggregation of one frame.  Tasks are groups of lines walked by one
// warp.  The rows of the horizontal directions, the longest lines, sit at every `stride`-th
// position of the task list, so every block draws about the same share of them and they do not
// pile up on a few SMs; the other positions hold the columns, then the diagonals from the middle
// outwards (longest first).
struct AggPlan {
  int n_h, n_v, n_d;           // line groups per direction of each class
  int nht, nvt, ntasks;        // horizontal and vertical tasks; task count
  int stride;                  // horizontal tasks at positions 0, stride, 2 stride, ...
  int nh, nv, nd;              // directions present in each class
  // byte i of each word: direction i of the class as r | (dx + 1) << 3 | (dy + 1) << 5, r its
  // output volume (bytes, not arrays: no local-memory copy of the parameter)
  uint32_t h_code, v_code, d_code;
};

__host__ __device__ __forceinline__ uint32_t dir_code(int r, int dx, int dy) {
  return (uint32_t)r | ((uint32_t)(dx + 1) << 3) | ((uint32_t)(dy + 1) << 5);
}

// Group index of rank r in middle-out order over n groups: the middle one, then alternately one
// below and one above, then the rest of the longer side.
__device__ __forceinline__ int middle_out(int r, int n) {
  const int mid = (n - 1) >> 1;
  if (r == 0) return mid;
  const int below = mid, above = n - 1 - mid;
  const int both = min(below, above);
  const int i = r - 1;
  if (i < 2 * both) return (i & 1) ? mid + 1 + (i >> 1) : mid - 1 - (i >> 1);
  const int j = i - 2 * both;
  return below > above ? mid - 1 - both - j : mid + 1 + both + j;
}

constexpr int kAggPWarps = 4;               // warps per block of the persistent aggregation
// The walkers of lines shorter than the rows sleep this long per step, so that the rows (the
// critical path of a landscape frame) that share their schedulers issue sooner: diagonals
// always, columns when H < W.  At 720p, D = 128 the aggregation took 0.328-0.330 ms with 16-48
// ns against 0.338 ms with none, and 0.346 ms with 200 ns.
constexpr unsigned kAggYieldNs = 32;
constexpr int kAggPRingUint4 = 512;         // 8 KB ring per warp

// Persistent aggregation of Eq. (8) over all directions of a frame.  Each warp repeatedly takes
// the next task from the counter; columns and diagonals are walked with GO = D/32 lanes of two
// 16-disparity groups each; rows with GH lanes, of one group each (D/16 lanes), or of half a group
// each when HALF (D/8 lanes, used at D = 32, where it measured faster; at D = 128 it measured
// slower).
template <int GH, int GO, bool HALF>
__global__ void __launch_bounds__(kAggPWarps * 32) k_aggregate_p(
    const uint8_t* __restrict__ cost, uint8_t* __restrict__ out, int W, int H, int D,
    AggPlan plan, uint32_t P1x2, uint32_t K21x2, size_t vol_bytes,
    unsigned int* __restrict__ counter) {
  extern __shared__ uint4 s_ring_p[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4* ring = s_ring_p + warp * kAggPRingUint4;
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(kFull, t, 0);
    if ((int)t >= plan.ntasks) break;
    const int ti = (int)t;
    uint32_t code;
    int k, cls;
    const int hq = ti / plan.stride;
    if (ti % plan.stride == 0 && hq < plan.nht) {  // a horizontal task
      cls = 0;
      code = plan.h_code >> (8 * (hq % plan.nh));
      k = hq / plan.nh;
    } else {
      const int j = ti - min(plan.nht, hq + 1);  // the other tasks in their own order
      if (j < plan.nvt) {
        cls = 1;
        code = plan.v_code >> (8 * (j % plan.nv));
        k = j / plan.nv;
      } else {
        cls = 2;
        const int i = j - plan.nvt;
        code = plan.d_code >> (8 * (i % plan.nd));
        k = middle_out(i / plan.nd, plan.n_d);
      }
    }
    uint8_t* dst = out + (size_t)(code & 7u) * vol_bytes;
    const int dx = (int)((code >> 3) & 3u) - 1, dy = (int)((code >> 5) & 3u) - 1;
    if (cls == 0) {
      if constexpr (HALF)
        agg_row_half<GH>(cost, dst, W, H, D, dx, P1x2, K21x2, k * (32 / GH), ring);
      else
        agg_walk<GH, 1, true>(cost, dst, W, H, D, dx, 0, P1x2, K21x2, k * (32 / GH), ring);
    }
    else if (cls == 1) {
      if (H < W)  // columns shorter than the rows
        agg_walk<GO, 2, true, kAggYieldNs>(cost, dst, W, H, D, 0, dy, P1x2, K21x2, k * (32 / GO),
                                           ring);
      else
        agg_walk<GO, 2, true>(cost, dst, W, H, D, 0, dy, P1x2, K21x2, k * (32 / GO), ring);
    }
    else
      agg_walk<GO, 2, false, kAggYieldNs>(cost, dst, W, H, D, dx, dy, P1x2, K21x2, k * (32 / GO),
                                          ring);
  }
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

namespace {
template <int GH, int GO, bool HALF>
void launch_agg_p(cudaStream_t s, const uint8_t* cost, uint8_t* out, int W, int H, int D,
                  const AggPlan& plan, uint32_t P1x2, uint32_t K21x2, size_t vol_bytes,
                  unsigned int* counter) {
  const size_t smem = (size_t)kAggPWarps * kAggPRingUint4 * sizeof(uint4);
  const void* f = (const void*)k_aggregate_p<GH, GO, HALF>;
  raise_smem_limit(f, smem);
  // one wave of resident blocks: per device, the SM count times the blocks an SM holds
  static std::mutex mu;
  static std::map<int, int> blocks;
  int dev = 0;
  cudaGetDevice(&dev);
  int nb = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = blocks.find(dev);
    if (it == blocks.end()) {
      int sms = 0, per = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_aggregate_p<GH, GO, HALF>,
                                                    kAggPWarps * 32, smem);
      nb = std::max(1, sms * std::max(1, per));
      blocks[dev] = nb;
    } else {
      nb = it->second;
    }
  }
  nb = std::min(nb, (plan.ntasks + kAggPWarps - 1) / kAggPWarps);
  cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
  k_aggregate_p<GH, GO, HALF><<<nb, kAggPWarps * 32, smem, s>>>(cost, out, W, H, D, plan, P1x2,
                                                             K21x2, vol_bytes, counter);
}
}  // namespace

void launch_aggregate_p(cudaStream_t s, const uint8_t* cost_il, int W, int H, int D,
                        const DirSet& dirs, int P1, int P2, uint8_t* out, size_t vol_bytes,
                        unsigned int* counter) {
  AggPlan plan;
  memset(&plan, 0, sizeof(plan));
  const int GH = D == 32 ? D / 8 : D / 16, GO = D / 32;
  const int lh = 32 / GH, lo = 32 / GO;
  plan.n_h = (H + lh - 1) / lh;
  plan.n_v = (W + lo - 1) / lo;
  plan.n_d = (W + H - 1 + lo - 1) / lo;
  for (int r = 0; r < dirs.n; ++r) {
    const int dx = dirs.dx[r], dy = dirs.dy[r];
    if (dy == 0)
      plan.h_code |= dir_code(r, dx, dy) << (8 * plan.nh++);
    else if (dx == 0)
      plan.v_code |= dir_code(r, dx, dy) << (8 * plan.nv++);
    else
      plan.d_code |= dir_code(r, dx, dy) << (8 * plan.nd++);
  }
  plan.nht = plan.nh * plan.n_h;
  plan.nvt = plan.nv * plan.n_v;
  plan.ntasks = plan.nht + plan.nvt + plan.nd * plan.n_d;
  // the last horizontal task must sit inside the list: stride * (nht - 1) < ntasks
  plan.stride = plan.nht > 1 ? std::max(1, (plan.ntasks - 1) / (plan.nht - 1)) : 1;
  const uint32_t P1x2 = (uint32_t)P1 * 0x10001u;
  const uint32_t K21x2 = (uint32_t)(P2 - P1) * 0x10001u;
  switch (D) {
    case 32: launch_agg_p<4, 1, true>(s, cost_il, out, W, H, D, plan, P1x2, K21x2, vol_bytes, counter); break;
    case 64: launch_agg_p<4, 2, false>(s, cost_il, out, W, H, D, plan, P1x2, K21x2, vol_bytes, counter); break;
    case 128: launch_agg_p<8, 4, false>(s, cost_il, out, W, H, D, plan, P1x2, K21x2, vol_bytes, counter); break;
    case 256: launch_agg_p<16, 8, false>(s, cost_il, out, W, H, D, plan, P1x2, K21x2, vol_bytes, counter); break;
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
  const size_t smem = wta_smem_bytes(D);
  k_wta<<<grid, kWtaThreads, smem, s>>>(vols, ndirs, vol_bytes, S, W, D, d_int, dsub, rkeys);
}

void launch_lr(cudaStream_t s, const int16_t* d_int, const float* dsub, const uint32_t* rkeys,
               const int32_t* kappa, int W, int H, int D, int lr_tol, float* D1) {
  dim3 grid((W + 255) / 256, H);
  k_lr<<<grid, 256, 0, s>>>(d_int, dsub, rkeys, kappa, W, H, D, lr_tol, D1);
}

}  // namespace pd
