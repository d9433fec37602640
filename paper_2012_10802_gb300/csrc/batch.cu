// Batched Sec. II-A / II-B over many stereo pairs of different sizes and disparity ranges.
//
// One launch per stage covers every pair of a wave: blocks find their pair in a prefix table of
// per-pair block counts and run the same block bodies as the single-pair kernels (sgm_body.cuh),
// so the results are identical to one pd_sgm call per pair.  The aggregation is one persistent
// launch: each warp repeatedly takes the next task (a group of lines of one pair and one
// direction) from an atomic counter over a task list ordered pair by pair, the largest pair
// first: a pair's directions then run together and share its cost rows in L2, and the warps
// flow on to the next pair without a barrier.  Eq. (9) is the exception: its blocks are short and wait on
// DRAM, and the search for the pair (dependent loads before the first volume load) cost them
// 15 % (8.6 against 7.4 ms over 64 mixed pairs), so it runs one launch per pair.  No kernel
// waits on another block.
#include "batch.cuh"
#include "sgm_body.cuh"

namespace pd {

namespace {

using namespace body;

__device__ __forceinline__ int find_pair(const int* __restrict__ starts, int npairs, int b) {
  int lo = 0, hi = npairs - 1;  // largest i with starts[i] <= b
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void k_kappa_b(const BatchPair* __restrict__ pairs, const int* __restrict__ starts,
                          int npairs) {
  const int i = find_pair(starts, npairs, blockIdx.x);
  const BatchPair& p = pairs[i];
  const int v = (blockIdx.x - starts[i]) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (v >= p.H) return;
  kappa_row(p.W, p.H, p.order, p.a0, p.a1, p.a2, p.cs, p.sn, p.delta_pt, p.kappa, v,
            threadIdx.x & 31);
}

// Blocks [0, total) census the left images, [total, 2 total) the row-shifted right images.
__global__ void k_census_b(const BatchPair* __restrict__ pairs, const int* __restrict__ starts,
                           int npairs, int total) {
  const bool right = (int)blockIdx.x >= total;
  const int b = right ? blockIdx.x - total : blockIdx.x;
  const int i = find_pair(starts, npairs, b);
  const BatchPair& p = pairs[i];
  const int t = b - starts[i];
  const int tx = (p.W + kCT_W - 1) / kCT_W;
  census_tile(right ? p.right : p.left, p.W, p.H, p.pitch, right ? p.kappa : nullptr,
              right ? p.cr : p.cl, t % tx, t / tx);
}

__global__ void __launch_bounds__(kCostThreads) k_cost_b(const BatchPair* __restrict__ pairs,
                                                         const int* __restrict__ starts,
                                                         int npairs) {
  const int i = find_pair(starts, npairs, blockIdx.x);
  const BatchPair& p = pairs[i];
  const int b = blockIdx.x - starts[i];
  const int nbx = cost_blocks_per_row(p.W, p.D);
  cost_il_block(p.cl, p.cr, p.W, p.D, p.cost, b % nbx, b / nbx);
}

__global__ void k_fill_b(const BatchPair* __restrict__ pairs, const int* __restrict__ starts,
                         int npairs) {
  const int i = find_pair(starts, npairs, blockIdx.x);
  const BatchPair& p = pairs[i];
  const size_t N = (size_t)p.W * p.H;
  for (size_t k = (size_t)(blockIdx.x - starts[i]) * blockDim.x + threadIdx.x; k < N;
       k += (size_t)(starts[i + 1] - starts[i]) * blockDim.x)
    p.rkeys[k] = 0xffffffffu;
}

// The walk of one task: rows with GH = D/16 lanes of one 16-disparity group each, columns and
// diagonals with GO = D/32 lanes of two groups each (as the single-pair aggregation).
template <int GH, int GO>
__device__ __forceinline__ void batch_walk(const BatchPair& p, uint8_t* dst, int dx, int dy,
                                           int local, uint32_t P1x2, uint32_t K21x2,
                                           uint4* ring) {
  if (dy == 0)
    agg_walk<GH, 1, true>(p.cost, dst, p.W, p.H, p.D, dx, 0, P1x2, K21x2, local * (32 / GH), ring);
  else if (dx == 0)
    agg_walk<GO, 2, true>(p.cost, dst, p.W, p.H, p.D, 0, dy, P1x2, K21x2, local * (32 / GO), ring);
  else
    agg_walk<GO, 2, false>(p.cost, dst, p.W, p.H, p.D, dx, dy, P1x2, K21x2, local * (32 / GO),
                           ring);
}

// Persistent aggregation.  Task t belongs to the segment s with seg[s].first <= t; its lines are
// (t - seg[s].first) * (lines per warp of the segment's direction) onwards.
__global__ void __launch_bounds__(256) k_aggregate_b(const BatchPair* __restrict__ pairs,
                                                     const BatchSegment* __restrict__ seg,
                                                     int nseg, int ntasks,
                                                     unsigned int* __restrict__ counter,
                                                     uint32_t P1x2, uint32_t K21x2) {
  extern __shared__ uint4 s_ring[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint4* ring = s_ring + (size_t)warp * kStages * 32;  // 8 KB per warp
  for (;;) {
    unsigned int t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((int)t >= ntasks) break;
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (seg[mid].first <= (int)t)
        lo = mid;
      else
        hi = mid - 1;
    }
    const BatchSegment sg = seg[lo];
    const BatchPair& p = pairs[sg.pair];
    uint8_t* dst = p.vols + (size_t)sg.r * p.vol_bytes;
    const int local = (int)t - sg.first;
    switch (p.D) {
      case 32: batch_walk<2, 1>(p, dst, sg.dx, sg.dy, local, P1x2, K21x2, ring); break;
      case 64: batch_walk<4, 2>(p, dst, sg.dx, sg.dy, local, P1x2, K21x2, ring); break;
      case 128: batch_walk<8, 4>(p, dst, sg.dx, sg.dy, local, P1x2, K21x2, ring); break;
      default: batch_walk<16, 8>(p, dst, sg.dx, sg.dy, local, P1x2, K21x2, ring); break;
    }
  }
}

// Eq. (9) and the right view for pair i of the wave: one launch per pair, so a block needs no
// search for its pair (the pair's row of the table is one load).
__global__ void __launch_bounds__(kWtaThreads) k_wta_pair(const BatchPair* __restrict__ pairs,
                                                          int i, int ndirs) {
  const BatchPair& p = pairs[i];
  wta_block(p.vols, ndirs, p.vol_bytes, nullptr, p.W, p.D, p.d_int, p.dsub, p.rkeys, blockIdx.x,
            blockIdx.y);
}

__global__ void k_lr_b(const BatchPair* __restrict__ pairs, const int* __restrict__ starts,
                       int npairs, int lr_tol) {
  const int i = find_pair(starts, npairs, blockIdx.x);
  const BatchPair& p = pairs[i];
  const int b = blockIdx.x - starts[i];
  const int nbx = (p.W + 255) / 256;
  lr_block(p.d_int, p.dsub, p.rkeys, p.kappa, p.W, p.D, lr_tol, p.D1, b % nbx, b / nbx);
}

}  // namespace

// Per-pair block counts of each stage (the host builds the prefix tables from these).
void batch_stage_blocks(int W, int H, int D, int counts[kBatchStages]) {
  counts[kStageKappa] = (H + 3) / 4;
  counts[kStageCensus] = ((W + kCT_W - 1) / kCT_W) * ((H + kCT_H - 1) / kCT_H);
  counts[kStageCost] = cost_blocks_per_row(W, D) * H;
  const size_t N = (size_t)W * H;
  counts[kStageFill] = (int)((N + 4095) / 4096);
  counts[kStageLr] = ((W + 255) / 256) * H;
}

int batch_lines_per_warp(int D, int dx, int dy) {
  return dy == 0 ? 32 / (D / 16) : 32 / (D / 32);  // rows: one group per lane; others: two
}

size_t batch_agg_smem(int warps_per_block) {
  return (size_t)warps_per_block * kStages * 32 * sizeof(uint4);
}

void launch_batch_wave(cudaStream_t s, const BatchWaveDev& w, int P1, int P2, int lr_tol,
                       int paths, int agg_warps, int agg_blocks) {
  const uint32_t P1x2 = (uint32_t)P1 * 0x10001u, K21x2 = (uint32_t)(P2 - P1) * 0x10001u;
  const int n = w.npairs;
  k_kappa_b<<<w.total[kStageKappa], 128, 0, s>>>(w.pairs, w.starts[kStageKappa], n);
  k_fill_b<<<w.total[kStageFill], 1024, 0, s>>>(w.pairs, w.starts[kStageFill], n);
  k_census_b<<<2 * w.total[kStageCensus], dim3(kCT_W, kCT_TY), 0, s>>>(w.pairs,
                                                                     w.starts[kStageCensus], n,
                                                                     w.total[kStageCensus]);
  k_cost_b<<<w.total[kStageCost], kCostThreads, 0, s>>>(w.pairs, w.starts[kStageCost], n);
  cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), s);
  const size_t smem = batch_agg_smem(agg_warps);
  raise_smem_limit((const void*)k_aggregate_b, smem);
  k_aggregate_b<<<agg_blocks, agg_warps * 32, smem, s>>>(w.pairs, w.segs, w.nseg, w.ntasks,
                                                         w.counter, P1x2, K21x2);
  for (int i = 0; i < n; ++i) {
    const BatchPair& hp = w.host_pairs[i];
    const int P = kWtaThreads / (hp.D / 16);
    k_wta_pair<<<dim3((hp.W + P - 1) / P, hp.H), kWtaThreads, wta_smem_bytes(hp.D), s>>>(
        w.pairs, i, paths);
  }
  k_lr_b<<<w.total[kStageLr], 256, 0, s>>>(w.pairs, w.starts[kStageLr], n, lr_tol);
}

void launch_batch_aggregate_only(cudaStream_t s, const BatchWaveDev& w, int P1, int P2,
                                 int agg_warps, int agg_blocks) {
  const uint32_t P1x2 = (uint32_t)P1 * 0x10001u, K21x2 = (uint32_t)(P2 - P1) * 0x10001u;
  cudaMemsetAsync(w.counter, 0, sizeof(unsigned int), s);
  const size_t smem = batch_agg_smem(agg_warps);
  raise_smem_limit((const void*)k_aggregate_b, smem);
  k_aggregate_b<<<agg_blocks, agg_warps * 32, smem, s>>>(w.pairs, w.segs, w.nseg, w.ntasks,
                                                         w.counter, P1x2, K21x2);
}

int batch_max_blocks_per_sm(int agg_warps) {
  raise_smem_limit((const void*)k_aggregate_b, batch_agg_smem(agg_warps));
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_aggregate_b, agg_warps * 32,
                                                batch_agg_smem(agg_warps));
  return n;
}

}  // namespace pd
