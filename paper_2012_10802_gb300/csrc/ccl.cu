// Sec. II-E: connected components of the pothole mask ("different potholes are labeled using
// connect component labeling"), their statistics, and the fake-pothole rule of Sec. III-B
// (detections at a corner of the image or made of a single superpixel are fake).
//
// Labelling is union-find over the pixel grid: every mask pixel starts as its own root, each
// pixel merges with its already-visited neighbours (left, up, and the two upper diagonals for
// 8-connectivity) by attaching the larger root under the smaller one with atomicMin, and a
// final pass points every pixel at its root.  The root of a component is therefore its smallest
// raster index.  The merges run first inside 16 x 16 tiles in shared memory and then only
// across tile borders in global memory, so a large pothole does not funnel every pixel's atomic
// into one root.  Components are numbered in the raster order of their roots (block counts, one
// scan, per-block ranks), so the numbering does not depend on thread timing.  Every find and
// merge loop has an iteration limit; exceeding it sets an error flag (reported as a component
// count of -1) instead of looping on.
#include <limits.h>

#include "common.cuh"

namespace pd {

namespace {

constexpr int kCclThreads = 1024;
static_assert(sizeof(pd_component) == 56, "pd_component layout");
constexpr int kLoopCap = 1 << 22;

__device__ __forceinline__ int find_root(const int32_t* L, int x, int* err) {
  for (int it = 0; it < kLoopCap; ++it) {
    const int y = __ldcg(L + x);  // parents change under other threads: read through L2
    if (y == x) return x;
    x = y;
  }
  atomicExch(err, 1);
  return x;
}

__device__ __forceinline__ void merge(int32_t* L, int a, int b, int* err) {
  for (int it = 0; it < kLoopCap; ++it) {
    a = find_root(L, a, err);
    b = find_root(L, b, err);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(L + b, a);  // attach root b under the smaller root a
    if (old == b) return;
    b = old;  // b stopped being a root meanwhile: retry from its new parent
  }
  atomicExch(err, 1);
}

// Running statistics of one component (atomics from the statistics pass).
struct CompAcc {
  int count, umin, vmin, umax, vmax, sp_first, multi, pad;
  unsigned long long sum_u, sum_v;
};

__device__ void acc_init_one(CompAcc* out) {
  CompAcc a;
  a.count = 0;
  a.umin = INT_MAX;
  a.vmin = INT_MAX;
  a.umax = -1;
  a.vmax = -1;
  a.sp_first = INT_MIN;
  a.multi = 0;
  a.pad = 0;
  a.sum_u = 0;
  a.sum_v = 0;
  *out = a;
}

// Labels inside one 16 x 16 tile, in shared memory: the same union-find on tile-local indices
// (local raster order within a tile agrees with the global raster order of its pixels), then
// every mask pixel gets the global raster index of its tile-local root.  Block 0 also clears the
// flags (component total and error) and, spread over all blocks, the component statistics for the
// later kernels.
constexpr int kTile = 16;

__device__ __forceinline__ int find_local(const int* s, int x) {
  const volatile int* vs = s;  // parents change under other threads of the block
  for (int it = 0; it < kTile * kTile; ++it) {
    const int y = vs[x];
    if (y == x) return x;
    x = y;
  }
  return x;
}

__device__ __forceinline__ void merge_local(int* s, int a, int b) {
  for (int it = 0; it < 4 * kTile * kTile; ++it) {
    a = find_local(s, a);
    b = find_local(s, b);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(s + b, a);
    if (old == b) return;
    b = old;
  }
}

__global__ void __launch_bounds__(kTile * kTile) k_ccl_local(const uint8_t* __restrict__ mask,
                                                             int W, int H, int conn,
                                                             int32_t* __restrict__ L, int* flags,
                                                             CompAcc* __restrict__ acc,
                                                             int max_comps) {
  __shared__ int s[kTile * kTile];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int u = blockIdx.x * kTile + tx, v = blockIdx.y * kTile + ty;
  const bool in = u < W && v < H;
  const bool m = in && mask[(size_t)v * W + u];
  const int me = threadIdx.x;
  s[me] = m ? me : -1;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < 2) flags[threadIdx.x] = 0;
  {
    const int nthreads = gridDim.x * gridDim.y * kTile * kTile;
    for (int k = (blockIdx.y * gridDim.x + blockIdx.x) * kTile * kTile + threadIdx.x;
         k < max_comps; k += nthreads)
      acc_init_one(acc + k);
  }
  __syncthreads();
  if (m) {
    if (tx > 0 && s[me - 1] >= 0) merge_local(s, me, me - 1);
    if (ty > 0) {
      if (s[me - kTile] >= 0) merge_local(s, me, me - kTile);
      if (conn == 8) {
        if (tx > 0 && s[me - kTile - 1] >= 0) merge_local(s, me, me - kTile - 1);
        if (tx < kTile - 1 && s[me - kTile + 1] >= 0) merge_local(s, me, me - kTile + 1);
      }
    }
  }
  __syncthreads();
  if (!in) return;
  int root = -1;
  if (m) {
    const int r = find_local(s, me);
    root = (blockIdx.y * kTile + r / kTile) * W + blockIdx.x * kTile + r % kTile;
  }
  L[(size_t)v * W + u] = root;
}

// Unions across tile borders: each mask pixel with an earlier neighbour (left, up, up-left,
// up-right) in another tile merges with it through the global union-find.
__global__ void __launch_bounds__(kTile * kTile) k_ccl_border(const uint8_t* __restrict__ mask,
                                                              int W, int H, int conn, int32_t* L,
                                                              int* err) {
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  if (tx != 0 && ty != 0 && tx != kTile - 1) return;  // interior pixels were merged locally
  const int u = blockIdx.x * kTile + tx, v = blockIdx.y * kTile + ty;
  if (u >= W || v >= H) return;
  const int p = v * W + u;
  if (!mask[p]) return;
  if (tx == 0 && u > 0 && mask[p - 1]) merge(L, p, p - 1, err);
  if (ty == 0 && v > 0 && mask[p - W]) merge(L, p, p - W, err);
  if (conn == 8 && v > 0) {
    if ((tx == 0 || ty == 0) && u > 0 && mask[p - W - 1]) merge(L, p, p - W - 1, err);
    if ((ty == 0 || tx == kTile - 1) && u < W - 1 && mask[p - W + 1]) merge(L, p, p - W + 1, err);
  }
}

// Every mask pixel points at its root; roots are counted per block of kCclThreads pixels.
__global__ void __launch_bounds__(kCclThreads) k_ccl_flatten_count(int32_t* L, int n, int* err,
                                                                   int* __restrict__ counts) {
  const int p = blockIdx.x * kCclThreads + threadIdx.x;
  bool root = false;
  if (p < n) {
    const int r = __ldcg(L + p);
    if (r >= 0) {
      root = r == p;
      if (!root) L[p] = find_root(L, p, err);
    }
  }
  const int c = __syncthreads_count(root);
  if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of the block counts in one block; total number of components in *total.
__global__ void __launch_bounds__(kCclThreads) k_ccl_scan(const int* __restrict__ counts, int nb,
                                                          int* __restrict__ offsets,
                                                          int* __restrict__ total) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < nb; base += kCclThreads) {
    const int i = base + threadIdx.x;
    const int x = i < nb ? counts[i] : 0;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
      int ws = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += y;
      }
      warp_sums[lane] = ws;  // inclusive over warps
    }
    __syncthreads();
    const int before = (w > 0 ? warp_sums[w - 1] : 0) + incl - x;
    if (i < nb) offsets[i] = carry + before;
    __syncthreads();
    if (threadIdx.x == kCclThreads - 1) carry += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Component number of every root (raster order of roots) and the root of every component.
__global__ void __launch_bounds__(kCclThreads) k_ccl_ids(const int32_t* __restrict__ L, int n,
                                                         const int* __restrict__ offsets,
                                                         int32_t* __restrict__ cid,
                                                         int32_t* __restrict__ root_of,
                                                         int max_comps) {
  __shared__ int warp_cnt[32];
  const int p = blockIdx.x * kCclThreads + threadIdx.x;
  const bool root = p < n && L[p] == p;
  const unsigned bal = __ballot_sync(0xffffffffu, root);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_cnt[w] = __popc(bal);
  __syncthreads();
  if (root) {
    int r = __popc(bal & ((1u << lane) - 1u));
    for (int k = 0; k < w; ++k) r += warp_cnt[k];
    const int id = offsets[blockIdx.x] + r;
    cid[p] = id;
    if (id < max_comps) root_of[id] = p;
  }
}

// Per mask pixel: the output label (component number) and its share of the statistics.
__global__ void k_ccl_stats(const int32_t* __restrict__ L, const int32_t* __restrict__ cid,
                            const int32_t* __restrict__ sp, int W, int H,
                            int32_t* __restrict__ labels, CompAcc* acc, int max_comps) {
  const unsigned FULL = 0xffffffffu;
  const int p = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
  int k = -1;
  if (p < W * H) {
    const int r = L[p];
    k = r < 0 ? -1 : cid[r];
    labels[p] = k;
  }
  // the lanes of a warp that share a component add their pixels in one set of atomics
  const bool valid = k >= 0 && k < max_comps;
  const int u = valid ? p % W : 0, v = valid ? p / W : 0, s = valid ? sp[p] : 0;
  unsigned pending = __ballot_sync(FULL, valid);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int kl = __shfl_sync(FULL, k, leader);
    const bool mine = valid && k == kl;
    const unsigned peers = __ballot_sync(FULL, mine);
    const int umin = __reduce_min_sync(FULL, mine ? u : INT_MAX);
    const int umax = __reduce_max_sync(FULL, mine ? u : -1);
    const int vmin = __reduce_min_sync(FULL, mine ? v : INT_MAX);
    const int vmax = __reduce_max_sync(FULL, mine ? v : -1);
    const unsigned su = __reduce_add_sync(FULL, mine ? (unsigned)u : 0u);  // < 32 * 4096
    const unsigned sv = __reduce_add_sync(FULL, mine ? (unsigned)v : 0u);
    const int smin = __reduce_min_sync(FULL, mine ? s : INT_MAX);
    const int smax = __reduce_max_sync(FULL, mine ? s : INT_MIN);
    if (lane == leader) {
      CompAcc* a = acc + kl;
      atomicAdd(&a->count, __popc(peers));
      atomicMin(&a->umin, umin);
      atomicMin(&a->vmin, vmin);
      atomicMax(&a->umax, umax);
      atomicMax(&a->vmax, vmax);
      atomicAdd(&a->sum_u, (unsigned long long)su);
      atomicAdd(&a->sum_v, (unsigned long long)sv);
      const int old = atomicCAS(&a->sp_first, INT_MIN, smin);
      if (smin != smax || (old != INT_MIN && old != smin)) a->multi = 1;
    }
    pending &= ~peers;
  }
}

// Statistics and the fake-pothole rule: the centroid lies in a corner cell of the image split
// 8 x 8 (compared exactly in integers), or every pixel carries the same superpixel label.
__global__ void k_ccl_finalize(const CompAcc* __restrict__ acc, const int32_t* __restrict__ root_of,
                               const int* __restrict__ total, const int* __restrict__ err, int W,
                               int H, int max_comps, pd_component* __restrict__ comps,
                               int* __restrict__ n_comps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = *total;
  if (k == 0) *n_comps = *err ? -1 : n;
  if (k >= n || k >= max_comps) return;
  const CompAcc a = acc[k];
  pd_component c;
  c.label = root_of[k];
  c.count = a.count;
  c.umin = a.umin;
  c.vmin = a.vmin;
  c.umax = a.umax;
  c.vmax = a.vmax;
  c.sum_u = (int64_t)a.sum_u;
  c.sum_v = (int64_t)a.sum_v;
  const int64_t cnt = a.count;
  const bool left = 8 * c.sum_u < (int64_t)W * cnt, right = 8 * c.sum_u >= (int64_t)7 * W * cnt;
  const bool top = 8 * c.sum_v < (int64_t)H * cnt, bottom = 8 * c.sum_v >= (int64_t)7 * H * cnt;
  c.superpixels = a.multi ? 2 : 1;
  c.corner = (left || right) && (top || bottom);
  c.single = !a.multi;
  c.fake = c.corner || c.single;
  comps[k] = c;
}

}  // namespace

size_t ccl_scratch_bytes(int W, int H, int max_comps) {
  const size_t n = (size_t)W * H, nb = (n + kCclThreads - 1) / kCclThreads;
  size_t acc = 0;
  carve_size<int32_t>(acc, n);         // L
  carve_size<int32_t>(acc, n);         // cid
  carve_size<int>(acc, nb);            // counts
  carve_size<int>(acc, nb);            // offsets
  carve_size<int>(acc, 2);             // total, err
  carve_size<int32_t>(acc, max_comps); // root_of
  carve_size<CompAcc>(acc, max_comps);
  return acc;
}

int launch_ccl(cudaStream_t s, const uint8_t* mask, const int32_t* sp, int W, int H, int conn,
               int32_t* labels, pd_component* comps, int max_comps, int* n_comps, void* scratch) {
  const int n = W * H, nb = (n + kCclThreads - 1) / kCclThreads;
  Carve c(scratch);
  int32_t* L = c.take<int32_t>(n);
  int32_t* cid = c.take<int32_t>(n);
  int* counts = c.take<int>(nb);
  int* offsets = c.take<int>(nb);
  int* flags = c.take<int>(2);  // total, err
  int32_t* root_of = c.take<int32_t>(max_comps);
  CompAcc* acc = c.take<CompAcc>(max_comps);
  const int T = 256, G = (n + T - 1) / T;
  const dim3 tiles((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  k_ccl_local<<<tiles, kTile * kTile, 0, s>>>(mask, W, H, conn, L, flags, acc, max_comps);
  k_ccl_border<<<tiles, kTile * kTile, 0, s>>>(mask, W, H, conn, L, flags + 1);
  k_ccl_flatten_count<<<nb, kCclThreads, 0, s>>>(L, n, flags + 1, counts);
  k_ccl_scan<<<1, kCclThreads, 0, s>>>(counts, nb, offsets, flags);
  k_ccl_ids<<<nb, kCclThreads, 0, s>>>(L, n, offsets, cid, root_of, max_comps);
  k_ccl_stats<<<G, T, 0, s>>>(L, cid, sp, W, H, labels, acc, max_comps);
  const int GK = (max_comps + T - 1) / T;
  k_ccl_finalize<<<GK > 0 ? GK : 1, T, 0, s>>>(acc, root_of, flags, flags + 1, W, H, max_comps,
                                               comps, n_comps);
  return 7;
}

}  // namespace pd
