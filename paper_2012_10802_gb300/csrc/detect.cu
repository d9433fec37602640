// Sec. II-D and II-E on the GPU: SLIC superpixels on the transformed disparity map, the
// superpixel-clustered map D3, the adaptive threshold of Eqs. (14)-(17) and the pothole mask.
//
// SLIC assignment is pixel-parallel: each 32x32 tile first gathers, in index order, the centres
// whose 2S x 2S search window can reach it, then every pixel scans that short list with the exact
// window test, so the result equals the centre-by-centre sweep of the original algorithm (the
// lower index wins ties).  Centre updates use exact integer sums (privatised per tile in shared
// memory) and one double division per coordinate.
#include <math.h>

#include "common.cuh"

namespace pd {

namespace {

constexpr int kTile = 32;                         // SLIC assignment tile (pixels per side)
constexpr int kTileThreads = 256;
constexpr int kRowsPerPass = kTileThreads / 32;  // rows of the tile one pass of the block covers
constexpr int kCandCap = 256;

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

__device__ float slic_gradient(const float* __restrict__ D2, int W, int H, int x, int y) {
  float gx = D2[(size_t)y * W + clampi(x + 1, 0, W - 1)] - D2[(size_t)y * W + clampi(x - 1, 0, W - 1)];
  float gy = D2[(size_t)clampi(y + 1, 0, H - 1) * W + x] - D2[(size_t)clampi(y - 1, 0, H - 1) * W + x];
  return gx * gx + gy * gy;
}

// Sums (count, x, y, q) over the lanes that share a label, one representative lane per label
// adding them into the tile's 32-bit shared slots (slot >= 0) or straight into the 64-bit global
// sums (slot < 0).  All 32 lanes must call it; lanes with valid == false contribute nothing.  q
// is summed in a 16-bit low part and a signed high part; the per-tile sums (at most 1024 pixels)
// are exact while |q| < 2^37, i.e. |D2| < 2^27 px.
__device__ void warp_accumulate(bool valid, int lab, int slot, int x, int y, long long q,
                                unsigned (*sacc)[5], unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(0xffffffffu, valid);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const int lab_l = __shfl_sync(0xffffffffu, lab, leader);
    const bool mine = valid && lab == lab_l;
    const unsigned peers = __ballot_sync(0xffffffffu, mine);
    const int xs = __reduce_add_sync(0xffffffffu, mine ? x : 0);
    const int ys = __reduce_add_sync(0xffffffffu, mine ? y : 0);
    const unsigned qlo = __reduce_add_sync(0xffffffffu, mine ? (unsigned)(q & 0xffff) : 0u);
    const int qhi = __reduce_add_sync(0xffffffffu, mine ? (int)(q >> 16) : 0);
    if (lane == leader) {
      if (slot >= 0) {  // per-tile 32-bit sums (exact for |q| < 2^37)
        unsigned* a = sacc[slot];
        atomicAdd(a + 0, (unsigned)__popc(peers));
        atomicAdd(a + 1, (unsigned)xs);
        atomicAdd(a + 2, (unsigned)ys);
        atomicAdd(a + 3, qlo);
        atomicAdd(a + 4, (unsigned)qhi);
      } else {
        const long long qs = (long long)qhi * 65536LL + (long long)qlo;
        unsigned long long* a = acc + 4 * (size_t)lab;
        atomicAdd(a + 0, (unsigned long long)__popc(peers));
        atomicAdd(a + 1, (unsigned long long)xs);
        atomicAdd(a + 2, (unsigned long long)ys);
        atomicAdd(a + 3, (unsigned long long)qs);
      }
    }
    pending &= ~peers;
  }
}

// Grid seeds moved to the lowest-gradient pixel of their 3x3 neighbourhood (seed wins ties).
__global__ void k_slic_seeds(const float* __restrict__ D2, int W, int H, int nx, int ny,
                             float* __restrict__ cx, float* __restrict__ cy,
                             float* __restrict__ cv) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx * ny) return;
  int i = k % nx, j = k / nx;
  int sx = (int)(((long long)(2 * i + 1) * W) / (2 * nx));
  int sy = (int)(((long long)(2 * j + 1) * H) / (2 * ny));
  int bx = sx, by = sy;
  float bg = slic_gradient(D2, W, H, sx, sy);
  for (int dy = -1; dy <= 1; ++dy)
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
  cx[k] = (float)bx;
  cy[k] = (float)by;
  cv[k] = D2[(size_t)by * W + bx];
}

__global__ void k_slic_init_labels(int W, int H, int nx, int ny, int32_t* __restrict__ labels) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  int y = blockIdx.y;
  if (x >= W) return;
  // y * ny and x * nx stay below 2^28 (W, H <= 16384): 32-bit divisions give the same floors
  labels[(size_t)y * W + x] = (int32_t)((y * ny / H) * nx + (x * nx / W));
}

// One assignment round (if do_assign) plus the per-centre sums of the resulting labels:
// acc[4k + 0..3] = members, sum x, sum y, sum rint(1024 D2).  A block covers a kTile x kTile tile;
// thread (tx, ty) handles pixels (x0 + tx, y0 + ty + kRowsPerPass * i), so a warp is one row of 32.
__global__ void __launch_bounds__(kTileThreads) k_slic_assign(
    const float* __restrict__ D2, int W, int H, int n, const float* __restrict__ cx,
    const float* __restrict__ cy, const float* __restrict__ cv, float Sf, float coef,
    int do_assign, int32_t* __restrict__ labels, unsigned long long* __restrict__ acc) {
  __shared__ int cand[kCandCap];
  __shared__ float ccx[kCandCap], ccy[kCandCap], ccv[kCandCap];
  __shared__ unsigned sacc[kCandCap][5];
  __shared__ int wcount[kTileThreads / 32];
  __shared__ int ncand;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  if (tid == 0) ncand = 0;
  __syncthreads();
  if (do_assign) {
    // conservative box test (1 px margin); the exact test runs per pixel below.  Thread t tests
    // centres 4t .. 4t+3 of each chunk of 4 * kTileThreads, and a block scan of the per-thread
    // counts places the hits, so the list stays in index order.
    const float bx0 = (float)x0 - 1.0f, bx1 = (float)(x0 + kTile), by0 = (float)y0 - 1.0f,
                by1 = (float)(y0 + kTile);
    for (int base = 0; base < n; base += 4 * kTileThreads) {  // block-uniform
      const int k0 = base + 4 * tid;
      float fx[4], fy[4], fv[4];
      if (k0 + 4 <= n) {  // 16-byte aligned: the arrays start on 256-byte boundaries
        const float4 X = *reinterpret_cast<const float4*>(cx + k0);
        const float4 Y = *reinterpret_cast<const float4*>(cy + k0);
        const float4 V = *reinterpret_cast<const float4*>(cv + k0);
        fx[0] = X.x, fx[1] = X.y, fx[2] = X.z, fx[3] = X.w;
        fy[0] = Y.x, fy[1] = Y.y, fy[2] = Y.z, fy[3] = Y.w;
        fv[0] = V.x, fv[1] = V.y, fv[2] = V.z, fv[3] = V.w;
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const bool in = k0 + b < n;
          fx[b] = in ? cx[k0 + b] : 0.0f;
          fy[b] = in ? cy[k0 + b] : 0.0f;
          fv[b] = in ? cv[k0 + b] : 0.0f;
        }
      }
      bool q[4];
      int cnt = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        q[b] = k0 + b < n && (fx[b] + Sf >= bx0) && (fx[b] - Sf <= bx1) && (fy[b] + Sf >= by0) &&
               (fy[b] - Sf <= by1);
        cnt += q[b] ? 1 : 0;
      }
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) wcount[warp] = incl;
      __syncthreads();
      int pos = ncand + incl - cnt;
      for (int w = 0; w < warp; ++w) pos += wcount[w];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (q[b]) {
          if (pos < kCandCap) {
            cand[pos] = k0 + b;
            ccx[pos] = fx[b];
            ccy[pos] = fy[b];
            ccv[pos] = fv[b];
          }
          ++pos;
        }
      __syncthreads();
      if (tid == 0) {
        int tot = ncand;
        for (int w = 0; w < kTileThreads / 32; ++w) tot += wcount[w];
        ncand = tot;
      }
      __syncthreads();
    }
  }
  const int nc = ncand;
  const bool overflow = nc > kCandCap;
  for (int i = tid; i < kCandCap; i += kTileThreads)
    sacc[i][0] = sacc[i][1] = sacc[i][2] = sacc[i][3] = sacc[i][4] = 0u;
  __syncthreads();

  // A thread takes NP pixels of its column, kTile / NP rows apart: each candidate's shared loads
  // and x distance then serve all of them.  The window test is a predicate, not a branch
  // (nearly every candidate passes for some lane of a row).  Expressions and the strict
  // first-index comparison are those of the centre-by-centre sweep.
  constexpr int NP = 4;
  constexpr int kHalf = kTile / NP;  // row spacing of a thread's pixels
#pragma unroll
  for (int pass = 0; pass < kHalf / kRowsPerPass; ++pass) {
    const int x = x0 + lane;
    int yy[NP], lab[NP], slot[NP];
    bool inside[NP];
    float val[NP];
    long long q[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      yy[h] = y0 + warp + kRowsPerPass * pass + kHalf * h;
      inside[h] = x < W && yy[h] < H;
      lab[h] = -1;
      slot[h] = -1;
      q[h] = 0;
      val[h] = 0.0f;
      if (inside[h]) {
        const size_t p = (size_t)yy[h] * W + x;
        val[h] = D2[p];
        lab[h] = labels[p];
      }
    }
    if (do_assign) {
      float best[NP], fyp[NP];
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        best[h] = INFINITY;
        fyp[h] = (float)yy[h];
      }
      const float fxp = (float)x;
      if (!overflow) {
        for (int i = 0; i < nc; ++i) {
          const float fx = fxp - ccx[i], cyi = ccy[i], cvi = ccv[i];
          const bool inx = fabsf(fx) <= Sf;
#pragma unroll
          for (int h = 0; h < NP; ++h) {
            const float fy = fyp[h] - cyi;
            const float dv = val[h] - cvi;
            const float dd = dv * dv + (fx * fx + fy * fy) * coef;
            if (inx && fabsf(fy) <= Sf && dd < best[h]) {
              best[h] = dd;
              slot[h] = i;
            }
          }
        }
#pragma unroll
        for (int h = 0; h < NP; ++h)
          if (slot[h] >= 0) lab[h] = cand[slot[h]];
      } else {  // rare: too many candidates for shared memory; scan every centre
#pragma unroll
        for (int h = 0; h < NP; ++h) {
          if (!inside[h]) continue;
          for (int k = 0; k < n; ++k) {
            float fx = fxp - cx[k];
            float fy = fyp[h] - cy[k];
            if (!(fabsf(fx) <= Sf && fabsf(fy) <= Sf)) continue;
            float dv = val[h] - cv[k];
            float dd = dv * dv + (fx * fx + fy * fy) * coef;
            if (dd < best[h]) {
              best[h] = dd;
              lab[h] = k;
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < NP; ++h)
        if (inside[h]) labels[(size_t)yy[h] * W + x] = lab[h];
    }
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      if (inside[h]) q[h] = rint_to_ll(val[h] * 1024.0f);  // exact scaling; rint's rounding
      // a label's slot is the same for every lane that has it, so grouping by label groups by
      // slot; lanes that kept an uncovered pixel's old label (slot -1) go straight to the global
      // sums
      warp_accumulate(inside[h] && slot[h] >= 0, lab[h], slot[h], x, yy[h], q[h], sacc, acc);
      warp_accumulate(inside[h] && slot[h] < 0, lab[h], -1, x, yy[h], q[h], sacc, acc);
    }
  }
  __syncthreads();
  if (!overflow)
    for (int i = tid; i < nc; i += kTileThreads) {
      if (sacc[i][0] == 0u) continue;
      unsigned long long* a = acc + 4 * (size_t)cand[i];
      const long long qs = (long long)(int)sacc[i][4] * 65536LL + (long long)sacc[i][3];
      atomicAdd(a + 0, (unsigned long long)sacc[i][0]);
      atomicAdd(a + 1, (unsigned long long)sacc[i][1]);
      atomicAdd(a + 2, (unsigned long long)sacc[i][2]);
      atomicAdd(a + 3, (unsigned long long)qs);
    }

}

// Centre update from the exact sums (empty clusters keep their centre); clears the sums.  It is
// a separate launch over many SMs because the three double divisions per centre are slow on one.
__global__ void k_slic_update(int n, unsigned long long* __restrict__ acc, float* __restrict__ cx,
                              float* __restrict__ cy, float* __restrict__ cv) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  unsigned long long* a = acc + 4 * (size_t)k;
  const long long cnt = (long long)a[0];
  const long long sx = (long long)a[1], sy = (long long)a[2], sq = (long long)a[3];
  if (cnt > 0) {
    const long long lim = 1LL << 24;
    if (cnt < lim && sx > -lim && sx < lim && sy > -lim && sy < lim && sq > -lim && sq < lim) {
      // Every operand is an exact float, so the correctly rounded float quotient equals the
      // double quotient rounded to float (double has at least 2 x 24 + 2 bits, which makes the
      // double rounding innocuous for a division), and /1024 scales exactly: the FP32 pipe
      // gives the result of the double expressions below without the slow FP64 one.
      const float fc = (float)(int)cnt;
      cx[k] = __fdiv_rn((float)(int)sx, fc);
      cy[k] = __fdiv_rn((float)(int)sy, fc);
      cv[k] = __fdiv_rn((float)(int)sq, fc) * (1.0f / 1024.0f);
    } else {
      cx[k] = (float)((double)sx / (double)cnt);
      cy[k] = (float)((double)sy / (double)cnt);
      cv[k] = (float)(((double)sq / (double)cnt) / 1024.0);
    }
  }
  a[0] = a[1] = a[2] = a[3] = 0ULL;
}

// D3: each pixel takes the mean of its superpixel, i.e. the value of the last centre update.
__global__ void k_slic_d3(const int32_t* __restrict__ labels, const float* __restrict__ cv,
                          size_t N, float* __restrict__ D3) {
  size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) D3[p] = cv[labels[p]];
}

__global__ void k_centres_out(int n, const float* __restrict__ cx, const float* __restrict__ cy,
                              const float* __restrict__ cv, float* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  out[3 * k] = cx[k];
  out[3 * k + 1] = cy[k];
  out[3 * k + 2] = cv[k];
}

// ------------------------------------------------------------------- Eqs. (14)-(17)
constexpr int kBins = 257;  // k = 0..255 plus an overflow bin for everything at or above 32 px

// Adds (1, a, b, a^2 + b^2) of the lanes sharing a bin into the shared histogram h.  The lanes
// of one bin form a group (match.any); each sum is one group-masked warp reduction, executed by
// every group at once, and the group's lowest lane adds the four sums.  All 32 lanes must call
// it.  The sums use the single-instruction warp reduction on 32-bit values; a and b (D2 below
// 2^16 px) fit, a^2 + b^2 is split into 16/16/32-bit parts.
__device__ void warp_hist(bool valid, int bin, long long a, long long b,
                          unsigned long long (*h)[4]) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? bin : -1);
  const unsigned long long sq = (unsigned long long)(a * a + b * b);
  const int sa = __reduce_add_sync(peers, (int)a);
  const int sb = __reduce_add_sync(peers, (int)b);
  const unsigned s0 = __reduce_add_sync(peers, (unsigned)(sq & 0xffffu));
  const unsigned s1 = __reduce_add_sync(peers, (unsigned)((sq >> 16) & 0xffffu));
  const unsigned s2 = __reduce_add_sync(peers, (unsigned)(sq >> 32));
  if (valid && lane == __ffs(peers) - 1) {
    const unsigned long long ssq = (unsigned long long)s0 + ((unsigned long long)s1 << 16) +
                                   ((unsigned long long)s2 << 32);
    atomicAdd(&h[bin][0], (unsigned long long)__popc(peers));
    atomicAdd(&h[bin][1], (unsigned long long)(long long)sa);
    atomicAdd(&h[bin][2], (unsigned long long)(long long)sb);
    atomicAdd(&h[bin][3], ssq);
  }
}

// Histograms of kmax = max(floor(a / 128), floor(b / 1024)) and kmin (the same with min), each
// with exact sums n, sum a, sum b, sum a^2 + b^2, over interior pixels with a valid 3x3 window;
// a = rint(1024 D2(p)), b = sum of rint(1024 D2) over the 8 neighbours.  Region 1 of threshold
// k/8 is {kmax < k}, region 2 is {kmin >= k}.  Blocks stride over rows.
__global__ void __launch_bounds__(256) k_thresh_hist(const float* __restrict__ D2,
                                                     const float* __restrict__ D1, int W, int H,
                                                     unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long sh[2][kBins][4];
  for (int i = threadIdx.x; i < 2 * kBins * 4; i += blockDim.x) (&sh[0][0][0])[i] = 0ULL;
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  for (int v = blockIdx.y; v < H; v += gridDim.y) {
    bool ok = u >= 1 && u < W - 1 && v >= 1 && v < H - 1;
    long long a = 0, b = 0;
    if (ok) {
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          size_t q = (size_t)(v + dy) * W + (u + dx);
          if (!(D1[q] >= 0.0f)) ok = false;
          long long qq = rint_to_ll(D2[q] * 1024.0f);
          if (dx == 0 && dy == 0)
            a = qq;
          else
            b += qq;
        }
    }
    long long ka = a >> 7, kb = b >> 10;
    long long kmax = ka > kb ? ka : kb, kmin = ka < kb ? ka : kb;
    int imax = (int)(kmax < 0 ? 0 : (kmax > 256 ? 256 : kmax));
    int imin = (int)(kmin < 0 ? 0 : (kmin > 256 ? 256 : kmin));
    warp_hist(ok, imax, a, b, sh[0]);
    warp_hist(ok, imin, a, b, sh[1]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kBins * 4; i += blockDim.x) {
    unsigned long long x = (&sh[0][0][0])[i];
    if (x) atomicAdd(hist + i, x);
  }
}

// E2(t) of Eq. (17) for t = k/8, k = 1..255: thread k forms the region sums from the histograms
// (region 1: kmax bins below k, region 2: kmin bins from k up), evaluates E2 in double, and the
// block takes the smallest minimising k; t_s from mode.
constexpr int kSolveThreads = 256;
static_assert(kSolveThreads == kBins - 1, "one solve thread per bin below the overflow bin");

// Inclusive block scan (sum) of one 64-bit value per thread; 256 threads.
__device__ long long block_scan_ll(long long v, long long* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) tmp[warp] = v;
  __syncthreads();
  long long off = 0;
  for (int w = 0; w < warp; ++w) off += tmp[w];
  __syncthreads();
  return v + off;
}

__global__ void __launch_bounds__(kSolveThreads) k_thresh_solve(
    const unsigned long long* __restrict__ hist, float delta_pd, int mode,
    double* __restrict__ thr, float* __restrict__ thr_up, double* __restrict__ E2) {
  __shared__ long long tmp[kSolveThreads / 32];
  __shared__ long long sKey[kSolveThreads];
  __shared__ int sK[kSolveThreads];
  __shared__ long long sA2[kSolveThreads], sN2[kSolveThreads];
  const int k = threadIdx.x;
  const unsigned long long(*hmax)[4] = reinterpret_cast<const unsigned long long(*)[4]>(hist);
  const unsigned long long(*hmin)[4] = reinterpret_cast<const unsigned long long(*)[4]>(hist + kBins * 4);
  // region 1 at threshold k: kmax bins 0..k-1 (exclusive prefix sums of bins 0..255);
  // region 2 at threshold k: kmin bins k..256 (total minus the exclusive prefix)
  // totals of the kmin histogram over all 257 bins: the last thread's inclusive prefix (bins
  // 0..255) plus the overflow bin
  __shared__ long long tot[4];
  long long r1[4], r2[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    long long xm = (long long)hmax[k][q];
    r1[q] = block_scan_ll(xm, tmp) - xm;
    long long xn = (long long)hmin[k][q];
    const long long incl = block_scan_ll(xn, tmp);
    r2[q] = incl - xn;  // exclusive prefix of kmin bins below k
    if (k == kSolveThreads - 1) tot[q] = incl + (long long)hmin[kBins - 1][q];
  }
  __syncthreads();
  double e = NAN;
  long long a2 = 0, n2 = 0;
  if (k >= 1) {
    long long n1 = r1[0], a1 = r1[1], b1 = r1[2];
    unsigned long long s1 = (unsigned long long)r1[3];
    n2 = tot[0] - r2[0];
    a2 = tot[1] - r2[1];
    long long b2 = tot[2] - r2[2];
    unsigned long long s2 = (unsigned long long)tot[3] - (unsigned long long)r2[3];
    if (n1 != 0 && n2 != 0) {
      double e1 = (double)s1 - ((double)a1 * (double)a1 + (double)b1 * (double)b1) / (double)n1;
      double e2 = (double)s2 - ((double)a2 * (double)a2 + (double)b2 * (double)b2) / (double)n2;
      e = e1 + e2;
    }
  }
  if (E2) E2[k] = e;
  // block argmin over the non-NaN energies, smallest k on ties, on integer keys (NaN: largest)
  sKey[k] = isnan(e) ? 0x7fffffffffffffffLL : f64_order_key(e);
  sK[k] = k;
  sA2[k] = a2;
  sN2[k] = n2;
  __syncthreads();
  for (int s = kSolveThreads / 2; s > 0; s >>= 1) {
    if (k < s) {
      const long long eo = sKey[k + s], em = sKey[k];
      const int ko = sK[k + s], km = sK[k];
      if (eo < em || (eo == em && ko < km)) {
        sKey[k] = eo;
        sK[k] = ko;
      }
    }
    __syncthreads();
  }
  if (k != 0) return;
  if (sKey[0] == 0x7fffffffffffffffLL) {  // no threshold splits the pixels into two regions
    thr[0] = NAN;
    thr[1] = -INFINITY;
    *thr_up = -INFINITY;
    return;
  }
  const int w = sK[0];
  // the mean of region 2 only for the winner (a double division costs ~560 cycles here)
  const double mean = ((double)sA2[w] / (double)sN2[w]) / 1024.0;
  thr[0] = (double)w * 0.125;
  thr[1] = (mode == 0 ? mean : thr[0]) - (double)delta_pd;
  *thr_up = __double2float_ru(thr[1]);
}

// D3 < t_s (Eq. 17's pothole rule) in float: for a float x and a double t, x < t exactly when
// x < tf with tf = t rounded up to a float (no float lies strictly between t and tf; infinities
// and NaN compare the same), which spares a per-pixel conversion on the FP64 pipe.
__global__ void k_mask(const float* __restrict__ D3, size_t N, const float* __restrict__ thr_up,
                       uint8_t* __restrict__ mask) {
  size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  mask[p] = D3[p] < *thr_up ? 1 : 0;
}

}  // namespace

void slic_grid(int W, int H, int K, int* nx, int* ny) {
  double S = sqrt((double)W * (double)H / (double)K);
  int a = (int)floor((double)W / S + 0.5);
  int b = (int)floor((double)H / S + 0.5);
  a = a < 1 ? 1 : (a > W ? W : a);
  b = b < 1 ? 1 : (b > H ? H : b);
  *nx = a;
  *ny = b;
}

size_t slic_scratch_bytes(int n) {
  size_t acc = 0;
  carve_size<float>(acc, n);
  carve_size<float>(acc, n);
  carve_size<float>(acc, n);
  carve_size<unsigned long long>(acc, 4 * (size_t)n);
  return acc;
}

int launch_slic(cudaStream_t s, const float* D2, int W, int H, int K, float m, int iters,
                int32_t* labels, float* D3, float* centres_out, void* scratch) {
  int nx, ny;
  slic_grid(W, H, K, &nx, &ny);
  int n = nx * ny;
  Carve cv_(scratch);
  float* cx = cv_.take<float>(n);
  float* cy = cv_.take<float>(n);
  float* cv = cv_.take<float>(n);
  unsigned long long* acc = cv_.take<unsigned long long>(4 * (size_t)n);
  float Sf = (float)sqrt((double)W * (double)H / (double)K);
  float coef = (float)((double)m * (double)m * (double)K / ((double)W * (double)H));
  cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 4 * (size_t)n, s);
  k_slic_seeds<<<(n + 127) / 128, 128, 0, s>>>(D2, W, H, nx, ny, cx, cy, cv);
  k_slic_init_labels<<<dim3((W + 255) / 256, H), 256, 0, s>>>(W, H, nx, ny, labels);
  dim3 tiles((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  int rounds = iters > 0 ? iters : 1;
  for (int it = 0; it < rounds; ++it) {
    k_slic_assign<<<tiles, kTileThreads, 0, s>>>(D2, W, H, n, cx, cy, cv, Sf, coef,
                                                 iters > 0 ? 1 : 0, labels, acc);
    k_slic_update<<<(n + 127) / 128, 128, 0, s>>>(n, acc, cx, cy, cv);
  }
  size_t N = (size_t)W * H;
  k_slic_d3<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(labels, cv, N, D3);
  if (centres_out) k_centres_out<<<(n + 127) / 128, 128, 0, s>>>(n, cx, cy, cv, centres_out);
  return 3 + 2 * rounds + (centres_out ? 1 : 0);
}

size_t threshold_scratch_bytes() {
  size_t acc = 0;
  carve_size<unsigned long long>(acc, 2 * kBins * 4);
  carve_size<double>(acc, 2);
  carve_size<float>(acc, 1);
  return acc;
}

int launch_threshold(cudaStream_t s, const float* D2, const float* D1, const float* D3, int W,
                     int H, float delta_pd, int mode, uint8_t* mask, double* thresholds,
                     double* E2, void* scratch) {
  Carve c(scratch);
  unsigned long long* hist = c.take<unsigned long long>(2 * kBins * 4);
  double* thr = c.take<double>(2);
  float* thr_up = c.take<float>(1);
  if (thresholds) thr = thresholds;
  cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 2 * kBins * 4, s);
  // one full wave of 8 resident blocks per SM (the register limit at 256 threads): many warps
  // in flight, and no second wave of a few blocks (rounding the grid up made one, of 4 blocks
  // at 720p, that doubled the kernel's time)
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int xb = (W + 255) / 256;
  int yb = (8 * (sms > 0 ? sms : 1)) / xb;
  yb = yb < 1 ? 1 : (yb < H ? yb : H);
  k_thresh_hist<<<dim3(xb, yb), 256, 0, s>>>(D2, D1, W, H, hist);
  k_thresh_solve<<<1, kSolveThreads, 0, s>>>(hist, delta_pd, mode, thr, thr_up, E2);
  size_t N = (size_t)W * H;
  k_mask<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(D3, N, thr_up, mask);
  return 3;
}

}  // namespace pd
