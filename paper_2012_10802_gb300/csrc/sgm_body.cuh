// Device-side bodies of the Sec. II-A / II-B kernels, shared by the single-pair kernels (sgm.cu) and
// the batched ones (batch.cu).  Each body takes its block coordinates explicitly.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace pd {
namespace body {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kBig2 = 0x3fff3fffu;  // "no neighbour": never the minimum, no u16 overflow

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

// ----------------------------------------------------------------------------- Eq. (6)
// One warp per row: minimum of f(x, v) - delta_pt over x = 0..W-1, each f evaluated in double in
// the fixed operation order of the model definition (the library is built without FMA
// contraction).  f is monotone in x for the linear model and convex or concave in x for the
// quadratic one, so the minimum over all x lies at an end point or, for a convex quadratic, next
// to the vertex: the warp evaluates both end points and the 64 columns around the vertex.
__device__ __forceinline__ double road_minus(double t1, double uc, double vc, double sn, int order,
                                             double a0, double a1, double a2, double delta_pt,
                                             int x) {
  double t2 = ((double)x - uc) * sn;
  double vp = (t1 - t2) + vc;
  double f = a0 + a1 * vp;
  if (order == 2) f = f + a2 * (vp * vp);
  return f - delta_pt;
}

// Row v of Eq. (6), computed by one warp (lane = the calling lane).
__device__ __forceinline__ void kappa_row(int W, int H, int order, double a0, double a1, double a2,
                                          double cs, double sn, double delta_pt,
                                          int32_t* __restrict__ kappa, int v, int lane) {
  double uc = (double)(W - 1) * 0.5, vc = (double)(H - 1) * 0.5;
  double t1 = ((double)v - vc) * cs;
  double best = 1e300;
  if (lane < 2) best = road_minus(t1, uc, vc, sn, order, a0, a1, a2, delta_pt, lane == 0 ? 0 : W - 1);
  if (order == 2 && a2 > 0.0 && sn != 0.0) {
    double xs = uc + ((t1 + vc) + a1 / (2.0 * a2)) / sn;  // column of the vertex vp = -a1 / (2 a2)
    if (xs > -64.0 && xs < (double)W + 64.0) {
      int xc = (int)floor(xs);
      for (int x = xc - 31 + 2 * lane; x <= xc - 30 + 2 * lane; ++x)
        if (x >= 0 && x < W) {
          double f = road_minus(t1, uc, vc, sn, order, a0, a1, a2, delta_pt, x);
          best = f < best ? f : best;
        }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double other = __shfl_xor_sync(kFull, best, o);
    best = other < best ? other : best;
  }
  if (lane == 0) kappa[v] = (int32_t)floor(best);
}

// ----------------------------------------------------------------------------- census
constexpr int kCT_W = 32, kCT_H = 32;  // census tile (pixels)
constexpr int kCT_TY = 8;              // thread rows of a census block: kCT_H / kCT_TY pixels each

// Census codes of one kCT_W x kCT_H tile (block of kCT_W x kCT_TY threads), tile (bx, by).
__device__ __forceinline__ void census_tile(const uint8_t* __restrict__ img, int W, int H,
                                            size_t pitch, const int32_t* __restrict__ kappa,
                                            uint32_t* __restrict__ codes, int bx, int by) {
  __shared__ uint8_t tile[kCT_H + 4][kCT_W + 4];
  const int u0 = bx * kCT_W, v0 = by * kCT_H;
  for (int i = threadIdx.y * kCT_W + threadIdx.x; i < (kCT_H + 4) * (kCT_W + 4);
       i += kCT_W * kCT_TY) {
    int ty = i / (kCT_W + 4), tx = i % (kCT_W + 4);
    int y = clampi(v0 + ty - 2, 0, H - 1);
    int x = clampi(u0 + tx - 2, 0, W - 1);
    if (kappa) x = clampi(x - kappa[y], 0, W - 1);  // the row-shifted image at (x, y)
    tile[ty][tx] = img[(size_t)y * pitch + x];
  }
  __syncthreads();
  const int u = u0 + threadIdx.x;
  if (u >= W) return;
#pragma unroll
  for (int r = 0; r < kCT_H / kCT_TY; ++r) {
    const int ly = threadIdx.y + kCT_TY * r, v = v0 + ly;
    if (v >= H) break;
    const uint8_t c = tile[ly + 2][threadIdx.x + 2];
    uint32_t code = 0;
    int k = 0;
#pragma unroll
    for (int dy = 0; dy < 5; ++dy)
#pragma unroll
      for (int dx = 0; dx < 5; ++dx) {
        if (dx == 2 && dy == 2) continue;
        code |= (uint32_t)(tile[ly + dy][threadIdx.x + dx] < c) << k;
        ++k;
      }
    codes[(size_t)v * W + u] = code;
  }
}

// ----------------------------------------------------------------------------- cost
// Interleaved layout, D % 16 == 0.  A block covers one segment of cost_seg(D) pixels of a row
// from one shared copy of the codes it needs.  A lane computes one 16-disparity group g for four
// consecutive pixels u .. u + 3: their right codes x = u + k - d, d in [16g, 16g + 16), are the 19
// consecutive words ending at x = u + 3 - 16g, read as five aligned 16-byte shared loads (the
// window starts at a multiple of 4 words because D and u - u0 are multiples of 4).  The lanes of
// a warp take the groups as the slow index, so a warp's stores for one k cover whole 16-byte
// chunks of D-byte pixel rows, and the window loads of 8 consecutive lanes fall in distinct
// banks.
constexpr int kCostThreads = 256;
constexpr int kCostWarps = kCostThreads / 32;
constexpr int kCostSlices = 8;

__host__ __device__ __forceinline__ int cost_seg(int D) {
  return kCostSlices * (kCostThreads / (D >> 4));
}
__host__ __device__ __forceinline__ int cost_blocks_per_row(int W, int D) {
  return (W + cost_seg(D) - 1) / cost_seg(D);
}

// Bytes (a, b, c, d) of the low bytes of four values.
__device__ __forceinline__ uint32_t pack4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}

// The 16 costs of group g for pixel u + k: word i holds d - 16g = 2i, 2i + 8, 2i + 1, 2i + 9 in
// its bytes 0..3 (byte 2j: d = 16g + j, byte 2j + 1: d = 16g + 8 + j).  w[m] is the right code
// of x = u + k - (16g + 15 + k - m), i.e. d - 16g = 15 + k - m.  CHECK: x may be negative
// (x0 = u - 16g, the x of k = 0, d = 16g).
template <bool CHECK>
__device__ __forceinline__ uint4 cost16_of(uint32_t c0, const uint32_t (&w)[20], int k, int x0) {
  uint32_t c[16];
#pragma unroll
  for (int dd = 0; dd < 16; ++dd) {
    c[dd] = (uint32_t)__popc(c0 ^ w[15 + k - dd]);
    if (CHECK && x0 + k - dd < 0) c[dd] = (uint32_t)kCensusBits;
  }
  return make_uint4(pack4(c[0], c[8], c[1], c[9]), pack4(c[2], c[10], c[3], c[11]),
                    pack4(c[4], c[12], c[5], c[13]), pack4(c[6], c[14], c[7], c[15]));
}

// Interleaved cost of the segment bx of row v.
__device__ __forceinline__ void cost_il_block(const uint32_t* __restrict__ cl,
                                              const uint32_t* __restrict__ cr, int W, int D,
                                              uint8_t* __restrict__ cost, int bx, int v) {
  __shared__ __align__(16) uint32_t sR[kCostSlices * kCostThreads + kMaxD];
  __shared__ __align__(16) uint32_t sL[kCostSlices * kCostThreads];
  const int seg = cost_seg(D);
  const int u0 = bx * seg;
  const int base = u0 - D + 1;  // x of sR[0]
  // the windows reach sR[seg + D - 1] (the last lane's fifth load); codes outside [0, W) read 0
  for (int i = threadIdx.x; i < seg + D; i += kCostThreads) {
    const int x = base + i;
    sR[i] = (x >= 0 && x < W) ? cr[(size_t)v * W + x] : 0u;
  }
  for (int i = threadIdx.x; i < seg; i += kCostThreads) {
    const int u = u0 + i;
    sL[i] = u < W ? cl[(size_t)v * W + u] : 0u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cpw = 32 / (D >> 4);  // 4-pixel chunks per warp and pass
  const int g = lane / cpw, ch = lane % cpw;
  const int step = kCostWarps * cpw * 4;
  for (int r = warp * cpw * 4 + 4 * ch; r < seg; r += step) {
    const int u = u0 + r;
    if (u >= W) break;  // later passes are further right
    const uint4 cq = *reinterpret_cast<const uint4*>(sL + r);
    const uint32_t c0[4] = {cq.x, cq.y, cq.z, cq.w};
    const int wb = r + D - 16 - 16 * g;  // sR index of x = u - 16g - 15, a multiple of 4
    uint32_t w[20];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const uint4 t = *reinterpret_cast<const uint4*>(sR + wb + 4 * q);
      w[4 * q] = t.x;
      w[4 * q + 1] = t.y;
      w[4 * q + 2] = t.z;
      w[4 * q + 3] = t.w;
    }
    const int x0 = u - 16 * g;
    const bool check = x0 - 15 < 0;
    uint8_t* dst = cost + ((size_t)v * W + u) * D + 16 * g;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 val = check ? cost16_of<true>(c0[k], w, k, x0) : cost16_of<false>(c0[k], w, k, x0);
      if (u + k < W) *reinterpret_cast<uint4*>(dst + (size_t)k * D) = val;
    }
  }
}

// ----------------------------------------------------------------------------- Eq. (8)
constexpr int kStages = 16;  // per-warp shared-memory ring of cost rows: kStages - 1 steps in flight

// Asynchronous 16-byte copy global -> shared (cp.async, L2 only); src_bytes = 0 writes zeros and
// reads nothing.
__device__ __forceinline__ void cp_async16(uint32_t smem, const void* gmem, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
// The same copy of 8 bytes (cp.async.ca: 4, 8 or 16 bytes); src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async8(uint32_t smem, const void* gmem, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(smem), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Every line of direction (dx, dy) is walked by a step index s; the pixel at step s moves by a
// constant byte stride through the [H][W][D] volumes, and the line lies inside the image for one
// contiguous range of s.  Horizontal lines are the rows (s runs along u); all other lines step
// one row per s (s runs along v, in the direction of dy), and diagonal lines are indexed by
// u - v (dx == dy) or u + v (dx == -dy).
struct LineWalk {
  long long off0;   // byte offset of step 0 (may lie outside the image)
  long long delta;  // byte stride per step
  int s_first, s_last, nsteps;
  int u0, v0;       // pixel of step 0; step s is (u0 + s dx, v0 + s dy)
};

__device__ __forceinline__ LineWalk line_walk(int dx, int dy, int W, int H, int D, int line,
                                              int first, int last, bool valid) {
  LineWalk w;
  if (dy == 0) {  // row `line`, s along u
    const int u0 = dx > 0 ? 0 : W - 1;
    w.off0 = ((long long)line * W + u0) * D;
    w.delta = (long long)dx * D;
    w.nsteps = W;
    w.s_first = 0;
    w.s_last = valid ? W - 1 : -1;
    w.u0 = u0;
    w.v0 = line;
    return w;
  }
  int vlo = 0, vhi = H - 1;
  if (dx != 0) {  // the rows any line of this warp touches
    if (dx == dy) {
      vlo = max(0, H - 1 - last);
      vhi = min(H - 1, W + H - 2 - first);
    } else {
      vlo = max(0, first - W + 1);
      vhi = min(H - 1, last);
    }
  }
  w.nsteps = vhi - vlo + 1;
  const int v0 = dy > 0 ? vlo : vhi;
  const int u0 = dx == 0 ? line : (dx == dy ? line - (H - 1) + v0 : line - v0);  // u at step 0
  w.off0 = ((long long)v0 * W + u0) * D;
  w.delta = ((long long)dy * W + dx) * D;
  // steps with 0 <= u0 + s*dx <= W-1 and 0 <= s < nsteps
  int lo = 0, hi = w.nsteps - 1;
  if (dx > 0) {
    lo = max(lo, -u0);
    hi = min(hi, W - 1 - u0);
  } else if (dx < 0) {
    lo = max(lo, u0 - (W - 1));
    hi = min(hi, u0);
  }
  w.s_first = lo;
  w.s_last = valid ? hi : -1;
  w.u0 = u0;
  w.v0 = v0;
  return w;
}

// The window of pixel (u, v) (see BandArgs).  tile_lo may point to global or shared memory
// (a generic load).
__device__ __forceinline__ void band_window(const BandArgs& b, int u, int v, int D, int& lo,
                                            int& hi) {
  const int t = b.tile_lo[(v >> 4) * b.tw + (u >> 4)];
  lo = t < 0 ? 0 : min(t, D - 1);
  hi = t < 0 ? D : min(lo + b.width, D);
}

// Bit i set for disparity 16 g + i inside [lo, hi).
__device__ __forceinline__ uint32_t group_in_mask(int g, int lo, int hi) {
  const int a = clampi(lo - 16 * g, 0, 16), b = clampi(hi - 16 * g, 0, 16);
  return ((1u << b) - 1u) & ~((1u << a) - 1u);
}

// The lines first .. first + 32/G - 1 of direction (dx, dy), walked by the calling warp (all 32
// lanes call it) with G lanes per line that each keep NG consecutive 16-disparity groups
// (G * NG = D / 16; NG = 1 or 2).  State: L of the previous pixel on the line (the oracle's
// normalised value) and its minimum over all disparities, replicated in both u16 halves; a line
// starts from L = 0, m = 0, which makes its first pixel's L equal to the cost.  Costs arrive
// through the warp's ring in shared memory (ring_base: ST = 16 / NG stages of 32 lanes x NG x 16
// bytes, 8 KB), ST - 1 steps ahead; L leaves with streaming 16-byte stores to dst_vol.  With two groups a lane
// carries 16 words: the step between its groups is a byte permutation inside the lane, so a line
// needs half the lanes, shuffles and per-step bookkeeping of one group per lane.  FULL: every
// line of the warp lies inside the image at every step (rows and columns), so a lane is active
// for the whole walk when its line exists and the per-step activity tests and state resets go.
template <int G, int NG, bool FULL, unsigned YIELD_NS = 0>
__device__ __forceinline__ void agg_walk(const uint8_t* __restrict__ cost,
                                         uint8_t* __restrict__ dst_vol, int W, int H, int D,
                                         int dx, int dy, uint32_t P1x2, uint32_t K21x2, int first,
                                         uint4* __restrict__ ring_base) {
  constexpr int LPW = 32 / G;  // lines per warp
  constexpr int NW = 8 * NG;   // u16x2 words per lane
  static_assert(NG == 1 || NG == 2, "one or two groups per lane");
  constexpr int ST = 16 / NG;  // ring stages
  const int nlines = dy == 0 ? H : (dx == 0 ? W : W + H - 1);
  const int lane = threadIdx.x & 31;
  const int g = lane % G;
  if (first >= nlines) return;  // the whole warp leaves together
  const int line = first + lane / G;
  const int last = min(first + LPW, nlines) - 1;
  const bool lvalid = line < nlines;
  const LineWalk lw = line_walk(dx, dy, W, H, D, line, first, last, lvalid);
  const uint8_t* csrc = cost + 16 * NG * g;
  uint8_t* dst = dst_vol + 16 * NG * g;

  uint32_t N[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) N[j] = 0;
  uint32_t mp = 0;

  // stage k of this lane: NG consecutive 16-byte slots at ring_base + (k * 32 + lane) * NG
  uint4* ring = ring_base + lane * NG;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  long long pf_off = lw.off0;
#pragma unroll
  for (int k = 0; k < ST - 1; ++k) {
    // only steps of the walk are read (a line may be shorter than the ring)
    const bool in = FULL ? (lvalid && k < lw.nsteps) : (k >= lw.s_first && k <= lw.s_last);
#pragma unroll
    for (int q = 0; q < NG; ++q)
      cp_async16(ring_s + (k * 32 * NG + q) * 16, csrc + (in ? pf_off : 0) + 16 * q,
                 in ? 16u : 0u);
    cp_async_commit();
    pf_off += lw.delta;
  }
  long long st_off = lw.off0;
  // Step s.  ALL: every lane's line is inside the image at this step (warp-uniform), so no
  // activity test, select or reset is needed.
  auto step = [&](const int s, auto all_tag) {
    constexpr bool ALL = decltype(all_tag)::value;
    const int k = s & (ST - 1);
    // rows and columns: a lane is active exactly when its line exists; diagonals: inside the
    // common range every lane is (all its lines exist there)
    const bool act = FULL ? lvalid : (ALL || (s >= lw.s_first && s <= lw.s_last));
    // YIELD_NS > 0: the walker sleeps that long each step, leaving its scheduler's issue slots
    // to the longer chains that share it
    if constexpr (YIELD_NS > 0) __nanosleep(YIELD_NS);
    cp_async_wait<ST - 2>();  // the copy of step s is complete
    uint32_t raw[4 * NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      const uint4 rv = ring[k * 32 * NG + q];
      raw[4 * q + 0] = rv.x;
      raw[4 * q + 1] = rv.y;
      raw[4 * q + 2] = rv.z;
      raw[4 * q + 3] = rv.w;
    }
    {
      const int sp = s + ST - 1;
      const bool in = FULL ? (lvalid && sp < lw.nsteps) : (sp >= lw.s_first && sp <= lw.s_last);
      const int kp = (k + ST - 1) & (ST - 1);
#pragma unroll
      for (int q = 0; q < NG; ++q)
        cp_async16(ring_s + (kp * 32 * NG + q) * 16, csrc + (in ? pf_off : 0) + 16 * q,
                   in ? 16u : 0u);
      cp_async_commit();
      pf_off += lw.delta;
    }
    uint32_t prevHi = kBig2, nextLo = kBig2;
    if constexpr (G > 1) {
      const uint32_t up = __shfl_up_sync(kFull, N[NW - 1], 1, G);
      const uint32_t dn = __shfl_down_sync(kFull, N[0], 1, G);
      if (g > 0) prevHi = up;
      if (g < G - 1) nextLo = dn;
    }
    const uint32_t K = mp + K21x2;
    uint32_t Lw[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const int q = j >> 3, i = j & 7;
      // d - 1 and d + 1 neighbours: inside the group the adjacent words; at a group's ends the
      // byte permutation with the neighbouring group (this lane's other group or the
      // neighbouring lane's)
      constexpr int kNW = NW;
      const uint32_t below = N[(j + kNW - 1) % kNW], above = N[(j + 1) % kNW];
      uint32_t lft, rgt;
      if (i == 0)
        lft = __byte_perm(q == 0 ? prevHi : below, N[(j + 7) % kNW], 0x5432);
      else
        lft = below;
      if (i == 7)
        rgt = __byte_perm(N[(j + kNW - 7) % kNW], q == NG - 1 ? nextLo : above, 0x5432);
      else
        rgt = above;
      uint32_t t = __vimin3_u16x2(lft, rgt, K);
      t = __viaddmin_u16x2(t, P1x2, N[j]);
      const uint32_t c = __byte_perm(raw[j >> 1], 0, (j & 1) ? 0x4342 : 0x4140);
      Lw[j] = t + c - mp;
    }
    uint32_t m;
    if constexpr (NW == 8) {
      m = __vimin3_u16x2(__vimin3_u16x2(Lw[0], Lw[1], Lw[2]), __vimin3_u16x2(Lw[3], Lw[4], Lw[5]),
                         __vminu2(Lw[6], Lw[7]));
    } else {
      const uint32_t a = __vimin3_u16x2(Lw[0], Lw[1], Lw[2]);
      const uint32_t b = __vimin3_u16x2(Lw[3], Lw[4], Lw[5]);
      const uint32_t c = __vimin3_u16x2(Lw[6], Lw[7], Lw[8]);
      const uint32_t d = __vimin3_u16x2(Lw[9], Lw[10], Lw[11]);
      const uint32_t e = __vimin3_u16x2(Lw[12], Lw[13], Lw[14]);
      m = __vminu2(__vimin3_u16x2(a, b, c), __vimin3_u16x2(d, e, Lw[15]));
    }
    m = __vminu2(m, __byte_perm(m, m, 0x1032));
#pragma unroll
    for (int o = 1; o < G; o <<= 1) m = __vminu2(m, __shfl_xor_sync(kFull, m, o, G));
    if (act) {
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        uint4 w;
        w.x = __byte_perm(Lw[8 * q + 0], Lw[8 * q + 1], 0x6420);
        w.y = __byte_perm(Lw[8 * q + 2], Lw[8 * q + 3], 0x6420);
        w.z = __byte_perm(Lw[8 * q + 4], Lw[8 * q + 5], 0x6420);
        w.w = __byte_perm(Lw[8 * q + 6], Lw[8 * q + 7], 0x6420);
        __stcs(reinterpret_cast<uint4*>(dst + st_off) + q, w);
      }
    }
    if (FULL || ALL || act) {
#pragma unroll
      for (int j = 0; j < NW; ++j) N[j] = Lw[j];
      mp = m;
    } else {
#pragma unroll
      for (int j = 0; j < NW; ++j) N[j] = 0;
      mp = 0;
    }
    st_off += lw.delta;
  };
  // The steps where every lane of the warp is active: all of them for rows and columns (FULL);
  // for diagonals the common part of the lines' ranges, almost the whole walk, as the warp's lines
  // are adjacent diagonals.  Steps outside it keep the per-lane activity test.
  int s_all_lo = 0, s_all_hi = lw.nsteps - 1;
  if constexpr (!FULL) {
    s_all_lo = __reduce_max_sync(kFull, lw.s_first);
    s_all_hi = __reduce_min_sync(kFull, lw.s_last);  // -1 when some lane has no line
    if (s_all_hi < s_all_lo) s_all_lo = s_all_hi = lw.nsteps;  // no common range
  }
  int s = 0;
  for (; s < s_all_lo; ++s) step(s, std::false_type{});
  // a 2x unrolled loop with a run-time ring slot keeps the code small: the persistent kernel
  // holds three variants of this walk, and fully unrolled they missed the instruction cache
#pragma unroll 2
  for (; s <= s_all_hi && s < lw.nsteps; ++s) step(s, std::true_type{});
  for (; s < lw.nsteps; ++s) step(s, std::false_type{});
  cp_async_wait<0>();  // no copy may still be in flight when the walk ends
}

// The rows (directions (+-1, 0), every line inside the image at every step) walked with G = D/8
// lanes per row that each keep half a 16-disparity group: lane h holds words 4c .. 4c + 3 of
// group h / 2 (c = h % 2), i.e. 8 disparities.  A row's step is then about half the instructions
// of agg_walk's one group per lane, at one more shuffle level for the minimum.  Costs arrive 8
// bytes per lane and step through the warp's ring (32 stages of 32 x 8 bytes, 8 KB); L leaves
// with streaming 8-byte stores.
template <int G>
__device__ __forceinline__ void agg_row_half(const uint8_t* __restrict__ cost,
                                             uint8_t* __restrict__ dst_vol, int W, int H, int D,
                                             int dx, uint32_t P1x2, uint32_t K21x2, int first,
                                             uint4* __restrict__ ring_base) {
  constexpr int LPW = 32 / G;  // rows per warp
  constexpr int ST = 32;       // ring stages
  const int lane = threadIdx.x & 31;
  const int h = lane % G, c = h & 1;
  if (first >= H) return;  // the whole warp leaves together
  const int line = first + lane / G;
  const bool lvalid = line < H;
  const LineWalk lw = line_walk(dx, 0, W, H, D, line, first, min(first + LPW, H) - 1, lvalid);
  const uint8_t* csrc = cost + 8 * h;  // this lane's 8 bytes of the pixel's D
  uint8_t* dst = dst_vol + 8 * h;
  uint32_t N[4] = {0, 0, 0, 0};
  uint32_t mp = 0;
  const uint32_t ring_s =
      (uint32_t)__cvta_generic_to_shared(reinterpret_cast<uint8_t*>(ring_base) + 8 * lane);
  const uint2* ring = reinterpret_cast<const uint2*>(ring_base) + lane;
  long long pf_off = lw.off0;
#pragma unroll
  for (int k = 0; k < ST - 1; ++k) {
    const bool in = lvalid && k < lw.nsteps;
    cp_async8(ring_s + k * 32 * 8, csrc + (in ? pf_off : 0), in ? 8u : 0u);
    cp_async_commit();
    pf_off += lw.delta;
  }
  long long st_off = lw.off0;
  const int src = c == 0 ? lane + 1 : lane - 1;  // the other half of the group
#pragma unroll 2
  for (int s = 0; s < lw.nsteps; ++s) {
    const int k = s & (ST - 1);
    cp_async_wait<ST - 2>();  // the copy of step s is complete
    const uint2 rv = ring[k * 32];
    {
      const int sp = s + ST - 1;
      const bool in = lvalid && sp < lw.nsteps;
      cp_async8(ring_s + ((k + ST - 1) & (ST - 1)) * 32 * 8, csrc + (in ? pf_off : 0),
                in ? 8u : 0u);
      cp_async_commit();
      pf_off += lw.delta;
    }
    // neighbours: the previous lane's last word, the next lane's first word and, across the
    // group's two halves, the group's word 7 (for c = 0) or word 0 (for c = 1)
    uint32_t A = __shfl_up_sync(kFull, N[3], 1, G);
    uint32_t Bn = __shfl_down_sync(kFull, N[0], 1, G);
    if (h == 0) A = kBig2;
    if (h == G - 1) Bn = kBig2;
    const uint32_t Y = __shfl_sync(kFull, c == 1 ? N[3] : N[0], src);
    const uint32_t lft0 = c == 0 ? __byte_perm(A, Y, 0x5432) : A;
    const uint32_t rgt3 = c == 1 ? __byte_perm(Y, Bn, 0x5432) : Bn;
    const uint32_t K = mp + K21x2;
    const uint32_t raw[2] = {rv.x, rv.y};
    uint32_t Lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t lft = j == 0 ? lft0 : N[j > 0 ? j - 1 : 0];
      const uint32_t rgt = j == 3 ? rgt3 : N[j < 3 ? j + 1 : 3];
      uint32_t t = __vimin3_u16x2(lft, rgt, K);
      t = __viaddmin_u16x2(t, P1x2, N[j]);
      const uint32_t cw = __byte_perm(raw[j >> 1], 0, (j & 1) ? 0x4342 : 0x4140);
      Lw[j] = t + cw - mp;
    }
    uint32_t m = __vminu2(__vimin3_u16x2(Lw[0], Lw[1], Lw[2]), Lw[3]);
    m = __vminu2(m, __byte_perm(m, m, 0x1032));
    if constexpr (G == 32) {
      m = __reduce_min_sync(kFull, m);  // both halves equal: the u32 order is the u16 order
    } else {
#pragma unroll
      for (int o = 1; o < G; o <<= 1) m = __vminu2(m, __shfl_xor_sync(kFull, m, o, G));
    }
    if (lvalid)
      __stcs(reinterpret_cast<uint2*>(dst + st_off),
             make_uint2(__byte_perm(Lw[0], Lw[1], 0x6420), __byte_perm(Lw[2], Lw[3], 0x6420)));
#pragma unroll
    for (int j = 0; j < 4; ++j) N[j] = Lw[j];
    mp = m;
    st_off += lw.delta;
  }
  cp_async_wait<0>();  // no copy may still be in flight when the walk ends
}

// ------------------------------------------------------------- volume sums and Eq. (9)
constexpr int kWtaThreads = 128;

// Loads this thread's 16 disparities of S as planar u16x2 pairs (d = 16g + j, 16g + 8 + j).
// All directions' loads are issued before the first sum (ndirs is 4 or 8), so a thread has up to
// 128 bytes in flight.
__device__ __forceinline__ void load_S_il(const uint8_t* __restrict__ vols, int ndirs,
                                          size_t vol_bytes, size_t off, uint32_t sw[8]) {
  uint4 a[8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
    if (r < ndirs) a[r] = __ldcs(reinterpret_cast<const uint4*>(vols + (size_t)r * vol_bytes + off));
#pragma unroll
  for (int j = 0; j < 8; ++j) sw[j] = 0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (r < ndirs) {
      const uint32_t raw[4] = {a[r].x, a[r].y, a[r].z, a[r].w};
#pragma unroll
      for (int j = 0; j < 8; ++j)
        sw[j] = __vadd2(sw[j], __byte_perm(raw[j >> 1], 0, (j & 1) ? 0x4342 : 0x4140));
    }
  }
}

__device__ __forceinline__ void load_S_nat(const uint16_t* __restrict__ S, size_t off,
                                           uint32_t sw[8]) {
  const uint4* src = reinterpret_cast<const uint4*>(S + off);
  uint4 q0 = __ldg(src), q1 = __ldg(src + 1);
  const uint32_t n[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};  // n[k]: d = 2k, 2k+1
#pragma unroll
  for (int j = 0; j < 8; ++j)
    sw[j] = __byte_perm(n[j >> 1], n[4 + (j >> 1)], (j & 1) ? 0x7632 : 0x5410);
}

// Natural-order u32 words k = 0..7 (d = 2k, 2k + 1) from planar pairs.
__device__ __forceinline__ void planar_to_natural(const uint32_t sw[8], uint32_t o[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    o[k] = __byte_perm(sw[2 * k], sw[2 * k + 1], 0x5410);
    o[4 + k] = __byte_perm(sw[2 * k], sw[2 * k + 1], 0x7632);
  }
}

// One block covers P = kWtaThreads / G pixels of one row; G = D / 16 threads per pixel.
// Writes d* (int16) and the sub-pixel value, and folds the right-view candidates of its pixels
// into rkeys[v][x] = min over d of (S(x + d, d) << 8 | d): every thread folds the keys of its 16
// disparities into a shared-memory minimum per column x = u - d, and the block then folds the
// columns it touched into rkeys with one atomicMin each.
// Shared memory: P * D u16 of S, then P + D - 1 u32 column minima (wta_smem_bytes).
__device__ __forceinline__ void wta_block(const uint8_t* __restrict__ vols, int ndirs,
                                          size_t vol_bytes, const uint16_t* __restrict__ S, int W,
                                          int D, int16_t* __restrict__ d_int,
                                          float* __restrict__ dsub, uint32_t* __restrict__ rkeys,
                                          int bx, int v) {
  extern __shared__ uint16_t sS[];  // [P][D], then the column minima
  const int G = D >> 4;
  const int P = kWtaThreads / G;
  const int u0 = bx * P;
  const int Peff = min(P, W - u0);
  const int ncol = Peff + D - 1;  // columns u0 - D + 1 .. u0 + Peff - 1
  uint32_t* sKey = reinterpret_cast<uint32_t*>(sS + P * D);
  for (int i = threadIdx.x; i < ncol; i += kWtaThreads) sKey[i] = 0xffffffffu;
  const int pix = threadIdx.x / G, g = threadIdx.x % G;
  const int u = u0 + pix;
  uint32_t key = 0xffffffffu;
  uint32_t sw[8];
  if (pix < Peff) {
    size_t off = ((size_t)v * W + u) * D + 16 * g;
    uint32_t o[8];
    if (S)
      load_S_nat(S, off, sw);
    else
      load_S_il(vols, ndirs, vol_bytes, off, sw);
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
  __syncthreads();  // column minima initialised, S of the block's pixels in shared memory
  if (pix < Peff) {
    // column of disparity d: u - d, at sKey[pix + D - 1 - d]
    uint32_t* col = sKey + (pix + D - 1 - 16 * g);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      atomicMin(col - j, ((sw[j] & 0xffffu) << 8) | (uint32_t)(16 * g + j));
      atomicMin(col - j - 8, ((sw[j] >> 16) << 8) | (uint32_t)(16 * g + 8 + j));
    }
  }
  if (pix < Peff && g == 0) {
    int ds = (int)(key & 0xffu);
    float sub = (float)ds;
    if (ds > 0 && ds < D - 1) {
      int a = sS[pix * D + ds - 1], b = sS[pix * D + ds], c = sS[pix * D + ds + 1];
      int num = a - c;
      int den = 2 * (a + c - 2 * b);
      if (den > 0) sub = (float)ds + (float)num / (float)den;
    }
    d_int[(size_t)v * W + u] = (int16_t)ds;
    dsub[(size_t)v * W + u] = sub;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ncol; i += kWtaThreads) {
    const int x = u0 - D + 1 + i;
    const uint32_t k = sKey[i];
    if (x >= 0 && k != 0xffffffffu) atomicMin(rkeys + (size_t)v * W + x, k);
  }
}

// Dynamic shared memory of wta_block for disparity range D.
__host__ __device__ constexpr size_t wta_smem_bytes(int D) {
  return (size_t)kWtaThreads * 16 * sizeof(uint16_t) +
         (size_t)(kWtaThreads * 16 / D + D - 1) * sizeof(uint32_t);
}

__device__ __forceinline__ void lr_block(const int16_t* __restrict__ d_int,
                                         const float* __restrict__ dsub,
                                         const uint32_t* __restrict__ rkeys,
                                         const int32_t* __restrict__ kappa, int W, int D, int lr_tol,
                                         float* __restrict__ D1, int bx, int v) {
  int u = bx * blockDim.x + threadIdx.x;
  if (u >= W) return;
  size_t p = (size_t)v * W + u;
  int ds = d_int[p];
  int xr = u - ds;
  bool valid = u >= D - 1 && xr >= 0;
  if (valid) {
    int dr = (int)(rkeys[(size_t)v * W + xr] & 0xffu);
    valid = abs(ds - dr) <= lr_tol;
  }
  float d1 = dsub[p] + (float)kappa[v];
  D1[p] = (valid && d1 >= 0.0f) ? d1 : -1.0f;
}

}  // namespace body
}  // namespace pd
