// Band-restricted SGM: the matching cost, Eq. (8) aggregation, Eq. (9) winner and the left-right
// check of Sec. II-B, each limited to a per-16x16-tile disparity window (an extension beyond the
// paper: the windows come from the band network in cnn.cu, or from the caller).  Outside its
// window a pixel's L is infinite.  The band's cost and L volumes are group-major,
// [D/16][H][W][16 bytes] (interleaved byte order inside each group, as in the full-range path),
// so that the groups of neighbouring pixels are neighbours in memory whatever their windows; only
// the groups that meet a pixel's window are computed, read and written.
#include "common.cuh"
#include "sgm_body.cuh"

namespace pd {

namespace {

using namespace body;

// The cost of a disparity outside its pixel's window.  With every in-window cost at most 24,
// an in-window L is at most 24 + P2 and m + P2 at most 24 + 2 P2; an L computed from a cost of
// 255 is at least 255.  For P2 <= 115 such a value therefore never wins a minimum of Eq. (8)
// over m + P2 and is never the pixel's minimum m: the in-window values are exactly those of the
// recurrence with L = infinity outside the window, and no masking is needed.
constexpr uint32_t kOutCost = 255;

// Interleaved cost of the groups meeting each pixel's window, for kCostBandPix pixels of row v
// per block.  A thread takes four consecutive pixels (one window: a 16-pixel tile holds four such
// chunks) and, as lane l of the chunk's pair, the groups b + l, b + l + 2, ... of the window
// (kOutCost outside the window within those groups).  As in the full-range cost, the four pixels'
// right codes for one group are 19 consecutive words, read as five aligned 16-byte shared loads.
constexpr int kCostBandPix = 256;

// Bytes of word i (d - 16g = 2i, 2i + 8, 2i + 1, 2i + 9) set to 0xff where d is outside the
// window (in16: bit dd set for d = 16g + dd inside it).
__device__ __forceinline__ uint32_t out_bytes(uint32_t in16, int i) {
  const uint32_t out = ~in16;
  return (((out >> (2 * i)) & 1u) * 0xffu) | (((out >> (2 * i + 8)) & 1u) * 0xff00u) |
         (((out >> (2 * i + 1)) & 1u) * 0xff0000u) | (((out >> (2 * i + 9)) & 1u) * 0xff000000u);
}

template <bool CHECK>
__device__ __forceinline__ uint4 cost16_band(uint32_t c0, const uint32_t (&w)[20], int k, int x0,
                                             const uint32_t (&om)[4]) {
  uint32_t c[16];
#pragma unroll
  for (int dd = 0; dd < 16; ++dd) {
    c[dd] = (uint32_t)__popc(c0 ^ w[15 + k - dd]);
    if (CHECK && x0 + k - dd < 0) c[dd] = (uint32_t)kCensusBits;
  }
  return make_uint4(pack4(c[0], c[8], c[1], c[9]) | om[0], pack4(c[2], c[10], c[3], c[11]) | om[1],
                    pack4(c[4], c[12], c[5], c[13]) | om[2], pack4(c[6], c[14], c[7], c[15]) | om[3]);
}

__global__ void __launch_bounds__(kCostBandPix / 2) k_cost_band(const uint32_t* __restrict__ cl,
                                                              const uint32_t* __restrict__ cr,
                                                              int W, int D, BandArgs band,
                                                              size_t plane,
                                                              uint8_t* __restrict__ cost) {
  __shared__ __align__(16) uint32_t sR[kCostBandPix + kMaxD];
  __shared__ __align__(16) uint32_t sL[kCostBandPix];
  const int v = blockIdx.y;
  const int u0 = blockIdx.x * kCostBandPix;
  const int base = u0 - D + 1;  // x of sR[0]; the windows reach sR[kCostBandPix + D - 1]
  for (int i = threadIdx.x; i < kCostBandPix + D; i += blockDim.x) {
    const int x = base + i;
    sR[i] = (x >= 0 && x < W) ? cr[(size_t)v * W + x] : 0u;
  }
  for (int i = threadIdx.x; i < kCostBandPix; i += blockDim.x) {
    const int u = u0 + i;
    sL[i] = u < W ? cl[(size_t)v * W + u] : 0u;
  }
  __syncthreads();
  const int r = 4 * (threadIdx.x >> 1), l = threadIdx.x & 1;  // chunk's first pixel, lane
  const int u = u0 + r;
  if (u >= W) return;
  int lo, hi;
  band_window(band, u, v, D, lo, hi);
  const int e = (hi - 1) >> 4;
  const uint4 cq = *reinterpret_cast<const uint4*>(sL + r);
  const uint32_t c0[4] = {cq.x, cq.y, cq.z, cq.w};
  for (int g = (lo >> 4) + l; g <= e; g += 2) {
    const uint32_t in16 = group_in_mask(g, lo, hi);
    const uint32_t om[4] = {out_bytes(in16, 0), out_bytes(in16, 1), out_bytes(in16, 2),
                            out_bytes(in16, 3)};
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
    uint8_t* dst = cost + plane * g + ((size_t)v * W + u) * 16;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 val = check ? cost16_band<true>(c0[k], w, k, x0, om)
                              : cost16_band<false>(c0[k], w, k, x0, om);
      if (u + k < W) *reinterpret_cast<uint4*>(dst + 16 * k) = val;
    }
  }
}

// ------------------------------------------------------------------ Eq. (8) over the windows
// Compact form: a line is owned by GL lanes, and lane l keeps the 16-disparity groups
// b + GL i + l (slot i = 0 .. NSM - 1) of the current pixel's window, relative to the window's
// first group b = lo / 16.  A 17-disparity window spans 2 groups, i.e. one slot per lane with
// GL = 2, while a full-range pixel uses all NSM = D / (16 GL) slots.  When the window's first group
// moves between consecutive pixels of a line (at a tile edge), the state is realigned: lanes
// exchange slots through shuffles and shift them, and disparities that leave the kept range are
// dropped, except the one just below the new range, which the next step still needs.
// Invariant between steps: slots at or above the current slot count hold the infinity marker.
// Ring depth of the compact kernel (15 steps in flight; a power of two).  Columns and diagonals
// wait on DRAM latency with a shallow ring: at 1920x1080 the band SGM took 0.93 ms with 6 stages,
// 0.83 ms with 12 and 0.715 ms with 16, 20 or 24, although 16 stages leave room for one block
// per SM.
constexpr int kCStages = 16;
static_assert((kCStages & (kCStages - 1)) == 0, "the ring depth is a power of two");
constexpr int kCWarps = 4;
constexpr uint32_t kInf2 = 0x3fff3fffu;

struct Win {
  int b, ns, ng;  // first group, slots in use, groups in the window
};

template <int GL>
__device__ __forceinline__ Win window_of(const BandArgs& band, int u, int v, int D, int& lo,
                                         int& hi) {
  band_window(band, u, v, D, lo, hi);
  Win w;
  w.b = lo >> 4;
  w.ng = ((hi - 1) >> 4) - w.b + 1;
  w.ns = (w.ng + GL - 1) / GL;
  return w;
}

template <int NSM>
__device__ __forceinline__ void shift_slots(uint32_t (&N)[NSM][8], int sh) {
#pragma unroll
  for (int t = 0; t < NSM; ++t) {
    if (sh > 0) {
#pragma unroll
      for (int i = 0; i + 1 < NSM; ++i)
#pragma unroll
        for (int w = 0; w < 8; ++w) N[i][w] = N[i + 1][w];
#pragma unroll
      for (int w = 0; w < 8; ++w) N[NSM - 1][w] = kInf2;
      --sh;
    } else if (sh < 0) {
#pragma unroll
      for (int i = NSM - 1; i > 0; --i)
#pragma unroll
        for (int w = 0; w < 8; ++w) N[i][w] = N[i - 1][w];
#pragma unroll
      for (int w = 0; w < 8; ++w) N[0][w] = kInf2;
      ++sh;
    }
  }
}

// Steps (this one included) that a line moving by (dx, dy) stays in the tile of pixel (u, v).
__device__ __forceinline__ int steps_in_tile(int u, int v, int dx, int dy) {
  const int su = dx > 0 ? 16 - (u & 15) : (dx < 0 ? (u & 15) + 1 : 1 << 30);
  const int sv = dy > 0 ? 16 - (v & 15) : (dy < 0 ? (v & 15) + 1 : 1 << 30);
  return min(su, sv);
}

// One slot of Eq. (8): the 8 words of N[i] with the neighbours prevHi (the word holding d - 1 of
// the slot's first disparity in its high half) and nextLo (d + 1 of the last, in its low half).
__device__ __forceinline__ void eq8_slot(const uint32_t (&n)[8], uint32_t prevHi, uint32_t nextLo,
                                         uint4 rv, uint32_t K, uint32_t P1x2, uint32_t mp,
                                         uint32_t (&Lw)[8]) {
  const uint32_t raw[4] = {rv.x, rv.y, rv.z, rv.w};
  const uint32_t left0 = __byte_perm(prevHi, n[7], 0x5432);
  const uint32_t right7 = __byte_perm(n[0], nextLo, 0x5432);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t lft = j == 0 ? left0 : n[j - 1];
    const uint32_t rgt = j == 7 ? right7 : n[j + 1];
    uint32_t t = __vimin3_u16x2(lft, rgt, K);
    t = __viaddmin_u16x2(t, P1x2, n[j]);
    const uint32_t c = __byte_perm(raw[j >> 1], 0, (j & 1) ? 0x4342 : 0x4140);
    Lw[j] = t + c - mp;
  }
}

__device__ __forceinline__ uint32_t min8(const uint32_t (&Lw)[8]) {
  return __vimin3_u16x2(__vimin3_u16x2(Lw[0], Lw[1], Lw[2]), __vimin3_u16x2(Lw[3], Lw[4], Lw[5]),
                        __vminu2(Lw[6], Lw[7]));
}

__device__ __forceinline__ void store8(uint8_t* p, const uint32_t (&Lw)[8]) {
  uint4 w;
  w.x = __byte_perm(Lw[0], Lw[1], 0x6420);
  w.y = __byte_perm(Lw[2], Lw[3], 0x6420);
  w.z = __byte_perm(Lw[4], Lw[5], 0x6420);
  w.w = __byte_perm(Lw[6], Lw[7], 0x6420);
  __stcs(reinterpret_cast<uint4*>(p), w);
}

// Lines of warp gw: horizontal and vertical lines are taken LPW at a time (16 rows or columns of
// one tile row or column); diagonal lines 16 apart (base + 16 j), so that the pixels of all the
// warp's lines enter new tiles at the same steps.
template <int LPW>
__device__ __forceinline__ void warp_lines(int gw, int dx, int dy, int& base, int& stride) {
  if (dx != 0 && dy != 0) {
    base = (gw >> 4) * (16 * LPW) + (gw & 15);
    stride = 16;
  } else {
    base = gw * LPW;
    stride = 1;
  }
}

template <int GL, int NSM>
__device__ __forceinline__ void agg_compact(const uint8_t* __restrict__ cost,
                                            uint8_t* __restrict__ dst, int W, int H, int D, int dx,
                                            int dy, uint32_t P1x2, uint32_t K21x2, int gw,
                                            int warp, const BandArgs& band, uint4* s_ring,
                                            size_t plane) {
  constexpr int LPW = 32 / GL;
  const int nlines = dy == 0 ? H : (dx == 0 ? W : W + H - 1);
  const int lane = threadIdx.x & 31;
  const int l = lane % GL;
  int first, stride;
  warp_lines<LPW>(gw, dx, dy, first, stride);
  if (first >= nlines) return;  // the whole warp leaves together
  const int line = first + stride * (lane / GL);
  const int last = min(first + stride * (LPW - 1), nlines - 1);
  // offsets of the line's pixels in 16-byte units of one group plane
  const LineWalk lw = line_walk(dx, dy, W, H, 16, line, first, last, line < nlines);

  uint4* ring = s_ring + (size_t)warp * kCStages * NSM * 32 + lane;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  constexpr uint32_t kStageBytes = NSM * 32 * 16;
  const uint4 kOut4 = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);

  // prefetch side: pointer to the prefetched pixel's group l, the window's group offset and the
  // number of slots to load, refreshed when the pixel enters a new tile
  const uint8_t* pf_ptr = cost + lw.off0 + plane * l;
  int p_left = 0, p_nl = 0;
  size_t p_off = 0;
  int pf_stage = 0;
  auto prefetch = [&](int sp) {
    if (sp >= lw.s_first && sp <= lw.s_last) {
      if (p_left == 0) {
        int lo, hi;
        const int pu = lw.u0 + sp * dx, pv = lw.v0 + sp * dy;
        const Win w = window_of<GL>(band, pu, pv, D, lo, hi);
        p_off = plane * w.b;
        p_nl = w.ns - (GL * (w.ns - 1) + l >= w.ng ? 1 : 0);  // slots whose group is in the window
        p_left = steps_in_tile(pu, pv, dx, dy);
      }
      --p_left;
      const uint32_t dsts = ring_s + pf_stage * kStageBytes;
      const uint8_t* src = pf_ptr + p_off;
      if (p_nl == 1) {  // a banded window: one slot
        cp_async16(dsts, src, 16u);
      } else {
#pragma unroll
        for (int i = 0; i < NSM; ++i)
          if (i < p_nl) cp_async16(dsts + i * 32 * 16, src + plane * (GL * i), 16u);
      }
    }
    cp_async_commit();
    pf_ptr += lw.delta;
    pf_stage = (pf_stage + 1) & (kCStages - 1);
  };
  for (int k = 0; k < kCStages - 1; ++k) prefetch(k);

  uint32_t N[NSM][8];
#pragma unroll
  for (int i = 0; i < NSM; ++i)
#pragma unroll
    for (int w = 0; w < 8; ++w) N[i][w] = 0;
  uint32_t mp = 0;
  int b_cur = -1, ns_prev = 0;  // b_cur < 0: the line starts at the next active step
  // consumption side: window of the current pixel, refreshed per tile
  int c_left = 0;
  Win cw{0, NSM, NSM * GL};
  uint8_t* st_ptr = dst + lw.off0 + plane * l;
  size_t st_off = 0;  // plane * cw.b
  int stage = 0;

  int s = 0;
  while (s < lw.nsteps) {  // warp-uniform
    // ---------------------------------------------------------------- one generic step
    const bool act = s >= lw.s_first && s <= lw.s_last;
    cp_async_wait<kCStages - 2>();  // the copies of step s are complete
    prefetch(s + kCStages - 1);     // into the stage of step s - 1, already consumed
    if (act) {
      if (c_left == 0) {
        int lo, hi;
        const int cu = lw.u0 + s * dx, cv = lw.v0 + s * dy;
        cw = window_of<GL>(band, cu, cv, D, lo, hi);
        c_left = steps_in_tile(cu, cv, dx, dy);
        st_off = plane * cw.b;
      }
      --c_left;
    }
    // A line starts from L = 0 and m = 0 at its first active step, which makes that pixel's L
    // equal to its cost.  (Lanes before their line starts may hold anything.)
    bool clear = act && b_cur < 0;
    if (clear) {
#pragma unroll
      for (int i = 0; i < NSM; ++i)
#pragma unroll
        for (int w = 0; w < 8; ++w) N[i][w] = 0;
      mp = 0;
    }
    // ---- realign the state when the window's first group moved (warp-uniform branch)
    uint32_t below = kInf2;
    const bool need = act && b_cur >= 0 && cw.b != b_cur;
    if (__any_sync(kFull, need)) {
      const int kk = need ? cw.b - b_cur : 0;  // new relative group r <- old r + kk
      const int rb = kk - 1;                   // old group just below the new range
      const bool has_b = rb >= 0 && rb < GL * NSM;
      const int sb = has_b ? rb / GL : -1;
      uint32_t v = 0;  // N[sb][7], selected with masks (an indexed read would go to local memory)
#pragma unroll
      for (int i = 0; i < NSM; ++i) v |= N[i][7] & (0u - (uint32_t)(i == sb));
      v = __shfl_sync(kFull, v, has_b ? rb % GL : l, GL);
      below = has_b ? v : kInf2;
      const int q = kk >= 0 ? kk / GL : -((-kk + GL - 1) / GL);  // floor(kk / GL)
      const int rem = kk - q * GL;
      const int src = (l + rem) % GL;
      if (__any_sync(kFull, rem != 0)) {
#pragma unroll
        for (int i = 0; i < NSM; ++i)
#pragma unroll
          for (int w = 0; w < 8; ++w) N[i][w] = __shfl_sync(kFull, N[i][w], src, GL);
      }
      shift_slots<NSM>(N, q + (l + rem >= GL ? 1 : 0));
      clear = clear || need;
    }

    const uint32_t K = mp + K21x2;
    const uint4* rs = ring + stage * (NSM * 32);
    uint32_t m = 0xffffffffu;
    // One slot in use now and before, no realignment: the neighbours outside the lane pair are
    // the infinity marker.
    bool lean = false;
    if constexpr (GL == 2)
      lean = __all_sync(kFull, !act || (cw.ns == 1 && ns_prev <= 1 && !need));
    if (lean) {
      const uint32_t x = __shfl_xor_sync(kFull, l == 0 ? N[0][7] : N[0][0], 1);
      uint32_t Lw[8];
      eq8_slot(N[0], l == 0 ? kInf2 : x, l == 0 ? x : kInf2, l < cw.ng ? rs[0] : kOut4, K, P1x2,
               mp, Lw);
      m = min8(Lw);
      if (act && l < cw.ng) store8(st_ptr + st_off, Lw);
#pragma unroll
      for (int j = 0; j < 8; ++j) N[0][j] = Lw[j];
    } else {
      // ---- generic step: the slots in use (the warp runs the largest count among its lines)
      const int ns_l = act ? cw.ns : 0;
      const int ns_w = __reduce_max_sync(kFull, ns_l);
      uint32_t a_prev = kInf2;                                          // A of slot i - 1
      uint32_t b_nxt = __shfl_sync(kFull, N[0][0], (l + 1) % GL, GL);   // B of slot i
#pragma unroll
      for (int i = 0; i < NSM; ++i) {
        if (i < ns_w) {  // warp-uniform
          const uint32_t a_cur = __shfl_sync(kFull, N[i][7], (l + GL - 1) % GL, GL);
          const uint32_t b_this = b_nxt;
          if (i + 1 < NSM)
            b_nxt = __shfl_sync(kFull, N[i + 1 < NSM ? i + 1 : i][0], (l + 1) % GL, GL);
          const uint32_t prevHi = l > 0 ? a_cur : (i == 0 ? below : a_prev);
          const uint32_t nextLo = l < GL - 1 ? b_this : (i + 1 < NSM ? b_nxt : kInf2);
          a_prev = a_cur;
          const bool ld = GL * i + l < cw.ng;  // groups past the window read as outside costs
          uint32_t Lw[8];
          eq8_slot(N[i], prevHi, nextLo, ld ? rs[i * 32] : kOut4, K, P1x2, mp, Lw);
          if (i < ns_l) {
            m = __vminu2(m, min8(Lw));
            if (ld) store8(st_ptr + st_off + plane * (GL * i), Lw);
#pragma unroll
            for (int j = 0; j < 8; ++j) N[i][j] = Lw[j];
          }
        }
      }
    }
    m = __vminu2(m, __byte_perm(m, m, 0x1032));
#pragma unroll
    for (int o = 1; o < GL; o <<= 1) m = __vminu2(m, __shfl_xor_sync(kFull, m, o, GL));
    if (act) {
      mp = m;
      if (clear || cw.ns < ns_prev) {
#pragma unroll
        for (int i = 0; i < NSM; ++i)
          if (i >= cw.ns)
#pragma unroll
            for (int w = 0; w < 8; ++w) N[i][w] = kInf2;
      }
      b_cur = cw.b;
      ns_prev = cw.ns;
    }
    st_ptr += lw.delta;
    stage = (stage + 1) & (kCStages - 1);
    ++s;

    // ------------------------------------------------ a run of lean steps (two lanes a line)
    // The next R steps keep every line of the warp in one tile, in a one-slot window, and
    // started or not started: no window lookup, realignment, path start or slot loop.
    if constexpr (GL == 2) {
      int r_lane;
      if (s > lw.s_last) {
        r_lane = 1 << 30;                                   // line finished
      } else if (s < lw.s_first) {
        r_lane = lw.s_first - s;                            // line not started yet
      } else {
        r_lane = (b_cur >= 0 && cw.ns == 1 && ns_prev == 1) ? min(c_left, lw.s_last - s + 1) : 0;
      }
      const int R = min((int)__reduce_min_sync(kFull, (unsigned)r_lane), lw.nsteps - s);
      const bool st_ok = s >= lw.s_first && s <= lw.s_last && l < cw.ng;
      const bool ld_ok = l < cw.ng;
      // unrolled twice: the state then alternates between two register sets instead of being
      // copied back every step
#pragma unroll 2
      for (int r = 0; r < R; ++r) {
        cp_async_wait<kCStages - 2>();
        prefetch(s + kCStages - 1);
        const uint32_t Kr = mp + K21x2;
        const uint32_t x = __shfl_xor_sync(kFull, l == 0 ? N[0][7] : N[0][0], 1);
        uint32_t Lw[8];
        eq8_slot(N[0], l == 0 ? kInf2 : x, l == 0 ? x : kInf2,
                 ld_ok ? ring[stage * (NSM * 32)] : kOut4, Kr, P1x2, mp, Lw);
        uint32_t mr = min8(Lw);
        mr = __vminu2(mr, __byte_perm(mr, mr, 0x1032));
        mr = __vminu2(mr, __shfl_xor_sync(kFull, mr, 1));
        if (st_ok) store8(st_ptr + st_off, Lw);
#pragma unroll
        for (int j = 0; j < 8; ++j) N[0][j] = Lw[j];
        mp = mr;
        st_ptr += lw.delta;
        stage = (stage + 1) & (kCStages - 1);
        ++s;
      }
      if (s - R >= lw.s_first && s - R <= lw.s_last) c_left -= R;
    }
  }
  cp_async_wait<0>();  // no copy may still be in flight when the warp exits
}

template <int GL, int NSM>
__global__ void __launch_bounds__(kCWarps * 32, NSM >= 4 ? 4 : 5) k_aggregate_band(
    const uint8_t* __restrict__ cost, uint8_t* __restrict__ out, int W, int H, int D, uint32_t dirs,
    uint32_t P1x2, uint32_t K21x2, size_t vol_bytes, BandArgs band, int ntiles_smem,
    size_t plane) {
  extern __shared__ uint4 s_dyn[];
  const int r = blockIdx.y;
  const uint32_t code = (dirs >> (4 * r)) & 0xfu;
  const int dx = (int)(code & 3u) - 1, dy = (int)(code >> 2) - 1;
  const int warp = threadIdx.x >> 5;
  // the window table, copied once per block when it fits (lookups then cost a shared load)
  if (ntiles_smem > 0) {
    int16_t* t = reinterpret_cast<int16_t*>(s_dyn + kCWarps * kCStages * NSM * 32);
    for (int i = threadIdx.x; i < ntiles_smem; i += blockDim.x) t[i] = band.tile_lo[i];
    __syncthreads();
    band.tile_lo = t;
  }
  agg_compact<GL, NSM>(cost, out + (size_t)r * vol_bytes, W, H, D, dx, dy, P1x2, K21x2,
                       blockIdx.x * kCWarps + warp, warp, band, s_dyn, plane);
}

// 0xFFFF in every u16 half of word j whose disparity lies outside the window.
__device__ __forceinline__ uint32_t out_fill(uint32_t in16, int j) {
  const uint32_t out = ~in16;
  return (((out >> j) & 1u) * 0xffffu) | (((out >> (8 + j)) & 1u) * 0xffff0000u);
}

// Eq. (9) over the windows: 64 pixels of row v per block, two lanes per pixel; lane l handles
// the window's groups b + 2 i + l (as in the aggregation).  S is marked 0xFFFF outside the window
// (in-window sums stay below 8 * (24 + 255)).  The parabola needs d* - 1 and d* + 1 inside the
// window.  The right view of column x takes only candidates d inside the window of pixel x + d:
// each lane folds the keys (S << 8 | d) of its in-window disparities into a shared-memory minimum
// per column, and the block then folds the touched columns into rkeys with one atomicMin each.
constexpr int kWtaBandPix = 64;

__global__ void __launch_bounds__(2 * kWtaBandPix) k_wta_band(const uint8_t* __restrict__ vols,
                                                              int ndirs, size_t vol_bytes, int W,
                                                              int D, BandArgs band, size_t plane,
                                                              int16_t* __restrict__ d_int,
                                                              float* __restrict__ dsub,
                                                              uint32_t* __restrict__ rkeys) {
  extern __shared__ uint16_t sS[];  // [kWtaBandPix][D] then the column minima (u32)
  const int v = blockIdx.y;
  const int u0 = blockIdx.x * kWtaBandPix;
  const int Peff = min(kWtaBandPix, W - u0);
  const int ncol = Peff + D - 1;
  uint32_t* sKey = reinterpret_cast<uint32_t*>(sS + kWtaBandPix * D);
  for (int i = threadIdx.x; i < ncol; i += 2 * kWtaBandPix) sKey[i] = 0xffffffffu;
  __syncthreads();
  const int pix = threadIdx.x >> 1, l = threadIdx.x & 1;
  const int u = u0 + pix;
  const int xbase = u0 - D + 1;  // column of sKey[0]
  uint32_t key = 0xffffffffu;
  int lo = 0, hi = D;
  if (pix < Peff) {
    band_window(band, u, v, D, lo, hi);
    const int b = lo >> 4, e = (hi - 1) >> 4;
    const size_t off = ((size_t)v * W + u) * 16;
    for (int g = b + l; g <= e; g += 2) {
      const uint32_t in16 = group_in_mask(g, lo, hi);
      uint32_t sw[8], o[8];
      load_S_il(vols, ndirs, vol_bytes, off + plane * g, sw);
#pragma unroll
      for (int j = 0; j < 8; ++j) sw[j] |= out_fill(in16, j);
      planar_to_natural(sw, o);
      uint4* row = reinterpret_cast<uint4*>(sS + pix * D + 16 * g);
      row[0] = make_uint4(o[0], o[1], o[2], o[3]);
      row[1] = make_uint4(o[4], o[5], o[6], o[7]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int d = 16 * g + j + 8 * h;
          const uint32_t sv = h ? (sw[j] >> 16) : (sw[j] & 0xffffu);
          const uint32_t kd = (sv << 8) | (uint32_t)d;
          if (sv != 0xffffu) {
            key = min(key, kd);
            if (u - d >= 0) atomicMin(sKey + (u - d - xbase), kd);
          }
        }
      }
    }
  }
  key = min(key, __shfl_xor_sync(kFull, key, 1));
  __syncthreads();
  if (pix < Peff && l == 0) {
    const int ds = (int)(key & 0xffu);
    float sub = (float)ds;
    if (ds - 1 >= lo && ds + 1 < hi) {
      const int a = sS[pix * D + ds - 1], bb = sS[pix * D + ds], c = sS[pix * D + ds + 1];
      const int num = a - c;
      const int den = 2 * (a + c - 2 * bb);
      if (den > 0) sub = (float)ds + (float)num / (float)den;
    }
    d_int[(size_t)v * W + u] = (int16_t)ds;
    dsub[(size_t)v * W + u] = sub;
  }
  for (int i = threadIdx.x; i < ncol; i += 2 * kWtaBandPix) {
    const uint32_t k = sKey[i];
    if (k != 0xffffffffu) atomicMin(rkeys + (size_t)v * W + xbase + i, k);
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
  k_cost_band<<<dim3((W + kCostBandPix - 1) / kCostBandPix, H), kCostBandPix / 2, 0, s>>>(
      cl, cr, W, D, band, (size_t)W * H * 16, cost);
}

constexpr int kMaxSmemTiles = 16384;  // 32 KB of window table in shared memory

template <int GL, int NSM>
void launch_compact(cudaStream_t s, dim3 grid, const uint8_t* cost_il, uint8_t* out, int W, int H,
                    int D, uint32_t packed, uint32_t P1x2, uint32_t K21x2, size_t vol_bytes,
                    const BandArgs& band) {
  const int ntiles = ((H + 15) / 16) * band.tw;
  const int nsm = ntiles <= kMaxSmemTiles ? ntiles : 0;
  const size_t ring = (size_t)kCWarps * kCStages * NSM * 32 * sizeof(uint4);
  const size_t smem = ring + (((size_t)nsm * sizeof(int16_t) + 15) & ~size_t(15));
  raise_smem_limit((const void*)k_aggregate_band<GL, NSM>, smem);
  k_aggregate_band<GL, NSM><<<grid, kCWarps * 32, smem, s>>>(cost_il, out, W, H, D, packed, P1x2,
                                                             K21x2, vol_bytes, band, nsm,
                                                             (size_t)W * H * 16);
}

void launch_aggregate_band(cudaStream_t s, const uint8_t* cost_il, int W, int H, int D,
                           const DirSet& dirs, int P1, int P2, uint8_t* out, size_t vol_bytes,
                           const BandArgs& band) {
  const int GL = D == 256 ? 4 : 2;
  const int LPW = 32 / GL;
  int maxwarps = 0;
  for (int r = 0; r < dirs.n; ++r) {
    const bool diag = dirs.dx[r] != 0 && dirs.dy[r] != 0;
    const int n = dirs.dy[r] == 0 ? H : (dirs.dx[r] == 0 ? W : W + H - 1);
    const int w = diag ? 16 * ((n + 16 * LPW - 1) / (16 * LPW)) : (n + LPW - 1) / LPW;
    maxwarps = w > maxwarps ? w : maxwarps;
  }
  dim3 grid((maxwarps + kCWarps - 1) / kCWarps, dirs.n);
  const uint32_t P1x2 = (uint32_t)P1 * 0x10001u;
  const uint32_t K21x2 = (uint32_t)(P2 - P1) * 0x10001u;
  uint32_t packed = 0;
  for (int r = 0; r < dirs.n; ++r)
    packed |= ((uint32_t)(dirs.dx[r] + 1) | ((uint32_t)(dirs.dy[r] + 1) << 2)) << (4 * r);
  switch (D) {
    case 32: launch_compact<2, 1>(s, grid, cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    case 64: launch_compact<2, 2>(s, grid, cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    case 128: launch_compact<2, 4>(s, grid, cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    case 256: launch_compact<4, 4>(s, grid, cost_il, out, W, H, D, packed, P1x2, K21x2, vol_bytes, band); break;
    default: break;  // the API admits D in {32, 64, 128, 256} only
  }
}

void launch_wta_band(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes, int W,
                     int H, int D, const BandArgs& band, int16_t* d_int, float* dsub,
                     uint32_t* rkeys) {
  const size_t smem = (size_t)kWtaBandPix * D * sizeof(uint16_t) +
                      (size_t)(kWtaBandPix + D - 1) * sizeof(uint32_t);
  raise_smem_limit((const void*)k_wta_band, smem);
  k_wta_band<<<dim3((W + kWtaBandPix - 1) / kWtaBandPix, H), 2 * kWtaBandPix, smem, s>>>(
      vols, ndirs, vol_bytes, W, D, band, (size_t)W * H * 16, d_int, dsub, rkeys);
}

void launch_lr_band(cudaStream_t s, const int16_t* d_int, const float* dsub, const uint32_t* rkeys,
                    const int32_t* kappa, int W, int H, int D, const BandArgs& band, int lr_tol,
                    float* D1) {
  k_lr_band<<<dim3((W + 255) / 256, H), 256, 0, s>>>(d_int, dsub, rkeys, kappa, W, D, band, lr_tol,
                                                    D1);
}

}  // namespace pd
