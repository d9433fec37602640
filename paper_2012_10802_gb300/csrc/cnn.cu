// The band network (an extension beyond the paper): predicts, per 16x16 tile, the centre of the
// tile's disparities after the perspective transformation of Sec. II-A and a confidence, so that
// the SGM of Sec. II-B can search a 17-disparity window instead of the full range.
//
// Network: 3x3 convolutions, zero padding 1, strides 1, 2, 2, 1, channels 2 -> 32 -> 32 -> 32 -> 2,
// ReLU after the first three, on the 4x-block-averaged row-shifted pair.  Activations are bf16,
// NHWC.  Every contraction runs on the fifth-generation tensor cores (bf16 operands in shared
// memory, fp32 accumulators in tensor memory, one issuing thread per CTA): each convolution is an
// implicit GEMM over the patch matrix (k = (ky * 3 + kx) * Cin + ci), and the backward pass computes
// dW = dZ^T Col (split over pixels, partial sums added in a fixed order) and dCol = dZ W with
// operands read in place
// (MN-major where the contraction runs along their rows), then a gather col2im that applies the
// previous layer's ReLU mask.  Training is Adam on fp32 master weights.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>
#include <string.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace pd {

namespace {

// ------------------------------------------------------------------- convolution on tcgen05
// One CTA computes 128 output pixels x all output channels of a 3x3 convolution (zero padding 1)
// as an implicit GEMM with K = Kp (k = (ky * 3 + kx) * Cin + ci, zeros up to Kp):
//  * the 128 x Kp patch matrix is gathered straight from the NHWC input into shared memory in
//    the K-major core-matrix layout (rows 8 r8 .. 8 r8 + 7 of k-group g at g * 2048 + r8 * 128
//    bytes), the weights [CoutP][Kp] likewise with N rows (rows >= CoutP zero), and the bias;
//  * one thread issues Kp / 16 MMAs of 128 x N x 16 into a TMEM accumulator of N fp32 columns and
//    commits them to an mbarrier, which every thread waits on (bounded);
//  * warp w reads rows 32 (w mod 4) .. + 31, columns 8 (w / 4) .. + 7 back, adds the bias and
//    stores bf16 [P][32] after ReLU (hidden layers) or fp32 [P][2] (output layer, N = 16).
// 16 warps per CTA: the grids of the later layers are small (64 CTAs at 1080p), so each CTA's
// gather and read-back are spread over as many threads as it has (row, 8-channel) pieces.
// With WRITE_COL the gathered patches also go to Col [P][Kp] for the backward pass.
constexpr int kConvM = 128, kConvThreads = 512;
constexpr long long kConvWaitCycles = 1ll << 31;  // about a second at the SM clock

struct ConvArgs {
  const __nv_bfloat16* X;  // [B][H][W][Cin]
  int B, H, W, Ho, Wo, stride;
  const __nv_bfloat16* Wt;  // [coutp][Kp]
  int coutp;
  const float* bias;  // [32], 16-byte aligned
  void* out;
  __nv_bfloat16* col;
  int* status;  // bit 0 set when the MMA wait ran out
  int P;        // B * Ho * Wo (< 2^31 / 36 by the network's size limit)
  long long wait_limit;
  int issue;  // 0 issues no MMA, so that the wait runs out (the timeout path's test)
};

__host__ __device__ constexpr int conv_kp(int cin) { return cin == 32 ? 288 : 32; }

// Dynamic shared memory of one CTA: the patch tile, the weight tile, the bias.
constexpr size_t conv_smem_bytes(int cin, int n) {
  return (size_t)(conv_kp(cin) / 8) * (kConvM + n) * 16 + 32 * sizeof(float);
}

template <int CIN, int N, bool F32OUT, bool WRITE_COL>
__global__ void __launch_bounds__(kConvThreads) k_conv_tc(ConvArgs a) {
  constexpr int KP = conv_kp(CIN), KG = KP / 8;
  constexpr uint32_t kGroupA = kConvM * 16, kGroupB = N * 16;  // bytes per k-group
  constexpr uint32_t kCols = N < 32 ? 32 : N;
  extern __shared__ __align__(128) uint8_t conv_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kConvM;
  const uint32_t sA = tc::smem_addr(conv_smem), sB = sA + KG * kGroupA;
  const uint32_t sBias = sB + KG * kGroupB;
  const float* bias_s = reinterpret_cast<const float*>(conv_smem + KG * kGroupA + KG * kGroupB);
  const uint32_t bar = tc::smem_addr(&mbar);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tslot), kCols);
  if (tid == 0) tc::mbar_init(bar, 1);

  for (int c = tid; c < KG * N; c += kConvThreads) {
    const int n = c % N, g = c / N;
    const bool ok = n < a.coutp;
    tc::cp_async16(sB + g * kGroupB + n * 16, a.Wt + (ok ? n * KP + g * 8 : 0), ok ? 16u : 0u);
  }
  if (tid < 8) tc::cp_async16(sBias + tid * 16, a.bias + tid * 4, 16u);
  if (CIN == 32) {
    // thread: channel quarter q of row tid / 4, all 9 taps (4 lanes read one 64-byte pixel)
    const int q = tid & 3, row = tid >> 2;
    const int p = m0 + row;
    const bool vp = p < a.P;
    int b = 0, oy = 0, ox = 0;
    if (vp) {
      ox = p % a.Wo;
      const int t = p / a.Wo;
      oy = t % a.Ho;
      b = t / a.Ho;
    }
    const int y0 = oy * a.stride - 1, x0 = ox * a.stride - 1;
    const __nv_bfloat16* base = a.X + ((size_t)b * a.H * a.W) * 32 + q * 8;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int y = y0 + tap / 3, x = x0 + tap % 3;
      const bool ok = vp && y >= 0 && y < a.H && x >= 0 && x < a.W;
      const __nv_bfloat16* src = ok ? base + ((size_t)y * a.W + x) * 32 : a.X;
      const uint32_t off = (tap * 4 + q) * kGroupA + row * 16;
      if (WRITE_COL) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (ok) v = *reinterpret_cast<const uint4*>(src);
        *reinterpret_cast<uint4*>(conv_smem + off) = v;
        if (vp) *reinterpret_cast<uint4*>(a.col + (size_t)p * KP + tap * 32 + q * 8) = v;
      } else {
        tc::cp_async16(sA + off, src, ok ? 16u : 0u);
      }
    }
  } else {
    // Cin = 2: thread = (row, k-group g); g holds taps 4 g .. 4 g + 3 (two channels each), taps
    // >= 9 are zero; one 16-byte shared store per thread (consecutive rows, consecutive bytes)
    const int row = tid & 127, g = tid >> 7;
    const int p = m0 + row;
    const bool vp = p < a.P;
    int b = 0, oy = 0, ox = 0;
    if (vp) {
      ox = p % a.Wo;
      const int t = p / a.Wo;
      oy = t % a.Ho;
      b = t / a.Ho;
    }
    const uint32_t* img = reinterpret_cast<const uint32_t*>(a.X) + (size_t)b * a.H * a.W;
    uint32_t v[4];
#pragma unroll
    for (int t4 = 0; t4 < 4; ++t4) {
      const int tap = 4 * g + t4;
      const int y = oy * a.stride + tap / 3 - 1, x = ox * a.stride + tap % 3 - 1;
      const bool ok = vp && tap < 9 && y >= 0 && y < a.H && x >= 0 && x < a.W;
      v[t4] = ok ? img[(size_t)y * a.W + x] : 0u;
    }
    const uint4 u = make_uint4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<uint4*>(conv_smem + g * kGroupA + row * 16) = u;
    if (WRITE_COL && vp) *reinterpret_cast<uint4*>(a.col + (size_t)p * KP + g * 8) = u;
  }
  tc::cp_async_wait_all();
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;

  if (tid == 0 && a.issue) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kConvM, N);
#pragma unroll 1
    for (int ks = 0; ks < KP / 16; ++ks) {
      const uint64_t ad = tc::smem_desc(sA + ks * 2 * kGroupA, kGroupA, 128);
      const uint64_t bd = tc::smem_desc(sB + ks * 2 * kGroupB, kGroupB, 128);
      tc::mma_bf16(taddr, ad, bd, idesc, ks > 0 ? 1u : 0u);
    }
    tc::mma_commit(bar);
  }
  const bool done = __all_sync(0xffffffffu, tc::mbar_wait_bounded(bar, 0, a.wait_limit));
  tc::fence_after_sync();
  const int quarter = warp & 3, cblk = warp >> 2;  // lanes 32 quarter .., columns 8 cblk ..
  if (!done) {
    if (lane == 0) atomicOr(a.status, 1);
  } else if (8 * cblk < N) {
    uint32_t r[8];
    tc::tmem_ld8(taddr + ((uint32_t)(quarter * 32) << 16) + 8 * cblk, r);
    const int p = m0 + quarter * 32 + lane;
    if (p < a.P) {
      if (!F32OUT) {
        uint32_t h[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int n = 8 * cblk + 2 * i;
          const float v0 = fmaxf(__uint_as_float(r[2 * i]) + bias_s[n], 0.0f);
          const float v1 = fmaxf(__uint_as_float(r[2 * i + 1]) + bias_s[n + 1], 0.0f);
          const __nv_bfloat162 t = __floats2bfloat162_rn(v0, v1);
          h[i] = *reinterpret_cast<const uint32_t*>(&t);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + (size_t)p * 32 +
                                  8 * cblk) = make_uint4(h[0], h[1], h[2], h[3]);
      } else if (cblk == 0) {
        reinterpret_cast<float2*>(a.out)[p] = make_float2(__uint_as_float(r[0]) + bias_s[0],
                                                          __uint_as_float(r[1]) + bias_s[1]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    // after a timeout the MMAs may still be running: give them another bounded wait
    if (!done && a.issue) tc::mbar_wait_bounded(bar, 0, a.wait_limit);
    tc::tmem_dealloc(taddr, kCols);
  }
}

template <int CIN, int N, bool F32OUT, bool WRITE_COL>
void conv_tc(cudaStream_t s, const ConvArgs& a) {
  const size_t smem = conv_smem_bytes(CIN, N);
  raise_smem_limit((const void*)k_conv_tc<CIN, N, F32OUT, WRITE_COL>, smem);
  const unsigned blocks = (unsigned)((a.P + kConvM - 1) / kConvM);
  k_conv_tc<CIN, N, F32OUT, WRITE_COL><<<blocks ? blocks : 1, kConvThreads, smem, s>>>(a);
}

// ----------------------------------------------------------------- backward GEMMs on tcgen05
constexpr int kBwdThreads = 256;

// dCol[p][k] = sum_co dZ[p][co] W[co][k] (layers 2-4, Kp = 288).  One CTA per 128 pixels:
//  * A = dZ rows, K-major (co-group g of row r at g * 2048 + r * 16); co-groups beyond ldz zero;
//  * B = W read MN-major: a core-matrix row is 8 consecutive k of one co, k-group ng and co-group
//    cg at ng * 512 + cg * 128 (no transpose on the way in);
//  * K = CoutP (32, or 16 with co >= 8 zero for the output layer); N = 288 as two MMAs of 144
//    columns into a 512-column accumulator; 8 warps read back 144 columns each.
struct DcolArgs {
  const __nv_bfloat16* dZ;  // [P][ldz]
  int ldz;                  // 32, or 8 for the output layer
  const __nv_bfloat16* Wt;  // [coutp][288]
  int coutp;
  float* dcol;  // [P][288]
  int* status;
  int P;
  long long wait_limit;
};

constexpr size_t dcol_smem_bytes() { return 4 * (size_t)kConvM * 16 + 36 * 512; }

__global__ void __launch_bounds__(kBwdThreads) k_dcol_tc(DcolArgs a) {
  constexpr int KP = 288, NG = KP / 8, KC = 32;
  constexpr uint32_t kGroupA = kConvM * 16, kNGroup = (KC / 8) * 128;
  extern __shared__ __align__(128) uint8_t bwd_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kConvM;
  const uint32_t sA = tc::smem_addr(bwd_smem), sB = sA + (KC / 8) * kGroupA;
  const uint32_t bar = tc::smem_addr(&mbar);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tslot), 512);
  if (tid == 0) tc::mbar_init(bar, 1);
  const int ksteps = a.coutp > 8 ? 2 : 1;
  for (int c = tid; c < kConvM * (KC / 8); c += kBwdThreads) {
    const int row = c & 127, g = c >> 7;
    const int p = m0 + row;
    const bool ok = p < a.P && g * 8 < a.ldz;
    tc::cp_async16(sA + g * kGroupA + row * 16, a.dZ + (ok ? (size_t)p * a.ldz + g * 8 : 0),
                   ok ? 16u : 0u);
  }
  for (int c = tid; c < NG * KC; c += kBwdThreads) {
    const int ng = c % NG, co = c / NG;
    const bool ok = co < a.coutp;
    tc::cp_async16(sB + ng * kNGroup + (co >> 3) * 128 + (co & 7) * 16,
                   a.Wt + (ok ? co * KP + ng * 8 : 0), ok ? 16u : 0u);
  }
  tc::cp_async_wait_all();
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  if (tid == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kConvM, 144, false, true);
    for (int j = 0; j < ksteps; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint64_t ad = tc::smem_desc(sA + j * 2 * kGroupA, kGroupA, 128);
        const uint64_t bd = tc::smem_desc(sB + 18 * h * kNGroup + j * 2 * 128, 128, kNGroup);
        tc::mma_bf16(taddr + 144 * h, ad, bd, idesc, j > 0 ? 1u : 0u);
      }
    tc::mma_commit(bar);
  }
  const bool done = __all_sync(0xffffffffu, tc::mbar_wait_bounded(bar, 0, a.wait_limit));
  tc::fence_after_sync();
  if (!done) {
    if (lane == 0) atomicOr(a.status, 1);
  } else {
    const int quarter = warp & 3, half = warp >> 2;
    const int p = m0 + quarter * 32 + lane;
    const uint32_t trow = taddr + ((uint32_t)(quarter * 32) << 16) + 144 * half;
    float4* dst = reinterpret_cast<float4*>(a.dcol + (size_t)p * KP + 144 * half);
#pragma unroll 1
    for (int i = 0; i < 9; ++i) {
      uint32_t r[16];
      tc::tmem_ld16(trow + 16 * i, r);
      if (p < a.P) {
#pragma unroll
        for (int v = 0; v < 4; ++v)
          dst[4 * i + v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                       __uint_as_float(r[4 * v + 2]),
                                       __uint_as_float(r[4 * v + 3]));
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    if (!done) tc::mbar_wait_bounded(bar, 0, a.wait_limit);
    tc::tmem_dealloc(taddr, 512);
  }
}

// part[r][co][k] = sum over pixel range r of Col[p][k] dZ[p][co].  Grid: (pixel ranges, k-tiles of
// 128); the CTA accumulates D[k][co] in TMEM over 64-pixel stages and writes its range's partial
// sums; k_sum_ranges then adds the ranges in a fixed order (no atomics: training is
// bit-reproducible run to run).
//  * A = Col read MN-major: a core-matrix row is 8 consecutive k of one pixel, k-group kg and
//    pixel-group pg of a stage at kg * 1024 + pg * 128;
//  * B = dZ read MN-major likewise (co-groups; those beyond ldz zero);
//  * two stage buffers: each is refilled once the commit of the MMAs that read it has arrived.
struct DwArgs {
  const __nv_bfloat16* col;  // [P][kp]
  int kp;                    // 32 or 288
  const __nv_bfloat16* dZ;   // [P][ldz]
  int ldz;
  float* part;  // [ranges][coutp][kp]: this CTA's pixel range's partial sums
  int coutp;
  int* status;
  int P, chunk;  // pixels per CTA, a multiple of 64
  long long wait_limit;
};

constexpr int kDwStage = 64;
constexpr int kBiasBlocks = 2048;  // at most this many blocks sum the bias gradient
constexpr size_t dw_smem_bytes(int n) { return 2 * (size_t)(16 + n / 8) * 1024; }

template <int N>  // co columns: 32, or 16 for the output layer
__global__ void __launch_bounds__(kBwdThreads) k_dw_tc(DwArgs a) {
  constexpr uint32_t kStageA = 16 * 1024, kStageB = (N / 8) * 1024;
  extern __shared__ __align__(128) uint8_t bwd_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k0 = blockIdx.y * 128;
  const int p_begin = blockIdx.x * a.chunk, p_end = min(a.P, p_begin + a.chunk);
  const int stages = (p_end - p_begin + kDwStage - 1) / kDwStage;
  const uint32_t s0 = tc::smem_addr(bwd_smem);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(&tslot), 32);
  if (tid == 0) {
    tc::mbar_init(tc::smem_addr(&mbar[0]), 1);
    tc::mbar_init(tc::smem_addr(&mbar[1]), 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, N, true, true);
  bool ok = true;
  int last = -1;  // last stage whose MMAs were committed
  for (int s = 0; s < stages; ++s) {
    const int buf = s & 1;
    if (s >= 2) {
      const bool w = tc::mbar_wait_bounded(tc::smem_addr(&mbar[buf]), ((s >> 1) - 1) & 1,
                                           a.wait_limit);
      if (__syncthreads_or(!w)) {
        ok = false;
        break;
      }
    }
    const uint32_t sa = s0 + buf * (kStageA + kStageB), sb = sa + kStageA;
    const int ps = p_begin + s * kDwStage;
    for (int c = tid; c < kDwStage * 16; c += kBwdThreads) {
      const int kg = 4 * (c >> 8) + (c & 3), pl = (c >> 2) & 63;
      const int p = ps + pl, k = k0 + kg * 8;
      const bool okc = p < p_end && k < a.kp;
      tc::cp_async16(sa + kg * 1024 + pl * 16, a.col + (okc ? (size_t)p * a.kp + k : 0),
                     okc ? 16u : 0u);
    }
    for (int c = tid; c < kDwStage * (N / 8); c += kBwdThreads) {
      const int cg = c % (N / 8), pl = c / (N / 8);
      const int p = ps + pl;
      const bool okc = p < p_end && cg * 8 < a.ldz;
      tc::cp_async16(sb + cg * 1024 + pl * 16, a.dZ + (okc ? (size_t)p * a.ldz + cg * 8 : 0),
                     okc ? 16u : 0u);
    }
    tc::cp_async_wait_all();
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int j = 0; j < kDwStage / 16; ++j)
        tc::mma_bf16(taddr, tc::smem_desc(sa + j * 256, 128, 1024),
                     tc::smem_desc(sb + j * 256, 128, 1024), idesc, (s > 0 || j > 0) ? 1u : 0u);
      tc::mma_commit(tc::smem_addr(&mbar[buf]));
    }
    last = s;
  }
  if (ok) {
    const bool w = tc::mbar_wait_bounded(tc::smem_addr(&mbar[last & 1]), (last >> 1) & 1,
                                         a.wait_limit);
    ok = !__syncthreads_or(!w);
  }
  tc::fence_after_sync();
  const int quarter = warp & 3, half = warp >> 2;
  if (!ok) {
    if (tid == 0) atomicOr(a.status, 1);
  } else if (16 * half < N) {
    uint32_t r[16];
    tc::tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + 16 * half, r);
    const int k = k0 + quarter * 32 + lane;
    if (k < a.kp)
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int co = 16 * half + i;
        if (co < a.coutp)
          a.part[((size_t)blockIdx.x * a.coutp + co) * a.kp + k] = __uint_as_float(r[i]);
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    // after a timeout the MMAs may still be running: give them another bounded wait
    if (!ok && last >= 0)
      tc::mbar_wait_bounded(tc::smem_addr(&mbar[last & 1]), (last >> 1) & 1, a.wait_limit);
    tc::tmem_dealloc(taddr, 32);
  }
}

void dcol_tc(cudaStream_t s, const DcolArgs& a) {
  raise_smem_limit((const void*)k_dcol_tc, dcol_smem_bytes());
  k_dcol_tc<<<(a.P + kConvM - 1) / kConvM, kBwdThreads, dcol_smem_bytes(), s>>>(a);
}

// out[i] = sum over r = 0 .. ranges - 1 of part[r][i], in that order.
__global__ void k_sum_ranges(const float* __restrict__ part, int ranges, int n,
                             float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float acc = 0.0f;
  for (int r = 0; r < ranges; ++r) acc += part[(size_t)r * n + i];
  out[i] = acc;
}

// Pixel ranges sized for about two CTAs per SM over all k-tiles (at most 2 sms ranges, the rows
// of the partial-sum buffer); dW = the ranges' sum.
template <int N>
void dw_tc(cudaStream_t s, DwArgs a, int sms, float* dW) {
  const int ktiles = (a.kp + 127) / 128;
  const int ranges = std::max(1, 2 * sms / ktiles);
  a.chunk = std::max(kDwStage, ((a.P + ranges - 1) / ranges + kDwStage - 1) / kDwStage * kDwStage);
  raise_smem_limit((const void*)k_dw_tc<N>, dw_smem_bytes(N));
  const int used = (a.P + a.chunk - 1) / a.chunk;  // <= ranges
  dim3 grid(used, ktiles);
  k_dw_tc<N><<<grid, kBwdThreads, dw_smem_bytes(N), s>>>(a);
  const int n = a.coutp * a.kp;
  k_sum_ranges<<<(n + 255) / 256, 256, 0, s>>>(a.part, used, n, dW);
}

// dA(b, y, x, c) = mask(b, y, x, c) * sum over taps with oy = (y + 1 - ky) / s, ox = (x + 1 - kx) / s
// integral and in range of dCol[(b, oy, ox)][(ky * 3 + kx) * 32 + c]; mask = (A > 0).  One thread
// per (pixel, 8 channels); bf16 out.
__global__ void k_col2im32(const float* __restrict__ dcol, const __nv_bfloat16* __restrict__ A,
                           int B, int H, int W, int Ho, int Wo, int stride,
                           __nv_bfloat16* __restrict__ dA) {
  const size_t total = (size_t)B * H * W * 4;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t & 3);
    const size_t p = t >> 2;
    const int x = (int)(p % W);
    const size_t by = p / W;
    const int y = (int)(by % H);
    const int b = (int)(by / H);
    float s[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = 0.0f;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int ny = y + 1 - ky;
      if (ny < 0 || ny % stride) continue;
      const int oy = ny / stride;
      if (oy >= Ho) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int nx = x + 1 - kx;
        if (nx < 0 || nx % stride) continue;
        const int ox = nx / stride;
        if (ox >= Wo) continue;
        const float4* src = reinterpret_cast<const float4*>(
            dcol + (((size_t)b * Ho + oy) * Wo + ox) * 288 + (ky * 3 + kx) * 32 + q * 8);
        const float4 u0 = src[0], u1 = src[1];
        s[0] += u0.x; s[1] += u0.y; s[2] += u0.z; s[3] += u0.w;
        s[4] += u1.x; s[5] += u1.y; s[6] += u1.z; s[7] += u1.w;
      }
    }
    const uint4 av = *reinterpret_cast<const uint4*>(A + p * 32 + q * 8);
    const __nv_bfloat16* a = reinterpret_cast<const __nv_bfloat16*>(&av);
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
      o[i] = __float2bfloat16_rn(__bfloat162float(a[i]) > 0.0f ? s[i] : 0.0f);
    *reinterpret_cast<uint4*>(dA + p * 32 + q * 8) = *reinterpret_cast<const uint4*>(o);
  }
}

// part[b][c] = sum over block b's rows of dZ[p][c] (C channels, ld columns per row); the blocks'
// sums are then added in block order by k_sum_ranges.
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dZ, size_t P, int C, int ld,
                            float* __restrict__ out_part) {
  __shared__ float part[256];
  const int c = threadIdx.x % C;
  const int rows_per_pass = blockDim.x / C;
  float s = 0.0f;
  for (size_t p = (size_t)blockIdx.x * rows_per_pass + threadIdx.x / C; p < P;
       p += (size_t)gridDim.x * rows_per_pass)
    s += __bfloat162float(dZ[p * ld + c]);
  part[threadIdx.x] = s;
  __syncthreads();
  if ((int)threadIdx.x < C) {
    float t = 0.0f;
    for (int r = 0; r < rows_per_pass; ++r) t += part[r * C + threadIdx.x];
    out_part[(size_t)blockIdx.x * C + threadIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------- loss
// Weight totals n_c = sum of centre weights, n_b = sum of confidence weights.
__global__ void k_loss_counts(const float* __restrict__ tgt, size_t P, float* __restrict__ cnt) {
  float a = 0.0f, b = 0.0f;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (size_t)gridDim.x * blockDim.x) {
    a += tgt[p * 4 + 2];
    b += tgt[p * 4 + 3];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(cnt, a);
    atomicAdd(cnt + 1, b);
  }
}

// Huber (delta 1) on out0 - centre / 16 over the centre weights plus the logistic loss of out1
// over the confidence weights, each divided by max(1, its weight total).  Writes dZ [P][8] (bf16,
// columns 2..7 zero) and adds the loss to *loss.
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ tgt, size_t P,
                       const float* __restrict__ cnt, __nv_bfloat16* __restrict__ dZ,
                       float* __restrict__ loss) {
  const float nc = fmaxf(1.0f, cnt[0]), nb = fmaxf(1.0f, cnt[1]);
  float l = 0.0f;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (size_t)gridDim.x * blockDim.x) {
    const float o0 = out[p * 2], z = out[p * 2 + 1];
    const float c = tgt[p * 4], y = tgt[p * 4 + 1], wc = tgt[p * 4 + 2], wb = tgt[p * 4 + 3];
    const float e = o0 - c * (1.0f / 16.0f);
    const float a = fabsf(e);
    l += wc * (a <= 1.0f ? 0.5f * e * e : a - 0.5f) / nc;
    l += wb * (fmaxf(z, 0.0f) - z * y + log1pf(expf(-fabsf(z)))) / nb;
    const float g0 = wc * fminf(fmaxf(e, -1.0f), 1.0f) / nc;
    const float g1 = wb * (1.0f / (1.0f + expf(-z)) - y) / nb;
    __align__(16) __nv_bfloat16 o[8];
    o[0] = __float2bfloat16_rn(g0);
    o[1] = __float2bfloat16_rn(g1);
#pragma unroll
    for (int i = 2; i < 8; ++i) o[i] = __float2bfloat16_rn(0.0f);
    *reinterpret_cast<uint4*>(dZ + p * 8) = *reinterpret_cast<const uint4*>(o);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// ----------------------------------------------------------------------- parameters
// Flat parameter index i -> (layer, co, k) or bias; gathers the gradient from the per-layer dW
// ([CoutP][Kp]) and db scratch, optionally applies Adam to the fp32 master copy, and refreshes the
// bf16 weights ([CoutP][Kp], padding untouched).
struct LayerDesc {
  int cin, cout, coutp, kp, stride, relu;
  int off;      // offset of this layer's weights in the flat vector
  int dw_off;   // offset of its [coutp][kp] gradient block
  int db_off;   // offset of its bias gradients
  int wb_off;   // offset of its bf16 weights
};

struct NetDesc {
  LayerDesc L[4];
  int n_params;
};

__device__ __forceinline__ bool locate(const NetDesc& d, int i, int& li, int& co, int& k,
                                       bool& is_bias) {
  for (li = 0; li < 4; ++li) {
    const LayerDesc& L = d.L[li];
    const int nw = L.cout * 9 * L.cin;
    if (i < L.off + nw) {
      const int r = i - L.off;
      co = r / (9 * L.cin);
      k = r % (9 * L.cin);
      is_bias = false;
      return true;
    }
    if (i < L.off + nw + L.cout) {
      co = i - L.off - nw;
      k = 0;
      is_bias = true;
      return true;
    }
  }
  return false;
}

__global__ void k_params_update(NetDesc d, float* __restrict__ theta, float* __restrict__ m,
                                float* __restrict__ v, const float* __restrict__ dW,
                                const float* __restrict__ db, float* __restrict__ grad_out,
                                __nv_bfloat16* __restrict__ wb, int adam, float lr, float bc1,
                                float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_params) return;
  int li, co, k;
  bool is_bias;
  if (!locate(d, i, li, co, k, is_bias)) return;
  const LayerDesc& L = d.L[li];
  const float g = is_bias ? db[L.db_off + co] : dW[L.dw_off + co * L.kp + k];
  if (grad_out) grad_out[i] = g;
  float th = theta[i];
  if (adam) {
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    th = th - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    theta[i] = th;
  }
  if (!is_bias) wb[L.wb_off + co * L.kp + k] = __float2bfloat16_rn(th);
}

// Bias vectors as fp32 arrays per layer (the GEMM epilogue reads them).
__global__ void k_bias_copy(NetDesc d, const float* __restrict__ theta, float* __restrict__ bias) {
  const int li = blockIdx.x, c = threadIdx.x;
  const LayerDesc& L = d.L[li];
  if (c < L.coutp) bias[li * 32 + c] = c < L.cout ? theta[L.off + L.cout * 9 * L.cin + c] : 0.0f;
}

// ------------------------------------------------------------------- band input, labels, windows
// x(y, x) = bf16((sum of the 4x4 block (edge repeated) - 2048) / 1024) for the left image and the
// row-shifted right image right(clamp(u - kappa(v))).
__global__ void k_band_input(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right,
                             int W, int H, size_t pitch, const int32_t* __restrict__ kappa,
                             int Wd, int Hd, __nv_bfloat16* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= Wd) return;
  int sl = 0, sr = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int v = min(4 * y + i, H - 1);
    const int k = kappa[v];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int u = min(4 * x + j, W - 1);
      sl += left[(size_t)v * pitch + u];
      const int ur = min(max(u - k, 0), W - 1);
      sr += right[(size_t)v * pitch + ur];
    }
  }
  __nv_bfloat162 o;
  o.x = __float2bfloat16_rn((float)(sl - 2048) / 1024.0f);
  o.y = __float2bfloat16_rn((float)(sr - 2048) / 1024.0f);
  reinterpret_cast<__nv_bfloat162*>(out)[(size_t)y * Wd + x] = o;
}

// One block of 256 threads per 16x16 tile: histogram of the valid (D1 >= 0) integer disparities,
// lower median c, count within [c - radius, c + radius].
__global__ void __launch_bounds__(256) k_band_labels(const int16_t* __restrict__ d_int,
                                                     const float* __restrict__ D1, int W, int H,
                                                     int D, int tw, int min_valid, int radius,
                                                     int frac_num, int frac_den,
                                                     float* __restrict__ tgt) {
  __shared__ int hist[kMaxD];
  const int tx = blockIdx.x, ty = blockIdx.y;
  for (int i = threadIdx.x; i < D; i += 256) hist[i] = 0;
  __syncthreads();
  const int u = tx * 16 + (threadIdx.x & 15), v = ty * 16 + (threadIdx.x >> 4);
  if (u < W && v < H) {
    const size_t p = (size_t)v * W + u;
    const int d = d_int[p];
    if (D1[p] >= 0.0f && d >= 0 && d < D) atomicAdd(&hist[d], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int i = 0; i < D; ++i) n += hist[i];
    float* o = tgt + ((size_t)ty * tw + tx) * 4;
    o[3] = 1.0f;
    if (n < min_valid) {
      o[0] = o[1] = o[2] = 0.0f;
      return;
    }
    const int rank = (n - 1) / 2;  // the lower median is the value of sorted index rank
    int c = 0, cum = 0;
    for (; c < D; ++c) {
      cum += hist[c];
      if (cum > rank) break;
    }
    int inside = 0;
    for (int i = max(0, c - radius); i <= min(D - 1, c + radius); ++i) inside += hist[i];
    o[0] = (float)c;
    o[1] = (long long)frac_den * inside >= (long long)frac_num * n ? 1.0f : 0.0f;
    o[2] = 1.0f;
  }
}

// Window of one tile from the network output: confident tiles (logit >= ln 9 in float) start at
// rint(16 o0) - band/2 moved into [0, D - band]; the others search the full range (-1).
__device__ __forceinline__ int16_t tile_window(const float* o, int D, int band) {
  const float c = rintf(o[0] * 16.0f) - (float)(band / 2);
  const float lo = fminf(fmaxf(c, 0.0f), (float)max(D - band, 0));
  return o[1] >= 2.19722457733621938f ? (int16_t)lo : (int16_t)-1;
}

// Per tile; an unconfident tile of the left border columns tx < t0 = ceil((D - 1) / 16), where the
// full-range search has no valid pixel (and the network no label), takes the window of tile
// (ty, t0).
__global__ void k_band_tiles(const float* __restrict__ out, int th, int tw, int D, int band,
                             int16_t* __restrict__ tile_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= th * tw) return;
  int16_t w = tile_window(out + 2 * i, D, band);
  const int ty = i / tw, tx = i % tw, t0 = (D - 1 + 15) / 16;
  if (w < 0 && tx < t0 && t0 < tw) w = tile_window(out + 2 * (ty * tw + t0), D, band);
  tile_lo[i] = w;
}

}  // namespace

// ---------------------------------------------------------------------------- the network object
}  // namespace pd

using namespace pd;

struct pd_cnn {
  int device = 0;
  int max_batch = 0, max_hd = 0, max_wd = 0;
  NetDesc desc;
  // parameters
  float* theta = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* bias = nullptr;     // [4][32]
  __nv_bfloat16* wb = nullptr;
  float* dW = nullptr;
  float* db = nullptr;
  float* part = nullptr;     // partial gradient sums: [2 sms][32][288] floats
  int sms = 0;               // SM count of the device (sizes the weight-gradient pixel ranges)
  float* scal = nullptr;     // loss, n_c, n_b
  int* status = nullptr;     // bit 0: a tensor-core wait of the convolutions ran out
  int step = 0;
  // activations and buffers (sized for max_batch x max_hd x max_wd)
  __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;
  __nv_bfloat16 *col1 = nullptr, *col2 = nullptr, *col3 = nullptr, *col4 = nullptr;
  __nv_bfloat16 *dz1 = nullptr, *dz2 = nullptr, *dz3 = nullptr, *dz4 = nullptr;
  float* out = nullptr;
  float* dcol = nullptr;
  size_t wb_elems = 0, dw_elems = 0;
};

namespace {

constexpr int kLayerCin[4] = {2, 32, 32, 32};
constexpr int kLayerCout[4] = {32, 32, 32, 2};
constexpr int kLayerStride[4] = {1, 2, 2, 1};

NetDesc make_desc() {
  NetDesc d;
  int off = 0, dw = 0, db = 0, wb = 0;
  for (int l = 0; l < 4; ++l) {
    LayerDesc& L = d.L[l];
    L.cin = kLayerCin[l];
    L.cout = kLayerCout[l];
    L.coutp = L.cout < 8 ? 8 : L.cout;
    L.kp = L.cin == 2 ? 32 : 9 * L.cin;
    L.stride = kLayerStride[l];
    L.relu = l < 3;
    L.off = off;
    off += L.cout * 9 * L.cin + L.cout;
    L.dw_off = dw;
    dw += L.coutp * L.kp;
    L.db_off = db;
    db += 32;
    L.wb_off = wb;
    wb += L.coutp * L.kp;
  }
  d.n_params = off;
  return d;
}

int conv_out(int n, int s) { return (n - 1) / s + 1; }

struct Shapes {
  int h[5], w[5];  // h[0] = input, h[l + 1] = output of layer l
};

Shapes shapes(int Hd, int Wd) {
  Shapes s;
  s.h[0] = Hd;
  s.w[0] = Wd;
  for (int l = 0; l < 4; ++l) {
    s.h[l + 1] = conv_out(s.h[l], kLayerStride[l]);
    s.w[l + 1] = conv_out(s.w[l], kLayerStride[l]);
  }
  return s;
}

unsigned grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 152 * 64 ? (b ? b : 1) : 152 * 64);
}

// Forward pass for B images of Hd x Wd at x.  With keep_col (training) the patch matrices of every
// layer are kept, with the activations, for the backward pass.
void cnn_forward(cudaStream_t s, pd_cnn* net, const __nv_bfloat16* x, int B, const Shapes& sh,
                 bool keep_col) {
  const NetDesc& d = net->desc;
  const __nv_bfloat16* in[4] = {x, net->a1, net->a2, net->a3};
  __nv_bfloat16* col[4] = {net->col1, net->col2, net->col3, net->col4};
  void* act[4] = {net->a1, net->a2, net->a3, net->out};
  for (int l = 0; l < 4; ++l) {
    const LayerDesc& L = d.L[l];
    ConvArgs a{};
    a.X = in[l];
    a.B = B;
    a.H = sh.h[l];
    a.W = sh.w[l];
    a.Ho = sh.h[l + 1];
    a.Wo = sh.w[l + 1];
    a.stride = L.stride;
    a.Wt = net->wb + L.wb_off;
    a.coutp = L.coutp;
    a.bias = net->bias + 32 * l;
    a.out = act[l];
    a.col = keep_col ? col[l] : nullptr;
    a.status = net->status;
    a.P = B * a.Ho * a.Wo;
    a.wait_limit = kConvWaitCycles;
    a.issue = 1;
    if (l == 0) {
      if (keep_col) conv_tc<2, 32, false, true>(s, a);
      else conv_tc<2, 32, false, false>(s, a);
    } else if (l < 3) {
      if (keep_col) conv_tc<32, 32, false, true>(s, a);
      else conv_tc<32, 32, false, false>(s, a);
    } else {
      if (keep_col) conv_tc<32, 16, true, true>(s, a);
      else conv_tc<32, 16, true, false>(s, a);
    }
  }
}

// Backward pass from dZ4 (in net->dz4): parameter gradients into net->dW / net->db.
void cnn_backward(cudaStream_t s, pd_cnn* net, int B, const Shapes& sh, int sms) {
  const NetDesc& d = net->desc;
  __nv_bfloat16* dz[4] = {net->dz1, net->dz2, net->dz3, net->dz4};
  __nv_bfloat16* col[4] = {net->col1, net->col2, net->col3, net->col4};
  const __nv_bfloat16* act_in[4] = {nullptr, net->a1, net->a2, net->a3};
  cudaMemsetAsync(net->dW, 0, net->dw_elems * sizeof(float), s);
  cudaMemsetAsync(net->db, 0, 4 * 32 * sizeof(float), s);
  for (int l = 3; l >= 0; --l) {
    const LayerDesc& L = d.L[l];
    const int Ho = sh.h[l + 1], Wo = sh.w[l + 1];
    const int P = B * Ho * Wo;
    const int ldz = l == 3 ? 8 : 32;
    // dW[co][k] = sum_p dZ[p][co] Col[p][k]
    DwArgs w{};
    w.col = col[l];
    w.kp = L.kp;
    w.dZ = dz[l];
    w.ldz = ldz;
    w.part = net->part;
    w.coutp = L.coutp;
    w.status = net->status;
    w.P = P;
    w.wait_limit = kConvWaitCycles;
    if (l == 3) dw_tc<16>(s, w, sms, net->dW + L.dw_off);
    else dw_tc<32>(s, w, sms, net->dW + L.dw_off);
    {
      const int threads = 256;
      const int blocks = (int)std::min<size_t>(((size_t)P * ldz + 4095) / 4096 + 1, kBiasBlocks);
      k_bias_grad<<<blocks, threads, 0, s>>>(dz[l], P, L.cout, ldz, net->part);
      k_sum_ranges<<<1, 32, 0, s>>>(net->part, blocks, L.cout, net->db + L.db_off);
    }
    if (l == 0) break;
    // dCol[p][k] = sum_co dZ[p][co] W[co][k]
    DcolArgs c{};
    c.dZ = dz[l];
    c.ldz = ldz;
    c.Wt = net->wb + L.wb_off;
    c.coutp = L.coutp;
    c.dcol = net->dcol;
    c.status = net->status;
    c.P = P;
    c.wait_limit = kConvWaitCycles;
    dcol_tc(s, c);
    const int H = sh.h[l], W = sh.w[l];
    const size_t Pin = (size_t)B * H * W;
    k_col2im32<<<grid_for(Pin * 4, 256), 256, 0, s>>>(net->dcol, act_in[l], B, H, W, Ho, Wo,
                                                       L.stride, dz[l - 1]);
  }
}

void refresh_weights(cudaStream_t s, pd_cnn* net, int adam, float lr, float* grad_out) {
  const NetDesc& d = net->desc;
  float bc1 = 1.0f, bc2 = 1.0f;
  if (adam) {
    net->step += 1;
    bc1 = 1.0f - powf(0.9f, (float)net->step);
    bc2 = 1.0f - powf(0.999f, (float)net->step);
  }
  k_params_update<<<(d.n_params + 255) / 256, 256, 0, s>>>(d, net->theta, net->adam_m, net->adam_v,
                                                           net->dW, net->db, grad_out, net->wb,
                                                           adam, lr, bc1, bc2);
  k_bias_copy<<<4, 32, 0, s>>>(d, net->theta, net->bias);
}

pd_status check_dims(pd_ctx* ctx, pd_cnn* net, int B, int Hd, int Wd) {
  if (!net) return fail(ctx, PD_ERR_INVALID_ARG, "network is NULL");
  if (B < 1 || B > net->max_batch || Hd < 1 || Hd > net->max_hd || Wd < 1 || Wd > net->max_wd)
    return fail(ctx, PD_ERR_INVALID_ARG,
                "batch %d x %d x %d outside the network's capacity %d x %d x %d", B, Hd, Wd,
                net->max_batch, net->max_hd, net->max_wd);
  return PD_OK;
}

pd_status loss_grad_enqueue(pd_ctx* ctx, pd_cnn* net, const __nv_bfloat16* x, const float* tgt,
                            int B, int Hd, int Wd) {
  cudaStream_t s = ctx->stream;
  const Shapes sh = shapes(Hd, Wd);
  const size_t P4 = (size_t)B * sh.h[4] * sh.w[4];
  cnn_forward(s, net, x, B, sh, true);
  cudaMemsetAsync(net->scal, 0, 4 * sizeof(float), s);
  k_loss_counts<<<grid_for(P4, 256), 256, 0, s>>>(tgt, P4, net->scal + 1);
  k_loss<<<grid_for(P4, 256), 256, 0, s>>>(net->out, tgt, P4, net->scal + 1, net->dz4, net->scal);
  cnn_backward(s, net, B, sh, net->sms);
  return PD_OK;
}

}  // namespace

namespace pd {

bool cnn_fits(const pd_cnn* net, int B, int Hd, int Wd) {
  return net && B >= 1 && B <= net->max_batch && Hd >= 1 && Hd <= net->max_hd && Wd >= 1 &&
         Wd <= net->max_wd;
}

const float* cnn_forward_enqueue(cudaStream_t s, pd_cnn* net, const void* x, int Hd, int Wd) {
  cnn_forward(s, net, reinterpret_cast<const __nv_bfloat16*>(x), 1, shapes(Hd, Wd), false);
  return net->out;
}

void launch_band_input(cudaStream_t s, const uint8_t* left, const uint8_t* right, int W, int H,
                       size_t pitch, const int32_t* kappa, void* x) {
  const int Wd = (W + 3) / 4, Hd = (H + 3) / 4;
  k_band_input<<<dim3((Wd + 127) / 128, Hd), 128, 0, s>>>(left, right, W, H, pitch, kappa, Wd, Hd,
                                                          reinterpret_cast<__nv_bfloat16*>(x));
}

void launch_band_tiles(cudaStream_t s, const float* cnn_out, int th, int tw, int D, int band_width,
                       int16_t* tile_lo) {
  k_band_tiles<<<(th * tw + 255) / 256, 256, 0, s>>>(cnn_out, th, tw, D, band_width, tile_lo);
}

}  // namespace pd

extern "C" {

pd_status pd_cnn_create(pd_cnn** out, int device, int max_batch, int max_hd, int max_wd) {
  if (!out) return PD_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_batch < 1 || max_hd < 1 || max_wd < 1 || max_hd > 4096 || max_wd > 4096 ||
      (size_t)max_batch * max_hd * max_wd > ((size_t)1 << 31) / 36)
    return PD_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return PD_ERR_CUDA;
  }
  pd_cnn* net = new pd_cnn();
  net->device = device;
  net->max_batch = max_batch;
  net->max_hd = max_hd;
  net->max_wd = max_wd;
  net->desc = make_desc();
  const NetDesc& d = net->desc;
  for (int l = 0; l < 4; ++l) {
    net->wb_elems += (size_t)d.L[l].coutp * d.L[l].kp;
  }
  net->dw_elems = net->wb_elems;
  const Shapes sh = shapes(max_hd, max_wd);
  const size_t B = (size_t)max_batch;
  size_t P[5];
  for (int l = 0; l < 5; ++l) P[l] = B * sh.h[l] * sh.w[l];
  bool ok = true;
  auto alloc = [&](auto*& p, size_t n) {
    if (!ok) return;
    if (cudaMalloc(reinterpret_cast<void**>(&p), n * sizeof(*p) + 16) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      p = nullptr;
    }
  };
  alloc(net->theta, (size_t)d.n_params);
  alloc(net->adam_m, (size_t)d.n_params);
  alloc(net->adam_v, (size_t)d.n_params);
  alloc(net->bias, 4 * 32);
  alloc(net->wb, net->wb_elems);
  alloc(net->dW, net->dw_elems);
  alloc(net->db, 4 * 32);
  if (cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      net->sms < 1) {
    cudaGetLastError();
    net->sms = 1;
  }
  // weight-gradient ranges (at most 2 sms rows of coutp x kp <= 32 x 288) and bias-gradient blocks
  alloc(net->part, std::max((size_t)2 * net->sms * 32 * 288, (size_t)kBiasBlocks * 32));
  alloc(net->scal, 4);
  alloc(net->status, 1);
  alloc(net->x0, P[0] * 2);
  alloc(net->a1, P[1] * 32);
  alloc(net->a2, P[2] * 32);
  alloc(net->a3, P[3] * 32);
  alloc(net->col1, P[1] * 32);
  alloc(net->col2, P[2] * 288);
  alloc(net->col3, P[3] * 288);
  alloc(net->col4, P[4] * 288);
  alloc(net->dz1, P[1] * 32);
  alloc(net->dz2, P[2] * 32);
  alloc(net->dz3, P[3] * 32);
  alloc(net->dz4, P[4] * 8);
  alloc(net->out, P[4] * 2);
  size_t dcol = std::max(P[2], std::max(P[3], P[4])) * 288;
  alloc(net->dcol, dcol);
  if (ok) {
    ok = cudaMemset(net->theta, 0, d.n_params * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->adam_m, 0, d.n_params * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->adam_v, 0, d.n_params * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->bias, 0, 4 * 32 * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->wb, 0, net->wb_elems * sizeof(__nv_bfloat16)) == cudaSuccess &&
         cudaMemset(net->dW, 0, net->dw_elems * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->db, 0, 4 * 32 * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->status, 0, sizeof(int)) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!ok) {
    pd_cnn_destroy(net);
    return PD_ERR_OOM;
  }
  *out = net;
  return PD_OK;
}

pd_status pd_cnn_destroy(pd_cnn* net) {
  if (!net) return PD_OK;
  cudaSetDevice(net->device);
  void* ptrs[] = {net->theta, net->adam_m, net->adam_v, net->bias, net->wb, net->dW, net->db,
                  net->part,
                  net->scal, net->status, net->x0, net->a1, net->a2, net->a3, net->col1, net->col2, net->col3,
                  net->col4, net->dz1, net->dz2, net->dz3, net->dz4, net->out, net->dcol};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete net;
  return PD_OK;
}

int pd_cnn_num_params(void) { return make_desc().n_params; }

}  // extern "C"

// ------------------------------------------------------------------------ training checkpoints
// File layout, all little-endian: magic "PDCNNCK" NUL (8 bytes), u32 format version, u32
// parameter count n, u64 Adam step, u64 caller-state byte count r, f32[n] master parameters,
// f32[n] Adam first moments, f32[n] second moments, r caller-state bytes, u32 CRC-32 of every
// byte before it.
namespace {

constexpr unsigned char kCkptMagic[8] = {'P', 'D', 'C', 'N', 'N', 'C', 'K', 0};
constexpr uint32_t kCkptVersion = 1;
constexpr size_t kCkptHeader = 32;
constexpr size_t kCkptMaxState = (size_t)1 << 20;

// CRC-32 of the IEEE 802.3 / zlib convention: reflected polynomial 0xEDB88320, initial value and
// final xor 0xFFFFFFFF, table-driven one byte at a time.
uint32_t crc32_ieee(const unsigned char* p, size_t n) {
  static const std::vector<uint32_t> table = [] {
    std::vector<uint32_t> t(256);
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      t[i] = c;
    }
    return t;
  }();
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xffu] ^ (c >> 8);
  return c ^ 0xFFFFFFFFu;
}

void put_u32(std::vector<unsigned char>& b, uint32_t v) {
  for (int i = 0; i < 4; ++i) b.push_back((unsigned char)(v >> (8 * i)));
}
void put_u64(std::vector<unsigned char>& b, uint64_t v) {
  for (int i = 0; i < 8; ++i) b.push_back((unsigned char)(v >> (8 * i)));
}
uint32_t get_u32(const unsigned char* p) {
  uint32_t v = 0;
  for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
  return v;
}
uint64_t get_u64(const unsigned char* p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}
void put_f32s(std::vector<unsigned char>& b, const std::vector<float>& x) {
  for (float f : x) {
    uint32_t u;
    memcpy(&u, &f, 4);
    put_u32(b, u);
  }
}
void get_f32s(const unsigned char* p, size_t n, std::vector<float>& x) {
  x.resize(n);
  for (size_t i = 0; i < n; ++i) {
    const uint32_t u = get_u32(p + 4 * i);
    memcpy(&x[i], &u, 4);
  }
}

struct Ckpt {
  uint32_t version = 0, n = 0;
  uint64_t step = 0, state_bytes = 0;
  const unsigned char* theta = nullptr;  // views into the file bytes
  const unsigned char* state = nullptr;
};

// Reads and checks a checkpoint file; on success `buf` holds it and `out` points into it.
bool read_ckpt(const char* path, std::vector<unsigned char>& buf, Ckpt& out, std::string& why) {
  FILE* f = fopen(path, "rb");
  if (!f) {
    why = "cannot open the file";
    return false;
  }
  buf.clear();
  unsigned char tmp[65536];
  size_t got;
  while ((got = fread(tmp, 1, sizeof(tmp), f)) > 0) {
    buf.insert(buf.end(), tmp, tmp + got);
    if (buf.size() > ((size_t)256 << 20)) break;
  }
  const bool err = ferror(f) != 0;
  fclose(f);
  if (err) {
    why = "read error";
    return false;
  }
  if (buf.size() < kCkptHeader + 4 || memcmp(buf.data(), kCkptMagic, 8) != 0) {
    why = "not a band-network checkpoint (magic)";
    return false;
  }
  out.version = get_u32(buf.data() + 8);
  out.n = get_u32(buf.data() + 12);
  out.step = get_u64(buf.data() + 16);
  out.state_bytes = get_u64(buf.data() + 24);
  if (out.version != kCkptVersion) {
    why = "unknown format version";
    return false;
  }
  if (out.state_bytes > kCkptMaxState || out.n > (1u << 24)) {
    why = "size fields out of range";
    return false;
  }
  const size_t want = kCkptHeader + (size_t)12 * out.n + (size_t)out.state_bytes + 4;
  if (buf.size() != want) {
    why = "file size does not match its header";
    return false;
  }
  if (crc32_ieee(buf.data(), want - 4) != get_u32(buf.data() + want - 4)) {
    why = "CRC-32 mismatch";
    return false;
  }
  out.theta = buf.data() + kCkptHeader;
  out.state = buf.data() + kCkptHeader + (size_t)12 * out.n;
  return true;
}

}  // namespace

extern "C" {

pd_status pd_cnn_checkpoint_info(const char* path, int* n_params, long long* step,
                                 size_t* state_bytes) {
  if (!path) return PD_ERR_INVALID_ARG;
  std::vector<unsigned char> buf;
  Ckpt c;
  std::string why;
  if (!read_ckpt(path, buf, c, why)) return PD_ERR_INVALID_ARG;
  if (n_params) *n_params = (int)c.n;
  if (step) *step = (long long)c.step;
  if (state_bytes) *state_bytes = (size_t)c.state_bytes;
  return PD_OK;
}

pd_status pd_cnn_save(pd_ctx* ctx, pd_cnn* net, const char* path, const void* state,
                      size_t state_bytes) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!net || !path) return fail(ctx, PD_ERR_INVALID_ARG, "NULL network or path");
  if (state_bytes > kCkptMaxState || (state_bytes && !state))
    return fail(ctx, PD_ERR_INVALID_ARG, "caller state of %zu bytes (at most %zu, non-NULL)",
                state_bytes, kCkptMaxState);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  const size_t n = (size_t)net->desc.n_params;
  std::vector<float> th(n), m(n), v(n);
  cudaStream_t s = ctx->stream;
  st = cuda_ok(ctx, cudaMemcpyAsync(th.data(), net->theta, n * 4, cudaMemcpyDeviceToHost, s),
               "checkpoint download");
  if (st == PD_OK)
    st = cuda_ok(ctx, cudaMemcpyAsync(m.data(), net->adam_m, n * 4, cudaMemcpyDeviceToHost, s),
                 "checkpoint download");
  if (st == PD_OK)
    st = cuda_ok(ctx, cudaMemcpyAsync(v.data(), net->adam_v, n * 4, cudaMemcpyDeviceToHost, s),
                 "checkpoint download");
  if (st == PD_OK) st = cuda_ok(ctx, cudaStreamSynchronize(s), "pd_cnn_save");
  if (st != PD_OK) return st;
  std::vector<unsigned char> b;
  b.reserve(kCkptHeader + 12 * n + state_bytes + 4);
  b.insert(b.end(), kCkptMagic, kCkptMagic + 8);
  put_u32(b, kCkptVersion);
  put_u32(b, (uint32_t)n);
  put_u64(b, (uint64_t)net->step);
  put_u64(b, (uint64_t)state_bytes);
  put_f32s(b, th);
  put_f32s(b, m);
  put_f32s(b, v);
  const unsigned char* sp = static_cast<const unsigned char*>(state);
  if (state_bytes) b.insert(b.end(), sp, sp + state_bytes);
  put_u32(b, crc32_ieee(b.data(), b.size()));
  // written whole to a temporary file, then renamed over the target
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(ctx, PD_ERR_INVALID_ARG, "cannot create %s", tmp.c_str());
  const bool ok = fwrite(b.data(), 1, b.size(), f) == b.size();
  const bool closed = fclose(f) == 0;
  if (!ok || !closed || rename(tmp.c_str(), path) != 0) {
    remove(tmp.c_str());
    return fail(ctx, PD_ERR_INVALID_ARG, "cannot write %s", path);
  }
  return PD_OK;
}

pd_status pd_cnn_load(pd_ctx* ctx, pd_cnn* net, const char* path, void* state, size_t state_cap,
                      size_t* state_bytes) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!net || !path) return fail(ctx, PD_ERR_INVALID_ARG, "NULL network or path");
  std::vector<unsigned char> buf;
  Ckpt c;
  std::string why;
  if (!read_ckpt(path, buf, c, why))
    return fail(ctx, PD_ERR_INVALID_ARG, "%s: %s", path, why.c_str());
  if ((int)c.n != net->desc.n_params)
    return fail(ctx, PD_ERR_INVALID_ARG, "%s holds %u parameters, the network has %d", path, c.n,
                net->desc.n_params);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  const size_t n = c.n;
  std::vector<float> th, m, v;
  get_f32s(c.theta, n, th);
  get_f32s(c.theta + 4 * n, n, m);
  get_f32s(c.theta + 8 * n, n, v);
  cudaStream_t s = ctx->stream;
  st = cuda_ok(ctx, cudaMemcpyAsync(net->theta, th.data(), n * 4, cudaMemcpyHostToDevice, s),
               "checkpoint upload");
  if (st == PD_OK)
    st = cuda_ok(ctx, cudaMemcpyAsync(net->adam_m, m.data(), n * 4, cudaMemcpyHostToDevice, s),
                 "checkpoint upload");
  if (st == PD_OK)
    st = cuda_ok(ctx, cudaMemcpyAsync(net->adam_v, v.data(), n * 4, cudaMemcpyHostToDevice, s),
                 "checkpoint upload");
  if (st != PD_OK) return st;
  net->step = (int)c.step;
  refresh_weights(s, net, 0, 0.0f, nullptr);
  // the host vectors must stay valid until the copies have run
  st = cuda_ok(ctx, cudaStreamSynchronize(s), "pd_cnn_load");
  if (st != PD_OK) return st;
  if (state && state_cap) memcpy(state, c.state, std::min(state_cap, (size_t)c.state_bytes));
  if (state_bytes) *state_bytes = (size_t)c.state_bytes;
  return PD_OK;
}

pd_status pd_cnn_set_params(pd_ctx* ctx, pd_cnn* net, const float* host_params, int n) {
  if (!ctx || !net || !host_params) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  if (n != net->desc.n_params)
    return fail(ctx, PD_ERR_INVALID_ARG, "expected %d parameters, got %d", net->desc.n_params, n);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  cudaStream_t s = ctx->stream;
  st = cuda_ok(ctx, cudaMemcpyAsync(net->theta, host_params, n * sizeof(float),
                                    cudaMemcpyHostToDevice, s),
               "parameter upload");
  if (st != PD_OK) return st;
  cudaMemsetAsync(net->adam_m, 0, n * sizeof(float), s);
  cudaMemsetAsync(net->adam_v, 0, n * sizeof(float), s);
  net->step = 0;
  refresh_weights(s, net, 0, 0.0f, nullptr);
  // the host buffer must stay valid until the copy has run
  return cuda_ok(ctx, cudaStreamSynchronize(s), "pd_cnn_set_params");
}

pd_status pd_cnn_get_params(pd_ctx* ctx, pd_cnn* net, float* host_params, int n) {
  if (!ctx || !net || !host_params) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  if (n != net->desc.n_params)
    return fail(ctx, PD_ERR_INVALID_ARG, "expected %d parameters, got %d", net->desc.n_params, n);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  st = cuda_ok(ctx, cudaMemcpyAsync(host_params, net->theta, n * sizeof(float),
                                    cudaMemcpyDeviceToHost, ctx->stream),
               "parameter download");
  if (st != PD_OK) return st;
  return cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "pd_cnn_get_params");
}

pd_status pd_cnn_forward(pd_ctx* ctx, pd_cnn* net, const void* x, int B, int Hd, int Wd,
                         float* out) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  pd_status st = check_dims(ctx, net, B, Hd, Wd);
  if (st != PD_OK) return st;
  if (!x || !out) return fail(ctx, PD_ERR_INVALID_ARG, "NULL input or output");
  st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  const Shapes sh = shapes(Hd, Wd);
  cnn_forward(ctx->stream, net, reinterpret_cast<const __nv_bfloat16*>(x), B, sh, false);
  const size_t n = (size_t)B * sh.h[4] * sh.w[4] * 2;
  cudaMemcpyAsync(out, net->out, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  return launched(ctx, "pd_cnn_forward");
}

pd_status pd_cnn_check(pd_ctx* ctx, pd_cnn* net) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!net) return fail(ctx, PD_ERR_INVALID_ARG, "network is NULL");
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  int flags = 0;
  st = cuda_ok(ctx, cudaMemcpyAsync(&flags, net->status, sizeof(int), cudaMemcpyDeviceToHost,
                                    ctx->stream),
               "status read");
  if (st != PD_OK) return st;
  st = cuda_ok(ctx, cudaStreamSynchronize(ctx->stream), "pd_cnn_check");
  if (st != PD_OK) return st;
  if (!flags) return PD_OK;
  cudaMemsetAsync(net->status, 0, sizeof(int), ctx->stream);
  return fail(ctx, PD_ERR_TIMEOUT, "a tensor-core wait of the band network ran out (flags %d)",
              flags);
}

pd_status pd_cnn_probe_timeout(pd_ctx* ctx, pd_cnn* net, long long limit_cycles) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!net) return fail(ctx, PD_ERR_INVALID_ARG, "network is NULL");
  if (limit_cycles < 0 || limit_cycles > kConvWaitCycles)
    return fail(ctx, PD_ERR_INVALID_ARG, "limit %lld outside [0, %lld]", limit_cycles,
                kConvWaitCycles);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  // one CTA of the hidden-layer convolution on a 1 x 1 image that issues no MMA
  ConvArgs a{};
  a.X = net->a1;
  a.B = a.H = a.W = a.Ho = a.Wo = a.stride = 1;
  a.Wt = net->wb + net->desc.L[1].wb_off;
  a.coutp = 32;
  a.bias = net->bias + 32;
  a.out = net->a2;
  a.status = net->status;
  a.P = 1;
  a.wait_limit = limit_cycles;
  a.issue = 0;
  conv_tc<32, 32, false, false>(ctx->stream, a);
  return launched(ctx, "pd_cnn_probe_timeout");
}

pd_status pd_cnn_loss_grad(pd_ctx* ctx, pd_cnn* net, const void* x, const float* targets, int B,
                           int Hd, int Wd, float* loss, float* grad) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  pd_status st = check_dims(ctx, net, B, Hd, Wd);
  if (st != PD_OK) return st;
  if (!x || !targets || !loss || !grad) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  loss_grad_enqueue(ctx, net, reinterpret_cast<const __nv_bfloat16*>(x), targets, B, Hd, Wd);
  refresh_weights(ctx->stream, net, 0, 0.0f, grad);
  cudaMemcpyAsync(loss, net->scal, sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  return launched(ctx, "pd_cnn_loss_grad");
}

pd_status pd_cnn_train_step(pd_ctx* ctx, pd_cnn* net, const void* x, const float* targets, int B,
                            int Hd, int Wd, float lr, float* loss) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  pd_status st = check_dims(ctx, net, B, Hd, Wd);
  if (st != PD_OK) return st;
  if (!x || !targets) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  if (!(lr > 0.0f) || !isfinite(lr)) return fail(ctx, PD_ERR_INVALID_ARG, "lr must be positive");
  st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  loss_grad_enqueue(ctx, net, reinterpret_cast<const __nv_bfloat16*>(x), targets, B, Hd, Wd);
  refresh_weights(ctx->stream, net, 1, lr, nullptr);
  if (loss)
    cudaMemcpyAsync(loss, net->scal, sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  return launched(ctx, "pd_cnn_train_step");
}

pd_status pd_band_input(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                        size_t pitch, const int32_t* kappa, void* x) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!left || !right || !kappa || !x) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  if (W < 1 || H < 1 || W > 16384 || H > 16384 || pitch < (size_t)W)
    return fail(ctx, PD_ERR_INVALID_ARG, "bad image size %dx%d or pitch %zu", W, H, pitch);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  launch_band_input(ctx->stream, left, right, W, H, pitch, kappa, x);
  return launched(ctx, "pd_band_input");
}

pd_status pd_band_labels(pd_ctx* ctx, const int16_t* d_int, const float* D1, int W, int H, int D,
                         float* targets) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!d_int || !D1 || !targets) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  if (W < 1 || H < 1 || W > 16384 || H > 16384 || D < 1 || D > kMaxD)
    return fail(ctx, PD_ERR_INVALID_ARG, "bad size %dx%d or D %d", W, H, D);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  const int tw = (W + 15) / 16, th = (H + 15) / 16;
  k_band_labels<<<dim3(tw, th), 256, 0, ctx->stream>>>(d_int, D1, W, H, D, tw, 64, 7, 995, 1000,
                                                       targets);
  return launched(ctx, "pd_band_labels");
}

pd_status pd_band_tiles(pd_ctx* ctx, const float* cnn_out, int tiles_h, int tiles_w, int D,
                        int band_width, int16_t* tile_lo) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (!cnn_out || !tile_lo) return fail(ctx, PD_ERR_INVALID_ARG, "NULL argument");
  if (tiles_h < 1 || tiles_w < 1 || D < 1 || D > kMaxD || band_width < 1 || band_width > D)
    return fail(ctx, PD_ERR_INVALID_ARG, "bad tile grid %dx%d, D %d or band %d", tiles_w, tiles_h,
                D, band_width);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  launch_band_tiles(ctx->stream, cnn_out, tiles_h, tiles_w, D, band_width, tile_lo);
  return launched(ctx, "pd_band_tiles");
}

}  // extern "C"
