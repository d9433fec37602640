// The band network (an extension beyond the paper): predicts, per 16x16 tile, the centre of the
// tile's disparities after the perspective transformation of Sec. II-A and a confidence, so that
// the SGM of Sec. II-B can search a 17-disparity window instead of the full range.
//
// Network: 3x3 convolutions, zero padding 1, strides 1, 2, 2, 1, channels 2 -> 32 -> 32 -> 32 -> 2,
// ReLU after the first three, on the 4x-block-averaged row-shifted pair.  Activations are bf16,
// NHWC; each convolution is an explicit im2col (k = (ky * 3 + kx) * Cin + ci) followed by a bf16
// tensor-core GEMM with fp32 accumulation (mma.m16n8k16, operands staged in shared memory and
// loaded with ldmatrix).  The backward pass uses the same GEMM with transposed operand layouts:
// dW = dZ^T Col (split over pixels, fp32 atomics), dCol = dZ W, and a gather col2im that applies
// the previous layer's ReLU mask.  Training is Adam on fp32 master weights.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"

namespace pd {

namespace {

// ------------------------------------------------------------------------------- GEMM
// C[M][N] = sum_k A(m, k) B(k, n), A and B bf16, fp32 accumulation.
//   A_ROW: A stored [M][lda] (k contiguous); otherwise [K][lda] (m contiguous).
//   B_NK:  B stored [N][ldb] (k contiguous); otherwise [K][ldb] (n contiguous).
// Contiguous extents must be multiples of 8 elements and rows 16-byte aligned; out-of-range
// rows and 8-element groups are read as zeros.  blockIdx.z splits K into chunks of k_chunk.
constexpr int kBM = 64, kBN = 32, kBK = 32, kGemmThreads = 128;
constexpr int kPad = 8;  // bf16 elements of padding per shared-memory row (bank spread)

enum Epilogue { kEpiBiasReluBf16 = 0, kEpiBiasF32 = 1, kEpiF32 = 2, kEpiAtomicF32 = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t r[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t r[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  void* C;
  const float* bias;
  int M, N, K, lda, ldb, ldc;
  int n_store;  // columns written (<= N)
  int k_chunk;
};

template <bool A_ROW, bool B_NK, int EPI>
__global__ void __launch_bounds__(kGemmThreads) k_gemm(GemmArgs g) {
  // A tile: A_ROW ? [kBM][kBK + kPad] : [kBK][kBM + kPad];  B tile: B_NK ? [kBN][kBK + kPad] : [kBK][kBN + kPad]
  __shared__ __align__(16) __nv_bfloat16 sA[kBM * (kBK + kPad) > kBK * (kBM + kPad) ? kBM * (kBK + kPad) : kBK * (kBM + kPad)];
  __shared__ __align__(16) __nv_bfloat16 sB[kBN * (kBK + kPad) > kBK * (kBN + kPad) ? kBN * (kBK + kPad) : kBK * (kBN + kPad)];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int k_begin = blockIdx.z * g.k_chunk;
  const int k_end = min(g.K, k_begin + g.k_chunk);
  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[j][i] = 0.0f;

  for (int k0 = k_begin; k0 < k_end; k0 += kBK) {
    // ---- stage A (kBM x kBK = 256 vectors of 8) and B (kBN x kBK = 128 vectors)
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int vi = tid + it * kGemmThreads;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (A_ROW) {
        const int r = vi >> 2, c = (vi & 3) * 8;  // row m0 + r, k0 + c .. + 7
        const int m = m0 + r, k = k0 + c;
        if (m < g.M && k < k_end)
          val = *reinterpret_cast<const uint4*>(g.A + (size_t)m * g.lda + k);
        *reinterpret_cast<uint4*>(sA + r * (kBK + kPad) + c) = val;
      } else {
        const int r = vi >> 3, c = (vi & 7) * 8;  // k row k0 + r, m0 + c .. + 7
        const int k = k0 + r, m = m0 + c;
        if (k < k_end && m < g.M)
          val = *reinterpret_cast<const uint4*>(g.A + (size_t)k * g.lda + m);
        *reinterpret_cast<uint4*>(sA + r * (kBM + kPad) + c) = val;
      }
    }
    {
      const int vi = tid;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (B_NK) {
        const int r = vi >> 2, c = (vi & 3) * 8;
        const int n = n0 + r, k = k0 + c;
        if (n < g.N && k < k_end)
          val = *reinterpret_cast<const uint4*>(g.B + (size_t)n * g.ldb + k);
        *reinterpret_cast<uint4*>(sB + r * (kBK + kPad) + c) = val;
      } else {
        const int r = vi >> 2, c = (vi & 3) * 8;
        const int k = k0 + r, n = n0 + c;
        if (k < k_end && n < g.N)
          val = *reinterpret_cast<const uint4*>(g.B + (size_t)k * g.ldb + n);
        *reinterpret_cast<uint4*>(sB + r * (kBN + kPad) + c) = val;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      uint32_t a[4];
      const int wm = warp * 16;
      if (A_ROW) {
        const int r = wm + (lane & 15), c = kk + (lane >> 4) * 8;
        ldsm_x4(smem_u32(sA + r * (kBK + kPad) + c), a);
      } else {
        const int q = lane >> 3, i = lane & 7;  // matrix q: m half q & 1, k half q >> 1
        const int r = kk + (q >> 1) * 8 + i, c = wm + (q & 1) * 8;
        ldsm_x4_t(smem_u32(sA + r * (kBM + kPad) + c), a);
      }
#pragma unroll
      for (int jp = 0; jp < 2; ++jp) {  // n tiles 2 jp and 2 jp + 1
        uint32_t b[4];
        const int q = lane >> 3, i = lane & 7;
        if (B_NK) {  // matrices: (n tile 2jp, k lo), (2jp, k hi), (2jp+1, k lo), (2jp+1, k hi)
          const int r = jp * 16 + (q >> 1) * 8 + i, c = kk + (q & 1) * 8;
          ldsm_x4(smem_u32(sB + r * (kBK + kPad) + c), b);
        } else {
          const int r = kk + (q & 1) * 8 + i, c = jp * 16 + (q >> 1) * 8;
          ldsm_x4_t(smem_u32(sB + r * (kBN + kPad) + c), b);
        }
        mma_bf16(acc[2 * jp], a, b[0], b[1]);
        mma_bf16(acc[2 * jp + 1], a, b[2], b[3]);
      }
    }
    __syncthreads();
  }

  // ---- epilogue: acc[j] covers rows m0 + 16 warp + lane/4 (+8), cols n0 + 8 j + 2 (lane%4) (+1)
  const int rbase = m0 + warp * 16 + (lane >> 2);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = rbase + 8 * h;
      if (m >= g.M) continue;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int n = n0 + 8 * j + 2 * (lane & 3) + e;
        if (n >= g.n_store) continue;
        float v = acc[j][2 * h + e];
        if (EPI == kEpiBiasReluBf16) {
          v = fmaxf(v + g.bias[n], 0.0f);
          reinterpret_cast<__nv_bfloat16*>(g.C)[(size_t)m * g.ldc + n] = __float2bfloat16_rn(v);
        } else if (EPI == kEpiBiasF32) {
          reinterpret_cast<float*>(g.C)[(size_t)m * g.ldc + n] = v + g.bias[n];
        } else if (EPI == kEpiF32) {
          reinterpret_cast<float*>(g.C)[(size_t)m * g.ldc + n] = v;
        } else {
          atomicAdd(reinterpret_cast<float*>(g.C) + (size_t)m * g.ldc + n, v);
        }
      }
    }
  }
}

template <bool A_ROW, bool B_NK, int EPI>
void gemm(cudaStream_t s, const GemmArgs& g, int splits) {
  dim3 grid((g.M + kBM - 1) / kBM, (g.N + kBN - 1) / kBN, splits);
  k_gemm<A_ROW, B_NK, EPI><<<grid, kGemmThreads, 0, s>>>(g);
}

// ------------------------------------------------------------------------------ im2col
// Col[p][k], p = (b, oy, ox), k = (ky * 3 + kx) * Cin + ci for k < 9 Cin, zero up to Kp.
// Cin = 32: one thread per (p, tap, 8 channels).
__global__ void k_im2col32(const __nv_bfloat16* __restrict__ X, int B, int H, int W, int Ho,
                           int Wo, int stride, __nv_bfloat16* __restrict__ col) {
  const size_t total = (size_t)B * Ho * Wo * 9 * 4;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t & 3);
    const size_t pt = t >> 2;
    const int tap = (int)(pt % 9);
    const size_t p = pt / 9;
    const int ox = (int)(p % Wo);
    const size_t bo = p / Wo;
    const int oy = (int)(bo % Ho);
    const int b = (int)(bo / Ho);
    const int y = oy * stride + tap / 3 - 1, x = ox * stride + tap % 3 - 1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (y >= 0 && y < H && x >= 0 && x < W)
      v = *reinterpret_cast<const uint4*>(X + (((size_t)b * H + y) * W + x) * 32 + q * 8);
    *reinterpret_cast<uint4*>(col + p * 288 + tap * 32 + q * 8) = v;
  }
}

// Cin = 2, Kp = 32: one thread per (p, k pair); pair j < 9 is tap j's two channels.
__global__ void k_im2col2(const __nv_bfloat16* __restrict__ X, int B, int H, int W, int Ho, int Wo,
                          __nv_bfloat16* __restrict__ col) {
  const size_t total = (size_t)B * Ho * Wo * 16;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t & 15);
    const size_t p = t >> 4;
    const int ox = (int)(p % Wo);
    const size_t bo = p / Wo;
    const int oy = (int)(bo % Ho);
    const int b = (int)(bo / Ho);
    uint32_t v = 0;
    if (j < 9) {
      const int y = oy + j / 3 - 1, x = ox + j % 3 - 1;
      if (y >= 0 && y < H && x >= 0 && x < W)
        v = *reinterpret_cast<const uint32_t*>(X + (((size_t)b * H + y) * W + x) * 2);
    }
    *reinterpret_cast<uint32_t*>(col + p * 32 + 2 * j) = v;
  }
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

// db[c] += sum over rows of dZ[p][c] (C channels, ld columns per row).
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dZ, size_t P, int C, int ld,
                            float* __restrict__ db) {
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
    atomicAdd(db + threadIdx.x, t);
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
  float* scal = nullptr;     // loss, n_c, n_b
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

// Forward pass for B images of Hd x Wd held in net->x0 (or x when given).  Leaves the
// activations and the im2col buffers of every layer in place for the backward pass.
void cnn_forward(cudaStream_t s, pd_cnn* net, const __nv_bfloat16* x, int B, const Shapes& sh) {
  const NetDesc& d = net->desc;
  const __nv_bfloat16* in[4] = {x, net->a1, net->a2, net->a3};
  __nv_bfloat16* col[4] = {net->col1, net->col2, net->col3, net->col4};
  __nv_bfloat16* act[3] = {net->a1, net->a2, net->a3};
  for (int l = 0; l < 4; ++l) {
    const LayerDesc& L = d.L[l];
    const int H = sh.h[l], W = sh.w[l], Ho = sh.h[l + 1], Wo = sh.w[l + 1];
    const size_t P = (size_t)B * Ho * Wo;
    if (L.cin == 2)
      k_im2col2<<<grid_for(P * 16, 256), 256, 0, s>>>(in[l], B, H, W, Ho, Wo, col[l]);
    else
      k_im2col32<<<grid_for(P * 36, 256), 256, 0, s>>>(in[l], B, H, W, Ho, Wo, L.stride, col[l]);
    GemmArgs g{};
    g.A = col[l];
    g.B = net->wb + L.wb_off;
    g.bias = net->bias + 32 * l;
    g.M = (int)P;
    g.N = L.coutp;
    g.K = L.kp;
    g.lda = L.kp;
    g.ldb = L.kp;
    g.k_chunk = L.kp;
    if (l < 3) {
      g.C = act[l];
      g.ldc = 32;
      g.n_store = 32;
      gemm<true, true, kEpiBiasReluBf16>(s, g, 1);
    } else {
      g.C = net->out;
      g.ldc = 2;
      g.n_store = 2;
      gemm<true, true, kEpiBiasF32>(s, g, 1);
    }
  }
}

// Backward pass from dZ4 (in net->dz4): parameter gradients into net->dW / net->db.
void cnn_backward(cudaStream_t s, pd_cnn* net, int B, const Shapes& sh) {
  const NetDesc& d = net->desc;
  __nv_bfloat16* dz[4] = {net->dz1, net->dz2, net->dz3, net->dz4};
  __nv_bfloat16* col[4] = {net->col1, net->col2, net->col3, net->col4};
  const __nv_bfloat16* act_in[4] = {nullptr, net->a1, net->a2, net->a3};
  cudaMemsetAsync(net->dW, 0, net->dw_elems * sizeof(float), s);
  cudaMemsetAsync(net->db, 0, 4 * 32 * sizeof(float), s);
  for (int l = 3; l >= 0; --l) {
    const LayerDesc& L = d.L[l];
    const int Ho = sh.h[l + 1], Wo = sh.w[l + 1];
    const size_t P = (size_t)B * Ho * Wo;
    const int ldz = l == 3 ? 8 : 32;
    // dW[co][k] = sum_p dZ[p][co] Col[p][k]: A = dZ as [K = P][M = coutp], B = Col as [K][N = kp]
    {
      GemmArgs g{};
      g.A = dz[l];
      g.B = col[l];
      g.C = net->dW + L.dw_off;
      g.M = L.coutp;
      g.N = L.kp;
      g.K = (int)P;
      g.lda = ldz;
      g.ldb = L.kp;
      g.ldc = L.kp;
      g.n_store = L.kp;
      const int chunk = 4096;
      g.k_chunk = chunk;
      gemm<false, false, kEpiAtomicF32>(s, g, (int)((P + chunk - 1) / chunk));
    }
    {
      const int threads = 256;
      const int blocks = (int)std::min<size_t>((P * ldz + 4095) / 4096 + 1, 2048);
      k_bias_grad<<<blocks, threads, 0, s>>>(dz[l], P, L.cout, ldz, net->db + L.db_off);
    }
    if (l == 0) break;
    // dCol[p][k] = sum_co dZ[p][co] W[co][k]: A = dZ [M = P][K = coutp], B = W as [K][N = kp]
    {
      GemmArgs g{};
      g.A = dz[l];
      g.B = net->wb + L.wb_off;
      g.C = net->dcol;
      g.M = (int)P;
      g.N = L.kp;
      g.K = L.coutp;
      g.lda = ldz;
      g.ldb = L.kp;
      g.ldc = L.kp;
      g.n_store = L.kp;
      g.k_chunk = L.coutp;
      gemm<true, false, kEpiF32>(s, g, 1);
    }
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
  cnn_forward(s, net, x, B, sh);
  cudaMemsetAsync(net->scal, 0, 4 * sizeof(float), s);
  k_loss_counts<<<grid_for(P4, 256), 256, 0, s>>>(tgt, P4, net->scal + 1);
  k_loss<<<grid_for(P4, 256), 256, 0, s>>>(net->out, tgt, P4, net->scal + 1, net->dz4, net->scal);
  cnn_backward(s, net, B, sh);
  return PD_OK;
}

}  // namespace

namespace pd {

bool cnn_fits(const pd_cnn* net, int B, int Hd, int Wd) {
  return net && B >= 1 && B <= net->max_batch && Hd >= 1 && Hd <= net->max_hd && Wd >= 1 &&
         Wd <= net->max_wd;
}

const float* cnn_forward_enqueue(cudaStream_t s, pd_cnn* net, const void* x, int Hd, int Wd) {
  cnn_forward(s, net, reinterpret_cast<const __nv_bfloat16*>(x), 1, shapes(Hd, Wd));
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
  alloc(net->scal, 4);
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
                  net->scal, net->x0, net->a1, net->a2, net->a3, net->col1, net->col2, net->col3,
                  net->col4, net->dz1, net->dz2, net->dz3, net->dz4, net->out, net->dcol};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete net;
  return PD_OK;
}

int pd_cnn_num_params(void) { return make_desc().n_params; }

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
  cnn_forward(ctx->stream, net, reinterpret_cast<const __nv_bfloat16*>(x), B, sh);
  const size_t n = (size_t)B * sh.h[4] * sh.w[4] * 2;
  cudaMemcpyAsync(out, net->out, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream);
  return launched(ctx, "pd_cnn_forward");
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
