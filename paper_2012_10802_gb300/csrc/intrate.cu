// Measured issue rate of the integer instruction class that the aggregation of Eq. (8) runs on:
// packed u16x2 DPX instructions (three-input minimum and fused add-minimum).  The aggregation's
// roofline divides its algorithmic integer operations by this rate, counted in u16 lanes.
//
// Every thread runs 8 registers through alternating __vimin3_u16x2 / __viaddmin_u16x2 steps;
// each step of a register reads another register, so a warp has four independent chains of
// two dependent instructions and the schedulers are never short of ready warps at 64 warps per
// SM.  Every block records its SM and the SM's clock at its start and end, so the per-SM rate
// comes out in instructions per clock, independent of the clock the GPU ran at.
#include <string.h>

#include <vector>

#include "common.cuh"

namespace pd {
namespace {

constexpr int kRateThreads = 256;
constexpr int kRateBlocksPerSM = 8;
constexpr int kRateInstrPerRep = 16;

__global__ void __launch_bounds__(kRateThreads) k_int_rate(int reps, uint32_t seed,
                                                           uint32_t* __restrict__ sink,
                                                           long long* __restrict__ span) {
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
    a[i] = seed ^ (threadIdx.x * 0x9E3779B9u + blockIdx.x * 0x85EBCA6Bu + (uint32_t)i * 0x27D4EB2Fu);
  const uint32_t k = 0x00200020u ^ (seed & 0x000f000fu);
  const uint32_t p1 = 0x00040004u ^ (seed & 0x00030003u);
  __syncthreads();
  const long long t0 = clock64();
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = __vimin3_u16x2(a[i], a[i ^ 1], k);
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = __viaddmin_u16x2(a[i], p1, a[i ^ 2]);
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) x ^= a[i];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
  if (threadIdx.x == 0) {
    uint32_t sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    span[3 * blockIdx.x + 0] = t0;
    span[3 * blockIdx.x + 1] = t1;
    span[3 * blockIdx.x + 2] = (long long)sm;
  }
}

}  // namespace
}  // namespace pd

using namespace pd;

extern "C" pd_status pd_int_rate(pd_ctx* ctx, int reps, double* lane_ops_per_s,
                                 double* instr_per_clk_sm) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  if (reps < 1 || reps > (1 << 20))
    return fail(ctx, PD_ERR_INVALID_ARG, "reps %d outside [1, 2^20]", reps);
  pd_status st = cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
  if (st != PD_OK) return st;
  const int nblocks = ctx->sm_count * kRateBlocksPerSM;
  size_t need = 0;
  carve_size<uint32_t>(need, (size_t)nblocks * kRateThreads);
  carve_size<long long>(need, (size_t)3 * nblocks);
  st = ensure_ws(ctx, need);
  if (st != PD_OK) return st;
  Carve c(ctx->ws);
  uint32_t* sink = c.take<uint32_t>((size_t)nblocks * kRateThreads);
  long long* span = c.take<long long>((size_t)3 * nblocks);
  // one launch to warm up, one timed
  k_int_rate<<<nblocks, kRateThreads, 0, ctx->stream>>>(reps, 0x1234u, sink, span);
  st = launched(ctx, "k_int_rate");
  if (st != PD_OK) return st;
  cudaEvent_t e0, e1;
  st = cuda_ok(ctx, cudaEventCreate(&e0), "cudaEventCreate");
  if (st != PD_OK) return st;
  st = cuda_ok(ctx, cudaEventCreate(&e1), "cudaEventCreate");
  if (st != PD_OK) {
    cudaEventDestroy(e0);
    return st;
  }
  cudaEventRecord(e0, ctx->stream);
  k_int_rate<<<nblocks, kRateThreads, 0, ctx->stream>>>(reps, 0x5678u, sink, span);
  cudaEventRecord(e1, ctx->stream);
  st = launched(ctx, "k_int_rate");
  if (st == PD_OK) st = cuda_ok(ctx, cudaEventSynchronize(e1), "k_int_rate");
  float ms = 0.f;
  if (st == PD_OK) st = cuda_ok(ctx, cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PD_OK) return st;
  std::vector<long long> h((size_t)3 * nblocks);
  st = cuda_ok(ctx, cudaMemcpy(h.data(), span, h.size() * sizeof(long long), cudaMemcpyDeviceToHost),
               "span copy");
  if (st != PD_OK) return st;
  const double per_block = (double)kRateThreads / 32.0 * reps * kRateInstrPerRep;  // warp instr
  if (lane_ops_per_s)  // u16 lanes: 32 threads x 2 halves per warp instruction
    *lane_ops_per_s = per_block * nblocks * 64.0 / (ms * 1e-3);
  if (instr_per_clk_sm) {
    // per SM: its warp instructions over the span from its first block's start to its last
    // block's end, in that SM's clocks; thread instructions per clock, averaged over the SMs
    std::vector<long long> lo(1024, -1), hi(1024, -1);
    std::vector<int> cnt(1024, 0);
    for (int b = 0; b < nblocks; ++b) {
      const long long t0 = h[3 * b], t1 = h[3 * b + 1];
      const int sm = (int)h[3 * b + 2];
      if (sm < 0 || sm >= 1024) continue;
      lo[sm] = lo[sm] < 0 ? t0 : (t0 < lo[sm] ? t0 : lo[sm]);
      hi[sm] = t1 > hi[sm] ? t1 : hi[sm];
      cnt[sm] += 1;
    }
    double sum = 0.0;
    int n = 0;
    for (int sm = 0; sm < 1024; ++sm)
      if (cnt[sm] > 0 && hi[sm] > lo[sm]) {
        sum += per_block * cnt[sm] * 32.0 / (double)(hi[sm] - lo[sm]);
        ++n;
      }
    *instr_per_clk_sm = n ? sum / n : 0.0;
  }
  return PD_OK;
}
