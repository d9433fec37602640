// Accuracy report against a ground truth (Sec. III): the percentage of error pixels e_p at three
// tolerances and the RMSE e_r of D1 against the ground-truth disparity D4 over the q pixels with a
// disparity (Sec. III-A), and pixel precision, recall, accuracy and F-score of the pothole mask
// against a ground-truth mask (Sec. III-B).  Counts are exact integers; the squared-error sum is
// accumulated in double precision (its summation order is not fixed).
#include <math.h>

#include "common.cuh"

namespace pd {

namespace {

struct AccSums {
  unsigned long long q, n1, n2, n3, tp, fp, fn, tn;
  double sse;
};

__global__ void k_accuracy(const float* __restrict__ D1, const float* __restrict__ D4,
                           const uint8_t* __restrict__ mask, const uint8_t* __restrict__ gt,
                           size_t n, float e1, float e2, float e3, AccSums* __restrict__ acc) {
  unsigned long long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double sse = 0.0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (size_t)gridDim.x * blockDim.x) {
    const float d1 = D1[p], d4 = D4[p];
    if (d1 >= 0.0f && isfinite(d4)) {
      const double e = (double)d1 - (double)d4;
      const double a = fabs(e);
      c[0] += 1;
      c[1] += a > (double)e1;
      c[2] += a > (double)e2;
      c[3] += a > (double)e3;
      sse += e * e;
    }
    const bool m = mask[p] != 0, g = gt[p] != 0;
    c[4] += m && g;
    c[5] += m && !g;
    c[6] += !m && g;
    c[7] += !m && !g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] += __shfl_xor_sync(0xffffffffu, c[k], o);
    sse += __shfl_xor_sync(0xffffffffu, sse, o);
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* dst = &acc->q;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (c[k]) atomicAdd(dst + k, c[k]);
    if (sse != 0.0) atomicAdd(&acc->sse, sse);
  }
}

__global__ void k_accuracy_final(const AccSums* __restrict__ a, double* __restrict__ out) {
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const double q = (double)a->q;
  out[0] = q;
  out[1] = a->q ? 100.0 * (double)a->n1 / q : nan;
  out[2] = a->q ? 100.0 * (double)a->n2 / q : nan;
  out[3] = a->q ? 100.0 * (double)a->n3 / q : nan;
  out[4] = a->q ? sqrt(a->sse / q) : nan;
  const double tp = (double)a->tp, fp = (double)a->fp, fn = (double)a->fn, tn = (double)a->tn;
  out[5] = tp;
  out[6] = fp;
  out[7] = fn;
  out[8] = tn;
  const double p = a->tp + a->fp ? tp / (tp + fp) : nan;
  const double r = a->tp + a->fn ? tp / (tp + fn) : nan;
  out[9] = p;
  out[10] = r;
  out[11] = (tp + tn) / (tp + fp + fn + tn);
  out[12] = a->tp ? 2.0 * p * r / (p + r) : nan;
}

}  // namespace

size_t accuracy_scratch_bytes() { return sizeof(AccSums); }

int launch_accuracy(cudaStream_t s, const float* D1, const float* D4, const uint8_t* mask,
                    const uint8_t* gt, int W, int H, const float eps[3], double* out,
                    void* scratch) {
  AccSums* acc = static_cast<AccSums*>(scratch);
  cudaMemsetAsync(acc, 0, sizeof(AccSums), s);
  const size_t n = (size_t)W * H;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_accuracy<<<(unsigned)blocks, 256, 0, s>>>(D1, D4, mask, gt, n, eps[0], eps[1], eps[2], acc);
  k_accuracy_final<<<1, 1, 0, s>>>(acc, out);
  return 2;
}

}  // namespace pd
