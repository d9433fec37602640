// Internal declarations shared by the libpothole translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pothole.h"

// Events of one profiled call: start, after prep, after aggregation, end of SGM, after the
// transform, after SLIC, after the mask.  Unused marks are null.
struct pd_prof_rec {
  cudaEvent_t ev[7];
  int used;  // bitmask of recorded marks
};

struct pd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  char err[512] = {0};
  void* ws = nullptr;  // device scratch owned by the context
  size_t ws_bytes = 0;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // batched path
  size_t batch_budget = (size_t)32 << 30;
  bool batch_graph = false, batch_autotune = true;
  void* pinned = nullptr;  // host staging of the batch tables (page-locked)
  size_t pinned_bytes = 0;
  cudaEvent_t batch_done = nullptr;
  bool batch_inflight = false;
  cudaGraphExec_t graph_exec = nullptr;
  void* graph_sig = nullptr;  // std::vector<long long>* signature of the captured batch
  void* tuned = nullptr;      // std::map<signature, warps per block>*
  bool prof = false;
  int prof_mask = 0x7f;  // the stage marks recorded while profiling (bit i: mark i)
  pd_prof_rec* recs = nullptr;  // kMaxProf records, events created on first use
  int nrec = 0;
  long long launches = 0;       // kernels launched by profiled calls
  // whole-path graph (pd_pipeline_config)
  bool pipe_graph = false;
  cudaStream_t cap_stream = nullptr;  // capture stream: the legacy stream cannot be captured
  cudaGraph_t pipe_src = nullptr;     // captured graph (its nodes address the exec's)
  cudaGraphExec_t pipe_exec = nullptr;
  void* pipe_key = nullptr;           // std::vector<unsigned char>* of the captured call
  long long pipe_kernels = 0;         // kernel nodes of the graph
  bool capturing = false;
  pd_prof_rec cap_rec = {};           // stands for the profiling record while capturing
  cudaEvent_t cap_ev[7] = {};         // events of the captured stage marks
  cudaGraphNode_t cap_node[7] = {};
  int cap_used = 0;
  // second stream of the learned band path (the census runs beside the network)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace pd {

// rint(x) (ties to even) as a 64-bit integer, equal to __float2ll_rn(x).  For |x| < 2^22 one
// float add puts rint(x) into the low mantissa bits of x + 1.5 * 2^23, whose unit in the last
// place is 1; larger or non-finite x take the 64-bit conversion instruction, which issues at the
// FP64 rate on this GPU.
__device__ __forceinline__ long long rint_to_ll(float x) {
  if (fabsf(x) < 4194304.0f) return (long long)(__float_as_int(x + 12582912.0f) - 0x4B400000);
  return __float2ll_rn(x);
}

constexpr int kCensusBits = 24;
constexpr int kMaxD = 256;
constexpr int kMaxImage = 4096;  // W, H limit of the exact moment sums

pd_status fail(pd_ctx* c, pd_status st, const char* fmt, ...);
pd_status cuda_ok(pd_ctx* c, cudaError_t e, const char* what);
// Checks the last launch; returns PD_OK or PD_ERR_CUDA with the message recorded.
pd_status launched(pd_ctx* c, const char* what);
// Makes sure the context holds at least `bytes` of device scratch.
pd_status ensure_ws(pd_ctx* c, size_t bytes);

// Bump allocator over the context scratch (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};
template <class T>
inline size_t carve_size(size_t& acc, size_t n) {
  acc = (acc + 255) & ~size_t(255);
  acc += n * sizeof(T);
  return acc;
}

// Key whose signed order is the order of the doubles (NaN excluded; -0 is folded to +0, so
// equal values tie): minimum searches compare it with integer instructions instead of FP64
// compares, which take about 63 cycles each on GB300.
__device__ __forceinline__ long long f64_order_key(double e) {
  long long b = __double_as_longlong(e);
  if (b == (long long)0x8000000000000000ULL) b = 0;
  return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}

// Raises kernel f's dynamic shared-memory limit to at least `bytes` on the current device.  The
// limit belongs to the device's context, so it is tracked per (kernel, device); repeated calls
// cost a lookup.
void raise_smem_limit(const void* f, size_t bytes);

// Aggregation directions (dx, dy): the first 4 are the axis paths, the last 4 the diagonals.
struct DirSet {
  int n;
  int8_t dx[8];
  int8_t dy[8];
};
DirSet dir_set(int paths);
DirSet one_dir(int dx, int dy);

// ------------------------------------------------------------------ SGM launchers (sgm.cu)
void launch_kappa(cudaStream_t s, int W, int H, int order, const double a[3], double cs,
                  double sn, double delta_pt, int32_t* kappa);
void launch_kappa_dev(cudaStream_t s, int W, int H, const pd_road_model* model, double delta_pt,
                      int32_t* kappa);
void launch_warp(cudaStream_t s, const uint8_t* right, int W, int H, size_t pitch,
                 const int32_t* kappa, uint8_t* out);
// Census of img, or of the row-shifted image when kappa != nullptr.
void launch_census(cudaStream_t s, const uint8_t* img, int W, int H, size_t pitch,
                   const int32_t* kappa, uint32_t* codes);
// Census codes of both images of a pair in one launch (the right one through kappa).
void launch_census_pair(cudaStream_t s, const uint8_t* left, const uint8_t* right, int W, int H,
                        size_t pitch, const int32_t* kappa, uint32_t* cl, uint32_t* cr);
// layout 0: natural [H][W][D]; layout 1: the interleaved layout of the aggregation kernels
// (D % 16 == 0): within each 16-disparity group g, byte 2j holds d = 16g + j and byte 2j+1 holds
// d = 16g + 8 + j.
void launch_cost(cudaStream_t s, const uint32_t* cl, const uint32_t* cr, int W, int H, int D,
                 int layout, uint8_t* cost);
void launch_to_interleaved(cudaStream_t s, const uint8_t* natural, size_t n_pix, int D,
                           uint8_t* out);
void launch_to_natural(cudaStream_t s, const uint8_t* inter, size_t n_pix, int D, uint8_t* out);
// Eq. (8) for every direction of `dirs`; volume r of `out` (stride vol_bytes) receives L_r in the
// interleaved layout.
// Eq. (8) over all directions of `dirs` into one interleaved L volume per direction (out + r
// vol_bytes), as one persistent launch (longest lines first; counter: one device word of
// scratch, reset on the stream before the launch).
void launch_aggregate_p(cudaStream_t s, const uint8_t* cost_il, int W, int H, int D,
                        const DirSet& dirs, int P1, int P2, uint8_t* out, size_t vol_bytes,
                        unsigned int* counter);
// S = sum of `ndirs` interleaved L volumes, written as natural uint16 [H][W][D].
void launch_sum_volumes(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes, int W,
                        int H, int D, uint16_t* S);
// Winner-take-all + sub-pixel + right-view keys, from interleaved L volumes (S == nullptr) or
// from a natural uint16 S.  rkeys must hold 0xFFFFFFFF on entry.
void launch_wta(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes,
                const uint16_t* S, int W, int H, int D, int16_t* d_int, float* dsub,
                uint32_t* rkeys);
void launch_lr(cudaStream_t s, const int16_t* d_int, const float* dsub, const uint32_t* rkeys,
               const int32_t* kappa, int W, int H, int D, int lr_tol, float* D1);

// ------------------------------------------------------------ transform launchers (dt.cu)
// Float coefficients of f for the D2 kernel, written by the roll solver on the device.
// Per-tile disparity windows of the band-restricted search: tile (u/16, v/16) searches
// [lo, min(lo + width, D)) with lo = min(tile_lo, D - 1), or all of [0, D) where tile_lo < 0.
struct BandArgs {
  const int16_t* tile_lo;  // [ceil(H/16)][tw], device
  int tw;
  int width;
};

void launch_cost_band(cudaStream_t s, const uint32_t* cl, const uint32_t* cr, int W, int H, int D,
                      const BandArgs& band, uint8_t* cost);
void launch_aggregate_band(cudaStream_t s, const uint8_t* cost_il, int W, int H, int D,
                           const DirSet& dirs, int P1, int P2, uint8_t* out, size_t vol_bytes,
                           const BandArgs& band);
void launch_wta_band(cudaStream_t s, const uint8_t* vols, int ndirs, size_t vol_bytes, int W,
                     int H, int D, const BandArgs& band, int16_t* d_int, float* dsub,
                     uint32_t* rkeys);
void launch_lr_band(cudaStream_t s, const int16_t* d_int, const float* dsub, const uint32_t* rkeys,
                    const int32_t* kappa, int W, int H, int D, const BandArgs& band, int lr_tol,
                    float* D1);

// Connected components (ccl.cu); returns the number of kernels launched.
size_t ccl_scratch_bytes(int W, int H, int max_comps);
int launch_ccl(cudaStream_t s, const uint8_t* mask, const int32_t* sp, int W, int H, int conn,
               int32_t* labels, pd_component* comps, int max_comps, int* n_comps, void* scratch);

// Accuracy report against a ground truth (report.cu).
size_t accuracy_scratch_bytes();
int launch_accuracy(cudaStream_t s, const float* D1, const float* D4, const uint8_t* mask,
                    const uint8_t* gt, int W, int H, const float eps[3], double* out,
                    void* scratch);

// The band network (cnn.cu).
bool cnn_fits(const pd_cnn* net, int B, int Hd, int Wd);
const float* cnn_forward_enqueue(cudaStream_t s, pd_cnn* net, const void* x, int Hd, int Wd);
void launch_band_input(cudaStream_t s, const uint8_t* left, const uint8_t* right, int W, int H,
                       size_t pitch, const int32_t* kappa, void* x);
void launch_band_tiles(cudaStream_t s, const float* cnn_out, int th, int tw, int D, int band_width,
                       int16_t* tile_lo);

struct RoadCoefF {
  float c, s, a0, a1, a2, uc, vc, pad;
};
size_t moments_scratch_bytes(int W, int H);
// fit != nullptr: only the inliers |D1 - f| <= tau of that fit count (the robust refit).
void launch_moments(cudaStream_t s, const float* D1, int W, int H, void* scratch, int64_t* sums,
                    const RoadCoefF* fit = nullptr, float tau = 0.0f);
size_t roll_scratch_bytes();
// Returns the number of kernels launched.
int launch_roll_solve(cudaStream_t s, const int64_t* sums, int order, int W, int H,
                      pd_road_model* fitted, RoadCoefF* coef, double* grid_scratch);
void launch_d2(cudaStream_t s, const float* D1, int W, int H, const RoadCoefF* coef,
               float delta_dt, float* D2);

// ------------------------------------------------------ superpixel / mask (detect.cu)
void slic_grid(int W, int H, int K, int* nx, int* ny);
size_t slic_scratch_bytes(int n_centres);
// Runs seeds + `iters` rounds of assignment/update; writes labels and D3.  Returns the number
// of kernels it launched.
int launch_slic(cudaStream_t s, const float* D2, int W, int H, int K, float m, int iters,
                int32_t* labels, float* D3, float* centres_out, void* scratch);
size_t threshold_scratch_bytes();
// Returns the number of kernels it launched.
int launch_threshold(cudaStream_t s, const float* D2, const float* D1, const float* D3, int W,
                     int H, float delta_pd, int mode, uint8_t* mask, double* thresholds,
                     double* E2, void* scratch);

}  // namespace pd
