// The C ABI of libpothole (declared in include/pothole.h): argument validation, scratch
// management and the launch sequences of each stage.  Every computation runs in the kernels of
// sgm.cu, dt.cu and detect.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "batch.cuh"
#include "common.cuh"

namespace pd {

pd_status fail(pd_ctx* c, pd_status st, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

pd_status cuda_ok(pd_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PD_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, PD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(c, PD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void raise_smem_limit(const void* f, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = set[{f, dev}];
  if (bytes <= cur) return;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
      cudaSuccess)
    cur = bytes;
}

pd_status launched(pd_ctx* c, const char* what) { return cuda_ok(c, cudaGetLastError(), what); }

pd_status ensure_ws(pd_ctx* c, size_t bytes) {
  if (bytes <= c->ws_bytes) return PD_OK;
  if (c->ws) {
    cudaFree(c->ws);  // synchronises the device, so no kernel still uses the old scratch
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  size_t want = bytes + (bytes >> 4);
  cudaError_t e = cudaMalloc(&c->ws, want);
  if (e != cudaSuccess) {
    c->ws = nullptr;
    cudaGetLastError();
    return fail(c, PD_ERR_OOM, "scratch of %zu bytes: %s", want, cudaGetErrorString(e));
  }
  c->ws_bytes = want;
  return PD_OK;
}

}  // namespace pd

using namespace pd;

namespace {

#define PD_TRY(x)                   \
  do {                              \
    pd_status _st = (x);            \
    if (_st != PD_OK) return _st;   \
  } while (0)

#define PD_REQUIRE(cond, ...)                                          \
  do {                                                                 \
    if (!(cond)) return fail(ctx, PD_ERR_INVALID_ARG, __VA_ARGS__);    \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------- profiling marks
constexpr int kMaxProf = 4096;

pd_prof_rec* prof_begin(pd_ctx* c) {
  if (!c->prof) return nullptr;
  if (!c->recs) c->recs = new pd_prof_rec[kMaxProf]();
  if (c->nrec >= kMaxProf) return nullptr;
  pd_prof_rec* r = &c->recs[c->nrec++];
  r->used = 0;
  return r;
}

void mark(pd_ctx* c, pd_prof_rec* r, int i) {
  if (!r || !(c->prof_mask >> i & 1)) return;
  if (r == &c->cap_rec) {  // capturing: an external event-record node, retargeted per replay
    cudaEventRecordWithFlags(c->cap_ev[i], c->stream, cudaEventRecordExternal);
    c->cap_used |= 1 << i;
    return;
  }
  if (!r->ev[i] && cudaEventCreate(&r->ev[i]) != cudaSuccess) {
    cudaGetLastError();
    r->ev[i] = nullptr;
    return;
  }
  cudaEventRecord(r->ev[i], c->stream);
  r->used |= 1 << i;
}

void count_launches(pd_ctx* c, long long n) {
  if (c->prof && !c->capturing) c->launches += n;
}
bool pow2_d(int D) { return D == 32 || D == 64 || D == 128 || D == 256; }

pd_status begin(pd_ctx* ctx) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  ctx->err[0] = 0;
  return cuda_ok(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
}

pd_status check_image(pd_ctx* ctx, int W, int H, size_t pitch) {
  PD_REQUIRE(W >= 1 && H >= 1, "image size %dx%d must be positive", W, H);
  PD_REQUIRE(W <= 16384 && H <= 16384, "image size %dx%d exceeds 16384", W, H);
  PD_REQUIRE(pitch >= (size_t)W, "pitch %zu is smaller than the width %d", pitch, W);
  return PD_OK;
}

pd_status check_model(pd_ctx* ctx, const pd_road_model* m) {
  PD_REQUIRE(m != nullptr, "road model is NULL");
  PD_REQUIRE(m->order == 1 || m->order == 2, "road model order %d must be 1 or 2", m->order);
  PD_REQUIRE(isfinite(m->a[0]) && isfinite(m->a[1]) && isfinite(m->a[2]) && isfinite(m->roll),
             "road model has a non-finite coefficient");
  return PD_OK;
}

pd_status check_penalties(pd_ctx* ctx, int P1, int P2) {
  PD_REQUIRE(P1 >= 0 && P1 < P2, "penalties must satisfy 0 <= P1 < P2 (got %d, %d)", P1, P2);
  PD_REQUIRE(kCensusBits + P2 <= 255, "P2 = %d too large: 24 + P2 must fit in a byte", P2);
  return PD_OK;
}

// Scratch layout of the fused SGM path.
struct SgmScratch {
  uint32_t* cl;
  uint32_t* cr;
  uint8_t* cost;
  uint8_t* vols;
  float* dsub;
  uint32_t* rkeys;
  int32_t* kappa;
  unsigned int* counter;  // task counter of the persistent aggregation
};

size_t sgm_scratch_bytes(int W, int H, int D, int paths) {
  size_t N = (size_t)W * H, acc = 0;
  carve_size<uint32_t>(acc, N);
  carve_size<uint32_t>(acc, N);
  carve_size<uint8_t>(acc, N * D);
  carve_size<uint8_t>(acc, N * D * paths);
  carve_size<float>(acc, N);
  carve_size<uint32_t>(acc, N);
  carve_size<int32_t>(acc, H);
  carve_size<unsigned int>(acc, 1);
  return acc;
}

SgmScratch sgm_carve(void* base, int W, int H, int D, int paths) {
  size_t N = (size_t)W * H;
  Carve c(base);
  SgmScratch s;
  s.cl = c.take<uint32_t>(N);
  s.cr = c.take<uint32_t>(N);
  s.cost = c.take<uint8_t>(N * D);
  s.vols = c.take<uint8_t>(N * D * paths);
  s.dsub = c.take<float>(N);
  s.rkeys = c.take<uint32_t>(N);
  s.kappa = c.take<int32_t>(H);
  s.counter = c.take<unsigned int>(1);
  return s;
}

pd_status check_sgm_params(pd_ctx* ctx, const pd_params* p) {
  PD_REQUIRE(p != nullptr, "params is NULL");
  PD_REQUIRE(pow2_d(p->D), "D = %d must be 32, 64, 128 or 256", p->D);
  PD_REQUIRE(p->paths == 4 || p->paths == 8, "paths = %d must be 4 or 8", p->paths);
  PD_TRY(check_penalties(ctx, p->P1, p->P2));
  PD_REQUIRE(p->lr_tol >= 0, "lr_tol = %d must be >= 0", p->lr_tol);
  PD_REQUIRE(isfinite(p->delta_pt), "delta_pt must be finite");
  return PD_OK;
}

// Enqueues the fused SGM (no validation; scratch already sized).
// The model is a host struct, or (model_dev != nullptr) one in device memory.
pd_status sgm_enqueue(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                      size_t pitch, const pd_road_model* model, const pd_params* p,
                      int32_t* kappa, int16_t* d_int, float* D1, pd_prof_rec* rec,
                      const pd_road_model* model_dev = nullptr) {
  cudaStream_t s = ctx->stream;
  SgmScratch sc = sgm_carve(ctx->ws, W, H, p->D, p->paths);
  int32_t* kap = kappa ? kappa : sc.kappa;
  size_t N = (size_t)W * H;
  size_t vol = N * p->D;
  mark(ctx, rec, 0);
  if (model_dev)
    launch_kappa_dev(s, W, H, model_dev, (double)p->delta_pt, kap);
  else
    launch_kappa(s, W, H, model->order, model->a, cos(model->roll), sin(model->roll),
                 (double)p->delta_pt, kap);
  launch_census_pair(s, left, right, W, H, pitch, kap, sc.cl, sc.cr);
  launch_cost(s, sc.cl, sc.cr, W, H, p->D, 1, sc.cost);
  cudaMemsetAsync(sc.rkeys, 0xff, N * sizeof(uint32_t), s);
  mark(ctx, rec, 1);
  launch_aggregate_p(s, sc.cost, W, H, p->D, dir_set(p->paths), p->P1, p->P2, sc.vols, vol,
                     sc.counter);
  mark(ctx, rec, 2);
  launch_wta(s, sc.vols, p->paths, vol, nullptr, W, H, p->D, d_int, sc.dsub, sc.rkeys);
  launch_lr(s, d_int, sc.dsub, sc.rkeys, kap, W, H, p->D, p->lr_tol, D1);
  mark(ctx, rec, 3);
  count_launches(ctx, 6);
  return launched(ctx, "pd_sgm");
}

// Enqueues the band-restricted SGM (no validation; scratch already sized).
// census_done: the row shifts and the census codes (sc.kappa or kappa, sc.cl, sc.cr) are already
// enqueued ahead of this call on ctx's stream.
pd_status sgm_band_enqueue(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                           size_t pitch, const pd_road_model* model, const pd_params* p,
                           const BandArgs& band, int32_t* kappa, int16_t* d_int, float* D1,
                           pd_prof_rec* rec, bool census_done = false) {
  cudaStream_t s = ctx->stream;
  SgmScratch sc = sgm_carve(ctx->ws, W, H, p->D, p->paths);
  int32_t* kap = kappa ? kappa : sc.kappa;
  size_t N = (size_t)W * H;
  size_t vol = N * p->D;
  mark(ctx, rec, 0);
  if (!census_done) {
    launch_kappa(s, W, H, model->order, model->a, cos(model->roll), sin(model->roll),
                 (double)p->delta_pt, kap);
    launch_census_pair(s, left, right, W, H, pitch, kap, sc.cl, sc.cr);
    count_launches(ctx, 2);
  }
  launch_cost_band(s, sc.cl, sc.cr, W, H, p->D, band, sc.cost);
  cudaMemsetAsync(sc.rkeys, 0xff, N * sizeof(uint32_t), s);
  mark(ctx, rec, 1);
  launch_aggregate_band(s, sc.cost, W, H, p->D, dir_set(p->paths), p->P1, p->P2, sc.vols, vol,
                        band);
  mark(ctx, rec, 2);
  launch_wta_band(s, sc.vols, p->paths, vol, W, H, p->D, band, d_int, sc.dsub, sc.rkeys);
  launch_lr_band(s, d_int, sc.dsub, sc.rkeys, kap, W, H, p->D, band, p->lr_tol, D1);
  mark(ctx, rec, 3);
  count_launches(ctx, 4);
  return launched(ctx, "pd_sgm_band");
}

size_t transform_scratch_bytes(int W, int H) {
  size_t acc = 0;
  carve_size<uint8_t>(acc, moments_scratch_bytes(W, H));
  carve_size<int64_t>(acc, 46);
  carve_size<pd_road_model>(acc, 1);
  carve_size<RoadCoefF>(acc, 1);
  carve_size<RoadCoefF>(acc, 1);
  carve_size<uint8_t>(acc, roll_scratch_bytes());
  return acc;
}

// Sec. II-C: the fit, then `iters` refits on the inliers (|D1 - f| <= tau) of the previous fit
// (reading R17; 0 iterations is the paper's fit), then Eq. (13).
pd_status transform_enqueue(pd_ctx* ctx, const float* D1, int W, int H, int order,
                            float delta_dt, pd_road_model* fitted, float* D2, void* base,
                            int iters = 0, float tau = 0.0f) {
  Carve c(base);
  void* part = c.take<uint8_t>(moments_scratch_bytes(W, H));
  int64_t* sums = c.take<int64_t>(46);
  pd_road_model* fit = c.take<pd_road_model>(1);
  RoadCoefF* coef = c.take<RoadCoefF>(1);
  RoadCoefF* prev = c.take<RoadCoefF>(1);
  double* grid = reinterpret_cast<double*>(c.take<uint8_t>(roll_scratch_bytes()));
  cudaStream_t s = ctx->stream;
  launch_moments(s, D1, W, H, part, sums);
  int n = launch_roll_solve(s, sums, order, W, H, fitted ? fitted : fit, coef, grid);
  for (int k = 0; k < iters; ++k) {
    cudaMemcpyAsync(prev, coef, sizeof(RoadCoefF), cudaMemcpyDeviceToDevice, s);
    launch_moments(s, D1, W, H, part, sums, prev, tau);
    n += 2 + launch_roll_solve(s, sums, order, W, H, fitted ? fitted : fit, coef, grid);
  }
  launch_d2(s, D1, W, H, coef, delta_dt, D2);
  count_launches(ctx, 3 + n);
  return launched(ctx, "pd_transform");
}

}  // namespace


// ------------------------------------------------------------------------- batched SGM

namespace {

struct WavePlan {
  int first, count;
  size_t table_off, table_bytes;  // within the table region
  size_t pairs_off, starts_off[kBatchStages], segs_off, counter_off;
  int nseg, ntasks;
  int total[kBatchStages];
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Launches the recorded waves (table upload first).
void batch_enqueue(pd_ctx* ctx, const std::vector<WavePlan>& waves, char* table_dev,
                   size_t table_bytes, const pd_params* p, int agg_warps, int agg_blocks) {
  cudaStream_t s = ctx->stream;
  cudaMemcpyAsync(table_dev, ctx->pinned, table_bytes, cudaMemcpyHostToDevice, s);
  for (const WavePlan& w : waves) {
    BatchWaveDev d;
    char* base = table_dev + w.table_off;
    d.pairs = reinterpret_cast<const BatchPair*>(base + w.pairs_off);
    d.host_pairs = reinterpret_cast<const BatchPair*>(static_cast<char*>(ctx->pinned) +
                                                      w.table_off + w.pairs_off);
    for (int k = 0; k < kBatchStages; ++k) d.starts[k] = reinterpret_cast<const int*>(base + w.starts_off[k]);
    d.segs = reinterpret_cast<const BatchSegment*>(base + w.segs_off);
    d.counter = reinterpret_cast<unsigned int*>(base + w.counter_off);
    d.npairs = w.count;
    d.nseg = w.nseg;
    d.ntasks = w.ntasks;
    for (int k = 0; k < kBatchStages; ++k) d.total[k] = w.total[k];
    launch_batch_wave(s, d, p->P1, p->P2, p->lr_tol, p->paths, agg_warps, agg_blocks);
  }
}

}  // namespace

extern "C" pd_status pd_batch_config(pd_ctx* ctx, size_t scratch_budget_bytes, int use_graph,
                                     int autotune) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  if (scratch_budget_bytes) ctx->batch_budget = scratch_budget_bytes;
  ctx->batch_graph = use_graph != 0;
  ctx->batch_autotune = autotune != 0;
  return PD_OK;
}

extern "C" pd_status pd_sgm_batch(pd_ctx* ctx, const pd_pair* pairs, int n, const pd_params* p) {
  PD_TRY(begin(ctx));
  PD_TRY(check_sgm_params(ctx, p));
  PD_REQUIRE(pairs != nullptr && n >= 1 && n <= 4096, "need 1..4096 pairs (got %d)", n);
  std::vector<size_t> need(n);
  for (int i = 0; i < n; ++i) {
    const pd_pair& q = pairs[i];
    PD_TRY(check_image(ctx, q.W, q.H, q.pitch));
    PD_TRY(check_model(ctx, &q.model));
    PD_REQUIRE(pow2_d(q.D), "pair %d: D = %d must be 32, 64, 128 or 256", i, q.D);
    PD_REQUIRE(q.left && q.right && q.d_int && q.D1, "pair %d: NULL image or output", i);
    need[i] = align256(sgm_scratch_bytes(q.W, q.H, q.D, p->paths));
  }
  // waves of consecutive pairs within the scratch budget
  std::vector<WavePlan> waves;
  size_t scratch_region = 0;
  for (int i = 0; i < n;) {
    WavePlan w{};
    w.first = i;
    size_t used = 0;
    while (i < n && (used == 0 || used + need[i] <= ctx->batch_budget)) used += need[i++];
    w.count = i - w.first;
    scratch_region = std::max(scratch_region, used);
    waves.push_back(w);
  }
  // table layout of every wave
  size_t table_bytes = 0;
  for (WavePlan& w : waves) {
    w.table_off = table_bytes;
    size_t o = 0;
    w.pairs_off = o;
    o = align256(o + sizeof(BatchPair) * w.count);
    for (int k = 0; k < kBatchStages; ++k) {
      w.starts_off[k] = o;
      o = align256(o + sizeof(int) * (w.count + 1));
    }
    w.segs_off = o;
    o = align256(o + sizeof(BatchSegment) * w.count * p->paths);
    w.counter_off = o;
    o = align256(o + sizeof(unsigned int));
    w.table_bytes = o;
    table_bytes += o;
  }
  PD_TRY(ensure_ws(ctx, table_bytes + scratch_region));
  char* table_dev = static_cast<char*>(ctx->ws);
  char* scratch = table_dev + align256(table_bytes);
  // the previous batch must have consumed the staging buffer before it is rewritten
  if (ctx->batch_inflight) {
    PD_TRY(cuda_ok(ctx, cudaEventSynchronize(ctx->batch_done), "pd_sgm_batch"));
    ctx->batch_inflight = false;
  }
  if (ctx->pinned_bytes < table_bytes) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
    size_t want = table_bytes + (table_bytes >> 2) + 4096;
    PD_TRY(cuda_ok(ctx, cudaHostAlloc(&ctx->pinned, want, cudaHostAllocDefault), "pinned staging"));
    ctx->pinned_bytes = want;
  }
  if (!ctx->batch_done)
    PD_TRY(cuda_ok(ctx, cudaEventCreateWithFlags(&ctx->batch_done, cudaEventDisableTiming),
                   "cudaEventCreate"));
  static const int kDx[8] = {1, -1, 0, 0, 1, -1, 1, -1};
  static const int kDy[8] = {0, 0, 1, -1, 1, -1, -1, 1};
  std::vector<long long> sig = {n, p->paths, p->P1, p->P2, p->lr_tol,
                                (long long)(double)p->delta_pt * 1000000};
  for (WavePlan& w : waves) {
    char* hbase = static_cast<char*>(ctx->pinned) + w.table_off;
    BatchPair* bp = reinterpret_cast<BatchPair*>(hbase + w.pairs_off);
    int* starts[kBatchStages];
    for (int k = 0; k < kBatchStages; ++k) {
      starts[k] = reinterpret_cast<int*>(hbase + w.starts_off[k]);
      starts[k][0] = 0;
    }
    struct Seg {
      BatchSegment s;
      int ntasks, nsteps;
      long long work;  // the pair's W * H * D
    };
    std::vector<Seg> segs;
    size_t off = 0;
    for (int j = 0; j < w.count; ++j) {
      const pd_pair& q = pairs[w.first + j];
      SgmScratch sc = sgm_carve(scratch + off, q.W, q.H, q.D, p->paths);
      off += need[w.first + j];
      BatchPair& b = bp[j];
      b.left = q.left;
      b.right = q.right;
      b.pitch = q.pitch;
      b.kappa = q.kappa ? q.kappa : sc.kappa;
      b.d_int = q.d_int;
      b.D1 = q.D1;
      b.cl = sc.cl;
      b.cr = sc.cr;
      b.cost = sc.cost;
      b.vols = sc.vols;
      b.dsub = sc.dsub;
      b.rkeys = sc.rkeys;
      b.vol_bytes = (size_t)q.W * q.H * q.D;
      b.a0 = q.model.a[0];
      b.a1 = q.model.a[1];
      b.a2 = q.model.a[2];
      b.cs = cos(q.model.roll);
      b.sn = sin(q.model.roll);
      b.delta_pt = (double)p->delta_pt;
      b.W = q.W;
      b.H = q.H;
      b.D = q.D;
      b.order = q.model.order;
      int cnt[kBatchStages];
      batch_stage_blocks(q.W, q.H, q.D, cnt);
      for (int k = 0; k < kBatchStages; ++k) starts[k][j + 1] = starts[k][j] + cnt[k];
      for (int r = 0; r < p->paths; ++r) {
        const int dx = kDx[r], dy = kDy[r];
        const int lpw = batch_lines_per_warp(q.D, dx, dy);
        const int nlines = dy == 0 ? q.H : (dx == 0 ? q.W : q.W + q.H - 1);
        const int nsteps = dy == 0 ? q.W : (dx == 0 ? q.H : std::min(q.W, q.H));
        Seg sg;
        sg.s = BatchSegment{0, j, r, dx, dy, 0};
        sg.ntasks = (nlines + lpw - 1) / lpw;
        sg.nsteps = nsteps;
        sg.work = (long long)q.W * q.H * q.D;
        segs.push_back(sg);
      }
      sig.insert(sig.end(), {q.W, q.H, q.D, (long long)q.pitch});
    }
    // pair by pair, the largest first, all directions of a pair together: a pair's tasks then run
    // at the same time, and its directions that sweep the same rows read them while L2 holds them
    std::stable_sort(segs.begin(), segs.end(), [](const Seg& a, const Seg& b) {
      return a.work != b.work ? a.work > b.work : a.s.pair < b.s.pair;
    });
    BatchSegment* hs = reinterpret_cast<BatchSegment*>(hbase + w.segs_off);
    int first = 0;
    for (size_t k = 0; k < segs.size(); ++k) {
      hs[k] = segs[k].s;
      hs[k].first = first;
      first += segs[k].ntasks;
    }
    w.nseg = (int)segs.size();
    w.ntasks = first;
    for (int k = 0; k < kBatchStages; ++k) w.total[k] = starts[k][w.count];
    *reinterpret_cast<unsigned int*>(hbase + w.counter_off) = 0;
  }
  // persistent aggregation: block shape from the tuning cache (4 warps until tuned)
  auto* tuned = static_cast<std::map<std::vector<long long>, int>*>(ctx->tuned);
  if (!tuned) ctx->tuned = tuned = new std::map<std::vector<long long>, int>();
  int agg_warps = 4;
  const bool known = tuned->count(sig) != 0;
  if (known) agg_warps = (*tuned)[sig];
  static bool smem_attr = false;
  if (!smem_attr) {  // the largest block (8 warps) sets the dynamic shared memory limit once
    batch_max_blocks_per_sm(8);
    smem_attr = true;
  }
  auto blocks_for = [&](int warps) { return ctx->sm_count * std::max(1, batch_max_blocks_per_sm(warps)); };
  cudaStream_t s = ctx->stream;
  if (ctx->batch_autotune && !known) {
    // run the batch once, then time the aggregation of the first wave with each block shape
    batch_enqueue(ctx, waves, table_dev, table_bytes, p, agg_warps, blocks_for(agg_warps));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int wc : {2, 4, 8}) {
      const WavePlan& w = waves[0];
      BatchWaveDev d;
      char* base = table_dev + w.table_off;
      d.pairs = reinterpret_cast<const BatchPair*>(base + w.pairs_off);
      d.host_pairs = nullptr;  // the aggregation alone needs no pair shapes on the host
      for (int k = 0; k < kBatchStages; ++k) d.starts[k] = reinterpret_cast<const int*>(base + w.starts_off[k]);
      d.segs = reinterpret_cast<const BatchSegment*>(base + w.segs_off);
      d.counter = reinterpret_cast<unsigned int*>(base + w.counter_off);
      d.npairs = w.count;
      d.nseg = w.nseg;
      d.ntasks = w.ntasks;
      cudaEventRecord(e0, s);
      launch_batch_aggregate_only(s, d, p->P1, p->P2, wc, blocks_for(wc));
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        agg_warps = wc;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (*tuned)[sig] = agg_warps;
    PD_TRY(launched(ctx, "pd_sgm_batch (tuning)"));
    cudaEventRecord(ctx->batch_done, s);
    ctx->batch_inflight = true;
    return PD_OK;
  }
  const int agg_blocks = blocks_for(agg_warps);
  if (ctx->batch_graph && s != nullptr) {
    // a captured graph holds the scratch, staging and stream addresses: they are part of its key
    std::vector<long long> gkey = sig;
    gkey.insert(gkey.end(), {(long long)(uintptr_t)ctx->ws, (long long)(uintptr_t)ctx->pinned,
                             (long long)(uintptr_t)s, agg_warps});
    auto* gsig = static_cast<std::vector<long long>*>(ctx->graph_sig);
    if (!ctx->graph_exec || !gsig || *gsig != gkey) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
      cudaGraph_t g = nullptr;
      PD_TRY(cuda_ok(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture"));
      batch_enqueue(ctx, waves, table_dev, table_bytes, p, agg_warps, agg_blocks);
      PD_TRY(cuda_ok(ctx, cudaStreamEndCapture(s, &g), "capture"));
      cudaError_t e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
      cudaGraphDestroy(g);
      PD_TRY(cuda_ok(ctx, e, "cudaGraphInstantiate"));
      delete gsig;
      ctx->graph_sig = new std::vector<long long>(gkey);
    }
    PD_TRY(cuda_ok(ctx, cudaGraphLaunch(ctx->graph_exec, s), "cudaGraphLaunch"));
  } else {
    batch_enqueue(ctx, waves, table_dev, table_bytes, p, agg_warps, agg_blocks);
  }
  PD_TRY(launched(ctx, "pd_sgm_batch"));
  cudaEventRecord(ctx->batch_done, s);
  ctx->batch_inflight = true;
  return PD_OK;
}

// ============================================================================== C ABI

extern "C" {

namespace {
void pipe_graph_free(pd_ctx* ctx);
}  // namespace

pd_status pd_create(pd_ctx** out, int device, void* stream) {
  if (!out) return PD_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return PD_ERR_INVALID_ARG;
  }
  pd_ctx* c = new pd_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return PD_ERR_CUDA;
  }
  *out = c;
  return PD_OK;
}

pd_status pd_destroy(pd_ctx* ctx) {
  if (!ctx) return PD_OK;
  cudaSetDevice(ctx->device);
  if (ctx->ws) cudaFree(ctx->ws);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->recs) {
    for (int i = 0; i < kMaxProf; ++i)
      for (auto& e : ctx->recs[i].ev)
        if (e) cudaEventDestroy(e);
    delete[] ctx->recs;
  }
  if (ctx->batch_done) cudaEventDestroy(ctx->batch_done);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  pipe_graph_free(ctx);
  for (auto& e : ctx->cap_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete static_cast<std::vector<long long>*>(ctx->graph_sig);
  delete static_cast<std::map<std::vector<long long>, int>*>(ctx->tuned);
  delete ctx;
  return PD_OK;
}

pd_status pd_set_stream(pd_ctx* ctx, void* stream) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return PD_OK;
}

const char* pd_last_error(const pd_ctx* ctx) { return ctx ? ctx->err : "context is NULL"; }

size_t pd_workspace_bytes(const pd_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

pd_status pd_default_params(pd_params* p) {
  if (!p) return PD_ERR_INVALID_ARG;
  p->D = 128;
  p->paths = 8;
  p->P1 = 4;
  p->P2 = 32;
  p->lr_tol = 1;
  p->delta_pt = 10.0f;
  p->delta_dt = 16.0f;
  p->delta_pd = 2.36f;
  p->slic_K = 1000;
  p->slic_m = 10.0f;
  p->slic_iters = 10;
  p->model_order = 2;
  p->threshold_mode = 0;
  p->fit_iters = 0;
  p->fit_tau = 1.0f;
  return PD_OK;
}

pd_status pd_warp(pd_ctx* ctx, const uint8_t* right, int W, int H, size_t pitch,
                  const pd_road_model* model, float delta_pt, uint8_t* right_warped,
                  int32_t* kappa) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_TRY(check_model(ctx, model));
  PD_REQUIRE(kappa != nullptr, "kappa is NULL");
  PD_REQUIRE(right_warped == nullptr || right != nullptr, "right is NULL");
  PD_REQUIRE(isfinite(delta_pt), "delta_pt must be finite");
  launch_kappa(ctx->stream, W, H, model->order, model->a, cos(model->roll), sin(model->roll),
               (double)delta_pt, kappa);
  if (right_warped) launch_warp(ctx->stream, right, W, H, pitch, kappa, right_warped);
  return launched(ctx, "pd_warp");
}

pd_status pd_census(pd_ctx* ctx, const uint8_t* img, int W, int H, size_t pitch,
                    uint32_t* codes) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_REQUIRE(img && codes, "NULL image or output");
  launch_census(ctx->stream, img, W, H, pitch, nullptr, codes);
  return launched(ctx, "pd_census");
}

pd_status pd_cost(pd_ctx* ctx, const uint8_t* left, const uint8_t* right_warped, int W, int H,
                  size_t pitch, int D, uint8_t* cost) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_REQUIRE(left && right_warped && cost, "NULL image or output");
  PD_REQUIRE(D >= 1 && D <= kMaxD, "D = %d must be in 1..256", D);
  size_t N = (size_t)W * H, need = 0;
  carve_size<uint32_t>(need, N);
  carve_size<uint32_t>(need, N);
  PD_TRY(ensure_ws(ctx, need));
  Carve c(ctx->ws);
  uint32_t* cl = c.take<uint32_t>(N);
  uint32_t* cr = c.take<uint32_t>(N);
  launch_census(ctx->stream, left, W, H, pitch, nullptr, cl);
  launch_census(ctx->stream, right_warped, W, H, pitch, nullptr, cr);
  launch_cost(ctx->stream, cl, cr, W, H, D, 0, cost);
  return launched(ctx, "pd_cost");
}

pd_status pd_aggregate_dir(pd_ctx* ctx, const uint8_t* cost, int W, int H, int D, int dx, int dy,
                           int P1, int P2, uint8_t* L) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(cost && L, "NULL cost or output");
  PD_REQUIRE(aligned16(cost) && aligned16(L), "cost and L must be 16-byte aligned");
  PD_REQUIRE(pow2_d(D), "D = %d must be 32, 64, 128 or 256", D);
  PD_REQUIRE(dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && (dx != 0 || dy != 0),
             "direction (%d, %d) must have components in {-1, 0, 1}, not both 0", dx, dy);
  PD_TRY(check_penalties(ctx, P1, P2));
  size_t vol = (size_t)W * H * D, need = 0;
  carve_size<uint8_t>(need, vol);
  carve_size<uint8_t>(need, vol);
  carve_size<unsigned int>(need, 1);
  PD_TRY(ensure_ws(ctx, need));
  Carve c(ctx->ws);
  uint8_t* cil = c.take<uint8_t>(vol);
  uint8_t* lil = c.take<uint8_t>(vol);
  unsigned int* counter = c.take<unsigned int>(1);
  launch_to_interleaved(ctx->stream, cost, (size_t)W * H, D, cil);
  launch_aggregate_p(ctx->stream, cil, W, H, D, one_dir(dx, dy), P1, P2, lil, vol, counter);
  launch_to_natural(ctx->stream, lil, (size_t)W * H, D, L);
  return launched(ctx, "pd_aggregate_dir");
}

pd_status pd_aggregate(pd_ctx* ctx, const uint8_t* cost, int W, int H, int D, int paths, int P1,
                       int P2, uint16_t* S) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(cost && S, "NULL cost or output");
  PD_REQUIRE(aligned16(cost) && aligned16(S), "cost and S must be 16-byte aligned");
  PD_REQUIRE(pow2_d(D), "D = %d must be 32, 64, 128 or 256", D);
  PD_REQUIRE(paths == 4 || paths == 8, "paths = %d must be 4 or 8", paths);
  PD_TRY(check_penalties(ctx, P1, P2));
  size_t vol = (size_t)W * H * D, need = 0;
  carve_size<uint8_t>(need, vol);
  carve_size<uint8_t>(need, vol * paths);
  carve_size<unsigned int>(need, 1);
  PD_TRY(ensure_ws(ctx, need));
  Carve c(ctx->ws);
  uint8_t* cil = c.take<uint8_t>(vol);
  uint8_t* vols = c.take<uint8_t>(vol * paths);
  unsigned int* counter = c.take<unsigned int>(1);
  launch_to_interleaved(ctx->stream, cost, (size_t)W * H, D, cil);
  launch_aggregate_p(ctx->stream, cil, W, H, D, dir_set(paths), P1, P2, vols, vol, counter);
  launch_sum_volumes(ctx->stream, vols, paths, vol, W, H, D, S);
  return launched(ctx, "pd_aggregate");
}

pd_status pd_disparity(pd_ctx* ctx, const uint16_t* S, int W, int H, int D, const int32_t* kappa,
                       int lr_tol, int16_t* d_int, float* D1) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(S && kappa && d_int && D1, "NULL input or output");
  PD_REQUIRE(aligned16(S), "S must be 16-byte aligned");
  PD_REQUIRE(pow2_d(D), "D = %d must be 32, 64, 128 or 256", D);
  PD_REQUIRE(lr_tol >= 0, "lr_tol = %d must be >= 0", lr_tol);
  size_t N = (size_t)W * H, need = 0;
  carve_size<float>(need, N);
  carve_size<uint32_t>(need, N);
  PD_TRY(ensure_ws(ctx, need));
  Carve c(ctx->ws);
  float* dsub = c.take<float>(N);
  uint32_t* rkeys = c.take<uint32_t>(N);
  cudaMemsetAsync(rkeys, 0xff, N * sizeof(uint32_t), ctx->stream);
  launch_wta(ctx->stream, nullptr, 0, 0, S, W, H, D, d_int, dsub, rkeys);
  launch_lr(ctx->stream, d_int, dsub, rkeys, kappa, W, H, D, lr_tol, D1);
  return launched(ctx, "pd_disparity");
}

pd_status pd_sgm(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                 size_t pitch, const pd_road_model* model, const pd_params* params,
                 int32_t* kappa, int16_t* d_int, float* D1) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_TRY(check_model(ctx, model));
  PD_TRY(check_sgm_params(ctx, params));
  PD_REQUIRE(left && right && d_int && D1, "NULL input or output");
  PD_TRY(ensure_ws(ctx, sgm_scratch_bytes(W, H, params->D, params->paths)));
  return sgm_enqueue(ctx, left, right, W, H, pitch, model, params, kappa, d_int, D1,
                     prof_begin(ctx));
}

pd_status pd_sgm_band(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                      size_t pitch, const pd_road_model* model, const pd_params* params,
                      const int16_t* tile_lo, int band_width, int32_t* kappa, int16_t* d_int,
                      float* D1) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_TRY(check_model(ctx, model));
  PD_TRY(check_sgm_params(ctx, params));
  PD_REQUIRE(left && right && d_int && D1 && tile_lo, "NULL input or output");
  PD_REQUIRE(band_width >= 1 && band_width <= params->D, "band width %d must be in 1..D",
             band_width);
  PD_REQUIRE(kCensusBits + 2 * params->P2 <= 255, "the band search needs 24 + 2 P2 <= 255");
  PD_TRY(ensure_ws(ctx, sgm_scratch_bytes(W, H, params->D, params->paths)));
  BandArgs band{tile_lo, (W + 15) / 16, band_width};
  return sgm_band_enqueue(ctx, left, right, W, H, pitch, model, params, band, kappa, d_int, D1,
                          prof_begin(ctx));
}

pd_status pd_sgm_learned(pd_ctx* ctx, pd_cnn* net, const uint8_t* left, const uint8_t* right,
                         int W, int H, size_t pitch, const pd_road_model* model,
                         const pd_params* params, int band_width, int16_t* tile_lo,
                         int32_t* kappa, int16_t* d_int, float* D1) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_TRY(check_model(ctx, model));
  PD_TRY(check_sgm_params(ctx, params));
  PD_REQUIRE(left && right && d_int && D1, "NULL input or output");
  PD_REQUIRE(band_width >= 1 && band_width <= params->D, "band width %d must be in 1..D",
             band_width);
  PD_REQUIRE(kCensusBits + 2 * params->P2 <= 255, "the band search needs 24 + 2 P2 <= 255");
  const int Hd = (H + 3) / 4, Wd = (W + 3) / 4, th = (H + 15) / 16, tw = (W + 15) / 16;
  PD_REQUIRE(cnn_fits(net, 1, Hd, Wd), "the network does not accept a %dx%d input", Wd, Hd);
  size_t acc = sgm_scratch_bytes(W, H, params->D, params->paths);
  const size_t x_off = (acc + 255) & ~size_t(255);
  const size_t t_off = (x_off + (size_t)Hd * Wd * 2 * 2 + 255) & ~size_t(255);
  PD_TRY(ensure_ws(ctx, t_off + (size_t)th * tw * sizeof(int16_t)));
  char* ws = static_cast<char*>(ctx->ws);
  void* x = ws + x_off;
  int16_t* tl = tile_lo ? tile_lo : reinterpret_cast<int16_t*>(ws + t_off);
  SgmScratch sc = sgm_carve(ctx->ws, W, H, params->D, params->paths);
  int32_t* kap = kappa ? kappa : sc.kappa;
  cudaStream_t s = ctx->stream;
  if (!ctx->side) {
    PD_TRY(cuda_ok(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking),
                   "side stream"));
    PD_TRY(cuda_ok(ctx, cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming),
                   "fork event"));
    PD_TRY(cuda_ok(ctx, cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming),
                   "join event"));
  }
  pd_prof_rec* rec = prof_begin(ctx);
  launch_kappa(s, W, H, model->order, model->a, cos(model->roll), sin(model->roll),
               (double)params->delta_pt, kap);
  // the census needs only the row shifts: it runs on the side stream beside the network
  cudaEventRecord(ctx->fork_ev, s);
  cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0);
  launch_census_pair(ctx->side, left, right, W, H, pitch, kap, sc.cl, sc.cr);
  cudaEventRecord(ctx->join_ev, ctx->side);
  launch_band_input(s, left, right, W, H, pitch, kap, x);
  const float* out = cnn_forward_enqueue(s, net, x, Hd, Wd);
  launch_band_tiles(s, out, th, tw, params->D, band_width, tl);
  cudaStreamWaitEvent(s, ctx->join_ev, 0);
  count_launches(ctx, 8);  // row shifts, census, network input, four convolutions, windows
  BandArgs band{tl, tw, band_width};
  return sgm_band_enqueue(ctx, left, right, W, H, pitch, model, params, band, kap, d_int, D1, rec,
                          true);
}

pd_status pd_transform_robust(pd_ctx* ctx, const float* D1, int W, int H, int order,
                              float delta_dt, int iters, float tau, pd_road_model* fitted,
                              float* D2) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(W <= kMaxImage && H <= kMaxImage, "transform needs W, H <= %d", kMaxImage);
  PD_REQUIRE(D1 && D2, "NULL input or output");
  PD_REQUIRE(order == 1 || order == 2, "order %d must be 1 or 2", order);
  PD_REQUIRE(isfinite(delta_dt), "delta_dt must be finite");
  PD_REQUIRE(iters >= 0 && iters <= 16, "iters = %d must be in 0..16", iters);
  PD_REQUIRE(isfinite(tau) && tau > 0.0f, "tau must be positive");
  PD_REQUIRE((reinterpret_cast<uintptr_t>(fitted) & 7u) == 0, "fitted must be 8-byte aligned");
  PD_TRY(ensure_ws(ctx, transform_scratch_bytes(W, H)));
  return transform_enqueue(ctx, D1, W, H, order, delta_dt, fitted, D2, ctx->ws, iters, tau);
}

pd_status pd_moments(pd_ctx* ctx, const float* D1, int W, int H, int64_t* sums) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(W <= kMaxImage && H <= kMaxImage, "moments need W, H <= %d", kMaxImage);
  PD_REQUIRE(D1 && sums, "NULL input or output");
  PD_TRY(ensure_ws(ctx, moments_scratch_bytes(W, H)));
  launch_moments(ctx->stream, D1, W, H, ctx->ws, sums);
  return launched(ctx, "pd_moments");
}

pd_status pd_transform(pd_ctx* ctx, const float* D1, int W, int H, int order, float delta_dt,
                       pd_road_model* fitted, float* D2) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(W <= kMaxImage && H <= kMaxImage, "transform needs W, H <= %d", kMaxImage);
  PD_REQUIRE(D1 && D2, "NULL input or output");
  PD_REQUIRE(order == 1 || order == 2, "order %d must be 1 or 2", order);
  PD_REQUIRE(isfinite(delta_dt), "delta_dt must be finite");
  PD_REQUIRE((reinterpret_cast<uintptr_t>(fitted) & 7u) == 0, "fitted must be 8-byte aligned");
  PD_TRY(ensure_ws(ctx, transform_scratch_bytes(W, H)));
  return transform_enqueue(ctx, D1, W, H, order, delta_dt, fitted, D2, ctx->ws);
}

pd_status pd_superpixels(pd_ctx* ctx, const float* D2, int W, int H, int K, float m, int iters,
                         int32_t* labels, float* D3, float* centres, int* n_centres) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(D2 && labels && D3, "NULL input or output");
  PD_REQUIRE(K >= 1 && (size_t)K <= (size_t)W * H, "K = %d must be in 1..W*H", K);
  PD_REQUIRE(isfinite(m) && m > 0.0f, "compactness m must be positive");
  PD_REQUIRE(iters >= 0 && iters <= 1000, "iters = %d must be in 0..1000", iters);
  int nx, ny;
  slic_grid(W, H, K, &nx, &ny);
  if (n_centres) *n_centres = nx * ny;
  PD_TRY(ensure_ws(ctx, slic_scratch_bytes(nx * ny)));
  count_launches(ctx, launch_slic(ctx->stream, D2, W, H, K, m, iters, labels, D3, centres, ctx->ws));
  return launched(ctx, "pd_superpixels");
}

pd_status pd_pothole_mask(pd_ctx* ctx, const float* D2, const float* D1, const float* D3, int W,
                          int H, float delta_pd, int mode, uint8_t* mask, double* thresholds,
                          double* E2) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(D2 && D1 && D3 && mask, "NULL input or output");
  PD_REQUIRE(mode == 0 || mode == 1, "mode %d must be 0 or 1", mode);
  PD_REQUIRE(isfinite(delta_pd), "delta_pd must be finite");
  PD_TRY(ensure_ws(ctx, threshold_scratch_bytes()));
  count_launches(ctx, launch_threshold(ctx->stream, D2, D1, D3, W, H, delta_pd, mode, mask,
                                       thresholds, E2, ctx->ws));
  return launched(ctx, "pd_pothole_mask");
}

pd_status pd_components(pd_ctx* ctx, const uint8_t* mask, const int32_t* sp_labels, int W, int H,
                        int connectivity, int32_t* labels, pd_component* comps, int max_comps,
                        int* n_comps) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(mask && sp_labels && labels && n_comps, "NULL input or output");
  PD_REQUIRE(connectivity == 4 || connectivity == 8, "connectivity %d must be 4 or 8",
             connectivity);
  PD_REQUIRE(max_comps >= 0 && (max_comps == 0 || comps), "max_comps %d needs a component buffer",
             max_comps);
  if (max_comps > W * H) max_comps = W * H;  // no mask has more components than pixels
  PD_TRY(ensure_ws(ctx, ccl_scratch_bytes(W, H, max_comps)));
  count_launches(ctx, launch_ccl(ctx->stream, mask, sp_labels, W, H, connectivity, labels, comps,
                                 max_comps, n_comps, ctx->ws));
  return launched(ctx, "pd_components");
}

pd_status pd_accuracy(pd_ctx* ctx, const float* D1, const float* D4, const uint8_t* mask,
                      const uint8_t* gt_mask, int W, int H, const float* eps, double* out) {
  PD_TRY(begin(ctx));
  PD_TRY(check_image(ctx, W, H, (size_t)W));
  PD_REQUIRE(D1 && D4 && mask && gt_mask && eps && out, "NULL input or output");
  PD_REQUIRE(isfinite(eps[0]) && isfinite(eps[1]) && isfinite(eps[2]), "non-finite tolerance");
  PD_TRY(ensure_ws(ctx, accuracy_scratch_bytes()));
  count_launches(ctx, launch_accuracy(ctx->stream, D1, D4, mask, gt_mask, W, H, eps, out,
                                      ctx->ws));
  return launched(ctx, "pd_accuracy");
}

namespace {

pd_status pipeline_impl(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                        size_t pitch, const pd_road_model* model, const pd_road_model* model_dev,
                        const pd_params* p, const pd_outputs* out, pd_stage_times* times);
pd_status pipeline_enqueue(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                           size_t pitch, const pd_road_model* model,
                           const pd_road_model* model_dev, const pd_params* p,
                           const pd_outputs* out, bool ccl, int conn, int max_comps,
                           pd_prof_rec* rec, pd_stage_times* times);
pd_status pipeline_graph_run(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                             size_t pitch, const pd_road_model* model,
                             const pd_road_model* model_dev, const pd_params* p,
                             const pd_outputs* out, bool ccl, int conn, int max_comps);
void pipe_graph_free(pd_ctx* ctx);

}  // namespace

pd_status pd_pipeline_config(pd_ctx* ctx, int use_graph) {
  PD_TRY(begin(ctx));
  ctx->pipe_graph = use_graph != 0;
  if (!ctx->pipe_graph) pipe_graph_free(ctx);
  return PD_OK;
}

pd_status pd_run_pipeline(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                          size_t pitch, const pd_road_model* model, const pd_params* p,
                          const pd_outputs* out, pd_stage_times* times) {
  PD_TRY(begin(ctx));
  PD_TRY(check_model(ctx, model));
  return pipeline_impl(ctx, left, right, W, H, pitch, model, nullptr, p, out, times);
}

pd_status pd_run_pipeline_dev(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W,
                              int H, size_t pitch, const pd_road_model* model_dev,
                              const pd_params* p, const pd_outputs* out, pd_stage_times* times) {
  PD_TRY(begin(ctx));
  PD_REQUIRE(model_dev != nullptr, "model is NULL");
  return pipeline_impl(ctx, left, right, W, H, pitch, nullptr, model_dev, p, out, times);
}

namespace {

pd_status pipeline_impl(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                        size_t pitch, const pd_road_model* model, const pd_road_model* model_dev,
                        const pd_params* p, const pd_outputs* out, pd_stage_times* times) {
  PD_TRY(check_image(ctx, W, H, pitch));
  PD_TRY(check_sgm_params(ctx, p));
  PD_REQUIRE(W <= kMaxImage && H <= kMaxImage, "the pipeline needs W, H <= %d", kMaxImage);
  PD_REQUIRE(left && right && out, "NULL input or outputs");
  PD_REQUIRE(out->d_int && out->D1 && out->D2 && out->labels && out->D3 && out->mask,
             "pd_outputs is missing a required buffer");
  PD_REQUIRE((reinterpret_cast<uintptr_t>(out->fitted) & 7u) == 0 &&
                 (reinterpret_cast<uintptr_t>(model_dev) & 7u) == 0,
             "road models in device memory must be 8-byte aligned");
  PD_REQUIRE(p->model_order == 1 || p->model_order == 2, "model_order must be 1 or 2");
  PD_REQUIRE(p->slic_K >= 1 && (size_t)p->slic_K <= (size_t)W * H, "slic_K out of range");
  PD_REQUIRE(isfinite(p->slic_m) && p->slic_m > 0.0f, "slic_m must be positive");
  PD_REQUIRE(p->slic_iters >= 0 && p->slic_iters <= 1000, "slic_iters out of range");
  PD_REQUIRE(p->threshold_mode == 0 || p->threshold_mode == 1, "threshold_mode must be 0 or 1");
  PD_REQUIRE(isfinite(p->delta_dt) && isfinite(p->delta_pd), "non-finite delta");
  PD_REQUIRE(p->fit_iters >= 0 && p->fit_iters <= 16 && isfinite(p->fit_tau) && p->fit_tau > 0.0f,
             "fit_iters must be in 0..16 and fit_tau positive");
  const bool ccl = out->components != nullptr;
  const int conn = out->connectivity == 0 ? 8 : out->connectivity;
  if (ccl) {
    PD_REQUIRE(out->n_comps != nullptr, "pd_outputs.components needs n_comps");
    PD_REQUIRE(conn == 4 || conn == 8, "connectivity %d must be 4 or 8", conn);
    PD_REQUIRE(out->max_comps >= 0 && (out->max_comps == 0 || out->comps != nullptr),
               "max_comps %d needs a component buffer of that size", out->max_comps);
  }
  const int max_comps = out->max_comps < W * H ? out->max_comps : W * H;
  int nx, ny;
  slic_grid(W, H, p->slic_K, &nx, &ny);
  size_t need = sgm_scratch_bytes(W, H, p->D, p->paths);
  size_t other = transform_scratch_bytes(W, H);
  if (slic_scratch_bytes(nx * ny) > other) other = slic_scratch_bytes(nx * ny);
  if (threshold_scratch_bytes() > other) other = threshold_scratch_bytes();
  if (ccl && ccl_scratch_bytes(W, H, max_comps) > other) other = ccl_scratch_bytes(W, H, max_comps);
  if (other > need) need = other;
  PD_TRY(ensure_ws(ctx, need));
  if (ctx->pipe_graph && !times)
    return pipeline_graph_run(ctx, left, right, W, H, pitch, model, model_dev, p, out, ccl, conn,
                              max_comps);
  if (times && !ctx->ev[0])
    for (auto& e : ctx->ev) PD_TRY(cuda_ok(ctx, cudaEventCreate(&e), "cudaEventCreate"));
  PD_TRY(pipeline_enqueue(ctx, left, right, W, H, pitch, model, model_dev, p, out, ccl, conn,
                          max_comps, prof_begin(ctx), times));
  if (times) {
    PD_TRY(cuda_ok(ctx, cudaEventSynchronize(ctx->ev[4]), "pipeline"));
    cudaEventElapsedTime(&times->sgm_ms, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&times->transform_ms, ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&times->superpixel_ms, ctx->ev[2], ctx->ev[3]);
    cudaEventElapsedTime(&times->mask_ms, ctx->ev[3], ctx->ev[4]);
    cudaEventElapsedTime(&times->total_ms, ctx->ev[0], ctx->ev[4]);
  }
  return PD_OK;
}

// The whole path's enqueued sequence (arguments validated, scratch sized).  rec: profiling
// record (or the capture stand-in, or NULL); times: record the stage events of pd_stage_times.
pd_status pipeline_enqueue(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                           size_t pitch, const pd_road_model* model,
                           const pd_road_model* model_dev, const pd_params* p,
                           const pd_outputs* out, bool ccl, int conn, int max_comps,
                           pd_prof_rec* rec, pd_stage_times* times) {
  cudaStream_t s = ctx->stream;
  if (times) cudaEventRecord(ctx->ev[0], s);
  PD_TRY(sgm_enqueue(ctx, left, right, W, H, pitch, model, p, out->kappa, out->d_int, out->D1,
                     rec, model_dev));
  if (times) cudaEventRecord(ctx->ev[1], s);
  PD_TRY(transform_enqueue(ctx, out->D1, W, H, p->model_order, p->delta_dt, out->fitted,
                           out->D2, ctx->ws, p->fit_iters, p->fit_tau));
  mark(ctx, rec, 4);
  if (times) cudaEventRecord(ctx->ev[2], s);
  count_launches(ctx, launch_slic(s, out->D2, W, H, p->slic_K, p->slic_m, p->slic_iters,
                                  out->labels, out->D3, nullptr, ctx->ws));
  mark(ctx, rec, 5);
  if (times) cudaEventRecord(ctx->ev[3], s);
  count_launches(ctx, launch_threshold(s, out->D2, out->D1, out->D3, W, H, p->delta_pd,
                                       p->threshold_mode, out->mask, out->thresholds, nullptr,
                                       ctx->ws));
  if (ccl)
    count_launches(ctx, launch_ccl(s, out->mask, out->labels, W, H, conn, out->components,
                                   out->comps, max_comps, out->n_comps, ctx->ws));
  mark(ctx, rec, 6);
  if (times) cudaEventRecord(ctx->ev[4], s);
  return launched(ctx, "pd_run_pipeline");
}

void pipe_graph_free(pd_ctx* ctx) {
  if (ctx->pipe_exec) cudaGraphExecDestroy(ctx->pipe_exec);
  if (ctx->pipe_src) cudaGraphDestroy(ctx->pipe_src);
  delete static_cast<std::vector<unsigned char>*>(ctx->pipe_key);
  ctx->pipe_exec = nullptr;
  ctx->pipe_src = nullptr;
  ctx->pipe_key = nullptr;
  ctx->pipe_kernels = 0;
  ctx->cap_used = 0;
}

// Captures the whole path on the capture stream into ctx->pipe_exec.  A held executable of the
// same shape (kernels, copies, marks) is updated in place, which is cheaper than a new
// instantiation; the graph it was instantiated from keeps addressing its nodes.
pd_status pipeline_capture(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                           size_t pitch, const pd_road_model* model,
                           const pd_road_model* model_dev, const pd_params* p,
                           const pd_outputs* out, bool ccl, int conn, int max_comps,
                           const std::vector<unsigned char>& key) {
  if (!ctx->cap_stream)
    PD_TRY(cuda_ok(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking),
                   "cudaStreamCreateWithFlags"));
  for (auto& e : ctx->cap_ev)
    if (!e) PD_TRY(cuda_ok(ctx, cudaEventCreate(&e), "cudaEventCreate"));
  cudaStream_t user = ctx->stream;
  ctx->stream = ctx->cap_stream;
  ctx->capturing = true;
  ctx->cap_used = 0;
  pd_status st = cuda_ok(ctx, cudaStreamBeginCapture(ctx->cap_stream,
                                                     cudaStreamCaptureModeThreadLocal),
                         "cudaStreamBeginCapture");
  cudaGraph_t g = nullptr;
  if (st == PD_OK) {
    st = pipeline_enqueue(ctx, left, right, W, H, pitch, model, model_dev, p, out, ccl, conn,
                          max_comps, ctx->prof ? &ctx->cap_rec : nullptr, nullptr);
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);  // always ends the capture
    if (st == PD_OK) st = cuda_ok(ctx, e, "cudaStreamEndCapture");
  }
  ctx->capturing = false;
  ctx->stream = user;
  if (st != PD_OK) {
    if (g) cudaGraphDestroy(g);
    pipe_graph_free(ctx);
    return st;
  }
  const int used = ctx->cap_used;
  if (ctx->pipe_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ctx->pipe_exec, g, &info) == cudaSuccess) {
      cudaGraphDestroy(g);
      *static_cast<std::vector<unsigned char>*>(ctx->pipe_key) = key;
      return PD_OK;
    }
    cudaGetLastError();  // a different shape: instantiate anew
  }
  pipe_graph_free(ctx);
  ctx->cap_used = used;
  st = cuda_ok(ctx, cudaGraphInstantiate(&ctx->pipe_exec, g, 0), "cudaGraphInstantiate");
  if (st != PD_OK) {
    cudaGraphDestroy(g);
    ctx->pipe_exec = nullptr;
    return st;
  }
  ctx->pipe_src = g;
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(g, nodes.data(), &n);
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType t;
    cudaGraphNodeGetType(node, &t);
    if (t == cudaGraphNodeTypeKernel) ++ctx->pipe_kernels;
    if (t == cudaGraphNodeTypeEventRecord) {
      cudaEvent_t ev = nullptr;
      cudaGraphEventRecordNodeGetEvent(node, &ev);
      for (int i = 0; i < 7; ++i)
        if (ev == ctx->cap_ev[i]) ctx->cap_node[i] = node;
    }
  }
  ctx->pipe_key = new std::vector<unsigned char>(key);
  return cuda_ok(ctx, cudaGetLastError(), "pipeline graph");
}

// Replays the captured path (capturing it first when the call differs from the captured one).
pd_status pipeline_graph_run(pd_ctx* ctx, const uint8_t* left, const uint8_t* right, int W, int H,
                             size_t pitch, const pd_road_model* model,
                             const pd_road_model* model_dev, const pd_params* p,
                             const pd_outputs* out, bool ccl, int conn, int max_comps) {
  std::vector<unsigned char> key;
  auto put = [&key](const void* v, size_t bytes) {
    const unsigned char* b = static_cast<const unsigned char*>(v);
    key.insert(key.end(), b, b + bytes);
  };
  put(&left, sizeof left);
  put(&right, sizeof right);
  put(&W, sizeof W);
  put(&H, sizeof H);
  put(&pitch, sizeof pitch);
  if (model)
    put(model, sizeof *model);
  else
    put(&model_dev, sizeof model_dev);
  put(p, sizeof *p);
  put(out, sizeof *out);
  put(&ctx->ws, sizeof ctx->ws);
  const int prof = ctx->prof ? ctx->prof_mask : 0;
  put(&prof, sizeof prof);
  const auto* held = static_cast<const std::vector<unsigned char>*>(ctx->pipe_key);
  if (!ctx->pipe_exec || !held || *held != key)
    PD_TRY(pipeline_capture(ctx, left, right, W, H, pitch, model, model_dev, p, out, ccl, conn,
                            max_comps, key));
  if (ctx->prof) {
    // this call's profiling record receives the stage marks; with the record ring full they go
    // back to the capture events so that no earlier record is overwritten
    pd_prof_rec* rec = prof_begin(ctx);
    for (int i = 0; i < 7; ++i) {
      if (!(ctx->cap_used >> i & 1)) continue;
      cudaEvent_t ev = ctx->cap_ev[i];
      if (rec) {
        if (!rec->ev[i]) PD_TRY(cuda_ok(ctx, cudaEventCreate(&rec->ev[i]), "cudaEventCreate"));
        ev = rec->ev[i];
        rec->used |= 1 << i;
      }
      PD_TRY(cuda_ok(ctx, cudaGraphExecEventRecordNodeSetEvent(ctx->pipe_exec, ctx->cap_node[i], ev),
                     "cudaGraphExecEventRecordNodeSetEvent"));
    }
  }
  PD_TRY(cuda_ok(ctx, cudaGraphLaunch(ctx->pipe_exec, ctx->stream), "cudaGraphLaunch"));
  count_launches(ctx, ctx->pipe_kernels);
  return PD_OK;
}

}  // namespace

pd_status pd_profile_enable(pd_ctx* ctx, int on) {
  if (!ctx) return PD_ERR_INVALID_ARG;
  ctx->prof = on != 0;
  // on == 2: only the two marks around the aggregation (after the prep, after the aggregation)
  ctx->prof_mask = on == 2 ? 0x6 : 0x7f;
  ctx->nrec = 0;
  ctx->launches = 0;
  return PD_OK;
}

pd_status pd_profile_read(pd_ctx* ctx, pd_profile* out) {
  PD_TRY(begin(ctx));
  PD_REQUIRE(out != nullptr, "out is NULL");
  memset(out, 0, sizeof(*out));
  double* slot[7] = {nullptr, &out->prep_ms, &out->aggregate_ms, &out->disparity_ms,
                     &out->transform_ms, &out->superpixel_ms, &out->mask_ms};
  for (int i = 0; i < ctx->nrec; ++i) {
    pd_prof_rec& r = ctx->recs[i];
    int first = -1, last = -1;
    for (int k = 0; k < 7; ++k)
      if (r.used & (1 << k)) {
        if (first < 0) first = k;
        last = k;
      }
    if (first < 0 || last <= first) continue;
    PD_TRY(cuda_ok(ctx, cudaEventSynchronize(r.ev[last]), "pd_profile_read"));
    int prev = first;
    for (int k = first + 1; k <= last; ++k) {
      if (!(r.used & (1 << k))) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.ev[prev], r.ev[k]);
      *slot[k] += ms;
      prev = k;
    }
    float tot = 0.f;
    cudaEventElapsedTime(&tot, r.ev[first], r.ev[last]);
    out->total_ms += tot;
    out->calls += 1;
  }
  out->launches = ctx->launches;
  ctx->nrec = 0;
  ctx->launches = 0;
  return PD_OK;
}

}  // extern "C"
