// Internal types of the batched Sec. II-A / II-B path (batch.cu, api.cu).
#pragma once

#include "common.cuh"

namespace pd {

// One pair of a wave, with its scratch pieces, as the device kernels read it.
struct BatchPair {
  const uint8_t* left;
  const uint8_t* right;
  size_t pitch;
  int32_t* kappa;
  int16_t* d_int;
  float* D1;
  uint32_t* cl;
  uint32_t* cr;
  uint8_t* cost;
  uint8_t* vols;
  float* dsub;
  uint32_t* rkeys;
  size_t vol_bytes;
  double a0, a1, a2, cs, sn, delta_pt;
  int W, H, D, order;
};

// A run of aggregation tasks: direction r = (dx, dy) of one pair; task `first` + j covers the
// j-th group of batch_lines_per_warp(D, dx, dy) lines.
struct BatchSegment {
  int first, pair, r, dx, dy, pad;
};

// Stages whose launch covers every pair of a wave (Eq. (9) runs one launch per pair).
enum { kStageKappa = 0, kStageCensus, kStageCost, kStageFill, kStageLr, kBatchStages };

// Device view of one wave: the tables live in the context scratch.
struct BatchWaveDev {
  const BatchPair* pairs;
  const BatchPair* host_pairs;      // the same table in host memory (shapes for per-pair grids)
  const int* starts[kBatchStages];  // per stage, npairs + 1 block prefixes
  const BatchSegment* segs;
  unsigned int* counter;
  int npairs, nseg, ntasks;
  int total[kBatchStages];
};

void batch_stage_blocks(int W, int H, int D, int counts[kBatchStages]);
// lines a warp walks in one aggregation task of direction (dx, dy)
int batch_lines_per_warp(int D, int dx, int dy);
size_t batch_agg_smem(int warps_per_block);
int batch_max_blocks_per_sm(int agg_warps);
void launch_batch_wave(cudaStream_t s, const BatchWaveDev& w, int P1, int P2, int lr_tol,
                       int paths, int agg_warps, int agg_blocks);
void launch_batch_aggregate_only(cudaStream_t s, const BatchWaveDev& w, int P1, int P2,
                                 int agg_warps, int agg_blocks);

}  // namespace pd
