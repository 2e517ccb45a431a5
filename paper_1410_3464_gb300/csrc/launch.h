// Internal launcher table: one entry per (storage precision, species count).
#pragma once
#include <cuda_runtime.h>
#include "device.cuh"

namespace pslbm {

struct Launchers {
  void (*bulk[NSHAPES])(cudaStream_t, const Tile*, int ntiles, const DevInst*, bool single);
  // TMA-staged bulk kernel (FP32 populations only; null for FP64); single is
  // the host parameter block when the tile list holds one simulation, else null
  void (*bulk_tma[NSHAPES])(cudaStream_t, const Tile*, int ntiles, const DevInst*, const DevParams* single);
  // TMA-staged bulk kernel with a single stage and three blocks per SM
  void (*bulk_tma1[NSHAPES])(cudaStream_t, const Tile*, int ntiles, const DevInst*, const DevParams* single);
  // chunk_map: (member, chunk) of every VOP chunk of a batch (null for one
  // simulation); nchunks: their number
  void (*vop)(cudaStream_t, const DevInst*, const int2* chunk_map, long long nchunks);
  void (*amend)(cudaStream_t, int ninst, const DevInst*);
  void (*init)(cudaStream_t, DevInst*, const uint8_t*, const double*, const double*, const double*, long long N);
  void (*fields)(cudaStream_t, const DevInst*, long long N, double*, double*, double*, double*, double*, uint8_t*);
  void (*budget)(cudaStream_t, const DevInst*, double* part, double* out);
};

// prec: 0 FP64, 1 FP32, 2 FP32 + half solutes, 3 FP32 + bfloat16 solutes; ns 0..MAXS
const Launchers* launchers(int prec, int ns);

}  // namespace pslbm
