// Explicit instantiation of the step kernels for one storage precision.
// Included by two translation units per precision with KTF (population
// storage), KTG (solute storage), KR (compute type), KNAME and KPART defined:
// KPART 1 holds the tile shapes of one node per thread and every other
// kernel, KPART 2 the bulk kernels of two nodes per thread (compiled apart so
// that the units build in parallel); the runtime merges the two tables.
#include "launch.h"
#include "bulk.cuh"
#include "interface.cuh"
#include "aux.cuh"

namespace pslbm {
namespace {

// Persistent grid: as many blocks as fit on the device at once (capped by the
// tile count); each block walks the tile list with a stride of the grid size.
template <class SH, int NS, bool SINGLE>
int bulk_grid(int ntiles) {
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bulk<SH, KTF, KTG, KR, NS, SINGLE>, NTHREADS, 0);
    cap = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return ntiles < cap ? ntiles : cap;
}
// single: the tile list covers one simulation (insts[0]) only.
template <class SH, int NS>
void bulk_l(cudaStream_t s, const Tile* tiles, int ntiles, const DevInst* insts, bool single) {
  if (ntiles <= 0) return;
  if (single)
    k_bulk<SH, KTF, KTG, KR, NS, true><<<bulk_grid<SH, NS, true>(ntiles), NTHREADS, 0, s>>>(tiles, ntiles, insts);
  else
    k_bulk<SH, KTF, KTG, KR, NS, false><<<bulk_grid<SH, NS, false>(ntiles), NTHREADS, 0, s>>>(tiles, ntiles, insts);
}
// Staged variants: grid of as many blocks as fit (two or three per SM, by
// the variant's shared memory and registers), dynamic shared memory opted in
// once.
template <class SH, int SHAPE, int NS, int MODE, bool SINGLE>
int bulk_tma_cap() {
  constexpr int smem = tma_smem<SH, KTG, NS, MODE>();
  static int cap = 0;
  if (cap == 0) {
    auto k = k_bulk_tma<SH, SHAPE, KTG, NS, MODE, SINGLE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, NTHREADS, smem);
    cap = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  return cap;
}
// single: the parameter block of the only simulation of the tile list (host
// copy, passed by value), or null for a batch.
template <class SH, int SHAPE, int NS, int MODE>
void bulk_tma_l(cudaStream_t s, const Tile* tiles, int ntiles, const DevInst* insts, const DevParams* single) {
  if (ntiles <= 0) return;
  constexpr int smem = tma_smem<SH, KTG, NS, MODE>();
  if (single) {
    const int cap = bulk_tma_cap<SH, SHAPE, NS, MODE, true>();
    k_bulk_tma<SH, SHAPE, KTG, NS, MODE, true>
        <<<ntiles < cap ? ntiles : cap, NTHREADS, smem, s>>>(tiles, ntiles, insts, *single);
  } else {
    static const DevParams unused{};
    const int cap = bulk_tma_cap<SH, SHAPE, NS, MODE, false>();
    k_bulk_tma<SH, SHAPE, KTG, NS, MODE, false>
        <<<ntiles < cap ? ntiles : cap, NTHREADS, smem, s>>>(tiles, ntiles, insts, unused);
  }
}
#if KPART == 1
// Grid over the chunks of VOP_CHUNK interface-bitmap words of all members
// (one chunk per warp), capped at one wave of resident blocks (warps then
// stride).
template <int NS>
void vop_l(cudaStream_t s, const DevInst* insts, const int2* chunk_map, long long nchunks) {
  if (nchunks <= 0) return;
  static int cap = 0;
  if (cap == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_vop<KTF, KTG, KR, NS>, NTHREADS, 0);
    cap = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }
  const long long need = (nchunks * 32 + NTHREADS - 1) / NTHREADS;
  k_vop<KTF, KTG, KR, NS><<<int(need < cap ? need : cap), NTHREADS, 0, s>>>(insts, chunk_map, nchunks);
}
template <int NS>
void amend_l(cudaStream_t s, int ninst, const DevInst* insts) {
  if (ninst <= 0) return;
  k_amend<KTF, KTG, KR, NS><<<ninst, NTHREADS, 0, s>>>(insts);
}
template <int NS>
void init_l(cudaStream_t s, DevInst* I, const uint8_t* m, const double* r1, const double* r2, const double* c,
            long long N) {
  long long blocks = (N + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  k_init<KTF, KTG, KR, NS><<<(int)blocks, 256, 0, s>>>(I, m, r1, r2, c);
}
template <int NS>
void fields_l(cudaStream_t s, const DevInst* I, long long N, double* r1, double* r2, double* ux, double* uy,
              double* c, uint8_t* t) {
  long long blocks = (N + 255) / 256;
  if (blocks > 65536) blocks = 65536;
  k_fields<KTF, KTG, KR, NS><<<(int)blocks, 256, 0, s>>>(I, r1, r2, ux, uy, c, t);
}
template <int NS>
void budget_l(cudaStream_t s, const DevInst* I, double* part, double* out) {
  k_budget_partial<KTF, KTG, KR, NS><<<BUD_BLOCKS, BUD_THREADS, 0, s>>>(I, part);
  k_budget_final<<<1, BUD_FINAL_THREADS, 0, s>>>(part, BUD_BLOCKS, out);
}
#endif

template <int NS>
constexpr Launchers make() {
#if KPART == 1
  if constexpr (sizeof(KTF) == 4) {
    return Launchers{{&bulk_l<ShapeA, NS>, &bulk_l<ShapeB, NS>, nullptr, nullptr},
                     {&bulk_tma_l<ShapeA, 0, NS, 1>, &bulk_tma_l<ShapeB, 1, NS, 1>, nullptr, nullptr},
                     {&bulk_tma_l<ShapeA, 0, NS, 2>, &bulk_tma_l<ShapeB, 1, NS, 2>, nullptr, nullptr},
                     &vop_l<NS>,
                     &amend_l<NS>, &init_l<NS>, &fields_l<NS>, &budget_l<NS>};
  } else {
    return Launchers{{&bulk_l<ShapeA, NS>, &bulk_l<ShapeB, NS>, nullptr, nullptr},
                     {nullptr, nullptr, nullptr, nullptr},
                     {nullptr, nullptr, nullptr, nullptr},
                     &vop_l<NS>,
                     &amend_l<NS>, &init_l<NS>, &fields_l<NS>, &budget_l<NS>};
  }
#else
  if constexpr (sizeof(KTF) == 4) {
    return Launchers{{nullptr, nullptr, &bulk_l<ShapeC, NS>, &bulk_l<ShapeD, NS>},
                     {nullptr, nullptr, nullptr, nullptr},
                     {nullptr, nullptr, &bulk_tma_l<ShapeC, 2, NS, 2>, &bulk_tma_l<ShapeD, 3, NS, 2>},
                     nullptr, nullptr, nullptr, nullptr, nullptr};
  } else {
    return Launchers{{nullptr, nullptr, &bulk_l<ShapeC, NS>, &bulk_l<ShapeD, NS>},
                     {nullptr, nullptr, nullptr, nullptr},
                     {nullptr, nullptr, nullptr, nullptr},
                     nullptr, nullptr, nullptr, nullptr, nullptr};
  }
#endif
}
const Launchers table[MAXS + 1] = {make<0>(), make<1>(), make<2>(), make<3>(), make<4>()};

}  // namespace

const Launchers* KNAME(int ns) { return (ns >= 0 && ns <= MAXS) ? &table[ns] : nullptr; }

}  // namespace pslbm
