// Budget read-out that allocates nothing.
//
// pslbm_read_fields(PSLBM_F_BUDGET) reduces the state into per-block partial
// sums held in a device buffer the library allocates on first use.  Some
// callers cannot allocate device memory at the point where they want the
// budget: hosts that hand the library a fixed memory pool and forbid any later
// allocation, and real-time loops where an allocation (which may synchronise
// the device or take a driver lock) could stall.  pslbm_budget_device_noalloc
// gives them the same numbers with the partial sums in a file-scope device
// array instead.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/pslbm.h"
#include "aux.cuh"
#include "launch.h"

using namespace pslbm;

namespace {

// Scratch: one partial-sum row per block of the budget reduction, with the
// same fixed grid of BUD_BLOCKS blocks that pslbm_read_fields uses, so both
// add the same numbers in the same order and give the same bits.  Each block
// covers a contiguous 1/BUD_BLOCKS of the lattice, so any lattice the library
// accepts fits.  The array is BUD_BLOCKS * NBUD doubles (36 KiB), held by every
// GPU that loads the library until the process exits.
static __device__ __align__(256) double g_noalloc_partials[BUD_BLOCKS * NBUD];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
double* g_partials_ptr[MAX_DEVICES] = {};

// Final pass: fixed-order sum of the partial rows into the caller's buffer, in
// the layout of the PSLBM_F_BUDGET field (max rho1, sum rho1, sum rho2, sum C_k,
// sum V_D, sum V_F, step count).
__global__ void __launch_bounds__(BUD_FINAL_THREADS) k_noalloc_final(const double* __restrict__ part, int nblocks,
                                                                     int ns, const DevInst* __restrict__ Ip,
                                                                     double* __restrict__ out) {
  double v[NBUD];
  budget_reduce(part, nblocks, v);
  if (threadIdx.x != 0) return;
  out[0] = v[0] > -1.0 / 0.0 ? v[0] : 0.0;
  out[1] = v[1];
  out[2] = v[2];
  for (int k = 0; k < ns; ++k) out[3 + k] = v[3 + k];
  out[3 + ns] = v[3 + MAXS];
  out[4 + ns] = v[4 + MAXS];
  out[5 + ns] = (double)Ip->scal[S_STEP];
}

template <class TF, class TG, class R, int NS>
void launch_partial(cudaStream_t s, const DevInst* I, double* part) {
  k_budget_partial<TF, TG, R, NS><<<BUD_BLOCKS, BUD_THREADS, 0, s>>>(I, part);
}

template <class TF, class TG, class R>
bool dispatch_ns(int ns, cudaStream_t s, const DevInst* I, double* part) {
  switch (ns) {
    case 0: launch_partial<TF, TG, R, 0>(s, I, part); return true;
    case 1: launch_partial<TF, TG, R, 1>(s, I, part); return true;
    case 2: launch_partial<TF, TG, R, 2>(s, I, part); return true;
    case 3: launch_partial<TF, TG, R, 3>(s, I, part); return true;
    case 4: launch_partial<TF, TG, R, 4>(s, I, part); return true;
  }
  return false;
}

// Device address of the scratch array for the current device, looked up once
// per device (host code cannot use the array's name as a device address).
cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_ptr[dev] = (double*)p;
  }
  *out = g_partials_ptr[dev];
  return cudaSuccess;
}

}  // namespace

namespace pslbm {
// Accessors into the handle (defined in runtime.cu).
const DevInst* handle_device_inst(pslbm_t h);
int handle_precision(pslbm_t h);
int handle_species(pslbm_t h);
pslbm_status handle_sticky(pslbm_t h);
pslbm_status handle_fail(pslbm_t h, pslbm_status s, const std::string& msg);
cudaStream_t library_stream();
}  // namespace pslbm

extern "C" pslbm_status pslbm_budget_device_noalloc(pslbm_t h, double* out) {
  if (!h) return handle_fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  // a handle whose state is poisoned (device error, non-finite or EOS-domain
  // state, timed-out wait) reports that error, as every other call does
  const pslbm_status sticky = handle_sticky(h);
  if (sticky != PSLBM_OK) return sticky;
  if (!out) return handle_fail(h, PSLBM_ERR_PARAM, "out is NULL");
  double* part = nullptr;
  cudaError_t e = partials_address(&part);
  if (e != cudaSuccess)
    return handle_fail(h, PSLBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t s = library_stream();
  const DevInst* I = handle_device_inst(h);
  const int ns = handle_species(h);
  bool ok = false;
  switch (handle_precision(h)) {
    case PSLBM_FP64: ok = dispatch_ns<double, double, double>(ns, s, I, part); break;
    case PSLBM_FP32: ok = dispatch_ns<float, float, float>(ns, s, I, part); break;
    case PSLBM_FP32_SOLUTE_F16: ok = dispatch_ns<float, __half, float>(ns, s, I, part); break;
    case PSLBM_FP32_SOLUTE_BF16: ok = dispatch_ns<float, __nv_bfloat16, float>(ns, s, I, part); break;
  }
  if (!ok) return handle_fail(h, PSLBM_ERR_PARAM, "no budget kernel for this precision / species count");
  k_noalloc_final<<<1, BUD_FINAL_THREADS, 0, s>>>(part, BUD_BLOCKS, ns, I, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return handle_fail(h, PSLBM_ERR_CUDA, std::string("budget launch: ") + cudaGetErrorString(e));
  return PSLBM_OK;
}
