// Host runtime behind the C ABI of include/pslbm.h: parameter validation,
// device allocation of the structure-of-arrays state, tile lists, CUDA-graph
// capture of whole steps, field read-out and batches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/pslbm.h"
#include "launch.h"

using namespace pslbm;

namespace {

std::mutex g_mu;
cudaStream_t g_own_stream = nullptr;
cudaStream_t g_user_stream = nullptr;
bool g_user_set = false;
std::string g_lib_err;

cudaStream_t lib_stream() {
  if (g_user_set) return g_user_stream;
  if (!g_own_stream) cudaStreamCreateWithFlags(&g_own_stream, cudaStreamNonBlocking);
  return g_own_stream;
}

size_t fsize(int prec) { return prec == PSLBM_FP64 ? 8 : 4; }
size_t gsize(int prec) { return prec == PSLBM_FP64 ? 8 : (prec == PSLBM_FP32 ? 4 : 2); }

struct GraphCache {
  std::map<int64_t, cudaGraphExec_t> exec;
  void clear() {
    for (auto& kv : exec) cudaGraphExecDestroy(kv.second);
    exec.clear();
  }
};

constexpr int NSTAGING = 3;

// Launch state shared by a single simulation and a batch: one tile list per
// tile shape (built on demand), the chosen bulk-kernel variant (tile shape and
// staging: plain loads or TMA-staged), and the captured graphs.
struct Stepper {
  const Launchers* L = nullptr;
  DevInst* d = nullptr;
  int ninst = 0;
  std::vector<std::pair<int, int>> dims;   // (nx, ny) per instance
  Tile* tiles[NSHAPES] = {};
  int ntiles[NSHAPES] = {};
  int shape = 0;
  int staged = 0;                          // 1: TMA-staged, two stages; 2: TMA-staged, one stage
  int fix_shape = -1;                      // caller's choice, -1: choose by timing
  int fix_staged = -1;
  bool staged_ok = false;                  // every instance has TMA descriptors
  const DevParams* single = nullptr;       // host parameters of a one-simulation stepper
  int2* chunk_map = nullptr;               // (instance, chunk) of every VOP chunk of a batch (device)
  long long nchunks = 0;                   // VOP chunks of all instances
  bool tuned = false;                      // variant chosen (by timing or by the caller)
  GraphCache graphs;
  double trial_ms[NSHAPES][NSTAGING] = {};
  void release() {
    graphs.clear();
    if (chunk_map) cudaFree(chunk_map);
    chunk_map = nullptr;
    for (int s = 0; s < NSHAPES; ++s) {
      if (tiles[s]) cudaFree(tiles[s]);
      tiles[s] = nullptr;
      ntiles[s] = 0;
    }
  }
};

}  // namespace

struct pslbm_s {
  pslbm_params p{};
  int prec = 0;
  int ns = 0;
  long long N = 0;
  DevInst h{};                 // host copy of the device descriptor
  DevInst* d = nullptr;        // device descriptor
  Stepper run;
  std::vector<void*> allocs;
  uint64_t bytes = 0;
  double* rb = nullptr;        // read-back scratch
  size_t rb_bytes = 0;
  std::string err;
  pslbm_status sticky = PSLBM_OK;
  int in_batch = 0;
  const Launchers* L = nullptr;
};

struct pslbm_batch_s {
  std::vector<pslbm_t> members;
  DevInst* d = nullptr;
  Stepper run;
  const Launchers* L = nullptr;
  std::string err;
  pslbm_status sticky = PSLBM_OK;
  unsigned long long* mon = nullptr;       // device: (step, status) per member, for pslbm_batch_monitor
  std::vector<unsigned long long> mon_h;
};

namespace {

pslbm_status fail(pslbm_t h, pslbm_status s, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (s == PSLBM_ERR_CUDA || s == PSLBM_ERR_NONFINITE || s == PSLBM_ERR_EOS_DOMAIN || s == PSLBM_ERR_TIMEOUT)
      h->sticky = s;
  } else {
    std::lock_guard<std::mutex> lk(g_mu);
    g_lib_err = msg;
  }
  return s;
}

#define CK(h, call)                                                                                   \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(h, PSLBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

pslbm_status check_device() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return PSLBM_ERR_NODEVICE;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return PSLBM_ERR_NODEVICE;
  if (!(prop.major == 10 && prop.minor == 3)) return PSLBM_ERR_NODEVICE;
  return PSLBM_OK;
}

std::string validate(const pslbm_params* p) {
  char buf[256];
  if (!p) return "params is NULL";
  if (p->struct_size != sizeof(pslbm_params)) {
    snprintf(buf, sizeof buf, "struct_size %u != %zu", p->struct_size, sizeof(pslbm_params));
    return buf;
  }
  if (p->nx < 1 || p->ny < 1 || (long long)p->nx * p->ny > 100000000LL)
    return "lattice size must be 1..100,000,000 nodes";
  if (p->precision < 0 || p->precision > 3) return "bad precision";
  for (int s = 0; s < 2; ++s)
    if (!(p->tau[s] > 0.5) || !std::isfinite(p->tau[s])) return "tau must be > 0.5";
  if (p->n_species < 0 || p->n_species > PSLBM_MAX_SPECIES) return "n_species out of range";
  if (p->precision >= 2 && p->n_species == 0) return "16-bit solute storage needs species";
  const int ns = p->n_species;
  auto okidx = [&](int i, bool allow_derived) {
    return i == PSLBM_IDX_ABSENT || (i >= 0 && i < ns) || (allow_derived && i == PSLBM_IDX_DERIVED);
  };
  if (!okidx(p->idx_A, true) || !okidx(p->idx_B, false) || !okidx(p->idx_E, false) || !okidx(p->idx_F, false))
    return "species index out of range";
  {
    int ids[4] = {p->idx_A, p->idx_B, p->idx_E, p->idx_F};
    for (int i = 0; i < 4; ++i)
      for (int j = i + 1; j < 4; ++j)
        if (ids[i] >= 0 && ids[i] == ids[j]) return "two roles share one species index";
  }
  for (int k = 0; k < ns; ++k) {
    if (!(p->J0[k] >= 0.0 && p->J0[k] < 1.0)) return "J0 must be in [0, 1)";
    if (!(p->tau_g[k] > 0.5)) return "tau_g must be > 0.5";
  }
  if (p->G11 != 0.0 && !(p->eos_b > 0 && p->eos_R > 0 && p->eos_T > 0)) return "bad EOS constants";
  if (!(p->rho10 != 0.0 && p->rho20 != 0.0)) return "rho10, rho20 must be nonzero";
  // reactive link rule needs kappa = k / (2 J_w) < 1
  if (p->idx_B >= 0 && p->k2 != 0.0 && !(p->k2 >= 0.0 && p->k2 < 0.5 * (1.0 - p->J0[p->idx_B])))
    return "k2 must be in [0, (1 - J0_B)/2)";
  if (p->idx_F >= 0 && p->k4 != 0.0 && !(p->k4 >= 0.0 && p->k4 < 0.5 * (1.0 - p->J0[p->idx_F])))
    return "k4 must be in [0, (1 - J0_F)/2)";
  if (!(p->V_split > 1.0)) return "V_split must be > 1";
  if (!(p->r1_surface_factor >= 0.0) || !std::isfinite(p->r1_surface_factor)) return "r1_surface_factor must be >= 0";
  for (int k = 0; k < PSLBM_MAX_SPECIES; ++k)
    if (!(p->conc_scale[k] >= 0.0) || !std::isfinite(p->conc_scale[k])) return "conc_scale must be >= 0 and finite";
  if (p->inlet_axis < 0 || p->inlet_axis > 1 || p->outlet_axis < 0 || p->outlet_axis > 1) return "axes must be 0 or 1";
  if (p->inlet_period_liq < 0 || p->inlet_period_gas < 0 ||
      (p->inlet_period_gas > 0 && p->inlet_period_liq + p->inlet_period_gas <= 0))
    return "bad inlet periods";
  if (p->inlet_ramp < 0 || (p->inlet_period_gas > 0 &&
                            (p->inlet_ramp > p->inlet_period_liq || p->inlet_ramp > p->inlet_period_gas)))
    return "inlet_ramp must be in [0, min(inlet periods)]";
  return "";
}

template <class R>
void fill_r(DevParamsR<R>& q, const DevParams& P) {
  for (int s = 0; s < 2; ++s) {
    q.tau[s] = R(P.tau[s]);
    q.inv_tau[s] = R(P.inv_tau[s]);
    q.w_adh[s] = R(P.w_adh[s]);
    q.shift_f[s] = R(P.shift_f[s]);
    q.shift_fg[s] = R(P.shift_fg[s]);
    q.rho_fill[s] = R(P.rho_fill[s]);
  }
  q.G11 = R(P.G11);
  q.G12 = R(P.G12);
  q.G21 = R(P.G21);
  q.a0 = R(P.a0);
  q.inv_rho10 = R(1.0 / P.rho10);
  q.inv_rho20 = R(1.0 / P.rho20);
  q.eos_a = R(P.eos_a);
  q.eos_b4 = R(P.eos_b / 4.0);
  q.eos_RT = R(P.eos_R * P.eos_T);
  q.six_over_G11 = R(P.G11 != 0.0 ? 6.0 / P.G11 : 0.0);
  q.gx = R(P.gx);
  q.gy = R(P.gy);
  for (int k = 0; k < MAXS; ++k) {
    q.J0[k] = R(P.J0[k]);
    q.Ja[k] = R(P.Ja[k]);
    q.inv_tau_g[k] = R(P.inv_tau_g[k]);
    q.shift_c[k] = R(P.shift_c[k]);
    q.conc_in[k] = R(P.conc_in[k]);
    q.cR1[k] = R(P.cR1[k]);
    q.cR3[k] = R(P.cR3[k]);
    q.gs_mul[k] = R(P.gs_scale[k]);
    q.gs_div[k] = R(1.0 / P.gs_scale[k]);
  }
  q.k1 = R(P.k1);
  q.k1_inv_Keq = R(P.k1 * P.inv_Keq);
  q.k1_s = R(P.k1 * P.r1_surface_factor);
  q.k1_inv_Keq_s = R(P.k1 * P.r1_surface_factor * P.inv_Keq);
  q.k3 = R(P.k3);
  q.k2 = R(P.k2);
  q.k4 = R(P.k4);
  q.C_F_sat = R(P.C_F_sat);
  q.gas_yield = R(P.gas_yield);
  q.inv_M_C = R(P.inv_M_C);
  q.c_total_per_rho1 = R(P.c_total_per_rho1);
  // link rule with kappa = k / (2 J_w), J_w = J_a: back = (out (1 - kappa) + k C_sat) / (1 + kappa),
  // flux q = out - back = out 2 kappa / (1 + kappa) - k C_sat / (1 + kappa) (no cancellation)
  q.vB_qa = q.vB_sh = q.vF_qa = q.vF_qc = q.vF_sh = R(0);
  if (P.iB >= 0) {
    const double kap = P.k2 / (2.0 * P.Ja[P.iB]);
    q.vB_qa = R(2.0 * kap / (1.0 + kap));
    q.vB_sh = R(P.Ja[P.iB] * P.shift_c[P.iB]);
  }
  if (P.iF >= 0) {
    const double kap = P.k4 / (2.0 * P.Ja[P.iF]);
    q.vF_qa = R(2.0 * kap / (1.0 + kap));
    q.vF_qc = R(P.k4 * P.C_F_sat / (1.0 + kap));
    q.vF_sh = R(P.Ja[P.iF] * P.shift_c[P.iF]);
  }
}

DevParams to_dev(const pslbm_params* p) {
  DevParams P{};
  P.nx = p->nx;
  P.ny = p->ny;
  P.px = p->periodic_x ? 1 : 0;
  P.py = p->periodic_y ? 1 : 0;
  P.ns = p->n_species;
  P.iA = p->idx_A;
  P.iB = p->idx_B;
  P.iE = p->idx_E;
  P.iF = p->idx_F;
  P.in_dx = p->inlet_axis == 1 ? 0 : 1;
  P.in_dy = p->inlet_axis == 1 ? 1 : 0;
  P.out_dx = p->outlet_axis == 1 ? 0 : -1;
  P.out_dy = p->outlet_axis == 1 ? -1 : 0;
  P.per_liq = p->inlet_period_liq;
  P.per_gas = p->inlet_period_gas;
  P.ramp = p->inlet_ramp;
  for (int s = 0; s < 2; ++s) {
    P.tau[s] = p->tau[s];
    P.w_adh[s] = p->w_adh[s];
    P.shift_f[s] = p->precision == PSLBM_FP64 ? 0.0 : p->rho_ref[s];
    P.shift_fg[s] = p->precision == PSLBM_FP64 ? 0.0 : p->rho_ref_gas[s];
    P.rho_fill[s] = p->rho_ref[s];
    P.rho_in_liq[s] = p->rho_in_liq[s];
    P.rho_in_gas[s] = p->rho_in_gas[s];
    P.rho_out[s] = p->rho_out[s];
    P.rho_out_gas[s] = p->rho_out_gas[s];
  }
  P.G11 = p->G11;
  P.G12 = p->G12;
  P.G21 = p->G21;
  P.a0 = p->a0;
  P.rho10 = p->rho10;
  P.rho20 = p->rho20;
  P.eos_a = p->eos_a;
  P.eos_b = p->eos_b;
  P.eos_R = p->eos_R;
  P.eos_T = p->eos_T;
  P.gx = p->body_force[0];
  P.gy = p->body_force[1];
  for (int k = 0; k < MAXS; ++k) {
    P.J0[k] = p->J0[k];
    P.tau_g[k] = k < p->n_species ? p->tau_g[k] : 1.0;
    P.shift_c[k] = p->precision == PSLBM_FP64 ? 0.0 : p->conc_ref[k];
    P.conc_in[k] = p->conc_in[k];
    // nearest power of two of conc_scale (0: 1), for 16-bit storage only
    double sc = 1.0;
    if (p->precision >= PSLBM_FP32_SOLUTE_F16 && p->conc_scale[k] > 0.0) {
      int e = (int)std::lround(std::log2(p->conc_scale[k]));
      e = std::max(-60, std::min(60, e));
      sc = std::ldexp(1.0, e);
    }
    P.gs_scale[k] = sc;
  }
  for (int s = 0; s < 2; ++s) P.inv_tau[s] = 1.0 / p->tau[s];
  for (int k = 0; k < MAXS; ++k) {
    P.Ja[k] = (1.0 - p->J0[k]) / 4.0;
    P.inv_tau_g[k] = 1.0 / P.tau_g[k];
    P.cR1[k] = (k == p->idx_A ? -1.0 : 0.0) + (k == p->idx_B ? 1.0 : 0.0);
    P.cR3[k] = (k == p->idx_B ? -1.0 : 0.0) + (k == p->idx_E ? -1.0 : 0.0) + (k == p->idx_F ? 1.0 : 0.0);
  }
  P.k1 = p->k1;
  P.r1_surface_factor = p->r1_surface_factor > 0.0 ? p->r1_surface_factor : 1.0;
  P.r1_surf = P.r1_surface_factor != 1.0;
  P.inv_Keq = p->inv_Keq;
  P.k3 = p->k3;
  P.k2 = p->k2;
  P.k4 = p->k4;
  P.C_F_sat = p->C_F_sat;
  P.gas_yield = p->gas_yield;
  P.inv_M_C = p->inv_M_C;
  P.c_total_per_rho1 = p->c_total_per_rho1;
  P.Vbar_D = p->Vbar_D;
  P.Vbar_F = p->Vbar_F;
  P.V_split = p->V_split;
  P.seed = p->seed;
  P.has_G11 = p->G11 != 0.0;
  P.has_rev = p->inv_Keq != 0.0;
  P.useB = p->idx_B >= 0 && p->k2 != 0.0;
  P.useF = p->idx_F >= 0 && p->k4 != 0.0;
  fill_r(P.rf, P);
  fill_r(P.rd, P);
  return P;
}

std::vector<Tile> make_tiles(int inst, int nx, int ny, int shape) {
  std::vector<Tile> t;
  for (int y0 = 0; y0 < ny; y0 += SHAPE_TY[shape])
    for (int x0 = 0; x0 < nx; x0 += SHAPE_TX[shape]) t.push_back(Tile{inst, x0, y0, 0});
  return t;
}

// Tile list of every instance of a stepper for one shape (device copy).
cudaError_t ensure_tiles(Stepper& st, int shape) {
  if (st.tiles[shape]) return cudaSuccess;
  std::vector<Tile> all;
  for (int i = 0; i < (int)st.dims.size(); ++i) {
    std::vector<Tile> t = make_tiles(i, st.dims[i].first, st.dims[i].second, shape);
    all.insert(all.end(), t.begin(), t.end());
  }
  Tile* d = nullptr;
  cudaError_t e = cudaMalloc(&d, all.size() * sizeof(Tile));
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, all.data(), all.size() * sizeof(Tile), cudaMemcpyHostToDevice, lib_stream());
  if (e == cudaSuccess) e = cudaStreamSynchronize(lib_stream());
  if (e != cudaSuccess) {
    cudaFree(d);
    return e;
  }
  st.tiles[shape] = d;
  st.ntiles[shape] = (int)all.size();
  return cudaSuccess;
}

pslbm_status dalloc(pslbm_t h, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(h, e == cudaErrorMemoryAllocation ? PSLBM_ERR_OOM : PSLBM_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(*ptr);
  h->bytes += bytes;
  return PSLBM_OK;
}

void free_all(pslbm_t h) {
  h->run.release();
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

// Enqueue one launch of the bulk kernel of a variant.
void enqueue_bulk(cudaStream_t s, const Stepper& st, int shape, int staged) {
  if (staged == 2)
    st.L->bulk_tma1[shape](s, st.tiles[shape], st.ntiles[shape], st.d, st.single);
  else if (staged == 1)
    st.L->bulk_tma[shape](s, st.tiles[shape], st.ntiles[shape], st.d, st.single);
  else
    st.L->bulk[shape](s, st.tiles[shape], st.ntiles[shape], st.d, st.single != nullptr);
}

// Enqueue n steps of the kernels for one bulk-kernel variant.
void enqueue_steps(cudaStream_t s, const Stepper& st, int shape, int staged, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    enqueue_bulk(s, st, shape, staged);
    st.L->vop(s, st.d, st.chunk_map, st.nchunks);
    st.L->amend(s, st.ninst, st.d);
  }
}

// n steps without graph capture, each kernel bracketed by CUDA events on the
// library stream: mean ms per step of the bulk, VOP and amendment kernels and
// of the whole step.
pslbm_status profile_steps(Stepper& st, int64_t n, double* kernel_ms, double* total_ms, std::string& err) {
  cudaStream_t s = lib_stream();
  cudaError_t te = ensure_tiles(st, st.shape);
  if (te != cudaSuccess) {
    err = std::string("tile list: ") + cudaGetErrorString(te);
    return PSLBM_ERR_CUDA;
  }
  cudaEvent_t ev[4] = {};
  for (int i = 0; i < 4; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
      err = "cudaEventCreate failed";
      return PSLBM_ERR_CUDA;
    }
  double acc[3] = {0, 0, 0}, tot = 0;
  pslbm_status st_ = PSLBM_OK;
  for (int64_t i = 0; i < n; ++i) {
    cudaEventRecord(ev[0], s);
    enqueue_bulk(s, st, st.shape, st.staged);
    cudaEventRecord(ev[1], s);
    st.L->vop(s, st.d, st.chunk_map, st.nchunks);
    cudaEventRecord(ev[2], s);
    st.L->amend(s, st.ninst, st.d);
    cudaEventRecord(ev[3], s);
    cudaError_t e = cudaEventSynchronize(ev[3]);
    if (e != cudaSuccess) {
      err = std::string("profile step: ") + cudaGetErrorString(e);
      st_ = PSLBM_ERR_CUDA;
      break;
    }
    float ms;
    for (int k = 0; k < 3; ++k) {
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      acc[k] += ms;
    }
    cudaEventElapsedTime(&ms, ev[0], ev[3]);
    tot += ms;
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  if (st_ != PSLBM_OK) return st_;
  for (int k = 0; k < 3; ++k) kernel_ms[k] = acc[k] / double(n);
  if (total_ms) *total_ms = tot / double(n);
  return PSLBM_OK;
}

// Initial solid volumes from the node types when the caller gives none:
// V_D = 1 at D(s) nodes, V_F = 1 at F(s) nodes, 0 elsewhere.
__global__ void k_vol_from_mask(const uint8_t* __restrict__ mask, double* __restrict__ V, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int t = mask[i] & 15;
    V[i] = t == PSLBM_SOLID_D ? 1.0 : 0.0;
    V[N + i] = t == PSLBM_SOLID_F ? 1.0 : 0.0;
  }
}

// First step's liquid threshold from the initial maximum of rho_1 over fluid
// nodes (res[0], -inf without fluid): the maximum in the ordered encoding of
// the step's slot, and half of it in both precisions, as the amendment kernel
// leaves them at the end of a step.
__global__ void k_first_threshold(const double* __restrict__ res, unsigned long long* __restrict__ scal) {
  const double m = res[0];
  const unsigned long long enc = m > -INFINITY ? ord_enc(m) : 0ULL;
  const double th = 0.5 * ord_dec(enc);
  scal[S_MAX0] = enc;
  scal[S_THETA] = (unsigned long long)__double_as_longlong(th);
  scal[S_THETAF] = (unsigned long long)(unsigned)__float_as_int(__double2float_rn(th));
}

// Step count and status bits of every member of a batch, gathered into one
// device buffer (out[2 i], out[2 i + 1]) for a single copy to the host.
__global__ void k_batch_monitor(const DevInst* __restrict__ insts, int n, unsigned long long* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    out[2 * i] = insts[i].scal[S_STEP];
    out[2 * i + 1] = insts[i].scal[S_STATUS];
  }
}

// Whether the bulk kernel of a variant is compiled (the staged kernels exist
// for the shapes of one node per thread).
bool variant_exists(const Stepper& st, int sh, int sg) {
  return sg == 0 ? st.L->bulk[sh] != nullptr : sg == 1 ? st.L->bulk_tma[sh] != nullptr : st.L->bulk_tma1[sh] != nullptr;
}

// Variants the stepper may use: every tile shape and staging the caller left
// open (staging only where every instance has TMA descriptors and the shape
// has a staged kernel).
std::vector<std::pair<int, int>> candidates(const Stepper& st) {
  std::vector<std::pair<int, int>> c;
  for (int sh = 0; sh < NSHAPES; ++sh) {
    if (st.fix_shape >= 0 && sh != st.fix_shape) continue;
    for (int sg = 0; sg < NSTAGING; ++sg) {
      if (st.fix_staged >= 0 && sg != st.fix_staged) continue;
      if (sg >= 1 && !st.staged_ok) continue;
      if (!variant_exists(st, sh, sg)) continue;
      c.push_back({sh, sg});
    }
  }
  return c;
}

// After a change of the caller's choices: a single candidate is taken at once;
// otherwise the variant is chosen by timing on the next long step call (until
// then the first candidate runs, with the two-box staging when it is open: the
// fastest staging on every large workload measured).
void choose(Stepper& st) {
  std::vector<std::pair<int, int>> c = candidates(st);
  int sh = c.empty() ? 0 : c[0].first, sg = c.empty() ? 0 : c[0].second;
  for (auto& v : c)
    if (v.first == sh && v.second == 1) sg = 1;
  if (sh != st.shape || sg != st.staged) st.graphs.clear();
  st.shape = sh;
  st.staged = sg;
  st.tuned = c.size() <= 1;
}

// Variant autotuning: the results do not depend on the variant (the per-node
// arithmetic and the fixed-order gathers are the same), so the first steps of
// a run are spent timing each candidate (one untimed step, then TUNE_STEPS
// timed steps each) in TUNE_ROUNDS passes, the second in reverse order, and
// the fastest by its best pass is kept (a run's first steps can be slower
// than its later ones, which a single pass would charge to the first
// candidates).
constexpr int TUNE_STEPS = 3;
constexpr int TUNE_ROUNDS = 2;
pslbm_status autotune(Stepper& st, std::string& err) {
  cudaStream_t s = lib_stream();
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    err = "cudaEventCreate failed";
    return PSLBM_ERR_CUDA;
  }
  std::vector<std::pair<int, int>> c = candidates(st);
  double best_ms = 0;
  int best = -1;
  const int nc = (int)c.size();
  for (int pass = 0; pass < TUNE_ROUNDS * nc; ++pass) {
    const int round = pass / nc;
    const int i = (round & 1) ? nc - 1 - pass % nc : pass % nc;
    const int sh = c[i].first, sg = c[i].second;
    cudaError_t e = ensure_tiles(st, sh);
    if (e != cudaSuccess) {
      err = std::string("tile list: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? PSLBM_ERR_OOM : PSLBM_ERR_CUDA;
    }
    enqueue_steps(s, st, sh, sg, 1);
    cudaEventRecord(a, s);
    enqueue_steps(s, st, sh, sg, TUNE_STEPS);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    if (e != cudaSuccess) {
      err = std::string("autotune: ") + cudaGetErrorString(e);
      return PSLBM_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double t = ms / TUNE_STEPS;
    if (round == 0 || t < st.trial_ms[sh][sg]) st.trial_ms[sh][sg] = t;
    if (best < 0 || t < best_ms) {
      best = i;
      best_ms = t;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (best >= 0) {
    if (c[best].first != st.shape || c[best].second != st.staged) st.graphs.clear();
    st.shape = c[best].first;
    st.staged = c[best].second;
  }
  st.tuned = true;
  return PSLBM_OK;
}

// Steps the autotuner spends (they advance the simulation like any others).
int64_t tune_cost(const Stepper& st) { return (int64_t)candidates(st).size() * (TUNE_STEPS + 1) * TUNE_ROUNDS; }

// Run n steps, replaying captured graphs of up to 32 steps.
pslbm_status run_steps(Stepper& st, int64_t n, std::string& err) {
  cudaStream_t s = lib_stream();
  if (!st.tuned && n >= tune_cost(st) + 1) {
    const int64_t spent = tune_cost(st);
    pslbm_status ts = autotune(st, err);
    if (ts != PSLBM_OK) return ts;
    n -= spent;
  }
  cudaError_t te = ensure_tiles(st, st.shape);
  if (te != cudaSuccess) {
    err = std::string("tile list: ") + cudaGetErrorString(te);
    return PSLBM_ERR_CUDA;
  }
  GraphCache& gc = st.graphs;
  const int64_t K = 32;
  while (n > 0) {
    const int64_t k = n >= K ? K : n;
    auto it = gc.exec.find(k);
    if (it == gc.exec.end()) {
      cudaGraph_t g;
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
        return PSLBM_ERR_CUDA;
      }
      enqueue_steps(s, st, st.shape, st.staged, k);
      e = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess) {
        err = std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
        return PSLBM_ERR_CUDA;
      }
      cudaGraphExec_t ex;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return PSLBM_ERR_CUDA;
      }
      it = gc.exec.emplace(k, ex).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second, s);
    if (e != cudaSuccess) {
      err = std::string("cudaGraphLaunch: ") + cudaGetErrorString(e);
      return PSLBM_ERR_CUDA;
    }
    n -= k;
  }
  return PSLBM_OK;
}

// Fix the tile shape (tx = ty = 0: leave it to timing).
pslbm_status set_shape(Stepper& st, int tx, int ty) {
  int idx = -2;
  if (tx == 0 && ty == 0) idx = -1;
  for (int sh = 0; sh < NSHAPES; ++sh)
    if (SHAPE_TX[sh] == tx && SHAPE_TY[sh] == ty) idx = sh;
  if (idx == -2) return PSLBM_ERR_PARAM;
  const int prev = st.fix_shape;
  st.fix_shape = idx;
  if (candidates(st).empty()) {
    // a fixed staging that this shape has no kernel for
    st.fix_shape = prev;
    return PSLBM_ERR_PARAM;
  }
  choose(st);
  return PSLBM_OK;
}

// Fix the staging (-1: leave it to timing, 0: plain loads, 1: TMA-staged,
// 2: TMA-staged with a single stage).
pslbm_status set_staging(Stepper& st, int mode) {
  if (mode < -1 || mode >= NSTAGING || (mode >= 1 && !st.staged_ok)) return PSLBM_ERR_PARAM;
  const int prev = st.fix_staged;
  st.fix_staged = mode;
  if (candidates(st).empty()) {
    // a fixed tile shape that has no kernel of this staging
    st.fix_staged = prev;
    return PSLBM_ERR_PARAM;
  }
  choose(st);
  return PSLBM_OK;
}

// TMA descriptors of an instance's population boxes (FP32 populations only):
// per tile shape and ping-pong buffer, a 3D map over (x, y, plane) whose box is
// the tile plus the staged kernel's ring (D2Q9) or the tile itself (D2Q5).
// Rows must be a multiple of 16 bytes; returns false when the instance does
// not qualify or the driver lacks the encoder.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)f;
  }
  return fn;
}

bool encode_maps(DevInst& I, const pslbm_params* p) {
  if (p->precision == PSLBM_FP64) return false;
  const size_t gs = gsize(p->precision);
  const uint64_t nx = (uint64_t)p->nx, ny = (uint64_t)p->ny, N = nx * ny;
  const int ns = p->n_species;
  if ((nx * 4) % 16 != 0 || (ns > 0 && (nx * gs) % 16 != 0)) return false;
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const CUtensorMapDataType gt = p->precision == PSLBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : p->precision == PSLBM_FP32_SOLUTE_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                         : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  for (int sh = 0; sh < NSHAPES; ++sh) {
    for (int b = 0; b < 2; ++b) {
      const cuuint64_t fdim[3] = {nx, ny, 18};
      const cuuint64_t fstr[2] = {nx * 4, N * 4};
      const cuuint32_t fbox[3] = {(cuuint32_t)(SHAPE_TX[sh] + 2 * stage_halo_x(SHAPE_NPT[sh])),
                                  (cuuint32_t)(SHAPE_TY[sh] + 2), 18};
      const cuuint32_t one[3] = {1, 1, 1};
      if (enc(&I.tmf[sh][b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, I.f[b], fdim, fstr, fbox, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
      if (ns > 0) {
        const cuuint64_t gdim[3] = {nx, ny, (cuuint64_t)(5 * ns)};
        const cuuint64_t gstr[2] = {nx * gs, N * gs};
        const cuuint32_t gbox[3] = {(cuuint32_t)SHAPE_TX[sh], (cuuint32_t)SHAPE_TY[sh], (cuuint32_t)(5 * ns)};
        if (enc(&I.tmg[sh][b], gt, 3, I.g[b], gdim, gstr, gbox, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
          return false;
      }
    }
  }
  return true;
}

pslbm_status device_status(pslbm_t h) {
  unsigned long long st = 0;
  CK(h, cudaMemcpyAsync(&st, h->h.scal + S_STATUS, sizeof st, cudaMemcpyDeviceToHost, lib_stream()));
  CK(h, cudaStreamSynchronize(lib_stream()));
  if (st & ST_NONFINITE) return fail(h, PSLBM_ERR_NONFINITE, "non-finite density on the device");
  if (st & ST_EOS) return fail(h, PSLBM_ERR_EOS_DOMAIN, "Eq. 13 square-root argument negative (rho_1 outside the EOS domain)");
  if (st & ST_TIMEOUT) return fail(h, PSLBM_ERR_TIMEOUT, "a bounded wait for staged populations gave up");
  return PSLBM_OK;
}

}  // namespace

extern "C" {

void* pslbm_get_stream(void) { return (void*)lib_stream(); }

pslbm_status pslbm_set_stream(void* s) {
  g_user_set = s != nullptr;
  g_user_stream = (cudaStream_t)s;
  return PSLBM_OK;
}

pslbm_status pslbm_create(const uint8_t* mask, const double* rho1, const double* rho2, const double* conc,
                          const double* vol, const pslbm_params* p, pslbm_t* out) {
  if (!out) return fail(nullptr, PSLBM_ERR_PARAM, "out is NULL");
  *out = nullptr;
  if (!mask || !rho1 || !rho2) return fail(nullptr, PSLBM_ERR_PARAM, "mask, rho1 and rho2 are required");
  std::string v = validate(p);
  if (!v.empty()) return fail(nullptr, PSLBM_ERR_PARAM, v);
  if (check_device() != PSLBM_OK) return fail(nullptr, PSLBM_ERR_NODEVICE, "no sm_103 CUDA device");
  const int ns = p->n_species;
  const Launchers* L = launchers(p->precision, ns);
  if (!L) return fail(nullptr, PSLBM_ERR_PARAM, "no kernels for this precision / species count");

  pslbm_t h = new (std::nothrow) pslbm_s();
  if (!h) return fail(nullptr, PSLBM_ERR_OOM, "host allocation failed");
  h->p = *p;
  h->prec = p->precision;
  h->ns = ns;
  h->L = L;
  const long long N = (long long)p->nx * p->ny;
  h->N = N;
  cudaStream_t s = lib_stream();
  DevInst& I = h->h;
  I.P = to_dev(p);
  I.N = N;
  I.evcap = (int)N;
  pslbm_status st = PSLBM_OK;
  {
    // one device allocation holds the instance's whole state, each part on a
    // 256-byte boundary (TMA wants 16-byte aligned bases); the initial
    // threshold's budget partial sums are the last part
    const size_t fb = (size_t)N * 18 * fsize(p->precision), gb = (size_t)N * 5 * ns * gsize(p->precision);
    const size_t sizes[] = {fb, fb, gb, gb, (size_t)N, (size_t)N, (size_t)N * 2 * sizeof(double), (size_t)N,
                            (size_t)N * sizeof(double), (size_t)N * 2 * sizeof(int), (size_t)N * sizeof(int),
                            (size_t)((N + 31) / 32) * sizeof(unsigned), S_NSCAL * sizeof(unsigned long long),
                            sizeof(DevInst), (size_t)(BUD_BLOCKS + 1) * NBUD * sizeof(double)};
    constexpr int NPARTS = sizeof(sizes) / sizeof(sizes[0]);
    size_t offs[NPARTS], total = 0;
    for (int i = 0; i < NPARTS; ++i) {
      offs[i] = total;
      total += ((sizes[i] ? sizes[i] : 16) + 255) / 256 * 256;
    }
    void* arena = nullptr;
    st = dalloc(h, &arena, total);
    if (st != PSLBM_OK) goto fail_cleanup;
    char* base = (char*)arena;
    I.f[0] = base + offs[0];
    I.f[1] = base + offs[1];
    I.g[0] = base + offs[2];
    I.g[1] = base + offs[3];
    I.type[0] = (uint8_t*)(base + offs[4]);
    I.type[1] = (uint8_t*)(base + offs[5]);
    I.V = (double*)(base + offs[6]);
    I.evt = (uint8_t*)(base + offs[7]);
    I.xs = (double*)(base + offs[8]);
    I.evlist = (int*)(base + offs[9]);
    I.claim = (int*)(base + offs[10]);
    I.vmask = (unsigned*)(base + offs[11]);
    I.scal = (unsigned long long*)(base + offs[12]);
    h->d = (DevInst*)(base + offs[13]);
    double* part = (double*)(base + offs[14]);
    double* res = part + (size_t)BUD_BLOCKS * NBUD;

    // the inputs are staged in the second population buffer (at least 72
    // bytes per node; they need 17 + 8 ns <= 49), which is cleared once the
    // initialisation kernel has read them
    double* dr1 = (double*)I.f[1];
    double* dr2 = dr1 + N;
    double* dc = (conc && ns) ? dr2 + N : nullptr;
    uint8_t* dmask = (uint8_t*)(dr2 + N + (dc ? (size_t)N * ns : 0));
    cudaError_t e = cudaMemcpyAsync(dmask, mask, N, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr1, rho1, N * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr2, rho2, N * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && dc) e = cudaMemcpyAsync(dc, conc, N * ns * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(I.evt, 0, (size_t)N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(I.claim, 0, (size_t)N * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(I.vmask, 0, (size_t)((N + 31) / 32) * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(I.scal, 0, S_NSCAL * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(I.scal + S_LIMIT, 0xff, sizeof(unsigned long long), s);
    if (e == cudaSuccess && ns) e = cudaMemsetAsync(I.g[1], 0, gb, s);
    if (e == cudaSuccess) {
      if (vol) {
        e = cudaMemcpyAsync(I.V, vol, (size_t)N * 2 * sizeof(double), cudaMemcpyHostToDevice, s);
      } else {
        k_vol_from_mask<<<(unsigned)std::min<long long>((N + 255) / 256, 65536), 256, 0, s>>>(dmask, I.V, N);
        e = cudaGetLastError();
      }
    }
    h->run.staged_ok = L->bulk_tma[0] != nullptr && encode_maps(I, p);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d, &I, sizeof(DevInst), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      L->init(s, h->d, dmask, dr1, dr2, dc, N);
      e = cudaGetLastError();
    }
    // initial liquid threshold: half the maximum initial rho_1 over fluid
    // nodes (the first budget entry), decoded on the device
    if (e == cudaSuccess) {
      L->budget(s, h->d, part, res);
      k_first_threshold<<<1, 1, 0, s>>>(res, I.scal);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(I.f[1], 0, fb, s);
    // the host copy of the descriptor is read by the copy above before the
    // call returns only for pageable memory; synchronise once for it and for
    // the errors of everything above
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = fail(nullptr, e == cudaErrorMemoryAllocation ? PSLBM_ERR_OOM : PSLBM_ERR_CUDA,
                std::string("create: ") + cudaGetErrorString(e));
      goto fail_cleanup;
    }
  }
  h->run.L = L;
  h->run.d = h->d;
  h->run.ninst = 1;
  h->run.dims.assign(1, {p->nx, p->ny});
  h->run.nchunks = ((N + 31) / 32 + VOP_CHUNK - 1) / VOP_CHUNK;
  h->run.single = &h->h.P;
  choose(h->run);
  {
    cudaError_t e = ensure_tiles(h->run, h->run.shape);
    if (e != cudaSuccess) {
      st = fail(nullptr, e == cudaErrorMemoryAllocation ? PSLBM_ERR_OOM : PSLBM_ERR_CUDA,
                std::string("tile list: ") + cudaGetErrorString(e));
      goto fail_cleanup;
    }
  }
  *out = h;
  return PSLBM_OK;
fail_cleanup : {
  std::string m = h->err;
  free_all(h);
  delete h;
  if (!m.empty()) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_lib_err = m;
  }
  return st;
}
}

pslbm_status pslbm_step(pslbm_t h, int64_t n) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (h->sticky) return h->sticky;
  if (n < 0) return fail(h, PSLBM_ERR_PARAM, "n < 0");
  if (h->in_batch) return fail(h, PSLBM_ERR_STATE, "handle is a member of a batch; step the batch");
  if (n == 0) return PSLBM_OK;
  std::string err;
  pslbm_status st = run_steps(h->run, n, err);
  if (st != PSLBM_OK) return fail(h, st, err);
  return PSLBM_OK;
}

pslbm_status pslbm_profile_step(pslbm_t h, int64_t n, double* kernel_ms, double* total_ms) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (h->sticky) return h->sticky;
  if (n < 1 || !kernel_ms) return fail(h, PSLBM_ERR_PARAM, "n < 1 or kernel_ms is NULL");
  if (h->in_batch) return fail(h, PSLBM_ERR_STATE, "handle is a member of a batch");
  std::string err;
  pslbm_status st = profile_steps(h->run, n, kernel_ms, total_ms, err);
  if (st != PSLBM_OK) return fail(h, st, err);
  return device_status(h);
}

pslbm_status pslbm_set_step_limit(pslbm_t h, int64_t limit) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (h->sticky) return h->sticky;
  const unsigned long long v = limit < 0 ? ~0ULL : (unsigned long long)limit;
  CK(h, cudaMemcpyAsync(h->h.scal + S_LIMIT, &v, sizeof v, cudaMemcpyHostToDevice, lib_stream()));
  CK(h, cudaStreamSynchronize(lib_stream()));
  return PSLBM_OK;
}

pslbm_status pslbm_estimate_device_bytes(const pslbm_params* p, uint64_t* bytes) {
  if (!bytes) return fail(nullptr, PSLBM_ERR_PARAM, "bytes is NULL");
  std::string v = validate(p);
  if (!v.empty()) return fail(nullptr, PSLBM_ERR_PARAM, v);
  const uint64_t N = (uint64_t)p->nx * (uint64_t)p->ny;
  const uint64_t per = 2 * 18 * fsize(p->precision) + 2 * 5 * (uint64_t)p->n_species * gsize(p->precision) +
                       2 /*types*/ + 16 /*V*/ + 1 /*events*/ + 8 /*excess*/ + 8 /*event lists*/ + 4 /*claims*/;
  const uint64_t vmask_bytes = ((N + 31) / 32) * 4;
  uint64_t tiles = 0;
  for (int sh = 0; sh < NSHAPES; ++sh)
    tiles += ((uint64_t)(p->nx + SHAPE_TX[sh] - 1) / SHAPE_TX[sh]) * ((uint64_t)(p->ny + SHAPE_TY[sh] - 1) / SHAPE_TY[sh]);
  *bytes = N * per + vmask_bytes + tiles * sizeof(Tile) + sizeof(DevInst) + S_NSCAL * 8 +
           (uint64_t)(BUD_BLOCKS + 1) * NBUD * sizeof(double) + 15 * 256;
  return PSLBM_OK;
}

pslbm_status pslbm_set_tile_shape(pslbm_t h, int32_t tile_x, int32_t tile_y) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (set_shape(h->run, tile_x, tile_y) != PSLBM_OK)
    return fail(h, PSLBM_ERR_PARAM,
                "unsupported tile shape (0x0, 16x16, 32x8, 16x32 or 32x16; the last two have no staged kernel)");
  return PSLBM_OK;
}

pslbm_status pslbm_get_tile_shape(pslbm_t h, int32_t* tile_x, int32_t* tile_y, int32_t* tuned) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (tile_x) *tile_x = SHAPE_TX[h->run.shape];
  if (tile_y) *tile_y = SHAPE_TY[h->run.shape];
  if (tuned) *tuned = h->run.tuned ? 1 : 0;
  return PSLBM_OK;
}

pslbm_status pslbm_set_staging(pslbm_t h, int32_t mode) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (set_staging(h->run, mode) != PSLBM_OK)
    return fail(h, PSLBM_ERR_PARAM, "staging must be -1, 0, 1 or 2 (1, 2 only where the handle has TMA descriptors)");
  return PSLBM_OK;
}

pslbm_status pslbm_get_staging(pslbm_t h, int32_t* staged, int32_t* available) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (staged) *staged = h->run.staged;
  if (available) *available = h->run.staged_ok ? 1 : 0;
  return PSLBM_OK;
}

pslbm_status pslbm_monitor(pslbm_t h, int64_t* steps, double* max_rho1, uint32_t* status) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (h->sticky) return h->sticky;
  unsigned long long sc[S_NSCAL];
  CK(h, cudaMemcpyAsync(sc, h->h.scal, sizeof sc, cudaMemcpyDeviceToHost, lib_stream()));
  CK(h, cudaStreamSynchronize(lib_stream()));
  const unsigned long long n = sc[S_STEP];
  if (steps) *steps = (int64_t)n;
  // the slot the last step filled (the initial maximum before the first step)
  if (max_rho1) *max_rho1 = ord_dec(sc[S_MAX0 + int(n & 1ULL)]);
  if (status) *status = (uint32_t)sc[S_STATUS];
  if (sc[S_STATUS] & ST_NONFINITE) return fail(h, PSLBM_ERR_NONFINITE, "non-finite density on the device");
  if (sc[S_STATUS] & ST_EOS)
    return fail(h, PSLBM_ERR_EOS_DOMAIN, "Eq. 13 square-root argument negative (rho_1 outside the EOS domain)");
  if (sc[S_STATUS] & ST_TIMEOUT) return fail(h, PSLBM_ERR_TIMEOUT, "a bounded wait for staged populations gave up");
  return PSLBM_OK;
}

pslbm_status pslbm_sync(pslbm_t h) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (h->sticky) return h->sticky;
  cudaError_t e = cudaStreamSynchronize(lib_stream());
  if (e != cudaSuccess) return fail(h, PSLBM_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
  return device_status(h);
}

pslbm_status pslbm_info(pslbm_t h, int64_t* steps, int32_t* nx, int32_t* ny, int32_t* n_species) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (steps) {
    unsigned long long t = 0;
    CK(h, cudaMemcpyAsync(&t, h->h.scal + S_STEP, sizeof t, cudaMemcpyDeviceToHost, lib_stream()));
    CK(h, cudaStreamSynchronize(lib_stream()));
    *steps = (int64_t)t;
  }
  if (nx) *nx = h->p.nx;
  if (ny) *ny = h->p.ny;
  if (n_species) *n_species = h->ns;
  return PSLBM_OK;
}

pslbm_status pslbm_device_bytes(pslbm_t h, uint64_t* bytes) {
  if (!h || !bytes) return fail(h, PSLBM_ERR_PARAM, "NULL argument");
  *bytes = h->bytes;
  return PSLBM_OK;
}

pslbm_status pslbm_read_fields(pslbm_t h, uint32_t fields, void* const* out) {
  if (!h) return fail(nullptr, PSLBM_ERR_PARAM, "handle is NULL");
  if (h->sticky) return h->sticky;
  if (fields & ~0xFFu) return fail(h, PSLBM_ERR_PARAM, "unknown field bits");
  if (fields && !out) return fail(h, PSLBM_ERR_PARAM, "out is NULL");
  const long long N = h->N;
  const int ns = h->ns;
  cudaStream_t s = lib_stream();
  // scratch: rho1, rho2, ux, uy (N each), conc (ns N), type (N bytes), budget partials
  const size_t need = (size_t)N * (4 + ns) * sizeof(double) + (size_t)N + (BUD_BLOCKS + 1) * NBUD * sizeof(double) + 64;
  if (h->rb_bytes < need) {
    if (h->rb) {
      cudaFree(h->rb);
      h->bytes -= h->rb_bytes;
    }
    h->rb = nullptr;
    h->rb_bytes = 0;
    cudaError_t e = cudaMalloc(&h->rb, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, PSLBM_ERR_OOM, "read-back scratch allocation failed");
    }
    h->rb_bytes = need;
    h->bytes += need;
  }
  double* r1 = h->rb;
  double* r2 = r1 + N;
  double* ux = r2 + N;
  double* uy = ux + N;
  double* cc = uy + N;
  double* part = cc + (size_t)N * ns;
  double* bud = part + BUD_BLOCKS * NBUD;
  uint8_t* ty = (uint8_t*)(bud + NBUD);
  h->L->fields(s, h->d, N, r1, r2, ux, uy, ns ? cc : nullptr, ty);
  CK(h, cudaGetLastError());
  if (fields & PSLBM_F_BUDGET) {
    h->L->budget(s, h->d, part, bud);
    CK(h, cudaGetLastError());
  }
  int i = 0;
  auto cp = [&](void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, s);
  };
  if (fields & PSLBM_F_RHO1) CK(h, cp(out[i++], r1, N * 8));
  if (fields & PSLBM_F_RHO2) CK(h, cp(out[i++], r2, N * 8));
  if (fields & PSLBM_F_UX) CK(h, cp(out[i++], ux, N * 8));
  if (fields & PSLBM_F_UY) CK(h, cp(out[i++], uy, N * 8));
  if (fields & PSLBM_F_CONC) {
    if (ns) CK(h, cp(out[i], cc, (size_t)N * ns * 8));
    ++i;
  }
  if (fields & PSLBM_F_TYPE) CK(h, cp(out[i++], ty, N));
  if (fields & PSLBM_F_VOL) CK(h, cp(out[i++], h->h.V, (size_t)N * 2 * 8));
  double budget_host[NBUD];
  unsigned long long stepc = 0;
  if (fields & PSLBM_F_BUDGET) {
    CK(h, cp(budget_host, bud, sizeof budget_host));
    CK(h, cp(&stepc, h->h.scal + S_STEP, sizeof stepc));
  }
  CK(h, cudaStreamSynchronize(s));
  if (fields & PSLBM_F_BUDGET) {
    double* o = (double*)out[i++];
    o[0] = budget_host[0] > -INFINITY ? budget_host[0] : 0.0;
    o[1] = budget_host[1];
    o[2] = budget_host[2];
    for (int k = 0; k < ns; ++k) o[3 + k] = budget_host[3 + k];
    o[3 + ns] = budget_host[3 + MAXS];
    o[4 + ns] = budget_host[4 + MAXS];
    o[5 + ns] = (double)stepc;
  }
  return device_status(h);
}

pslbm_status pslbm_destroy(pslbm_t h) {
  if (!h) return PSLBM_OK;
  cudaStreamSynchronize(lib_stream());
  if (h->rb) cudaFree(h->rb);
  free_all(h);
  delete h;
  return PSLBM_OK;
}

const char* pslbm_last_error(pslbm_t h) {
  if (h) return h->err.c_str();
  return g_lib_err.c_str();
}

// ------------------------------------------------------------------ batches

pslbm_status pslbm_batch_create(int32_t n, const pslbm_t* members, int32_t tile_x, int32_t tile_y,
                                pslbm_batch_t* out) {
  if (!out) return fail(nullptr, PSLBM_ERR_PARAM, "out is NULL");
  *out = nullptr;
  if (n < 1 || !members) return fail(nullptr, PSLBM_ERR_PARAM, "empty batch");
  for (int i = 0; i < n; ++i) {
    if (!members[i] || members[i]->sticky) return fail(nullptr, PSLBM_ERR_PARAM, "invalid member");
    if (members[i]->in_batch) return fail(nullptr, PSLBM_ERR_STATE, "member already in a batch");
    if (members[i]->prec != members[0]->prec || members[i]->ns != members[0]->ns)
      return fail(nullptr, PSLBM_ERR_PARAM, "members differ in precision or species count");
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return fail(nullptr, PSLBM_ERR_PARAM, "duplicate member");
  }
  pslbm_batch_t b = new (std::nothrow) pslbm_batch_s();
  if (!b) return fail(nullptr, PSLBM_ERR_OOM, "host allocation failed");
  b->run.staged_ok = true;
  for (int i = 0; i < n; ++i) b->run.staged_ok = b->run.staged_ok && members[i]->run.staged_ok;
  b->L = members[0]->L;
  b->run.L = b->L;
  if (set_shape(b->run, tile_x, tile_y) != PSLBM_OK) {
    delete b;
    return fail(nullptr, PSLBM_ERR_PARAM, "unsupported tile shape (0x0, 16x16, 32x8, 16x32 or 32x16)");
  }
  std::vector<DevInst> di;
  for (int i = 0; i < n; ++i) {
    b->members.push_back(members[i]);
    di.push_back(members[i]->h);
    b->run.dims.push_back({members[i]->p.nx, members[i]->p.ny});
  }
  // VOP chunks of all members, in member order
  std::vector<int2> cmap;
  for (int i = 0; i < n; ++i) {
    const long long nc = ((members[i]->N + 31) / 32 + VOP_CHUNK - 1) / VOP_CHUNK;
    for (long long c = 0; c < nc; ++c) cmap.push_back(make_int2(i, (int)c));
  }
  b->run.nchunks = (long long)cmap.size();
  cudaStream_t s = lib_stream();
  cudaError_t e = cudaMalloc(&b->d, di.size() * sizeof(DevInst));
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d, di.data(), di.size() * sizeof(DevInst), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMalloc(&b->run.chunk_map, cmap.size() * sizeof(int2));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->run.chunk_map, cmap.data(), cmap.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  b->L = members[0]->L;
  b->run.L = b->L;
  b->run.d = b->d;
  b->run.ninst = n;
  if (e == cudaSuccess) e = ensure_tiles(b->run, b->run.shape);
  if (e != cudaSuccess) {
    b->run.release();
    if (b->d) cudaFree(b->d);
    delete b;
    return fail(nullptr, e == cudaErrorMemoryAllocation ? PSLBM_ERR_OOM : PSLBM_ERR_CUDA,
                std::string("batch create: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < n; ++i) members[i]->in_batch = 1;
  *out = b;
  return PSLBM_OK;
}

pslbm_status pslbm_batch_step(pslbm_batch_t b, int64_t n) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (b->sticky) return b->sticky;
  if (n < 0) return fail(nullptr, PSLBM_ERR_PARAM, "n < 0");
  if (n == 0) return PSLBM_OK;
  std::string err;
  pslbm_status st = run_steps(b->run, n, err);
  if (st != PSLBM_OK) {
    b->sticky = st;
    b->err = err;
    return fail(nullptr, st, err);
  }
  return PSLBM_OK;
}

pslbm_status pslbm_batch_get_tile_shape(pslbm_batch_t b, int32_t* tile_x, int32_t* tile_y, int32_t* tuned) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (tile_x) *tile_x = SHAPE_TX[b->run.shape];
  if (tile_y) *tile_y = SHAPE_TY[b->run.shape];
  if (tuned) *tuned = b->run.tuned ? 1 : 0;
  return PSLBM_OK;
}

pslbm_status pslbm_batch_set_staging(pslbm_batch_t b, int32_t mode) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (set_staging(b->run, mode) != PSLBM_OK)
    return fail(nullptr, PSLBM_ERR_PARAM, "staging must be -1, 0, 1 or 2 (1, 2 only where every member has TMA descriptors)");
  return PSLBM_OK;
}

pslbm_status pslbm_batch_get_staging(pslbm_batch_t b, int32_t* staged, int32_t* available) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (staged) *staged = b->run.staged;
  if (available) *available = b->run.staged_ok ? 1 : 0;
  return PSLBM_OK;
}

pslbm_status pslbm_batch_sync(pslbm_batch_t b) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (b->sticky) return b->sticky;
  cudaError_t e = cudaStreamSynchronize(lib_stream());
  if (e != cudaSuccess) return fail(nullptr, PSLBM_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
  for (pslbm_t m : b->members) {
    pslbm_status st = device_status(m);
    if (st != PSLBM_OK) return st;
  }
  return PSLBM_OK;
}

pslbm_status pslbm_batch_profile_step(pslbm_batch_t b, int64_t n, double* kernel_ms, double* total_ms) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (b->sticky) return b->sticky;
  if (n < 1 || !kernel_ms) return fail(nullptr, PSLBM_ERR_PARAM, "n < 1 or kernel_ms is NULL");
  std::string err;
  pslbm_status st = profile_steps(b->run, n, kernel_ms, total_ms, err);
  if (st != PSLBM_OK) {
    b->sticky = st;
    b->err = err;
    return fail(nullptr, st, err);
  }
  return PSLBM_OK;
}

pslbm_status pslbm_batch_monitor(pslbm_batch_t b, int64_t* min_steps, uint32_t* status) {
  if (!b) return fail(nullptr, PSLBM_ERR_PARAM, "batch is NULL");
  if (b->sticky) return b->sticky;
  const int n = (int)b->members.size();
  cudaStream_t s = lib_stream();
  if (!b->mon) {
    cudaError_t e = cudaMalloc(&b->mon, (size_t)n * 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->mon = nullptr;
      return fail(nullptr, PSLBM_ERR_OOM, "batch monitor buffer");
    }
    b->mon_h.assign((size_t)n * 2, 0ULL);
  }
  k_batch_monitor<<<(n + 255) / 256, 256, 0, s>>>(b->d, n, b->mon);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->mon_h.data(), b->mon, (size_t)n * 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(nullptr, PSLBM_ERR_CUDA, std::string("batch monitor: ") + cudaGetErrorString(e));
  unsigned long long lo = ~0ULL, bits = 0;
  for (int i = 0; i < n; ++i) {
    lo = std::min(lo, b->mon_h[2 * i]);
    bits |= b->mon_h[2 * i + 1];
  }
  if (min_steps) *min_steps = (int64_t)lo;
  if (status) *status = (uint32_t)bits;
  return PSLBM_OK;
}

pslbm_status pslbm_batch_destroy(pslbm_batch_t b) {
  if (!b) return PSLBM_OK;
  cudaStreamSynchronize(lib_stream());
  b->run.release();
  if (b->d) cudaFree(b->d);
  if (b->mon) cudaFree(b->mon);
  for (pslbm_t m : b->members) m->in_batch = 0;
  delete b;
  return PSLBM_OK;
}

}  // extern "C"

namespace pslbm {

const Launchers* launchers_f64(int ns);
const Launchers* launchers_f32(int ns);
const Launchers* launchers_f32h(int ns);
const Launchers* launchers_f32b(int ns);
const Launchers* launchers_f64_n2(int ns);
const Launchers* launchers_f32_n2(int ns);
const Launchers* launchers_f32h_n2(int ns);
const Launchers* launchers_f32b_n2(int ns);

// The two halves of a precision's table (one and two nodes per thread) merged:
// every slot takes the entry that is set.
static Launchers merge_launchers(const Launchers& a, const Launchers& b) {
  Launchers m = a;
  for (int s = 0; s < NSHAPES; ++s) {
    if (!m.bulk[s]) m.bulk[s] = b.bulk[s];
    if (!m.bulk_tma[s]) m.bulk_tma[s] = b.bulk_tma[s];
    if (!m.bulk_tma1[s]) m.bulk_tma1[s] = b.bulk_tma1[s];
  }
  return m;
}
struct MergedLauncherTables {
  Launchers t[4][MAXS + 1];
  MergedLauncherTables() {
    const Launchers* (*one[4])(int) = {launchers_f64, launchers_f32, launchers_f32h, launchers_f32b};
    const Launchers* (*two[4])(int) = {launchers_f64_n2, launchers_f32_n2, launchers_f32h_n2, launchers_f32b_n2};
    for (int p = 0; p < 4; ++p)
      for (int ns = 0; ns <= MAXS; ++ns) t[p][ns] = merge_launchers(*one[p](ns), *two[p](ns));
  }
};

const Launchers* launchers(int prec, int ns) {
  static const MergedLauncherTables tables;
  if (ns < 0 || ns > MAXS) return nullptr;
  switch (prec) {
    case PSLBM_FP64: return &tables.t[0][ns];
    case PSLBM_FP32: return &tables.t[1][ns];
    case PSLBM_FP32_SOLUTE_F16: return &tables.t[2][ns];
    case PSLBM_FP32_SOLUTE_BF16: return &tables.t[3][ns];
  }
  return nullptr;
}

}  // namespace pslbm

// Accessors used by the allocation-free budget entry point (noalloc.cu).
namespace pslbm {
const DevInst* handle_device_inst(pslbm_t h) { return h->d; }
long long handle_nodes(pslbm_t h) { return h->N; }
int handle_precision(pslbm_t h) { return h->prec; }
int handle_species(pslbm_t h) { return h->ns; }
pslbm_status handle_sticky(pslbm_t h) { return h->sticky; }
pslbm_status handle_fail(pslbm_t h, pslbm_status s, const std::string& msg) { return fail(h, s, msg); }
cudaStream_t library_stream() { return lib_stream(); }
}  // namespace pslbm
