// Device-side data structures and per-node helpers of the reactive two-phase
// LBM (Chen, Kang et al., arXiv 1410.3464, Sections 3-4).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace pslbm {

constexpr int MAXS = 4;
constexpr uint8_t T_LIQUID = 0, T_GAS = 1, T_SOLID_D = 2, T_SOLID_F = 3, T_WALL = 4, T_INLET = 5,
                  T_OUTLET = 6;
constexpr uint8_t T_MASK = 0x0F;     // low nibble: node type
constexpr uint8_t T_NEW = 0x40;      // flag set by the amendment kernel: solid -> liquid this step
constexpr uint8_t T_VANISH = 0x80;   // flag: liquid -> solid this step

// Tile shapes of the step kernels: 256 threads, a tile of TX x TY nodes and a
// one-node ring.  Thread (tx, ty) of a TX x RY block computes the NPT nodes
// (tx, ty + k RY) of the tile, k < NPT (nodes per thread).  The runtime picks
// the fastest shape per handle or batch by timing its first steps (results do
// not depend on the shape).
constexpr int NTHREADS = 256;
// Interface-bitmap words per warp chunk of the VOP kernel.
constexpr int VOP_CHUNK = 4;
template <int TX_, int RY_, int NPT_ = 1>
struct TileShape {
  static constexpr int TX = TX_, RY = RY_, NPT = NPT_, TY = RY_ * NPT_;
  static constexpr int EXT_X = TX + 2, EXT_Y = TY + 2;
  static constexpr int EXT = EXT_X * EXT_Y;
  static constexpr int RING = EXT - TX * TY;
  static_assert(TX * RY == NTHREADS, "one thread per column position and row of a pass");
  static_assert(RING <= NTHREADS, "one ring node per thread");
};
using ShapeA = TileShape<16, 16>;      // 16 x 16, one node per thread
using ShapeB = TileShape<32, 8>;       // 32 x 8, one node per thread
using ShapeC = TileShape<16, 16, 2>;   // 16 x 32, two nodes per thread
using ShapeD = TileShape<32, 8, 2>;    // 32 x 16, two nodes per thread
constexpr int NSHAPES = 4;
constexpr int SHAPE_TX[NSHAPES] = {ShapeA::TX, ShapeB::TX, ShapeC::TX, ShapeD::TX};
constexpr int SHAPE_TY[NSHAPES] = {ShapeA::TY, ShapeB::TY, ShapeC::TY, ShapeD::TY};
constexpr int SHAPE_NPT[NSHAPES] = {ShapeA::NPT, ShapeB::NPT, ShapeC::NPT, ShapeD::NPT};
// The staged bulk kernel's D2Q9 box reaches this many nodes left and right of
// a tile of one node per thread (one ring node is needed; four keep the box's
// x origin on a 16-byte boundary for FP32 rows), and one node above and below.
// The box of a tile of two nodes per thread has no x halo (the tile's own x
// origin is aligned; its side ring columns are read from global memory), so
// that two blocks with two stages each fit on an SM.
constexpr int STAGE_HALO_X = 4;
__host__ __device__ constexpr int stage_halo_x(int npt) { return npt == 1 ? STAGE_HALO_X : 0; }

// Per-instance scalar slots (unsigned long long each).
enum {
  S_STEP = 0,      // steps taken
  S_MAX0 = 1,      // ordered-encoded max rho_1, slot for even steps
  S_MAX1 = 2,      // slot for odd steps
  S_STATUS = 3,    // error bits
  S_NEVENT = 4,    // events recorded by the VOP kernel this step
  S_LIMIT = 5,     // step limit: an instance at or past it is frozen (kernels skip it)
  S_THETA = 6,     // this step's liquid threshold (half the previous maximum), FP64 bits
  S_THETAF = 7,    // the same rounded to FP32 (bits in the low word)
  S_TILES = 8,     // tiles claimed so far by the bulk launch in progress (first instance of a
                   // launch only; the amendment kernel sets it back to zero after every launch)
  S_NSCAL = 9
};
enum { ST_NONFINITE = 1, ST_EOS = 2, ST_EVOVERFLOW = 4, ST_TIMEOUT = 8 };

// Budget reduction: [max rho1, sum rho1, sum rho2, sum C_k (MAXS), sum V_D, sum V_F].
constexpr int NBUD = 5 + MAXS;
constexpr int BUD_BLOCKS = 512;
constexpr int BUD_THREADS = 256;

// Event codes written by the VOP kernel.
enum { EV_NONE = 0, EV_DISSOLVE = 1, EV_OVERFLOW = 2 };   // overflow: code | (dir << 4)

// Parameters used in arithmetic, stored in the compute precision so that no
// kernel converts FP64 values at run time (FP64 runs at a small fraction of the
// FP32 rate on GB300).  Reciprocals replace divisions where a parameter divides.
template <class R>
struct DevParamsR {
  R tau[2], inv_tau[2], G11, G12, G21, a0, inv_rho10, inv_rho20, w_adh[2];
  R eos_a, eos_b4, eos_RT, six_over_G11;
  R gx, gy, shift_f[2], shift_fg[2], rho_fill[2];
  R J0[MAXS], Ja[MAXS], inv_tau_g[MAXS], shift_c[MAXS], conc_in[MAXS], cR1[MAXS], cR3[MAXS];
  R k1, k1_inv_Keq, k3, k2, k4, C_F_sat, gas_yield, inv_M_C, c_total_per_rho1;
  R k1_s, k1_inv_Keq_s;   // R1 constants at liquid nodes touching D(s) (surface factor applied)
  // reactive link rule (Eqs. 29-31 as a halfway wall): link flux q = out * qa - qc,
  // returning population out - q, out = stored + sh (the stored shift J_a C_0 undone)
  R vB_qa, vB_sh, vF_qa, vF_qc, vF_sh;
  // 16-bit solute storage: stored value = shifted population * gs_mul[k];
  // loaded value * gs_div[k] (powers of two, so both are exact)
  R gs_mul[MAXS], gs_div[MAXS];
};

struct DevParams {
  int nx, ny, px, py, ns;
  int iA, iB, iE, iF;
  int per_liq, per_gas, ramp;
  int has_G11, has_rev, useB, useF;   // G11 != 0, inv_Keq != 0, R2 active, R4 active
  int r1_surf;                        // R1 surface factor differs from 1
  int in_dx, in_dy, out_dx, out_dy;   // node downstream of an inlet / upstream of an outlet
  double tau[2], G11, G12, G21, a0, rho10, rho20, w_adh[2];
  double eos_a, eos_b, eos_R, eos_T;
  double gx, gy;
  double shift_f[2];       // population shift of liquid nodes, rho_ref (0 in FP64 storage)
  double shift_fg[2];      // population shift of gas nodes, rho_ref_gas (0 in FP64 storage)
  double rho_fill[2];      // density of a refilled node without fluid neighbours
  double J0[MAXS], tau_g[MAXS], shift_c[MAXS];
  double inv_tau[2], Ja[MAXS], inv_tau_g[MAXS];  // 1/tau, (1 - J0)/4, 1/tau_g
  double cR1[MAXS], cR3[MAXS];                     // S_k = cR1[k] R1 + cR3[k] R3 (Eq. 28)
  double k1, inv_Keq, k3, k2, k4, C_F_sat, gas_yield, inv_M_C, c_total_per_rho1;
  double r1_surface_factor;
  double Vbar_D, Vbar_F, V_split;
  unsigned long long seed;
  double rho_in_liq[2], rho_in_gas[2], rho_out[2], rho_out_gas[2];
  double conc_in[MAXS];
  double gs_scale[MAXS];   // 16-bit solute storage scale per species (a power of two; 1 otherwise)
  DevParamsR<float> rf;
  DevParamsR<double> rd;
};

template <class R> __host__ __device__ __forceinline__ const DevParamsR<R>& rp(const DevParams& P);
template <> __host__ __device__ __forceinline__ const DevParamsR<float>& rp<float>(const DevParams& P) { return P.rf; }
template <> __host__ __device__ __forceinline__ const DevParamsR<double>& rp<double>(const DevParams& P) { return P.rd; }

struct DevInst {
  // TMA descriptors of the population boxes of the staged bulk kernel, per tile
  // shape and ping-pong buffer (encoded only when the instance qualifies:
  // FP32 populations and rows a multiple of 16 bytes; zero otherwise)
  CUtensorMap tmf[NSHAPES][2];
  CUtensorMap tmg[NSHAPES][2];
  DevParams P;
  void* f[2];                 // [2][9][N] populations, ping-pong
  void* g[2];                 // [ns][5][N] solute populations, ping-pong
  uint8_t* type[2];           // [N] node types, ping-pong
  double* V;                  // [2][N] V_D, V_F
  uint8_t* evt;               // [N] VOP events (zero except during a step)
  double* xs;                 // [N] overflow excess of an event node
  int* evlist;                // [evcap] event node indices
  int* claim;                 // [N] zero except while the amendment kernel runs
  unsigned* vmask;            // [(N + 31) / 32] bit per node: a mineral a liquid node touched this
                              // step (set by the bulk kernel, consumed and cleared by k_vop)
  unsigned long long* scal;   // [S_NSCAL]
  long long N;
  int evcap;
};

struct Tile {
  int inst, x0, y0, pad;
};

// D2Q9 velocity set of Eq. 7 (the D2Q5 set is directions 0-4).
__host__ __device__ constexpr int ex_(int a) {
  return (a == 1 || a == 5 || a == 8) ? 1 : (a == 3 || a == 6 || a == 7) ? -1 : 0;
}
__host__ __device__ constexpr int ey_(int a) {
  return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp_(int a) {
  return a == 0 ? 0 : a == 1 ? 3 : a == 2 ? 4 : a == 3 ? 1 : a == 4 ? 2 : a == 5 ? 7 : a == 6 ? 8 : a == 7 ? 5 : 6;
}
#define EX(a) ex_(a)
#define EY(a) ey_(a)
#define OPP(a) opp_(a)

template <class R> __device__ __forceinline__ R w9(int a) {
  return a == 0 ? R(4.0 / 9.0) : (a < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}
// interaction weights w(|e|^2): 1/9 axis, 1/36 diagonal (sum w e_x^2 = c_s^2)
template <class R> __device__ __forceinline__ R wf(int a) {
  return a == 0 ? R(0) : (a < 5 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}

__device__ __forceinline__ bool is_fluid(uint8_t t) { return t <= T_GAS; }
__device__ __forceinline__ bool is_res(uint8_t t) { return t == T_INLET || t == T_OUTLET; }
__device__ __forceinline__ bool is_live(uint8_t t) { return t <= T_GAS || t == T_INLET || t == T_OUTLET; }
__device__ __forceinline__ bool is_mineral(uint8_t t) { return t == T_SOLID_D || t == T_SOLID_F; }

// Storage conversion.
template <class T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class R, class T> __device__ __forceinline__ R ld(const T* p) { return R(to_f<T>(__ldg(p))); }
template <> __device__ __forceinline__ double ld<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<float, float>(const float* p) { return __ldg(p); }
template <class T, class R> __device__ __forceinline__ void st(T* p, R v);
template <> __device__ __forceinline__ void st<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void st<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }
template <> __device__ __forceinline__ void st<__nv_bfloat16, float>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}
// Solute populations in 16-bit storage carry a per-species power-of-two
// scale (pslbm_params.conc_scale); FP32 and FP64 storage carry none.
template <class T> struct Is16 { static constexpr bool value = false; };
template <> struct Is16<__half> { static constexpr bool value = true; };
template <> struct Is16<__nv_bfloat16> { static constexpr bool value = true; };

// plain (coherent) loads for data written earlier in the same kernel sequence
template <class R, class T> __device__ __forceinline__ R ldc(const T* p) { return R(to_f<T>(*p)); }
template <> __device__ __forceinline__ double ldc<double, double>(const double* p) { return *p; }
template <> __device__ __forceinline__ float ldc<float, float>(const float* p) { return *p; }

// Solute population of species k as the compute precision sees it: the
// stored value times the species' storage scale (16-bit storage only).
// gld: read-only path (__ldg); gldc: coherent load; gst: store.
template <class R, class TG>
__device__ __forceinline__ R gld(const DevParams& P, int k, const TG* p) {
  if constexpr (Is16<TG>::value) return ld<R>(p) * rp<R>(P).gs_div[k];
  else return ld<R>(p);
}
template <class R, class TG>
__device__ __forceinline__ R gldc(const DevParams& P, int k, const TG* p) {
  if constexpr (Is16<TG>::value) return ldc<R>(p) * rp<R>(P).gs_div[k];
  else return ldc<R>(p);
}
template <class TG, class R>
__device__ __forceinline__ void gst(const DevParams& P, int k, TG* p, R v) {
  if constexpr (Is16<TG>::value) st<TG, R>(p, v * rp<R>(P).gs_mul[k]);
  else st<TG, R>(p, v);
}

// Neighbour coordinate with periodic wrap; false outside a non-periodic edge.
__device__ __forceinline__ bool nbr(const DevParams& P, int x, int y, int dx, int dy, int& xn, int& yn) {
  xn = x + dx;
  yn = y + dy;
  if (xn < 0 || xn >= P.nx) {
    if (!P.px) return false;
    xn %= P.nx;
    if (xn < 0) xn += P.nx;
  }
  if (yn < 0 || yn >= P.ny) {
    if (!P.py) return false;
    yn %= P.ny;
    if (yn < 0) yn += P.ny;
  }
  return true;
}

// Order-preserving map of doubles to unsigned 64-bit (for atomicMax).
__device__ __forceinline__ unsigned long long ord_enc(double v) {
  unsigned long long b = __double_as_longlong(v);
  return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__host__ __device__ inline double ord_dec(unsigned long long e) {
  unsigned long long b = (e & 0x8000000000000000ULL) ? (e & 0x7FFFFFFFFFFFFFFFULL) : ~e;
  union { unsigned long long u; double d; } c;
  c.u = b;
  return c.d;
}

// The liquid threshold of the current step in the compute precision, decoded
// once per step by the amendment kernel (no FP64 arithmetic in the FP32 bulk).
template <class R> __device__ __forceinline__ R theta_of(const DevInst* Ip);
template <> __device__ __forceinline__ double theta_of<double>(const DevInst* Ip) {
  return __longlong_as_double((long long)Ip->scal[S_THETA]);
}
template <> __device__ __forceinline__ float theta_of<float>(const DevInst* Ip) {
  return __int_as_float((int)(unsigned)Ip->scal[S_THETAF]);
}

// Eq. 9a with the population shift: delta rho summed in direction order.
template <class R, class TF>
__device__ __forceinline__ R density_shifted(const TF* f, long long N, long long node) {
  R s = ld<R>(f + node);
#pragma unroll
  for (int a = 1; a < 9; ++a) s += ld<R>(f + a * N + node);
  return s;
}

// Same sum through plain (coherent) loads, for data written by an earlier kernel
// of the same step.
template <class R, class TF>
__device__ __forceinline__ R density_c(const TF* f, long long N, long long node) {
  R s = ldc<R>(f + node);
#pragma unroll
  for (int a = 1; a < 9; ++a) s += ldc<R>(f + a * N + node);
  return s;
}

// Reservoir densities at step t.  The inlet alternates liquid slugs of
// per_liq steps and gas slugs of per_gas steps; the last `ramp` steps of each
// slug blend linearly into the next state.  The outlet holds the liquid or the
// gas state according to the marking of the node upstream of it (x - 1, or
// y - 1 for outlets along y).
__device__ __forceinline__ void reservoir_rho(const DevParams& P, uint8_t t, unsigned long long step, bool up_liquid,
                                              double& r1, double& r2) {
  if (t == T_INLET) {
    double wg = 0.0;   // weight of the gas state
    if (P.per_gas > 0) {
      const long long per = P.per_liq + P.per_gas;
      const long long ph = (long long)(step % (unsigned long long)per);
      const long long R = P.ramp;
      if (ph < P.per_liq) {
        wg = (R > 0 && ph >= P.per_liq - R) ? double(ph - (P.per_liq - R) + 1) / double(R + 1) : 0.0;
      } else {
        wg = (R > 0 && ph >= per - R) ? 1.0 - double(ph - (per - R) + 1) / double(R + 1) : 1.0;
      }
    }
    r1 = (1.0 - wg) * P.rho_in_liq[0] + wg * P.rho_in_gas[0];
    r2 = (1.0 - wg) * P.rho_in_liq[1] + wg * P.rho_in_gas[1];
  } else {
    // outlet: the coexistence state of the phase arriving from upstream
    r1 = up_liquid ? P.rho_out[0] : P.rho_out_gas[0];
    r2 = up_liquid ? P.rho_out[1] : P.rho_out_gas[1];
  }
}

// Population shift of a node of type t: the reference density of its phase
// (gas-marked nodes: the gas reference; every other type: the liquid one).
template <class R>
__device__ __forceinline__ R fshift(const DevParams& P, int comp, uint8_t t) {
  return (t & T_MASK) == T_GAS ? rp<R>(P).shift_fg[comp] : rp<R>(P).shift_f[comp];
}

// Marking of an arbitrary node from global memory (same arithmetic as the
// shared-memory path, so both give the same answer bit for bit).
template <class R, class TF>
__device__ __forceinline__ bool liquid_at(const DevParams& P, const uint8_t* tin, const TF* fin, int N, int node,
                                          R theta) {
  uint8_t t = tin[node] & T_MASK;
  if (!is_fluid(t)) return false;
  R rho1 = fshift<R>(P, 0, t) + density_shifted<R>(fin, (long long)N, node);
  return rho1 > theta;
}

// Marking of the node upstream of an outlet node at index idx.
template <class R, class TF>
__device__ __forceinline__ bool outlet_up_liquid(const DevParams& P, const uint8_t* tin, const TF* fin, int N, int idx,
                                                 R theta) {
  int xn, yn;
  if (!nbr(P, idx % P.nx, idx / P.nx, P.out_dx, P.out_dy, xn, yn)) return false;
  return liquid_at<R, TF>(P, tin, fin, N, yn * P.nx + xn, theta);
}

// Explicitly rounded operations.  The hot formulas are written with these
// (fused where a product feeds a sum) so that the compiler cannot contract
// them differently in different kernel variants: every variant -- plain
// loads, TMA stages, parameters from global memory or from the constant bank
// -- evaluates exactly the same operations and gives bit-identical results.
template <class R> __device__ __forceinline__ R radd(R a, R b);
template <class R> __device__ __forceinline__ R rsub(R a, R b);
template <class R> __device__ __forceinline__ R rmul(R a, R b);
template <class R> __device__ __forceinline__ R rdiv(R a, R b);
template <class R> __device__ __forceinline__ R rfma(R a, R b, R c);
template <> __device__ __forceinline__ float radd<float>(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ float rsub<float>(float a, float b) { return __fsub_rn(a, b); }
template <> __device__ __forceinline__ float rmul<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ float rdiv<float>(float a, float b) { return __fdiv_rn(a, b); }
template <> __device__ __forceinline__ float rfma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double radd<double>(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ double rsub<double>(double a, double b) { return __dsub_rn(a, b); }
template <> __device__ __forceinline__ double rmul<double>(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ double rdiv<double>(double a, double b) { return __ddiv_rn(a, b); }
template <> __device__ __forceinline__ double rfma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// Eq. 12 (C-S EOS) and the Eq. 13 square-root argument 6/G11 (p - rho/3).
template <class R> __device__ __forceinline__ R psi_arg(const DevParams& P, R rho) {
  // Eq. 12 with 1 + eta + eta^2 - eta^3 = 1 + eta (1 + eta (1 - eta))
  const DevParamsR<R>& Q = rp<R>(P);
  const R eta = rmul<R>(Q.eos_b4, rho);
  const R om = rsub<R>(R(1), eta);
  const R poly = rfma<R>(eta, rfma<R>(eta, om, R(1)), R(1));
  const R num = rmul<R>(rmul<R>(rho, Q.eos_RT), poly);
  const R p = rfma<R>(-rmul<R>(Q.eos_a, rho), rho, rdiv<R>(num, rmul<R>(rmul<R>(om, om), om)));
  return rmul<R>(Q.six_over_G11, rsub<R>(p, rmul<R>(rho, R(1.0 / 3.0))));
}

template <class R> __device__ __forceinline__ R rrcp(R v);
template <> __device__ __forceinline__ double rrcp<double>(double v) { return 1.0 / v; }
template <> __device__ __forceinline__ float rrcp<float>(float v) { return __frcp_rn(v); }
template <class R> __device__ __forceinline__ R rmax(R a, R b);
template <> __device__ __forceinline__ double rmax<double>(double a, double b) { return fmax(a, b); }
template <> __device__ __forceinline__ float rmax<float>(float a, float b) { return fmaxf(a, b); }
template <class R> __device__ __forceinline__ R rexp(R v);
template <> __device__ __forceinline__ double rexp<double>(double v) { return exp(v); }
template <> __device__ __forceinline__ float rexp<float>(float v) { return expf(v); }

// The interaction stencils of Eqs. 11, 14 and 16 at one node, from the values
// of psi_1, phi_1, phi_2 at the node (index 0) and its eight neighbours (1-8,
// Eq. 7 order) and the neighbours' liveness (fluid or reservoir):
//   S = sum_a w(|e_a|^2) v(x + e_a) e_a  (w = 1/9 axis, 1/36 diagonal)
// for each field, and the wall-density sums sum_a w s(x + e_a) e_a with s = 1
// at non-live neighbours.  A non-live (solid or wall) neighbour takes the value
// of its mirror image across the wall: the node itself for an axis link, and
// for a diagonal link the live one of the two axis neighbours beside it when
// exactly one is live (a flat wall), else the node itself (a corner).  Since
// sum_a w e_a = 0 the sums are formed from differences of opposite neighbours,
// (v1 - v3)/9 + ((v5 - v7) + (v8 - v6))/36 along x and (v2 - v4)/9 +
// ((v5 - v7) - (v8 - v6))/36 along y, which are free of cancellation in a bulk
// phase.  Outputs: ps (x, y), p2 (x, y) for F_12, p1 (x, y) for F_21, walls (x, y).
template <class R>
struct Stencils {
  R psx, psy, p2x, p2y, p1x, p1y, ssx, ssy;
};
template <class R>
__device__ __forceinline__ void pair_sums(const R* v, R& sx, R& sy) {
  const R d13 = rsub<R>(v[1], v[3]), d24 = rsub<R>(v[2], v[4]);
  const R d57 = rsub<R>(v[5], v[7]), d86 = rsub<R>(v[8], v[6]);
  sx = rfma<R>(R(1.0 / 9.0), d13, rmul<R>(R(1.0 / 36.0), radd<R>(d57, d86)));
  sy = rfma<R>(R(1.0 / 9.0), d24, rmul<R>(R(1.0 / 36.0), rsub<R>(d57, d86)));
}
template <class R>
__device__ __forceinline__ Stencils<R> force_stencils(R (&ps)[9], R (&p1)[9], R (&p2)[9], const bool (&lv)[9]) {
  int ix = 0, iy = 0;   // wall-density sums in units of 1/36
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if (a >= 5 && !lv[a]) {
      // ah, av are constants once the loop is unrolled: selects, no indexing
      const int ah = EX(a) > 0 ? 1 : 3, av = EY(a) > 0 ? 2 : 4;
      const bool flat = lv[ah] != lv[av], h = lv[ah];
      ps[a] = flat ? (h ? ps[ah] : ps[av]) : ps[0];
      p1[a] = flat ? (h ? p1[ah] : p1[av]) : p1[0];
      p2[a] = flat ? (h ? p2[ah] : p2[av]) : p2[0];
    } else if (!lv[a]) {
      ps[a] = ps[0];
      p1[a] = p1[0];
      p2[a] = p2[0];
    }
    const int sw = lv[a] ? 0 : (a < 5 ? 4 : 1);
    ix += EX(a) * sw;
    iy += EY(a) * sw;
  }
  Stencils<R> S;
  pair_sums<R>(ps, S.psx, S.psy);
  pair_sums<R>(p2, S.p2x, S.p2y);
  pair_sums<R>(p1, S.p1x, S.p1y);
  S.ssx = rmul<R>(R(ix), R(1.0 / 36.0));
  S.ssy = rmul<R>(R(iy), R(1.0 / 36.0));
  return S;
}

// F_1 (Eqs. 11, 14a, 16 and the body force) from its stencil sums, and F_2
// (Eqs. 14b, 16), in a fixed operation order.
template <class R>
__device__ __forceinline__ R force1(R G11, R G12, R w1, R psc, R p1c, R sp, R s2, R ss, R rho1, R g) {
  R F = -rmul<R>(rmul<R>(G11, psc), sp);
  F = rfma<R>(-rmul<R>(G12, p1c), s2, F);
  F = rfma<R>(-rmul<R>(w1, psc), ss, F);
  return rfma<R>(rho1, g, F);
}
template <class R>
__device__ __forceinline__ R force2(R G21, R w2, R p2c, R s1, R ss, R rho2, R g) {
  R F = -rmul<R>(rmul<R>(G21, p2c), s1);
  F = rfma<R>(-rmul<R>(w2, rho2), ss, F);
  return rfma<R>(rho2, g, F);
}

// Common velocity u' (Eq. 18) of one axis, and u_r (Eq. 19).
template <class R>
__device__ __forceinline__ R u_common(R j1, R j2, R it1, R it2, R rden) {
  return rmul<R>(rfma<R>(j1, it1, rmul<R>(j2, it2)), rden);
}
template <class R>
__device__ __forceinline__ R u_phys(R j1, R j2, R F1, R F2, R rrt) {
  return rmul<R>(rfma<R>(R(0.5), radd<R>(F1, F2), radd<R>(j1, j2)), rrt);
}

// D2Q9 equilibrium relative to a node's shift (Eq. 8): w (dr + rho (3 eu +
// 4.5 eu^2 - uu)) with dr = rho - shift and uu = 1.5 |u|^2, and the BGK
// collision with source (Eq. 6): f - (f - feq) / tau + w S.
template <class R>
__device__ __forceinline__ R feq_shifted(R w, R dr, R rho, R eu, R uu) {
  const R t = rsub<R>(rfma<R>(rmul<R>(R(4.5), eu), eu, rmul<R>(R(3), eu)), uu);
  return rmul<R>(w, rfma<R>(rho, t, dr));
}
template <class R>
__device__ __forceinline__ R bgk(R fa, R feq, R itau, R w, R S) {
  return rfma<R>(w, S, rfma<R>(-rsub<R>(fa, feq), itau, fa));
}
template <class R>
__device__ __forceinline__ R half_u2(R ux, R uy) {
  return rmul<R>(R(1.5), rfma<R>(ux, ux, rmul<R>(uy, uy)));
}
// D2Q5 equilibrium relative to the solute shift (Eq. 21) and collision with
// the homogeneous source (Eq. 20): geq = J (C - shift) + C e.u / 2.
template <class R>
__device__ __forceinline__ R geq_shifted(R ja, R C, R sh, R eu) {
  return rfma<R>(ja, rsub<R>(C, sh), rmul<R>(rmul<R>(R(0.5), C), eu));
}

// The nine D2Q9 equilibria of Eq. 8 relative to a node's shift, dr = rho -
// shift, uu = 1.5 |u|^2, evaluated for opposite directions together: the part
// even in e.u, w (dr + rho (4.5 (e.u)^2 - uu)), is shared and the odd part
// 3 w rho e.u is added and subtracted.
template <class R>
__device__ __forceinline__ void feq_pairs(R dr, R rho, R ux, R uy, R uu, R* feq) {
  const R ws = R(1.0 / 9.0), wd = R(1.0 / 36.0);
  feq[0] = rmul<R>(R(4.0 / 9.0), rfma<R>(rho, -uu, dr));
  const R a3s = rmul<R>(R(1.0 / 3.0), rho), a3d = rmul<R>(R(1.0 / 12.0), rho);   // 3 w rho
  // (1, 3): e.u = ux; (2, 4): uy; (5, 7): ux + uy; (6, 8): uy - ux
  const R e[4] = {ux, uy, radd<R>(ux, uy), rsub<R>(uy, ux)};
  constexpr int pa[4] = {1, 2, 5, 6}, pb[4] = {3, 4, 7, 8};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const R w = q < 2 ? ws : wd, a3 = q < 2 ? a3s : a3d;
    const R sym = rmul<R>(w, rfma<R>(rho, rfma<R>(R(4.5), rmul<R>(e[q], e[q]), -uu), dr));
    const R asym = rmul<R>(a3, e[q]);
    feq[pa[q]] = radd<R>(sym, asym);
    feq[pb[q]] = rsub<R>(sym, asym);
  }
}

// The five D2Q5 equilibria of Eq. 21 relative to the species' shift sh:
// J_a (C - sh) + C e.u / 2, opposite directions together.
template <class R>
__device__ __forceinline__ void geq_pairs(R J0, R Ja, R C, R sh, R ux, R uy, R* geq) {
  const R cs = rsub<R>(C, sh), hc = rmul<R>(R(0.5), C);
  const R sa = rmul<R>(Ja, cs), ax = rmul<R>(hc, ux), ay = rmul<R>(hc, uy);
  geq[0] = rmul<R>(J0, cs);
  geq[1] = radd<R>(sa, ax);
  geq[3] = rsub<R>(sa, ax);
  geq[2] = radd<R>(sa, ay);
  geq[4] = rsub<R>(sa, ay);
}

// exp(v) - 1 without the cancellation of evaluating exp(v) first (phi_1 of
// Eq. 15a at the small rho_2 of the liquid phase would lose most of its FP32
// digits otherwise)
template <class R> __device__ __forceinline__ R rexpm1(R v);
template <> __device__ __forceinline__ double rexpm1<double>(double v) { return expm1(v); }
template <> __device__ __forceinline__ float rexpm1<float>(float v) { return expm1f(v); }
template <class R> __device__ __forceinline__ R rsqrt_(R v);
template <> __device__ __forceinline__ double rsqrt_<double>(double v) { return sqrt(v); }
template <> __device__ __forceinline__ float rsqrt_<float>(float v) { return sqrtf(v); }

// psi_1 (Eq. 13), phi_1, phi_2 (Eq. 15) of a live node; sets status bits on a bad argument.
template <class R>
__device__ __forceinline__ void potentials(const DevParams& P, R rho1, R rho2, R& psi, R& phi1, R& phi2,
                                           unsigned& status) {
  const DevParamsR<R>& Q = rp<R>(P);
  if (P.has_G11) {
    R arg = psi_arg<R>(P, rho1);
    if (!(arg >= R(0))) {
      status |= (arg == arg) ? ST_EOS : ST_NONFINITE;
      arg = R(0);
    }
    psi = rsqrt_<R>(arg);
  } else {
    psi = R(0);
  }
  phi1 = -rexpm1<R>(-rmul<R>(rho2, Q.inv_rho20));
  phi2 = rsub<R>(Q.a0, rexp<R>(-rmul<R>(rho1, Q.inv_rho10)));
}

// Same as potentials(), with the parameters taken from a block already staged
// in the compute precision (shared memory in the bulk kernel).
template <class R>
__device__ __forceinline__ void potentials_q(const DevParamsR<R>& Q, bool has_G11, R rho1, R rho2, R& psi, R& phi1,
                                             R& phi2, unsigned& status) {
  if (has_G11) {
    const R eta = Q.eos_b4 * rho1;
    const R om = R(1) - eta;
    const R p = rho1 * Q.eos_RT * (R(1) + eta + eta * eta - eta * eta * eta) / (om * om * om) - Q.eos_a * rho1 * rho1;
    R arg = Q.six_over_G11 * (p - rho1 / R(3));
    if (!(arg >= R(0))) {
      status |= (arg == arg) ? ST_EOS : ST_NONFINITE;
      arg = R(0);
    }
    psi = rsqrt_<R>(arg);
  } else {
    psi = R(0);
  }
  phi1 = -rexpm1<R>(-rmul<R>(rho2, Q.inv_rho20));
  phi2 = rsub<R>(Q.a0, rexp<R>(-rmul<R>(rho1, Q.inv_rho10)));
}

// SplitMix64 output for a given state (Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long s) {
  unsigned long long z = s + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace pslbm
