// Fused bulk kernel of one time step (Chen, Kang et al., arXiv 1410.3464,
// Sections 3-4, numerical procedure of Section 4.7):
//   moments (Eq. 9) -> liquid/gas marking (Section 4.5) -> psi/phi (Eqs. 13,
//   15) staged in shared memory with a one-node ring -> forces (Eqs. 11, 14,
//   16) -> velocities (Eqs. 17-19) -> concentration amendment at marking
//   changes (Step 2) -> homogeneous sources (Eqs. 5a, 5c, 27, 28) -> D2Q9
//   collide and push (Eq. 6, halfway bounce-back) -> D2Q5 collide and push
//   (Eqs. 20-22), bouncing back at every non-liquid neighbour (no-flux links,
//   Eq. 26; the reactive rule of Eqs. 29-31 is applied to the bounced
//   populations of liquid-mineral links by the interface kernel).
//
// State between steps is the pre-collision populations; streaming is a push
// into the other buffer of a ping-pong pair, so every population is read once
// and written once.  The ring nodes' densities are recomputed from their
// populations (read through L2), so psi at radius 2 is never stored in HBM.
//
// The kernel is persistent: each block walks a strided list of 32x8 tiles.
// Node types of the next tile are loaded while the current tile computes, so
// a tile costs one dependent DRAM round trip (its populations); the shared
// stage is double-buffered, so a tile costs one block barrier.  Rare paths
// (marking amendment, reservoir nodes, wrap-around indices) are out of line
// to keep the hot loop small.
#pragma once
#include "device.cuh"
#include "tma.cuh"

namespace pslbm {

// Ring position r (0..SH::RING-1) -> ext coordinates.
template <class SH>
__device__ __forceinline__ void ring_pos(int r, int& ex, int& ey) {
  if (r < SH::EXT_X) {
    ex = r;
    ey = 0;
  } else if (r < 2 * SH::EXT_X) {
    ex = r - SH::EXT_X;
    ey = SH::EXT_Y - 1;
  } else if (r < 2 * SH::EXT_X + (SH::EXT_Y - 2)) {
    ex = 0;
    ey = 1 + (r - 2 * SH::EXT_X);
  } else {
    ex = SH::EXT_X - 1;
    ey = 1 + (r - 2 * SH::EXT_X - (SH::EXT_Y - 2));
  }
}

template <class R, class TG, int NS>
__device__ __forceinline__ void conc_at(const TG* gin, int N, int node, const DevParams& P, R* C) {
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const TG* gk = gin + k * 5 * N;
    R s = gld<R>(P, k, gk + node);
#pragma unroll
    for (int a = 1; a < 5; ++a) s += gld<R>(P, k, gk + a * N + node);
    C[k] = rp<R>(P).shift_c[k] + s;
  }
}

// Raw type of the node at ext position (ex, ey) of a tile (WALL outside a
// non-periodic edge), and its global index (-1 outside).
__device__ __forceinline__ uint8_t ext_type(const DevParams& P, const uint8_t* tin, int x0, int y0, int ex, int ey,
                                            int& idx) {
  int xn, yn;
  if (!nbr(P, x0 - 1, y0 - 1, ex, ey, xn, yn)) {
    idx = -1;
    return T_WALL;
  }
  idx = yn * P.nx + xn;
  return tin[idx] & T_MASK;
}

// Types of one tile for this thread: its own ext positions (one per node it
// computes) and (tid < SH::RING) one ring position.
template <int NPT>
struct TileTypes {
  uint8_t own[NPT], ring;
  int own_idx[NPT], ring_idx;
};

template <class SH>
__device__ __forceinline__ TileTypes<SH::NPT> load_types(const Tile& tl, const DevParams& P, const uint8_t* tin,
                                                         int tid) {
  TileTypes<SH::NPT> tt;
  const int tx = tid % SH::TX, ty = tid / SH::TX;
#pragma unroll
  for (int k = 0; k < SH::NPT; ++k)
    tt.own[k] = ext_type(P, tin, tl.x0, tl.y0, tx + 1, ty + 1 + k * SH::RY, tt.own_idx[k]);
  tt.ring = T_WALL;
  tt.ring_idx = -1;
  if (tid < SH::RING) {
    int ex, ey;
    ring_pos<SH>(tid, ex, ey);
    tt.ring = ext_type(P, tin, tl.x0, tl.y0, ex, ey, tt.ring_idx);
  }
  return tt;
}

// What one bulk launch needs of an instance: the buffers of the current step,
// the step and the liquid threshold.  All are fixed for the launch (the step
// counter and the threshold advance in the amendment kernel), so a launch over
// one simulation reads them once.
template <class TF, class TG, class R>
struct StepView {
  const TF* fin;
  TF* fout;
  const TG* gin;
  TG* gout;
  const uint8_t* tin;
  uint8_t* tout;
  unsigned* vmask;
  unsigned long long* scal;
  unsigned long long step;
  int cur, N;
  R theta;
};

template <class TF, class TG, class R>
__device__ __forceinline__ StepView<TF, TG, R> step_view(const DevInst* Ip) {
  StepView<TF, TG, R> v;
  v.step = Ip->scal[S_STEP];
  v.cur = int(v.step & 1ULL);
  v.fin = (const TF*)Ip->f[v.cur];
  v.fout = (TF*)Ip->f[v.cur ^ 1];
  v.gin = (const TG*)Ip->g[v.cur];
  v.gout = (TG*)Ip->g[v.cur ^ 1];
  v.tin = Ip->type[v.cur];
  v.tout = Ip->type[v.cur ^ 1];
  v.vmask = Ip->vmask;
  v.scal = Ip->scal;
  v.N = (int)Ip->N;
  v.theta = theta_of<R>(Ip);
  return v;
}

// Per-thread maximum of rho_1 and status bits of the tiles a thread has done
// since the last flush.
template <class R>
struct TileAcc {
  R mx;
  unsigned status;
};

// a[k] of a small register array at a run-time index, as a chain of selects
// over constant indices (the array stays in registers).
template <int NA, class T>
__device__ __forceinline__ T pick(const T (&a)[NA], int k) {
  T v = a[0];
#pragma unroll
  for (int i = 1; i < NA; ++i) v = (k == i) ? a[i] : v;
  return v;
}

// Warp reduction of the accumulators into the instance's slots: the exact
// maximum (the atomic only when it can raise the slot) and the status bits.
// Called by all lanes of the warp.
template <class R>
__device__ __forceinline__ void flush_acc(TileAcc<R>& acc, unsigned long long* scal, int cur) {
  R m = acc.mx;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = rmax<R>(m, __shfl_xor_sync(0xffffffffu, m, o));
  const unsigned st = __reduce_or_sync(0xffffffffu, acc.status);
  if ((threadIdx.x & 31) == 0) {
    if (m > R(-1.0 / 0.0)) {
      const unsigned long long enc = ord_enc(double(m));
      unsigned long long* slot = &scal[S_MAX0 + (cur ^ 1)];
      if (enc > *(volatile unsigned long long*)slot) atomicMax(slot, enc);
    }
    if (st) atomicOr(&scal[S_STATUS], (unsigned long long)st);
  }
  acc.mx = R(-1.0 / 0.0);
  acc.status = 0;
}

// Index of the neighbour (x + dx, y + dy) with wrap (out of line: used only by
// tiles whose ring crosses the domain edge).
static __device__ __noinline__ int nbr_index(const DevParams& P, int x, int y, int dx, int dy) {
  int xn, yn;
  nbr(P, x, y, dx, dy, xn, yn);
  return yn * P.nx + xn;
}

// Section 4.5 amendment at a node whose neighbourhood changed marking (out of
// line, rare).  dC[k] receives the solute handed over by vanishing (liquid ->
// gas) neighbours, each giving C / (number of its liquid neighbours); for an
// appearing (gas -> liquid) node, cb[k] receives the mean C of its surviving
// liquid neighbours (0 if none).
template <class SH, class R, class TF, class TG, int NS>
__device__ __noinline__ void amend_marking(const DevParams& P, const uint8_t* tin, const TF* fin, const TG* gin,
                                           int N, int x, int y, bool appear, const uint8_t* s_t,
                                           const uint8_t* s_m, int eo, R theta, R* dC, R* cb) {
  R base[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) { base[k] = R(0); dC[k] = R(0); }
  int nsrc = 0;
#pragma unroll
  for (int b = 1; b < 5; ++b) {
    const int en = eo + EY(b) * SH::EXT_X + EX(b);
    int xn, yn;
    if (!nbr(P, x, y, EX(b), EY(b), xn, yn)) continue;
    const int nn = yn * P.nx + xn;
    if (appear && s_t[en] == T_LIQUID && s_m[en]) {
      R Cn[NS];
      conc_at<R, TG, NS>(gin, N, nn, P, Cn);
#pragma unroll
      for (int k = 0; k < NS; ++k) base[k] += Cn[k];
      ++nsrc;
    }
    if (s_t[en] == T_LIQUID && s_m[en] == 0) {
      int nrec = 0;
#pragma unroll
      for (int c = 1; c < 5; ++c) {
        int xz, yz;
        if (!nbr(P, xn, yn, EX(c), EY(c), xz, yz)) continue;
        nrec += liquid_at<R, TF>(P, tin, fin, N, yz * P.nx + xz, theta) ? 1 : 0;
      }
      R Cn[NS];
      conc_at<R, TG, NS>(gin, N, nn, P, Cn);
#pragma unroll
      for (int k = 0; k < NS; ++k) dC[k] += Cn[k] / R(nrec);
    }
  }
#pragma unroll
  for (int k = 0; k < NS; ++k) cb[k] = nsrc ? base[k] / R(nsrc) : R(0);
}

// Densities of a reservoir node at this step (out of line: only inlet and
// outlet nodes take this path).
template <class R, class TF>
__device__ __noinline__ void res_density(const DevParams& P, uint8_t t, unsigned long long step, const uint8_t* tin,
                                         const TF* fin, int N, int idx, R theta, R& r1, R& r2) {
  double a, b;
  reservoir_rho(P, t, step, t == T_OUTLET && outlet_up_liquid<R, TF>(P, tin, fin, N, idx, theta), a, b);
  r1 = R(a);
  r2 = R(b);
}

// Reservoir node: push its equilibrium state (densities of reservoir_rho,
// velocity of the node downstream of an inlet / upstream of an outlet) into
// its fluid neighbours, and the solute equilibrium into its liquid neighbours
// when it is itself liquid.
template <class SH, class R, class TF, class TG, int NS>
__device__ __noinline__ void reservoir_push(const DevParams& P, const uint8_t* tin, const TF* fin, const TG* gin,
                                            TF* fout, TG* gout, int N, int x, int y, uint8_t t,
                                            unsigned long long step, R theta, const uint8_t* s_t,
                                            const uint8_t* s_m, int eo) {
  const int node = y * P.nx + x;
  double a_, b_;
  reservoir_rho(P, t, step, t == T_OUTLET && outlet_up_liquid<R, TF>(P, tin, fin, N, node, theta), a_, b_);
  const R r1 = R(a_), r2 = R(b_);
  R ux = R(0), uy = R(0);
  int xn, yn;
  const int dx = (t == T_INLET) ? P.in_dx : P.out_dx, dy = (t == T_INLET) ? P.in_dy : P.out_dy;
  if (nbr(P, x, y, dx, dy, xn, yn)) {
    const int nn = yn * P.nx + xn;
    const uint8_t tnn = tin[nn] & T_MASK;
    if (is_fluid(tnn)) {
      R q1[9], q2[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        q1[a] = ld<R>(fin + a * N + nn);
        q2[a] = ld<R>(fin + (9 + a) * N + nn);
      }
      R e1 = q1[0], e2 = q2[0];
#pragma unroll
      for (int a = 1; a < 9; ++a) { e1 += q1[a]; e2 += q2[a]; }
      const R jx = (q1[1] - q1[3]) + (q1[5] - q1[6]) + (q1[8] - q1[7]) + (q2[1] - q2[3]) + (q2[5] - q2[6]) +
                   (q2[8] - q2[7]);
      const R jy = (q1[2] - q1[4]) + (q1[5] - q1[8]) + (q1[6] - q1[7]) + (q2[2] - q2[4]) + (q2[5] - q2[8]) +
                   (q2[6] - q2[7]);
      const R rt = (fshift<R>(P, 0, tnn) + e1) + (fshift<R>(P, 1, tnn) + e2);
      ux = jx / rt;
      uy = jy / rt;
    }
  }
  const R uu = half_u2<R>(ux, uy);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const R rho = s == 0 ? r1 : r2;
    TF* fo = fout + s * 9 * N;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const int en = eo + EY(a) * SH::EXT_X + EX(a);
      if (!is_fluid(s_t[en])) continue;
      // stored relative to the shift of the receiving node's new phase
      const R dr = rho - (s_m[en] ? rp<R>(P).shift_f[s] : rp<R>(P).shift_fg[s]);
      const R eu = R(EX(a)) * ux + R(EY(a)) * uy;   // exact: e has components 0, +-1
      const R w = w9<R>(a);
      const R feq = feq_shifted<R>(w, dr, rho, eu, uu);
      nbr(P, x, y, EX(a), EY(a), xn, yn);
      st<TF, R>(fo + a * N + yn * P.nx + xn, feq);
    }
  }
  if constexpr (NS > 0) {
    if (s_m[eo]) {
      R Cr[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) Cr[k] = rp<R>(P).conc_in[k];
      if (t == T_OUTLET) {
        const int ew = eo + P.out_dy * SH::EXT_X + P.out_dx;
#pragma unroll
        for (int k = 0; k < NS; ++k) Cr[k] = R(0);
        if (is_fluid(s_t[ew]) && s_m[ew] && nbr(P, x, y, P.out_dx, P.out_dy, xn, yn))
          conc_at<R, TG, NS>(gin, N, yn * P.nx + xn, P, Cr);
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const R Ja = rp<R>(P).Ja[k];
#pragma unroll
        for (int a = 1; a < 5; ++a) {
          const int en = eo + EY(a) * SH::EXT_X + EX(a);
          if (!(is_fluid(s_t[en]) && s_m[en])) continue;
          const R eu = R(EX(a)) * ux + R(EY(a)) * uy;   // exact
          const R geq = geq_shifted<R>(Ja, Cr[k], rp<R>(P).shift_c[k], eu);
          nbr(P, x, y, EX(a), EY(a), xn, yn);
          gst<TG, R>(P, k, gout + (k * 5 + a) * N + yn * P.nx + xn, geq);
        }
      }
    }
  }
}

// Minimum resident blocks per SM the register allocation targets: FP32
// compute with one node per thread keeps three 256-thread blocks per SM; two
// nodes per thread (twice the moments carried across the tile's barrier) and
// FP64 (twice the registers per value, bound by FP64 arithmetic anyway) two.
#ifndef PSLBM_BULK_MINB
#define PSLBM_BULK_MINB 3
#endif
template <class R, int NPT>
constexpr int bulk_min_blocks() {
  return (sizeof(R) == 8 || NPT > 1) ? 2 : PSLBM_BULK_MINB;
}

// Shared-memory record of one ext node: psi_1, phi_1, phi_2 (zero where not
// live) and a code of its type and liquid marking, read by a neighbour with
// one vector load.
template <class R>
struct alignas(4 * sizeof(R)) Pot {
  R ps, p1, p2, code;
};
// Code bits: the low nibble holds what a push needs of a neighbour (fluid,
// liquid marking, reservoir, mineral), then live, an axis-link pair (raw
// type liquid, raw type D(s)) and the raw type.
constexpr int C_FLUID = 1, C_MARK = 2, C_RES = 4, C_MIN = 8, C_LIVE = 16, C_OLDLIQ = 32, C_SOLD = 64;
__device__ __forceinline__ int node_code(uint8_t t, bool mark) {
  return (is_fluid(t) ? C_FLUID : 0) | (mark ? C_MARK : 0) | (is_res(t) ? C_RES : 0) | (is_mineral(t) ? C_MIN : 0) |
         (is_live(t) ? C_LIVE : 0) | (t == T_LIQUID ? C_OLDLIQ : 0) | (t == T_SOLID_D ? C_SOLD : 0) | (int(t) << 8);
}
template <class R> __device__ __forceinline__ R code_bits(int c);
template <> __device__ __forceinline__ float code_bits<float>(int c) { return __int_as_float(c); }
template <> __device__ __forceinline__ double code_bits<double>(int c) { return __longlong_as_double((long long)c); }
template <class R> __device__ __forceinline__ int code_of(R v);
template <> __device__ __forceinline__ int code_of<float>(float v) { return __float_as_int(v); }
template <> __device__ __forceinline__ int code_of<double>(double v) { return (int)__double_as_longlong(v); }

// Population source of the plain kernel: loads from global memory (L2 for
// the ring).  own() loads the node's D2Q9 and D2Q5 populations (as stored,
// i.e. shifted in the reduced precisions); ring_density() returns the two
// stored density sums of a ring node.
template <class TF, class TG, class R, int NS>
struct GlobalSrc {
  static constexpr bool kReread = false;
  const TF* fin;
  const TG* gin;
  int N;
  // ly: the node's row in its tile (unused here)
  __device__ __forceinline__ void own_f(int idx, int, R* f1, R* f2) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      f1[a] = ld<R>(fin + a * N + idx);
      f2[a] = ld<R>(fin + (9 + a) * N + idx);
    }
  }
  // one component's populations (an L1 hit when re-read within the tile)
  __device__ __forceinline__ void own_fc(int idx, int, int comp, R* f) const {
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = ld<R>(fin + (comp * 9 + a) * N + idx);
  }
  __device__ __forceinline__ void own_g(int node, R (*gs)[5]) const {
#pragma unroll
    for (int k = 0; k < NS; ++k)
#pragma unroll
      for (int a = 0; a < 5; ++a) gs[k][a] = ld<R>(gin + (k * 5 + a) * N + node);
  }
  __device__ __forceinline__ void ring_density(int ring_idx, int, int, R& d1, R& d2) const {
    d1 = density_shifted<R>(fin, (long long)N, ring_idx);
    d2 = density_shifted<R>(fin + 9 * N, (long long)N, ring_idx);
  }
};

// One tile of the bulk step (Sections 3-4; the order of Section 4.7 with the
// cut after the streaming of Step 1).  `src` delivers the populations,
// `after_sync` runs once the block has passed the tile's barrier (all reads of
// the tile's staged populations are done by then), `tt` holds this tile's node
// types on entry and the next tile's on return (`next_types(tt)` loads them).
// The tile's maximum of rho_1 and its status bits go into `acc`.  Returns true
// when the block must stop (a bounded wait of the staged kernel gave up in
// some thread).
//
// Each thread computes SH::NPT nodes, rows ty + k RY of the tile.  Before the
// barrier it loads all of them (their loads in flight together) and keeps
// their moments; after it, the nodes run one after the other through the same
// code.  The D2Q9 populations are held in registers across the barrier only
// with one node per thread and a source that does not re-read them (kHold);
// otherwise the collision reads them again (from the stage, or from L1).
template <class SH, class TF, class TG, class R, int NS, class Src, class AfterSync, class NextTypes>
__device__ __forceinline__ bool bulk_tile(const Tile& tl, const StepView<TF, TG, R>& V, const DevParams& P,
                                          const Src& src, AfterSync after_sync, NextTypes next_types, bool waited_ok,
                                          TileTypes<SH::NPT>& tt, TileAcc<R>& acc, Pot<R>* spot, uint8_t* st_,
                                          uint8_t* sm_) {
  constexpr int NPT = SH::NPT;
  constexpr bool kHold = NPT == 1 && !Src::kReread;
  const int tid = threadIdx.x;
  const int tx = tid % SH::TX, ty = tid / SH::TX;
  int er = -1, rex = 0, rey = 0;
  if (tid < SH::RING) {
    ring_pos<SH>(tid, rex, rey);
    er = rey * SH::EXT_X + rex;
  }
  const int N = V.N;
  const int nx = P.nx;
  const unsigned long long step = V.step;
  const TF* __restrict__ fin = V.fin;
  TF* __restrict__ fout = V.fout;
  const TG* __restrict__ gin = V.gin;
  TG* __restrict__ gout = V.gout;
  const uint8_t* __restrict__ tin = V.tin;
  uint8_t* __restrict__ tout = V.tout;
  const R theta = V.theta;
  // neighbour indices need wrap arithmetic only on a tile whose ring crosses
  // a periodic edge: across a non-periodic edge the neighbour is a wall, and
  // a push toward a wall bounces back without using the neighbour's index
  const bool inner = (!P.px || (tl.x0 >= 1 && tl.x0 + SH::TX + 1 <= nx)) &&
                     (!P.py || (tl.y0 >= 1 && tl.y0 + SH::TY + 1 <= P.ny));
  unsigned status = 0;

  // ---- phase 1: population loads (own nodes and one ring node)
  uint8_t own_tv[NPT];
  int own_iv[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    own_tv[k] = tt.own[k];
    own_iv[k] = tt.own_idx[k];
  }
  const uint8_t ring_t = tt.ring;
  const int ring_idx = tt.ring_idx;
  // populations are stored relative to the reference density of the node's
  // phase (0 in FP64)
  R q1[NPT][9], q2[NPT][9];
  R gs[NS > 0 ? NS : 1][5];
#pragma unroll
  for (int k = 0; k < NPT; ++k)
    if (is_fluid(own_tv[k]) && own_iv[k] >= 0) src.own_f(own_iv[k], ty + k * SH::RY, q1[k], q2[k]);
  // solute populations of a liquid node (undoing the species' storage scale,
  // a power of two: exact); loaded here only when the populations are held
  auto load_g = [&](bool own, uint8_t own_t, int node) {
    if constexpr (NS > 0) {
      if (own && own_t == T_LIQUID) {
        src.own_g(node, gs);
        if constexpr (Is16<TG>::value) {
#pragma unroll
          for (int k = 0; k < NS; ++k)
#pragma unroll
            for (int a = 0; a < 5; ++a) gs[k][a] = gs[k][a] * rp<R>(P).gs_div[k];
        }
      }
    }
  };
  if constexpr (kHold) {
    const int x = tl.x0 + tx, y = tl.y0 + ty;
    load_g(x < nx && y < P.ny, own_tv[0], y * nx + x);
  }
  R r1r = R(0), r2r = R(0);
  if (tid < SH::RING && is_fluid(ring_t)) {
    R d1r, d2r;
    src.ring_density(ring_idx, tl.x0 - 1 + rex, tl.y0 - 1 + rey, d1r, d2r);
    r1r = fshift<R>(P, 0, ring_t) + d1r;
    r2r = fshift<R>(P, 1, ring_t) + d2r;
  }
  // prefetch the next tile's node types
  next_types(tt);

  // ---- moments of the own nodes (Eq. 9)
  R rho1v[NPT], rho2v[NPT], d1v[NPT], d2v[NPT], j1xv[NPT], j1yv[NPT], j2xv[NPT], j2yv[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    R rho1 = R(0), rho2 = R(0), d1 = R(0), d2 = R(0), j1x = R(0), j1y = R(0), j2x = R(0), j2y = R(0);
    if (is_fluid(own_tv[k]) && own_iv[k] >= 0) {
      const R* f1 = q1[k];
      const R* f2 = q2[k];
      d1 = f1[0];
      d2 = f2[0];
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        d1 += f1[a];
        d2 += f2[a];
      }
      j1x = (f1[1] - f1[3]) + (f1[5] - f1[6]) + (f1[8] - f1[7]);
      j1y = (f1[2] - f1[4]) + (f1[5] - f1[8]) + (f1[6] - f1[7]);
      j2x = (f2[1] - f2[3]) + (f2[5] - f2[6]) + (f2[8] - f2[7]);
      j2y = (f2[2] - f2[4]) + (f2[5] - f2[8]) + (f2[6] - f2[7]);
      rho1 = fshift<R>(P, 0, own_tv[k]) + d1;
      rho2 = fshift<R>(P, 1, own_tv[k]) + d2;
      if (!(rho1 == rho1 && rho2 == rho2)) status |= ST_NONFINITE;
    }
    rho1v[k] = rho1;
    rho2v[k] = rho2;
    d1v[k] = d1;
    d2v[k] = d2;
    j1xv[k] = j1x;
    j1yv[k] = j1y;
    j2xv[k] = j2x;
    j2yv[k] = j2y;
  }
  // ---- potentials of the own nodes and (tid < RING) one ring node -> shared.
  // One loop body, not unrolled, serves all, so the equation of state, the
  // exponentials and the reservoir path are emitted once.
#pragma unroll 1
  for (int w = 0; w <= NPT; ++w) {
    const bool ring = w == NPT;
    if (ring && tid >= SH::RING) break;
    const uint8_t tw = ring ? ring_t : pick(own_tv, w);
    R r1 = ring ? r1r : pick(rho1v, w), r2 = ring ? r2r : pick(rho2v, w);
    if (is_res(tw)) res_density<R, TF>(P, tw, step, tin, fin, N, ring ? ring_idx : pick(own_iv, w), theta, r1, r2);
    R ps = R(0), p1 = R(0), p2 = R(0);
    if (is_live(tw)) potentials<R>(P, r1, r2, ps, p1, p2, status);
    const bool mk = is_live(tw) && r1 > theta;
    const int slot = ring ? er : (ty + 1 + w * SH::RY) * SH::EXT_X + (tx + 1);
    spot[slot] = Pot<R>{ps, p1, p2, code_bits<R>(node_code(tw, mk))};
    st_[slot] = tw;
    sm_[slot] = mk ? 1 : 0;
  }
  if (__syncthreads_or(waited_ok ? 0 : 1)) return true;
  after_sync();

  // ---- phase 2, node by node
#pragma unroll 1
  for (int kn = 0; kn < NPT; ++kn) {
    const int ly = ty + kn * SH::RY;
    const int x = tl.x0 + tx, y = tl.y0 + ly;
    const bool own = x < nx && y < P.ny;
    const int node = y * nx + x;
    const int eo = (ly + 1) * SH::EXT_X + (tx + 1);
    const uint8_t own_t = pick(own_tv, kn);
    const int own_idx = pick(own_iv, kn);
    const uint8_t t = own ? own_t : T_WALL;
    const R sh1 = fshift<R>(P, 0, own_t), sh2 = fshift<R>(P, 1, own_t);
    const R rho1 = pick(rho1v, kn), rho2 = pick(rho2v, kn), d1 = pick(d1v, kn), d2 = pick(d2v, kn);
    const R j1x = pick(j1xv, kn), j1y = pick(j1yv, kn), j2x = pick(j2xv, kn), j2y = pick(j2yv, kn);
    R f1[9], f2[9];
    if constexpr (kHold) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        f1[a] = q1[0][a];
        f2[a] = q2[0][a];
      }
    }
    R mymax = R(-1.0 / 0.0);
    if (own && is_fluid(t)) {
      mymax = rho1;
      // ---- forces (Eqs. 11, 14a/b, 16) with mirror-image solid neighbours
      // (force_stencils).
      const Pot<R> pc = spot[eo];
      const R psc = pc.ps, p1c = pc.p1, p2c = pc.p2;
      // neighbour codes kept for the pushes: the low nibble of each of the eight
      // neighbours (nbits, 4 bits per direction) and the raw-type pair of the four
      // axis neighbours (abits, 2 bits per direction)
      unsigned nbits = 0u, abits = 0u;
      const int c0 = code_of<R>(pc.code);
      R vps[9], vp1[9], vp2[9];
      bool lv[9];
      vps[0] = psc;
      vp1[0] = p1c;
      vp2[0] = p2c;
      lv[0] = true;
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        const Pot<R> q = spot[eo + EY(a) * SH::EXT_X + EX(a)];
        const int ca = code_of<R>(q.code);
        nbits |= unsigned(ca & 0xF) << (4 * (a - 1));
        if (a < 5) abits |= unsigned((ca >> 5) & 0x3) << (2 * (a - 1));
        lv[a] = (ca & C_LIVE) != 0;
        vps[a] = q.ps;
        vp1[a] = q.p1;
        vp2[a] = q.p2;
      }
      const Stencils<R> S = force_stencils<R>(vps, vp1, vp2, lv);
      const R spx = S.psx, spy = S.psy, s2x = S.p2x, s2y = S.p2y, s1x = S.p1x, s1y = S.p1y, ssx = S.ssx,
              ssy = S.ssy;
      const R G11 = rp<R>(P).G11, G12 = rp<R>(P).G12, G21 = rp<R>(P).G21, w1 = rp<R>(P).w_adh[0],
              w2 = rp<R>(P).w_adh[1];
      const R F1x = force1<R>(G11, G12, w1, psc, p1c, spx, s2x, ssx, rho1, rp<R>(P).gx);
      const R F1y = force1<R>(G11, G12, w1, psc, p1c, spy, s2y, ssy, rho1, rp<R>(P).gy);
      const R F2x = force2<R>(G21, w2, p2c, s1x, ssx, rho2, rp<R>(P).gx);
      const R F2y = force2<R>(G21, w2, p2c, s1y, ssy, rho2, rp<R>(P).gy);
      // ---- velocities (Eqs. 17-19)
      const R it1 = rp<R>(P).inv_tau[0], it2 = rp<R>(P).inv_tau[1];
      const R rden = rrcp<R>(rfma<R>(rho1, it1, rmul<R>(rho2, it2)));
      const R upx = u_common<R>(j1x, j2x, it1, it2, rden);
      const R upy = u_common<R>(j1y, j2y, it1, it2, rden);
      const R q1 = rho1 != R(0) ? rmul<R>(rp<R>(P).tau[0], rrcp<R>(rho1)) : R(0);
      const R q2 = rho2 != R(0) ? rmul<R>(rp<R>(P).tau[1], rrcp<R>(rho2)) : R(0);
      const R u1x = rfma<R>(F1x, q1, upx), u1y = rfma<R>(F1y, q1, upy);
      const R u2x = rfma<R>(F2x, q2, upx), u2y = rfma<R>(F2y, q2, upy);
      const R rrt = rrcp<R>(radd<R>(rho1, rho2));
      const R urx = u_phys<R>(j1x, j2x, F1x, F2x, rrt);
      const R ury = u_phys<R>(j1y, j2y, F1y, F2y, rrt);

      const bool liq = (c0 & C_MARK) != 0;
      tout[node] = liq ? T_LIQUID : T_GAS;

      // neighbour indices for the push (constant offsets away from the edges)
      int nb[9];
#pragma unroll
      for (int a = 1; a < 9; ++a) nb[a] = inner ? node + EX(a) + EY(a) * nx : nbr_index(P, x, y, EX(a), EY(a));

      // ---- solutes: concentration with the Step-2 amendment, sources
      if constexpr (!kHold) load_g(own, own_t, node);
      R S1 = R(0), S2 = R(0);
      R C[NS > 0 ? NS : 1];
      R Sk[NS > 0 ? NS : 1];
      if constexpr (NS > 0) {
        if (liq) {
          const bool appear = (t == T_GAS);
          bool vnb = false;
#pragma unroll
          for (int b = 1; b < 5; ++b) {
            // a neighbour that was liquid and is no longer marked liquid
            vnb |= ((abits >> (2 * (b - 1))) & 1u) && !((nbits >> (4 * (b - 1))) & C_MARK);
          }
          if (appear || vnb) {
            R dC[NS], cb[NS];
            amend_marking<SH, R, TF, TG, NS>(P, tin, fin, gin, N, x, y, appear, st_, sm_, eo, theta, dC, cb);
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              const R J0 = rp<R>(P).J0[k], Ja = rp<R>(P).Ja[k];
#pragma unroll
              for (int a = 0; a < 5; ++a) {
                const R ja = a == 0 ? J0 : Ja;
                gs[k][a] = appear ? rfma<R>(ja, radd<R>(cb[k], dC[k]), -rmul<R>(ja, rp<R>(P).shift_c[k]))
                                  : rfma<R>(ja, dC[k], gs[k][a]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            R s = gs[k][0];
#pragma unroll
            for (int a = 1; a < 5; ++a) s += gs[k][a];
            C[k] = rp<R>(P).shift_c[k] + s;
          }
          // homogeneous reactions (Eqs. 5a, 5c; sources Eqs. 27, 28)
          R CA = R(0), CB = R(0), CE = R(0), tot = R(0);
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            if (k == P.iA) CA = C[k];
            if (k == P.iB) CB = C[k];
            if (k == P.iE) CE = C[k];
            tot += C[k];
          }
          if (P.iA == -2) CA = rmax<R>(R(0), rfma<R>(rp<R>(P).c_total_per_rho1, rho1, -tot));
          // Section 2: R1 is faster at the surface of D(s) (a liquid node with a
          // D(s) node on an axis link)
          bool surf = false;
          if (P.r1_surf) {
#pragma unroll
            for (int b = 1; b < 5; ++b) surf |= ((abits >> (2 * (b - 1) + 1)) & 1u) != 0;
          }
          R R1 = rmul<R>(surf ? rp<R>(P).k1_s : rp<R>(P).k1, CA);
          if (P.has_rev)
            R1 = rsub<R>(R1, rmul<R>(rmul<R>(surf ? rp<R>(P).k1_inv_Keq_s : rp<R>(P).k1_inv_Keq, CB),
                                     rsqrt_<R>(rmax<R>(rmul<R>(rho2, rp<R>(P).inv_M_C), R(0)))));
          const R R3 = rmul<R>(rmul<R>(rp<R>(P).k3, CB), CE);
#pragma unroll
          for (int k = 0; k < NS; ++k) Sk[k] = rfma<R>(rp<R>(P).cR1[k], R1, rmul<R>(rp<R>(P).cR3[k], R3));
          S1 = -rmul<R>(rp<R>(P).gas_yield, R1);
          S2 = rmul<R>(rp<R>(P).gas_yield, R1);
        }
      }

      // ---- push targets, shared by both components: the slot that the
      // population moving along a lands in (slot a of the fluid neighbour, or
      // slot OPP(a) here when it bounces back from a solid or wall), whether it
      // is stored (nothing goes into a reservoir), and whether the node that
      // receives it is marked liquid (the shift it is stored relative to)
      int pdst[9];
      unsigned pkeep = 0u, pliq = 0u;
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        const int c = int((nbits >> (4 * (a - 1))) & 0xFu);
        const bool fl = (c & C_FLUID) != 0;
        pdst[a] = fl ? a * N + nb[a] : OPP(a) * N + node;
        pkeep |= (fl || !(c & C_RES)) ? (1u << a) : 0u;
        pliq |= (fl ? (c & C_MARK) != 0 : liq) ? (1u << a) : 0u;
        // a liquid node flags the minerals on its axis links for the VOP kernel
        if (a < 5 && liq && (c & C_MIN)) atomicOr(&V.vmask[nb[a] >> 5], 1u << (nb[a] & 31));
      }

      // ---- fluid collision (Eq. 6, Eq. 8 at u_eq) and push streaming.  The
      // collision runs relative to this node's shift; a value pushed into a node
      // whose new phase has another shift is re-based by w (shift - shift').
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const R rho = s == 0 ? rho1 : rho2;
        const R dr = s == 0 ? d1 : d2;
        const R ux = s == 0 ? u1x : u2x, uy = s == 0 ? u1y : u2y;
        const R itau = s == 0 ? it1 : it2;
        const R Ssrc = s == 0 ? S1 : S2;
        const R uu = half_u2<R>(ux, uy);
        const R shs = s == 0 ? sh1 : sh2;
        const R dl = shs - rp<R>(P).shift_f[s], dg = shs - rp<R>(P).shift_fg[s];
        const R down = liq ? dl : dg;
        if constexpr (!kHold) {
          // read the component's populations again (from the stage, or from L1)
          // rather than keeping them in registers across the barrier
          src.own_fc(own_idx, ly, s, s == 0 ? f1 : f2);
        }
        TF* fo = fout + s * 9 * N;
        // Eq. 8 relative to the node's shift, for opposite directions a, a'
        // together: w (dr + rho (4.5 (e.u)^2 - 1.5 u^2)) +- 3 w rho e.u
        R feq[9];
        feq_pairs<R>(dr, rho, ux, uy, uu, feq);
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          const R fa = s == 0 ? f1[a] : f2[a];
          const R w = w9<R>(a);
          const R fs = bgk<R>(fa, feq[a], itau, w, Ssrc);
          if (a == 0) {
            st<TF, R>(fo + node, rfma<R>(w, down, fs));
            continue;
          }
          // into a fluid neighbour (re-based to its new phase), or bounced back
          // here from a solid or wall; nothing into a reservoir
          const R sto = ((pliq >> a) & 1u) ? dl : dg;
          if ((pkeep >> a) & 1u) st<TF, R>(fo + pdst[a], rfma<R>(w, sto, fs));
        }
      }

      // ---- solute collision (Eqs. 20-22 with u_r) and push streaming
      if constexpr (NS > 0) {
        if (liq) {
          // Eq. 21 relative to the species' shift, opposite directions together:
          // J_a (C - shift) +- C e.u / 2
          R geq[NS][5];
#pragma unroll
          for (int k = 0; k < NS; ++k) geq_pairs<R>(rp<R>(P).J0[k], rp<R>(P).Ja[k], C[k], rp<R>(P).shift_c[k], urx, ury,
                                                    geq[k]);
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            // the rest population stays; a moving one goes into a liquid
            // neighbour, out into a liquid reservoir, or bounces back here
            // (no-flux / mineral link)
            // so: slot * N + destination node, the same for every species
            int so = a * N + node;
            bool keep = true;
            if (a > 0) {
              const int c = int((nbits >> (4 * (a - 1))) & 0xFu);
              const bool into = (c & (C_FLUID | C_MARK)) == (C_FLUID | C_MARK);
              const bool out = (c & (C_RES | C_MARK)) == (C_RES | C_MARK);
              so = ((into || out) ? a : OPP(a)) * N + (into ? nb[a] : node);
              keep = !out;
            }
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              const R ja = a == 0 ? rp<R>(P).J0[k] : rp<R>(P).Ja[k];
              const R gs_ = bgk<R>(gs[k][a], geq[k][a], rp<R>(P).inv_tau_g[k], ja, Sk[k]);
              if (keep) gst<TG, R>(P, k, gout + k * 5 * N + so, gs_);
            }
          }
        } else {
          // gas node: no solute
#pragma unroll
          for (int k = 0; k < NS; ++k) {
#pragma unroll
            for (int a = 0; a < 5; ++a)
              gst<TG, R>(P, k, gout + (k * 5 + a) * N + node,
                         -(a == 0 ? rp<R>(P).J0[k] : rp<R>(P).Ja[k]) * rp<R>(P).shift_c[k]);
          }
        }
      }
    } else if (own) {
      if (is_res(t))
        reservoir_push<SH, R, TF, TG, NS>(P, tin, fin, gin, fout, gout, N, x, y, t, step, theta, st_, sm_, eo);
      tout[node] = t;
    }

    // ---- max of rho_1 over fluid nodes (next step's threshold)
    acc.mx = rmax<R>(acc.mx, mymax);
  }
  acc.status |= status;
  return false;
}

// Plain bulk kernel: persistent over the tile list, populations loaded from
// global memory by each thread.  The shared stage is double-buffered, so a
// tile costs one block barrier.  Blocks claim their tiles in list order from
// a counter, so that blocks that meet cheap tiles take more of them.
//
// SINGLE: every tile belongs to the one simulation at insts[0]; its step view
// is read once, the next tile's descriptor is loaded a tile ahead, and the
// maximum and status are flushed once at the end.  Otherwise (a batch) the
// view and step limit are read, and the accumulators flushed, once per run of
// consecutive tiles of one instance.
template <class SH, class TF, class TG, class R, int NS, bool SINGLE>
__global__ void __launch_bounds__(NTHREADS, bulk_min_blocks<R, SH::NPT>()) k_bulk(const Tile* __restrict__ tiles, int ntiles,
                                                                         const DevInst* __restrict__ insts) {
  __shared__ Pot<R> s_pot[2][SH::EXT];
  __shared__ uint8_t s_t[2][SH::EXT], s_m[2][SH::EXT];
  __shared__ int s_claim[2];
  const int stride = gridDim.x;
  TileAcc<R> acc{R(-1.0 / 0.0), 0u};
  int buf = 0;
  TileTypes<SH::NPT> tt;
  // after its first tile (blockIdx.x) a block claims its tiles in list order
  // from the launch's counter (in the first instance), one tile ahead: lane 0
  // of the last warp (no ring node) claims tile j+2 during tile j and shares it
  // through shared memory, read after the tile's barrier
  constexpr int CLAIMER = NTHREADS - 32;
  auto claim = [&] { return stride + (int)atomicAdd(insts->scal + S_TILES, 1ULL); };
  if constexpr (SINGLE) {
    // one simulation: all tiles are live or none is
    if (!(insts->scal[S_STEP] < insts->scal[S_LIMIT])) return;
    const StepView<TF, TG, R> V = step_view<TF, TG, R>(insts);
    const DevParams& P = insts->P;
    const GlobalSrc<TF, TG, R, NS> src{V.fin, V.gin, V.N};
    int ti = blockIdx.x;
    Tile tl = ti < ntiles ? tiles[ti] : Tile{};
    if (threadIdx.x == CLAIMER) s_claim[0] = claim();
    if (ti < ntiles) tt = load_types<SH>(tl, P, V.tin, threadIdx.x);
    __syncthreads();
    int j = 0;
    while (ti < ntiles) {
      const int nt = s_claim[j & 1];
      const Tile tn = nt < ntiles ? tiles[nt] : Tile{};
      if (threadIdx.x == CLAIMER) s_claim[(j & 1) ^ 1] = claim();
      auto next_types = [&](TileTypes<SH::NPT>& t) {
        if (nt < ntiles) t = load_types<SH>(tn, P, V.tin, threadIdx.x);
      };
      bulk_tile<SH, TF, TG, R, NS>(tl, V, P, src, [] {}, next_types, true, tt, acc, s_pot[buf], s_t[buf],
                                   s_m[buf]);
      buf ^= 1;
      ++j;
      ti = nt;
      tl = tn;
    }
    flush_acc(acc, V.scal, V.cur);
  } else {
    // a batch: consecutive tiles of a block often belong to one instance (a
    // large member spans many tiles), so the instance's view and step limit
    // are read, and its maximum and status flushed, only when the instance
    // changes; tile descriptors ride a tile ahead
    int ti = blockIdx.x;
    Tile tl = ti < ntiles ? tiles[ti] : Tile{};
    int vinst = -1;            // instance of the run in progress
    bool vlive = false;        // ... below its step limit
    bool have_tt = false;      // tt holds the current tile's types
    StepView<TF, TG, R> V{};
    if (threadIdx.x == CLAIMER) s_claim[0] = claim();
    __syncthreads();
    int j = 0;
    while (ti < ntiles) {
      const int nt = s_claim[j & 1];
      const Tile tn = nt < ntiles ? tiles[nt] : Tile{};
      if (threadIdx.x == CLAIMER) s_claim[(j & 1) ^ 1] = claim();
      if (tl.inst != vinst) {
        if (vlive) flush_acc(acc, V.scal, V.cur);
        vinst = tl.inst;
        const DevInst* I = insts + vinst;
        vlive = I->scal[S_STEP] < I->scal[S_LIMIT];
        if (vlive) V = step_view<TF, TG, R>(I);
        have_tt = false;
      }
      if (vlive) {
        const DevParams& P = insts[vinst].P;
        if (!have_tt) tt = load_types<SH>(tl, P, V.tin, threadIdx.x);
        const bool same = nt < ntiles && tn.inst == vinst;
        auto next_types = [&](TileTypes<SH::NPT>& t) {
          if (same) t = load_types<SH>(tn, P, V.tin, threadIdx.x);
        };
        const GlobalSrc<TF, TG, R, NS> src{V.fin, V.gin, V.N};
        bulk_tile<SH, TF, TG, R, NS>(tl, V, P, src, [] {}, next_types, true, tt, acc, s_pot[buf], s_t[buf],
                                     s_m[buf]);
        buf ^= 1;
        have_tt = same;
      } else {
        // a frozen member: nothing to compute, but the claim made during this
        // tile is read after a barrier
        __syncthreads();
      }
      ++j;
      ti = nt;
      tl = tn;
    }
    if (vlive) flush_acc(acc, V.scal, V.cur);
  }
}

// ---------------------------------------------------------------- staged

// Shared-memory stage of the staged kernel: the D2Q9 box of a tile (both
// components, the tile plus a ring of one node in y and four in x, so that
// the box's x origin stays on a 16-byte boundary) and, when STAGE_G, the D2Q5
// box of the tile itself, as the TMA unit writes them (x fastest, then y,
// then plane).
template <class SH, class TG, int NS, bool STAGE_G = true>
struct StageCfg {
  static constexpr int HX = stage_halo_x(SH::NPT);
  static constexpr int BX = SH::TX + 2 * HX, BY = SH::TY + 2;
  static constexpr int FBYTES = BX * BY * 18 * 4;
  static constexpr int GBYTES = (NS > 0 && STAGE_G) ? SH::TX * SH::TY * 5 * NS * (int)sizeof(TG) : 0;
  static constexpr int FOFF = 0;
  static constexpr int GOFF = ((FBYTES + 127) / 128) * 128;
  static constexpr int STAGE = GOFF + ((GBYTES + 127) / 128) * 128;
  static constexpr uint32_t TX_BYTES = FBYTES + GBYTES;
};

// Population source of the staged kernel: the tile's own populations and the
// ring densities come from the shared stage; nodes that lie across a periodic
// edge (outside the box) are read from global memory.  Without STAGE_G the
// solute populations are read from global memory, and the kernel re-reads the
// D2Q9 populations from the stage where it needs them instead of holding them
// in registers across the tile's barrier (kReread).
template <class SH, class TG, int NS, bool STAGE_G = true>
struct StageSrc {
  using C = StageCfg<SH, TG, NS, STAGE_G>;
  static constexpr bool kReread = !STAGE_G;
  const float* fs;     // stage D2Q9 box
  const TG* gs_;       // stage D2Q5 box (STAGE_G) or the solute populations in global memory
  const float* fin;
  int N, nx, ny, x0, y0;
  static_assert(!STAGE_G || SH::NPT == 1, "the staged D2Q5 box is indexed by thread");
  // A thread position beyond the lattice edge of a partial tile stands for the
  // wrapped node across a periodic edge (idx >= 0 only then): not in the box.
  // ly: the node's row in the tile.
  __device__ __forceinline__ void own_f(int idx, int ly, float* f1, float* f2) const {
    const int tx = threadIdx.x % SH::TX;
    if (x0 + tx < nx && y0 + ly < ny) {
      const float* b = fs + (ly + 1) * C::BX + (tx + C::HX);
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        f1[a] = b[a * C::BX * C::BY];
        f2[a] = b[(9 + a) * C::BX * C::BY];
      }
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        f1[a] = ld<float>(fin + a * N + idx);
        f2[a] = ld<float>(fin + (9 + a) * N + idx);
      }
    }
  }
  // one component's populations (as own_f)
  __device__ __forceinline__ void own_fc(int idx, int ly, int comp, float* f) const {
    const int tx = threadIdx.x % SH::TX;
    if (x0 + tx < nx && y0 + ly < ny) {
      const float* b = fs + (ly + 1) * C::BX + (tx + C::HX) + comp * 9 * C::BX * C::BY;
#pragma unroll
      for (int a = 0; a < 9; ++a) f[a] = b[a * C::BX * C::BY];
    } else {
#pragma unroll
      for (int a = 0; a < 9; ++a) f[a] = ld<float>(fin + (comp * 9 + a) * N + idx);
    }
  }
  __device__ __forceinline__ void own_g(int node, float (*g)[5]) const {
    if constexpr (STAGE_G) {
      const int i = threadIdx.x;
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int a = 0; a < 5; ++a) g[k][a] = ldc<float>(gs_ + (k * 5 + a) * SH::TX * SH::TY + i);
    } else {
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int a = 0; a < 5; ++a) g[k][a] = ld<float>(gs_ + (k * 5 + a) * N + node);
    }
  }
  // a ring node inside the lattice and the box: from the box; otherwise
  // (across a periodic edge, or a side column of a box without x halo) from
  // global memory
  __device__ __forceinline__ void ring_density(int ring_idx, int rx, int ry, float& d1, float& d2) const {
    const bool in_box = C::HX > 0 || (rx >= x0 && rx < x0 + SH::TX);
    if (rx >= 0 && rx < nx && ry >= 0 && ry < ny && in_box) {
      const float* b = fs + (ry - y0 + 1) * C::BX + (rx - x0 + C::HX);
      float s1 = b[0], s2 = b[9 * C::BX * C::BY];
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        s1 += b[a * C::BX * C::BY];
        s2 += b[(9 + a) * C::BX * C::BY];
      }
      d1 = s1;
      d2 = s2;
    } else {
      d1 = density_shifted<float>(fin, (long long)N, ring_idx);
      d2 = density_shifted<float>(fin + 9 * N, (long long)N, ring_idx);
    }
  }
};

// Issue the TMA copies of the tile `d` into a stage (one thread), from the
// population maps of its step.
template <class SH, class TG, int NS, bool STAGE_G>
__device__ __forceinline__ void stage_issue(const Tile& d, const CUtensorMap* mf, const CUtensorMap* mg,
                                            unsigned char* stage, uint64_t* bar) {
  using C = StageCfg<SH, TG, NS, STAGE_G>;
  mbar_arrive_expect_tx(bar, C::TX_BYTES);
  tma_load_3d(stage + C::FOFF, mf, bar, d.x0 - C::HX, d.y0 - 1, 0);
  if constexpr (NS > 0 && STAGE_G) tma_load_3d(stage + C::GOFF, mg, bar, d.x0, d.y0, 0);
}

// Staged bulk kernel (FP32 populations): the TMA unit brings each tile's
// population box into shared memory ahead of its use, so the populations'
// DRAM latency overlaps arithmetic instead of stalling it.  Two stages in
// both modes; the arithmetic is the plain kernel's, value for value.
//   MODE 1: each stage holds the tile's D2Q9 box and its D2Q5 box; a tile
//     reads its stage only before the tile's barrier (into registers), so the
//     copy of tile j+2 is issued into tile j's stage right after tile j's
//     barrier; two blocks per SM fit.
//   MODE 2: each stage holds the D2Q9 box only; the solute populations are
//     read from global memory where they are used, and the D2Q9 populations
//     are read from the stage again for the collision instead of being held
//     in registers across the barrier, so the kernel fits three blocks per SM
//     (fewer registers, 70 KB of shared memory).  The stage of tile j is read
//     until the end of tile j, so the copy of tile j+1 goes into tile j-1's
//     stage right after tile j's barrier.
// Each block takes tiles blockIdx.x and blockIdx.x + gridDim.x, then claims
// further tiles in list order from a counter (lane 0 of the last warp, which
// has no ring node and so time to spare before the barrier, claims tile j+2
// while the block computes tile j-1 and shares it through shared memory), so
// that blocks that meet cheap tiles take more of them and the launch does not
// end with a few blocks still working; tile descriptors ride two tiles ahead
// in registers.  SINGLE: every tile belongs to the one simulation
// at insts[0], whose parameter block comes as a kernel argument (read from the
// constant bank, uniform across the grid); its step view and population maps
// are read once and the maximum and status flushed once at the end.
// Otherwise (a batch) the view and step limit are read, the population maps
// acquired and the accumulators flushed once per run of consecutive tiles of
// one instance; tiles of a member frozen at its step limit are copied but not
// computed.
//
// Smem bytes of the dynamic stages of a mode.
template <class SH, class TG, int NS, int MODE>
constexpr int tma_smem() {
  return 2 * StageCfg<SH, TG, NS, MODE == 1>::STAGE;
}

// Resident blocks per SM of a staged variant: MODE 1 two; MODE 2 three with
// one node per thread, two with two (a larger box, more registers).
template <class SH, int MODE>
constexpr int tma_min_blocks() {
  return (MODE == 1 || SH::NPT > 1) ? 2 : 3;
}

template <class SH, int SHAPE, class TG, int NS, int MODE, bool SINGLE>
__global__ void __launch_bounds__(NTHREADS, tma_min_blocks<SH, MODE>())
    k_bulk_tma(const Tile* __restrict__ tiles, int ntiles, const DevInst* __restrict__ insts,
               const __grid_constant__ DevParams Pk) {
  constexpr bool SG = MODE == 1;   // solute box staged too
  using C = StageCfg<SH, TG, NS, SG>;
  using R = float;
  using View = StepView<float, TG, R>;
  extern __shared__ __align__(128) unsigned char dyn[];
  __shared__ Pot<R> s_pot[2][SH::EXT];
  __shared__ uint8_t s_t[2][SH::EXT], s_m[2][SH::EXT];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int s_claim[2];

  const int stride = gridDim.x;
  constexpr int CLAIMER = NTHREADS - 32;   // the thread that claims tiles
  View V{};
  if constexpr (SINGLE) {
    // one simulation: all tiles are live or none is
    if (!(insts->scal[S_STEP] < insts->scal[S_LIMIT])) return;
    V = step_view<float, TG, R>(insts);
  }
  // the instance whose population maps the issuing thread acquired last (batch)
  int iss_inst = -1, iss_cur = 0;
  // copies of a tile into a stage (thread 0)
  auto issue = [&](const Tile& d, unsigned char* stage, uint64_t* bar) {
    const DevInst* Ip = insts + (SINGLE ? 0 : d.inst);
    int cur = V.cur;
    if constexpr (!SINGLE) {
      if (d.inst != iss_inst) {
        iss_inst = d.inst;
        iss_cur = int(Ip->scal[S_STEP] & 1ULL);
        tensormap_acquire(&Ip->tmf[SHAPE][iss_cur]);
        if constexpr (NS > 0 && SG) tensormap_acquire(&Ip->tmg[SHAPE][iss_cur]);
      }
      cur = iss_cur;
    }
    stage_issue<SH, TG, NS, SG>(d, &Ip->tmf[SHAPE][cur], &Ip->tmg[SHAPE][cur], stage, bar);
  };
  // the next tile of this block from the launch's claim counter (in the first
  // instance; V.scal is that instance's for one simulation)
  auto claim = [&] {
    unsigned long long* c = (SINGLE ? V.scal : insts->scal) + S_TILES;
    return 2 * stride + (int)atomicAdd(c, 1ULL);
  };
  // tile descriptors ride two tiles ahead in registers
  int ti = blockIdx.x;
  int t1 = ti + stride;
  Tile d0 = ti < ntiles ? tiles[ti] : Tile{};
  Tile d1 = t1 < ntiles ? tiles[t1] : Tile{};
  if (threadIdx.x == CLAIMER) s_claim[0] = claim();
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
    if constexpr (SINGLE) {
      tensormap_acquire(&insts->tmf[SHAPE][V.cur]);
      if constexpr (NS > 0 && SG) tensormap_acquire(&insts->tmg[SHAPE][V.cur]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ti < ntiles) issue(d0, dyn, &bars[0]);
    if (t1 < ntiles) issue(d1, dyn + C::STAGE, &bars[1]);
  }
  TileTypes<SH::NPT> tt;
  bool have_tt = false;             // tt holds the current tile's types
  int vinst = SINGLE ? 0 : -1;      // instance of the run in progress (batch)
  bool vlive = SINGLE;              // ... below its step limit
  TileAcc<R> acc{R(-1.0 / 0.0), 0u};
  int j = 0;                        // tiles processed by this block
  uint32_t phase = 0;               // parity bit per stage
  while (ti < ntiles) {
    const int b = j & 1;                          // stage and shared buffers of this tile
    // tile j+2 was claimed during tile j-1 (or before the first tile); claim
    // tile j+3 now (read at the top of tile j+1, after this tile's barrier)
    const int t2 = s_claim[b];
    const Tile d2 = t2 < ntiles ? tiles[t2] : Tile{};
    if (threadIdx.x == CLAIMER) s_claim[b ^ 1] = claim();
    const bool ok = mbar_wait_bounded(&bars[b], (phase >> b) & 1u);
    phase ^= 1u << b;
    if constexpr (!SINGLE) {
      if (d0.inst != vinst) {
        // a new run of tiles of one instance: close the previous one and read
        // this instance's view once
        if (vlive) flush_acc(acc, V.scal, V.cur);
        vinst = d0.inst;
        const DevInst* I = insts + vinst;
        vlive = I->scal[S_STEP] < I->scal[S_LIMIT];
        if (vlive) V = step_view<float, TG, R>(I);
        have_tt = false;
      }
    }
    unsigned char* stage = dyn + b * C::STAGE;
    // after the tile's barrier: MODE 1 refills this tile's stage with tile
    // j+2; MODE 2 refills the other stage (tile j-1 is done with it: every
    // thread has passed this barrier) with tile j+1, from the second tile on
    auto refill = [&] {
      if (threadIdx.x != 0) return;
      if constexpr (MODE == 1) {
        if (t2 < ntiles) issue(d2, stage, &bars[b]);
      } else {
        if (j >= 1 && t1 < ntiles) issue(d1, dyn + (b ^ 1) * C::STAGE, &bars[b ^ 1]);
      }
    };
    bool stop;
    if (vlive) {
      const DevParams& P = SINGLE ? Pk : insts[vinst].P;
      if (!have_tt) tt = load_types<SH>(d0, P, V.tin, threadIdx.x);
      const bool same = t1 < ntiles && (SINGLE || d1.inst == vinst);
      auto next_types = [&](TileTypes<SH::NPT>& t) {
        if (same) t = load_types<SH>(d1, P, V.tin, threadIdx.x);
      };
      const StageSrc<SH, TG, NS, SG> src{(const float*)(stage + C::FOFF),
                                         SG ? (const TG*)(stage + C::GOFF) : V.gin, V.fin, V.N, P.nx, P.ny, d0.x0,
                                         d0.y0};
      stop = bulk_tile<SH, float, TG, R, NS>(d0, V, P, src, refill, next_types, ok, tt, acc, s_pot[b], s_t[b],
                                             s_m[b]);
      have_tt = same;
    } else {
      // a member frozen at its step limit: its copy landed, nothing to
      // compute; once every thread is past its wait the stage may be reused
      stop = __syncthreads_or(ok ? 0 : 1) != 0;
      if (!stop) refill();
    }
    if (stop) {
      // a wait gave up: record it, let the copies still in flight land
      // (bounded waits: this tile's stage, and the other stage when it holds
      // a copy not waited for yet: always in MODE 1 (tile j+1), in MODE 2
      // only on the first tile (tile 1, issued up front)), and leave
      if (vlive) flush_acc(acc, V.scal, V.cur);
      if (threadIdx.x == 0) {
        atomicOr(&insts[SINGLE ? 0 : d0.inst].scal[S_STATUS], (unsigned long long)ST_TIMEOUT);
        mbar_wait_bounded(&bars[b], ((phase >> b) & 1u) ^ 1u);
        if ((MODE == 1 || j == 0) && t1 < ntiles) mbar_wait_bounded(&bars[b ^ 1], (phase >> (b ^ 1)) & 1u);
      }
      return;
    }
    ++j;
    ti = t1;
    t1 = t2;
    d0 = d1;
    d1 = d2;
  }
  if (vlive) flush_acc(acc, V.scal, V.cur);
}

}  // namespace pslbm
