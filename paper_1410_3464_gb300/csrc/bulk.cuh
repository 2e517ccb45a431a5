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
    R s = ld<R>(gk + node);
#pragma unroll
    for (int a = 1; a < 5; ++a) s += ld<R>(gk + a * N + node);
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

// Types of one tile for this thread: its own ext position and (tid < SH::RING)
// one ring position.
struct TileTypes {
  uint8_t own, ring;
  int own_idx, ring_idx;
};

template <class SH>
__device__ __forceinline__ TileTypes load_types(const Tile* tiles, const DevInst* insts, int ti, int tid) {
  TileTypes tt;
  const Tile tl = tiles[ti];
  const DevInst* Ip = insts + tl.inst;
  const int cur = int(Ip->scal[S_STEP] & 1ULL);
  const uint8_t* tin = Ip->type[cur];
  const int tx = tid % SH::TX, ty = tid / SH::TX;
  tt.own = ext_type(Ip->P, tin, tl.x0, tl.y0, tx + 1, ty + 1, tt.own_idx);
  tt.ring = T_WALL;
  tt.ring_idx = -1;
  if (tid < SH::RING) {
    int ex, ey;
    ring_pos<SH>(tid, ex, ey);
    tt.ring = ext_type(Ip->P, tin, tl.x0, tl.y0, ex, ey, tt.ring_idx);
  }
  return tt;
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

// Reservoir node: push its equilibrium state (densities of reservoir_rho,
// velocity of the node next to it along x) into its fluid neighbours, and the
// solute equilibrium into its liquid neighbours when it is itself liquid.
template <class SH, class R, class TF, class TG, int NS>
__device__ __noinline__ void reservoir_push(const DevParams& P, const uint8_t* tin, const TF* fin, const TG* gin,
                                            TF* fout, TG* gout, int N, int x, int y, uint8_t t,
                                            unsigned long long step, R theta, const uint8_t* s_t,
                                            const uint8_t* s_m, int eo) {
  const int node = y * P.nx + x;
  const R sh1 = rp<R>(P).shift_f[0], sh2 = rp<R>(P).shift_f[1];
  double a_, b_;
  reservoir_rho(P, t, step, t == T_OUTLET && outlet_up_liquid<R, TF>(P, tin, fin, N, node, theta), a_, b_);
  const R r1 = R(a_), r2 = R(b_);
  R ux = R(0), uy = R(0);
  int xn, yn;
  const int dx = (t == T_INLET) ? 1 : -1;
  if (nbr(P, x, y, dx, 0, xn, yn)) {
    const int nn = yn * P.nx + xn;
    if (is_fluid(tin[nn] & T_MASK)) {
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
      const R rt = (sh1 + e1) + (sh2 + e2);
      ux = jx / rt;
      uy = jy / rt;
    }
  }
  const R uu = R(1.5) * (ux * ux + uy * uy);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const R rho = s == 0 ? r1 : r2;
    const R dr = rho - (s == 0 ? sh1 : sh2);
    TF* fo = fout + s * 9 * N;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const int en = eo + EY(a) * SH::EXT_X + EX(a);
      if (!is_fluid(s_t[en])) continue;
      const R eu = R(EX(a)) * ux + R(EY(a)) * uy;
      const R w = w9<R>(a);
      const R feq = w * (dr + rho * (R(3) * eu + R(4.5) * eu * eu - uu));
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
        const int ew = eo - 1;
#pragma unroll
        for (int k = 0; k < NS; ++k) Cr[k] = R(0);
        if (is_fluid(s_t[ew]) && s_m[ew] && nbr(P, x, y, -1, 0, xn, yn))
          conc_at<R, TG, NS>(gin, N, yn * P.nx + xn, P, Cr);
      }
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const R Ja = rp<R>(P).Ja[k];
#pragma unroll
        for (int a = 1; a < 5; ++a) {
          const int en = eo + EY(a) * SH::EXT_X + EX(a);
          if (!(is_fluid(s_t[en]) && s_m[en])) continue;
          const R eu = R(EX(a)) * ux + R(EY(a)) * uy;
          const R geq = Ja * (Cr[k] - rp<R>(P).shift_c[k]) + R(0.5) * Cr[k] * eu;
          nbr(P, x, y, EX(a), EY(a), xn, yn);
          st<TG, R>(gout + (k * 5 + a) * N + yn * P.nx + xn, geq);
        }
      }
    }
  }
}

// Minimum resident blocks per SM the register allocation targets: FP32
// compute keeps three 256-thread blocks per SM; FP64 (twice the registers per
// value, bound by FP64 arithmetic anyway) two.
#ifndef PSLBM_BULK_MINB
#define PSLBM_BULK_MINB 3
#endif
template <class R>
constexpr int bulk_min_blocks() {
  return sizeof(R) == 8 ? 2 : PSLBM_BULK_MINB;
}

template <class SH, class TF, class TG, class R, int NS>
__global__ void __launch_bounds__(NTHREADS, bulk_min_blocks<R>()) k_bulk(const Tile* __restrict__ tiles, int ntiles,
                                                                         const DevInst* __restrict__ insts) {
  __shared__ R s_psi[2][SH::EXT], s_phi1[2][SH::EXT], s_phi2[2][SH::EXT];
  __shared__ uint8_t s_t[2][SH::EXT], s_m[2][SH::EXT];

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int tx = tid % SH::TX, ty = tid / SH::TX;
  const int eo = (ty + 1) * SH::EXT_X + (tx + 1);
  int er = -1;
  if (tid < SH::RING) {
    int ex, ey;
    ring_pos<SH>(tid, ex, ey);
    er = ey * SH::EXT_X + ex;
  }

  int ti = blockIdx.x;
  int buf = 0;
  TileTypes tt;
  if (ti < ntiles) tt = load_types<SH>(tiles, insts, ti, tid);

  for (; ti < ntiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const DevInst* Ip = insts + tl.inst;
    const DevParams& P = Ip->P;
    const int N = (int)Ip->N;
    const int nx = P.nx;
    const unsigned long long step = Ip->scal[S_STEP];
    if (step >= Ip->scal[S_LIMIT]) {
      // frozen instance: keep the type prefetch in step with the tile walk; the
      // stage buffer is not toggled, so no barrier is skipped for it
      if (ti + (int)gridDim.x < ntiles) tt = load_types<SH>(tiles, insts, ti + gridDim.x, tid);
      continue;
    }
    const int cur = int(step & 1ULL);
    const TF* __restrict__ fin = (const TF*)Ip->f[cur];
    TF* __restrict__ fout = (TF*)Ip->f[cur ^ 1];
    const TG* __restrict__ gin = (const TG*)Ip->g[cur];
    TG* __restrict__ gout = (TG*)Ip->g[cur ^ 1];
    const uint8_t* __restrict__ tin = Ip->type[cur];
    uint8_t* __restrict__ tout = Ip->type[cur ^ 1];
    const R theta = R(0.5 * ord_dec(Ip->scal[S_MAX0 + cur]));
    const R sh1 = rp<R>(P).shift_f[0], sh2 = rp<R>(P).shift_f[1];
    // tiles whose ring is inside the domain need no wrap arithmetic
    const bool inner = tl.x0 >= 1 && tl.y0 >= 1 && tl.x0 + SH::TX + 1 <= nx && tl.y0 + SH::TY + 1 <= P.ny;
    R* sp = s_psi[buf];
    R* sq1 = s_phi1[buf];
    R* sq2 = s_phi2[buf];
    uint8_t* st_ = s_t[buf];
    uint8_t* sm_ = s_m[buf];
    unsigned status = 0;

    // ---- phase 1: issue population loads (own node and one ring node)
    const int x = tl.x0 + tx, y = tl.y0 + ty;
    const bool own = x < nx && y < P.ny;
    const int node = y * nx + x;
    const uint8_t own_t = tt.own;
    const uint8_t ring_t = tt.ring;
    const int own_idx = tt.own_idx, ring_idx = tt.ring_idx;
    const uint8_t t = own ? own_t : T_WALL;
    R f1[9], f2[9];
    R gs[NS > 0 ? NS : 1][5];
    const bool own_fluid = is_fluid(own_t) && own_idx >= 0;
    if (own_fluid) {
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        f1[a] = ld<R>(fin + a * N + own_idx);
        f2[a] = ld<R>(fin + (9 + a) * N + own_idx);
      }
    }
    if constexpr (NS > 0) {
      if (own && own_t == T_LIQUID) {
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int a = 0; a < 5; ++a) gs[k][a] = ld<R>(gin + (k * 5 + a) * N + node);
      }
    }
    R r1r = R(0), r2r = R(0);
    if (tid < SH::RING && is_fluid(ring_t)) {
      r1r = sh1 + density_shifted<R>(fin, (long long)N, ring_idx);
      r2r = sh2 + density_shifted<R>(fin + 9 * N, (long long)N, ring_idx);
    }
    // prefetch the next tile's node types
    if (ti + (int)gridDim.x < ntiles) tt = load_types<SH>(tiles, insts, ti + gridDim.x, tid);

    // ---- moments of the own node (Eq. 9), potentials -> shared
    R rho1 = R(0), rho2 = R(0), d1 = R(0), d2 = R(0), j1x = R(0), j1y = R(0), j2x = R(0), j2y = R(0);
    {
      R r1 = R(0), r2 = R(0);
      if (own_fluid) {
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
        rho1 = sh1 + d1;
        rho2 = sh2 + d2;
        r1 = rho1;
        r2 = rho2;
        if (!(rho1 == rho1 && rho2 == rho2)) status |= ST_NONFINITE;
      } else if (is_res(own_t)) {
        double a, b;
        reservoir_rho(P, own_t, step,
                      own_t == T_OUTLET && outlet_up_liquid<R, TF>(P, tin, fin, N, own_idx, theta), a, b);
        r1 = R(a);
        r2 = R(b);
      }
      R ps = R(0), p1 = R(0), p2 = R(0);
      if (is_live(own_t)) potentials<R>(P, r1, r2, ps, p1, p2, status);
      sp[eo] = ps;
      sq1[eo] = p1;
      sq2[eo] = p2;
      st_[eo] = own_t;
      sm_[eo] = (is_live(own_t) && r1 > theta) ? 1 : 0;
    }
    if (tid < SH::RING) {
      R r1 = r1r, r2 = r2r;
      if (is_res(ring_t)) {
        double a, b;
        reservoir_rho(P, ring_t, step,
                      ring_t == T_OUTLET && outlet_up_liquid<R, TF>(P, tin, fin, N, ring_idx, theta), a, b);
        r1 = R(a);
        r2 = R(b);
      }
      R ps = R(0), p1 = R(0), p2 = R(0);
      if (is_live(ring_t)) potentials<R>(P, r1, r2, ps, p1, p2, status);
      sp[er] = ps;
      sq1[er] = p1;
      sq2[er] = p2;
      st_[er] = ring_t;
      sm_[er] = (is_live(ring_t) && r1 > theta) ? 1 : 0;
    }
    __syncthreads();

    R mymax = R(-1.0 / 0.0);
    if (own && is_fluid(t)) {
      mymax = rho1;
      // ---- forces (Eqs. 11, 14a/b, 16) with neutral solid neighbours
      const R psc = sp[eo], p1c = sq1[eo], p2c = sq2[eo];
      R spx = 0, spy = 0, s2x = 0, s2y = 0, s1x = 0, s1y = 0, ssx = 0, ssy = 0;
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        const int en = eo + EY(a) * SH::EXT_X + EX(a);
        const bool lv = is_live(st_[en]);
        const R w = wf<R>(a);
        const R vp = w * (lv ? sp[en] : psc);
        const R v2 = w * (lv ? sq2[en] : p2c);
        const R v1 = w * (lv ? sq1[en] : p1c);
        const R vs = lv ? R(0) : w;
        if (EX(a) > 0) { spx += vp; s2x += v2; s1x += v1; ssx += vs; }
        if (EX(a) < 0) { spx -= vp; s2x -= v2; s1x -= v1; ssx -= vs; }
        if (EY(a) > 0) { spy += vp; s2y += v2; s1y += v1; ssy += vs; }
        if (EY(a) < 0) { spy -= vp; s2y -= v2; s1y -= v1; ssy -= vs; }
      }
      const R G11 = rp<R>(P).G11, G12 = rp<R>(P).G12, G21 = rp<R>(P).G21, w1 = rp<R>(P).w_adh[0], w2 = rp<R>(P).w_adh[1];
      const R F1x = -G11 * psc * spx - G12 * p1c * s2x - w1 * psc * ssx + rho1 * rp<R>(P).gx;
      const R F1y = -G11 * psc * spy - G12 * p1c * s2y - w1 * psc * ssy + rho1 * rp<R>(P).gy;
      const R F2x = -G21 * p2c * s1x - w2 * rho2 * ssx + rho2 * rp<R>(P).gx;
      const R F2y = -G21 * p2c * s1y - w2 * rho2 * ssy + rho2 * rp<R>(P).gy;
      // ---- velocities (Eqs. 17-19)
      const R it1 = rp<R>(P).inv_tau[0], it2 = rp<R>(P).inv_tau[1];
      const R rden = rrcp<R>(rho1 * it1 + rho2 * it2);
      const R upx = (j1x * it1 + j2x * it2) * rden;
      const R upy = (j1y * it1 + j2y * it2) * rden;
      const R q1 = rho1 != R(0) ? rp<R>(P).tau[0] * rrcp<R>(rho1) : R(0);
      const R q2 = rho2 != R(0) ? rp<R>(P).tau[1] * rrcp<R>(rho2) : R(0);
      const R u1x = upx + F1x * q1, u1y = upy + F1y * q1;
      const R u2x = upx + F2x * q2, u2y = upy + F2y * q2;
      const R rrt = rrcp<R>(rho1 + rho2);
      const R urx = (j1x + j2x + R(0.5) * (F1x + F2x)) * rrt;
      const R ury = (j1y + j2y + R(0.5) * (F1y + F2y)) * rrt;

      const bool liq = sm_[eo] != 0;
      tout[node] = liq ? T_LIQUID : T_GAS;

      // neighbour indices for the push (constant offsets away from the edges)
      int nb[9];
#pragma unroll
      for (int a = 1; a < 9; ++a) nb[a] = inner ? node + EX(a) + EY(a) * nx : nbr_index(P, x, y, EX(a), EY(a));

      // ---- solutes: concentration with the Step-2 amendment, sources
      R S1 = R(0), S2 = R(0);
      R C[NS > 0 ? NS : 1];
      R Sk[NS > 0 ? NS : 1];
      if constexpr (NS > 0) {
        if (liq) {
          const bool appear = (t == T_GAS);
          bool vnb = false;
#pragma unroll
          for (int b = 1; b < 5; ++b) {
            const int en = eo + EY(b) * SH::EXT_X + EX(b);
            vnb |= (st_[en] == T_LIQUID && sm_[en] == 0);
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
                gs[k][a] = appear ? ja * (cb[k] + dC[k]) - ja * rp<R>(P).shift_c[k] : gs[k][a] + ja * dC[k];
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
          if (P.iA == -2) CA = rmax<R>(R(0), rp<R>(P).c_total_per_rho1 * rho1 - tot);
          R R1 = rp<R>(P).k1 * CA;
          if (P.has_rev) R1 -= rp<R>(P).k1_inv_Keq * CB * rsqrt_<R>(rmax<R>(rho2 * rp<R>(P).inv_M_C, R(0)));
          const R R3 = rp<R>(P).k3 * CB * CE;
#pragma unroll
          for (int k = 0; k < NS; ++k) Sk[k] = rp<R>(P).cR1[k] * R1 + rp<R>(P).cR3[k] * R3;
          S1 = -rp<R>(P).gas_yield * R1;
          S2 = rp<R>(P).gas_yield * R1;
        }
      }

      // ---- fluid collision (Eq. 6, Eq. 8 at u_eq) and push streaming
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const R rho = s == 0 ? rho1 : rho2;
        const R dr = s == 0 ? d1 : d2;
        const R ux = s == 0 ? u1x : u2x, uy = s == 0 ? u1y : u2y;
        const R itau = s == 0 ? it1 : it2;
        const R Ssrc = s == 0 ? S1 : S2;
        const R uu = R(1.5) * (ux * ux + uy * uy);
        TF* fo = fout + s * 9 * N;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
          const R fa = s == 0 ? f1[a] : f2[a];
          const R eu = R(EX(a)) * ux + R(EY(a)) * uy;
          const R w = w9<R>(a);
          const R feq = w * (dr + rho * (R(3) * eu + R(4.5) * eu * eu - uu));
          const R fs = fa - (fa - feq) * itau + w * Ssrc;
          if (a == 0) {
            st<TF, R>(fo + node, fs);
            continue;
          }
          const uint8_t tn = st_[eo + EY(a) * SH::EXT_X + EX(a)];
          if (is_fluid(tn))
            st<TF, R>(fo + a * N + nb[a], fs);
          else if (!is_res(tn))
            st<TF, R>(fo + OPP(a) * N + node, fs);
        }
      }

      // ---- solute collision (Eqs. 20-22 with u_r) and push streaming
      if constexpr (NS > 0) {
        if (liq) {
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            const R eu = R(EX(a)) * urx + R(EY(a)) * ury;
            int dst = node, slot = a;            // rest population stays
            bool keep = true;
            if (a > 0) {
              const int en = eo + EY(a) * SH::EXT_X + EX(a);
              const uint8_t tn = st_[en];
              const bool mn = sm_[en] != 0;
              if (is_fluid(tn) && mn) {
                dst = nb[a];                     // into a liquid neighbour
              } else if (is_res(tn) && mn) {
                keep = false;                    // outflow into a liquid reservoir
              } else {
                slot = OPP(a);                   // no-flux / mineral: bounce back
              }
            }
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              const R ja = a == 0 ? rp<R>(P).J0[k] : rp<R>(P).Ja[k];
              const R geq = ja * (C[k] - rp<R>(P).shift_c[k]) + R(0.5) * C[k] * eu;
              const R gst = gs[k][a] - (gs[k][a] - geq) * rp<R>(P).inv_tau_g[k] + ja * Sk[k];
              if (keep) st<TG, R>(gout + (k * 5 + slot) * N + dst, gst);
            }
          }
        } else {
          // gas node: no solute
#pragma unroll
          for (int k = 0; k < NS; ++k) {
#pragma unroll
            for (int a = 0; a < 5; ++a)
              st<TG, R>(gout + (k * 5 + a) * N + node, -(a == 0 ? rp<R>(P).J0[k] : rp<R>(P).Ja[k]) * rp<R>(P).shift_c[k]);
          }
        }
      }
    } else if (own) {
      if (is_res(t)) reservoir_push<SH, R, TF, TG, NS>(P, tin, fin, gin, fout, gout, N, x, y, t, step, theta, st_, sm_, eo);
      tout[node] = t;
    }

    // ---- warp max of rho_1 over fluid nodes (next step's threshold) and status
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = rmax<R>(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0) {
      if (mymax > R(-1.0 / 0.0)) {
        // exact maximum; the atomic only when it can raise the slot
        const unsigned long long enc = ord_enc(double(mymax));
        unsigned long long* slot = &Ip->scal[S_MAX0 + (cur ^ 1)];
        if (enc > *(volatile unsigned long long*)slot) atomicMax(slot, enc);
      }
      if (status) atomicOr(&Ip->scal[S_STATUS], (unsigned long long)status);
    }
    buf ^= 1;
  }
}

}  // namespace pslbm
