// Fused bulk kernel of one time step (Chen, Kang et al., arXiv 1410.3464,
// Sections 3-4, numerical procedure of Section 4.7):
//   moments (Eq. 9) -> liquid/gas marking (Section 4.5) -> psi/phi (Eqs. 13,
//   15) staged in shared memory with a one-node ring -> forces (Eqs. 11, 14,
//   16) -> velocities (Eqs. 17-19) -> concentration amendment at marking
//   changes (Step 2) -> homogeneous sources (Eqs. 5a, 5c, 27, 28) -> D2Q9
//   collide and push (Eq. 6, halfway bounce-back) -> D2Q5 collide and push
//   (Eqs. 20-22) with no-flux and reactive links (Eqs. 29-31).
//
// State between steps is the pre-collision populations; streaming is a push
// into the other buffer of a ping-pong pair, so every population is read once
// and written once.  The ring nodes' densities are recomputed from their
// populations (read through L2), so psi at radius 2 is never stored in HBM.
#pragma once
#include "device.cuh"

namespace pslbm {

// Ring position r (0..RING-1) -> ext coordinates.
__device__ __forceinline__ void ring_pos(int r, int& ex, int& ey) {
  if (r < EXT_X) {
    ex = r;
    ey = 0;
  } else if (r < 2 * EXT_X) {
    ex = r - EXT_X;
    ey = EXT_Y - 1;
  } else if (r < 2 * EXT_X + (EXT_Y - 2)) {
    ex = 0;
    ey = 1 + (r - 2 * EXT_X);
  } else {
    ex = EXT_X - 1;
    ey = 1 + (r - 2 * EXT_X - (EXT_Y - 2));
  }
}

// Marking of an arbitrary node from global memory (same arithmetic as the
// shared-memory path, so both give the same answer bit for bit).
template <class R, class TF>
__device__ __forceinline__ bool liquid_at(const DevParams& P, const uint8_t* tin, const TF* fin, long long N,
                                          long long node, double theta) {
  uint8_t t = tin[node] & T_MASK;
  if (!is_fluid(t)) return false;
  R rho1 = R(P.shift_f[0]) + density_shifted<R>(fin, N, node);
  return double(rho1) > theta;
}

template <class R, class TG, int NS>
__device__ __forceinline__ void conc_at(const TG* gin, long long N, long long node, const DevParams& P, R* C) {
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const TG* gk = gin + (long long)k * 5 * N;
    R s = ld<R>(gk + node);
#pragma unroll
    for (int a = 1; a < 5; ++a) s += ld<R>(gk + a * N + node);
    C[k] = R(P.shift_c[k]) + s;
  }
}

template <class TF, class TG, class R, int NS>
__global__ void __launch_bounds__(NTHREADS) k_bulk(const Tile* __restrict__ tiles, int ntiles,
                                                    const DevInst* __restrict__ insts) {
  __shared__ R s_psi[EXT], s_phi1[EXT], s_phi2[EXT];
  __shared__ uint8_t s_t[EXT], s_m[EXT];
  __shared__ double s_max[NTHREADS / 32];
  __shared__ unsigned s_status;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int eo = (ty + 1) * EXT_X + (tx + 1);

  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const DevInst* Ip = insts + tl.inst;
    const DevParams& P = Ip->P;
    const long long N = Ip->N;
    const unsigned long long step = Ip->scal[S_STEP];
    const int cur = int(step & 1ULL);
    const TF* __restrict__ fin = (const TF*)Ip->f[cur];
    TF* __restrict__ fout = (TF*)Ip->f[cur ^ 1];
    const TG* __restrict__ gin = (const TG*)Ip->g[cur];
    TG* __restrict__ gout = (TG*)Ip->g[cur ^ 1];
    const uint8_t* __restrict__ tin = Ip->type[cur];
    uint8_t* __restrict__ tout = Ip->type[cur ^ 1];
    const double theta = 0.5 * ord_dec(Ip->scal[S_MAX0 + cur]);
    unsigned status = 0;
    if (tid == 0) s_status = 0;

    // ---- phase 1: own node moments, ring densities, potentials -> shared
    const int x = tl.x0 + tx, y = tl.y0 + ty;
    const bool own = x < P.nx && y < P.ny;
    const long long node = (long long)y * P.nx + x;
    uint8_t t = T_WALL;
    R f1[9], f2[9];
    R rho1 = R(0), rho2 = R(0), d1 = R(0), d2 = R(0), j1x = R(0), j1y = R(0), j2x = R(0), j2y = R(0);
    {
      int xn, yn;
      bool in = nbr(P, tl.x0 - 1, tl.y0 - 1, tx + 1, ty + 1, xn, yn);
      long long nn = (long long)yn * P.nx + xn;
      uint8_t te = in ? (tin[nn] & T_MASK) : T_WALL;
      R r1 = R(0), r2 = R(0);
      if (own) t = te;
      if (is_fluid(te)) {
        if (own) {
#pragma unroll
          for (int a = 0; a < 9; ++a) {
            f1[a] = ld<R>(fin + a * N + node);
            f2[a] = ld<R>(fin + (9 + a) * N + node);
          }
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
          rho1 = R(P.shift_f[0]) + d1;
          rho2 = R(P.shift_f[1]) + d2;
          r1 = rho1;
          r2 = rho2;
        } else {
          r1 = R(P.shift_f[0]) + density_shifted<R>(fin, N, nn);
          r2 = R(P.shift_f[1]) + density_shifted<R>(fin + 9 * N, N, nn);
        }
      } else if (is_res(te)) {
        double a, b;
        reservoir_rho(P, te, step, a, b);
        r1 = R(a);
        r2 = R(b);
      }
      R ps = R(0), p1 = R(0), p2 = R(0);
      if (is_live(te)) potentials<R>(P, r1, r2, ps, p1, p2, status);
      s_psi[eo] = ps;
      s_phi1[eo] = p1;
      s_phi2[eo] = p2;
      s_t[eo] = te;
      s_m[eo] = (is_live(te) && double(r1) > theta) ? 1 : 0;
      if (is_fluid(te) && !(double(r1) == double(r1) && double(r2) == double(r2))) status |= ST_NONFINITE;
    }
    for (int r = tid; r < RING; r += NTHREADS) {
      int ex, ey;
      ring_pos(r, ex, ey);
      int xn, yn;
      bool in = nbr(P, tl.x0 - 1, tl.y0 - 1, ex, ey, xn, yn);
      long long nn = (long long)yn * P.nx + xn;
      uint8_t te = in ? (tin[nn] & T_MASK) : T_WALL;
      R r1 = R(0), r2 = R(0);
      if (is_fluid(te)) {
        r1 = R(P.shift_f[0]) + density_shifted<R>(fin, N, nn);
        r2 = R(P.shift_f[1]) + density_shifted<R>(fin + 9 * N, N, nn);
      } else if (is_res(te)) {
        double a, b;
        reservoir_rho(P, te, step, a, b);
        r1 = R(a);
        r2 = R(b);
      }
      R ps = R(0), p1 = R(0), p2 = R(0);
      if (is_live(te)) potentials<R>(P, r1, r2, ps, p1, p2, status);
      const int e = ey * EXT_X + ex;
      s_psi[e] = ps;
      s_phi1[e] = p1;
      s_phi2[e] = p2;
      s_t[e] = te;
      s_m[e] = (is_live(te) && double(r1) > theta) ? 1 : 0;
    }
    __syncthreads();

    double mymax = -1.0 / 0.0;
    if (own) {
      if (is_fluid(t)) {
        mymax = double(rho1);
        // ---- forces (Eqs. 11, 14a/b, 16) with neutral solid neighbours
        const R psc = s_psi[eo], p1c = s_phi1[eo], p2c = s_phi2[eo];
        R spx = 0, spy = 0, s2x = 0, s2y = 0, s1x = 0, s1y = 0, ssx = 0, ssy = 0;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
          const int en = eo + EY(a) * EXT_X + EX(a);
          const bool lv = is_live(s_t[en]);
          const R w = wf<R>(a);
          const R vp = w * (lv ? s_psi[en] : psc);
          const R v2 = w * (lv ? s_phi2[en] : p2c);
          const R v1 = w * (lv ? s_phi1[en] : p1c);
          const R vs = lv ? R(0) : w;
          if (EX(a) > 0) { spx += vp; s2x += v2; s1x += v1; ssx += vs; }
          if (EX(a) < 0) { spx -= vp; s2x -= v2; s1x -= v1; ssx -= vs; }
          if (EY(a) > 0) { spy += vp; s2y += v2; s1y += v1; ssy += vs; }
          if (EY(a) < 0) { spy -= vp; s2y -= v2; s1y -= v1; ssy -= vs; }
        }
        const R G11 = R(P.G11), G12 = R(P.G12), G21 = R(P.G21), w1 = R(P.w_adh[0]), w2 = R(P.w_adh[1]);
        const R F1x = -G11 * psc * spx - G12 * p1c * s2x - w1 * psc * ssx + rho1 * R(P.gx);
        const R F1y = -G11 * psc * spy - G12 * p1c * s2y - w1 * psc * ssy + rho1 * R(P.gy);
        const R F2x = -G21 * p2c * s1x - w2 * rho2 * ssx + rho2 * R(P.gx);
        const R F2y = -G21 * p2c * s1y - w2 * rho2 * ssy + rho2 * R(P.gy);
        // ---- velocities (Eqs. 17-19)
        const R t1 = R(P.tau[0]), t2 = R(P.tau[1]);
        const R den = rho1 / t1 + rho2 / t2;
        const R upx = (j1x / t1 + j2x / t2) / den;
        const R upy = (j1y / t1 + j2y / t2) / den;
        const R u1x = upx + (rho1 != R(0) ? t1 * F1x / rho1 : R(0));
        const R u1y = upy + (rho1 != R(0) ? t1 * F1y / rho1 : R(0));
        const R u2x = upx + (rho2 != R(0) ? t2 * F2x / rho2 : R(0));
        const R u2y = upy + (rho2 != R(0) ? t2 * F2y / rho2 : R(0));
        const R rt = rho1 + rho2;
        const R urx = (j1x + j2x + R(0.5) * (F1x + F2x)) / rt;
        const R ury = (j1y + j2y + R(0.5) * (F1y + F2y)) / rt;

        const bool liq = s_m[eo] != 0;
        tout[node] = liq ? T_LIQUID : T_GAS;

        // ---- solutes: concentration with the Step-2 amendment, sources
        R S1 = R(0), S2 = R(0);
        R gs[NS > 0 ? NS : 1][5];
        R C[NS > 0 ? NS : 1];
        R Sk[NS > 0 ? NS : 1];
        if constexpr (NS > 0) {
          if (liq) {
            const bool appear = (t == T_GAS);
            bool vnb = false;
#pragma unroll
            for (int b = 1; b < 5; ++b) {
              const int en = eo + EY(b) * EXT_X + EX(b);
              vnb |= (s_t[en] == T_LIQUID && s_m[en] == 0);
            }
            if (!appear) {
#pragma unroll
              for (int k = 0; k < NS; ++k)
#pragma unroll
                for (int a = 0; a < 5; ++a) gs[k][a] = ld<R>(gin + ((long long)k * 5 + a) * N + node);
            }
            if (appear || vnb) {
              // Section 4.5 amendment (rare): appearing node takes the mean C
              // of its surviving liquid neighbours; each vanishing neighbour
              // hands C / (number of its liquid neighbours) to this node.
              R base[NS], dC[NS];
#pragma unroll
              for (int k = 0; k < NS; ++k) { base[k] = R(0); dC[k] = R(0); }
              int nsrc = 0;
#pragma unroll
              for (int b = 1; b < 5; ++b) {
                const int en = eo + EY(b) * EXT_X + EX(b);
                int xn, yn;
                if (!nbr(P, x, y, EX(b), EY(b), xn, yn)) continue;
                const long long nn = (long long)yn * P.nx + xn;
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
                    nrec += liquid_at<R, TF>(P, tin, fin, N, (long long)yz * P.nx + xz, theta) ? 1 : 0;
                  }
                  R Cn[NS];
                  conc_at<R, TG, NS>(gin, N, nn, P, Cn);
#pragma unroll
                  for (int k = 0; k < NS; ++k) dC[k] += Cn[k] / R(nrec);
                }
              }
#pragma unroll
              for (int k = 0; k < NS; ++k) {
                const R J0 = R(P.J0[k]), Ja = (R(1) - J0) / R(4);
                if (appear) {
                  const R cb = (nsrc ? base[k] / R(nsrc) : R(0)) + dC[k];
#pragma unroll
                  for (int a = 0; a < 5; ++a) {
                    const R ja = a == 0 ? J0 : Ja;
                    gs[k][a] = ja * cb - ja * R(P.shift_c[k]);
                  }
                } else {
#pragma unroll
                  for (int a = 0; a < 5; ++a) gs[k][a] += (a == 0 ? J0 : Ja) * dC[k];
                }
              }
            }
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              R s = gs[k][0];
#pragma unroll
              for (int a = 1; a < 5; ++a) s += gs[k][a];
              C[k] = R(P.shift_c[k]) + s;
            }
            // homogeneous reactions (Eqs. 5a, 5c; sources Eqs. 27, 28)
            R CA = R(0), CB = R(0), CE = R(0), tot = R(0);
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              if (k == P.iA) CA = C[k];
              if (k == P.iB) CB = C[k];
              if (k == P.iE) CE = C[k];
              tot += C[k];
              Sk[k] = R(0);
            }
            if (P.iA == -2) CA = fmax(R(0), R(P.c_total_per_rho1) * rho1 - tot);
            const R CC = rho2 * R(P.inv_M_C);
            const R R1 = R(P.k1) * (CA - R(P.inv_Keq) * CB * rsqrt_<R>(fmax(CC, R(0))));
            const R R3 = R(P.k3) * CB * CE;
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              if (k == P.iA) Sk[k] -= R1;
              if (k == P.iB) Sk[k] += R1 - R3;
              if (k == P.iE) Sk[k] -= R3;
              if (k == P.iF) Sk[k] += R3;
            }
            S1 = -R(P.gas_yield) * R1;
            S2 = R(P.gas_yield) * R1;
          }
        }

        // ---- fluid collision (Eq. 6, Eq. 8 at u_eq) and push streaming
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const R rho = s == 0 ? rho1 : rho2;
          const R dr = s == 0 ? d1 : d2;
          const R ux = s == 0 ? u1x : u2x, uy = s == 0 ? u1y : u2y;
          const R itau = R(1) / (s == 0 ? t1 : t2);
          const R Ssrc = s == 0 ? S1 : S2;
          const R uu = ux * ux + uy * uy;
          TF* fo = fout + (long long)s * 9 * N;
#pragma unroll
          for (int a = 0; a < 9; ++a) {
            const R fa = s == 0 ? f1[a] : f2[a];
            const R eu = R(EX(a)) * ux + R(EY(a)) * uy;
            const R w = w9<R>(a);
            const R feq = w * (dr + rho * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
            const R fs = fa - (fa - feq) * itau + w * Ssrc;
            if (a == 0) {
              st<TF, R>(fo + node, fs);
              continue;
            }
            const int en = eo + EY(a) * EXT_X + EX(a);
            const uint8_t tn = s_t[en];
            if (is_fluid(tn)) {
              int xn, yn;
              nbr(P, x, y, EX(a), EY(a), xn, yn);
              st<TF, R>(fo + a * N + (long long)yn * P.nx + xn, fs);
            } else if (!is_res(tn)) {
              st<TF, R>(fo + OPP(a) * N + node, fs);
            }
          }
        }

        // ---- solute collision (Eqs. 20-22 with u_r) and push streaming
        if constexpr (NS > 0) {
          if (liq) {
#pragma unroll
            for (int a = 0; a < 5; ++a) {
              R gst[NS];
              const R eu = R(EX(a)) * urx + R(EY(a)) * ury;
#pragma unroll
              for (int k = 0; k < NS; ++k) {
                const R J0 = R(P.J0[k]);
                const R ja = a == 0 ? J0 : (R(1) - J0) / R(4);
                const R geq = ja * (C[k] - R(P.shift_c[k])) + R(0.5) * C[k] * eu;
                gst[k] = gs[k][a] - (gs[k][a] - geq) / R(P.tau_g[k]) + ja * Sk[k];
              }
              if (a == 0) {
#pragma unroll
                for (int k = 0; k < NS; ++k) st<TG, R>(gout + (long long)k * 5 * N + node, gst[k]);
                continue;
              }
              const int en = eo + EY(a) * EXT_X + EX(a);
              const uint8_t tn = s_t[en];
              const bool mn = s_m[en] != 0;
              if (is_fluid(tn) && mn) {
                int xn, yn;
                nbr(P, x, y, EX(a), EY(a), xn, yn);
                const long long nn = (long long)yn * P.nx + xn;
#pragma unroll
                for (int k = 0; k < NS; ++k) st<TG, R>(gout + ((long long)k * 5 + a) * N + nn, gst[k]);
              } else if (is_res(tn) && mn) {
                // outflow into a liquid reservoir
              } else {
                // no-flux (gas, wall, gas reservoir) or reactive (mineral) link
                if (is_mineral(tn)) {
                  R qB = R(0);
                  bool rB = false;
#pragma unroll
                  for (int k = 0; k < NS; ++k) {
                    const R Ja = (R(1) - R(P.J0[k])) / R(4);
                    const R out = gst[k] + Ja * R(P.shift_c[k]);
                    if (k == P.iB && P.k2 != 0.0 && tn == T_SOLID_D) {
                      // R2 at D(s): consumption k2 C_w, C_w = (out + back) / (2 J_w)
                      const R kap = R(P.k2) / (R(2) * Ja);
                      const R bk = out * (R(1) - kap) / (R(1) + kap);
                      qB = out - bk;
                      rB = true;
                      gst[k] = bk - Ja * R(P.shift_c[k]);
                      Ip->q[(0LL * 4 + (a - 1)) * N + node] = double(qB);
                    } else if (k == P.iF && P.k4 != 0.0) {
                      // R4 at D(s) or F(s): consumption k4 (C_w - C_sat)
                      const R kap = R(P.k4) / (R(2) * Ja);
                      const R bk = (out * (R(1) - kap) + R(P.k4) * R(P.C_F_sat)) / (R(1) + kap);
                      gst[k] = bk - Ja * R(P.shift_c[k]);
                      Ip->q[(1LL * 4 + (a - 1)) * N + node] = double(out - bk);
                    }
                  }
                  if (rB) {
#pragma unroll
                    for (int k = 0; k < NS; ++k)
                      if (k == P.iE) gst[k] += qB;   // product E of R2 leaves the wall
                  }
                }
#pragma unroll
                for (int k = 0; k < NS; ++k) st<TG, R>(gout + ((long long)k * 5 + OPP(a)) * N + node, gst[k]);
              }
            }
          } else {
            // gas node: no solute
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              const R J0 = R(P.J0[k]), Ja = (R(1) - J0) / R(4);
#pragma unroll
              for (int a = 0; a < 5; ++a)
                st<TG, R>(gout + ((long long)k * 5 + a) * N + node, -(a == 0 ? J0 : Ja) * R(P.shift_c[k]));
            }
          }
        }
      } else if (is_res(t)) {
        // ---- reservoir node: push its equilibrium into fluid neighbours
        double a_, b_;
        reservoir_rho(P, t, step, a_, b_);
        const R r1 = R(a_), r2 = R(b_);
        R ux = R(0), uy = R(0);
        int xn, yn;
        const int dx = (t == T_INLET) ? 1 : -1;
        if (nbr(P, x, y, dx, 0, xn, yn)) {
          const long long nn = (long long)yn * P.nx + xn;
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
            const R rt = (R(P.shift_f[0]) + e1) + (R(P.shift_f[1]) + e2);
            ux = jx / rt;
            uy = jy / rt;
          }
        }
        const R uu = ux * ux + uy * uy;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const R rho = s == 0 ? r1 : r2;
          const R dr = rho - R(P.shift_f[s]);
          TF* fo = fout + (long long)s * 9 * N;
#pragma unroll
          for (int a = 1; a < 9; ++a) {
            const int en = eo + EY(a) * EXT_X + EX(a);
            if (!is_fluid(s_t[en])) continue;
            const R eu = R(EX(a)) * ux + R(EY(a)) * uy;
            const R w = w9<R>(a);
            const R feq = w * (dr + rho * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
            nbr(P, x, y, EX(a), EY(a), xn, yn);
            st<TF, R>(fo + a * N + (long long)yn * P.nx + xn, feq);
          }
        }
        if constexpr (NS > 0) {
          if (s_m[eo]) {
            R Cr[NS];
#pragma unroll
            for (int k = 0; k < NS; ++k) Cr[k] = R(P.conc_in[k]);
            if (t == T_OUTLET) {
              const int ew = eo - 1;
#pragma unroll
              for (int k = 0; k < NS; ++k) Cr[k] = R(0);
              if (is_fluid(s_t[ew]) && s_m[ew] && nbr(P, x, y, -1, 0, xn, yn))
                conc_at<R, TG, NS>(gin, N, (long long)yn * P.nx + xn, P, Cr);
            }
#pragma unroll
            for (int k = 0; k < NS; ++k) {
              const R J0 = R(P.J0[k]), Ja = (R(1) - J0) / R(4);
#pragma unroll
              for (int a = 1; a < 5; ++a) {
                const int en = eo + EY(a) * EXT_X + EX(a);
                if (!(is_fluid(s_t[en]) && s_m[en])) continue;
                const R eu = R(EX(a)) * ux + R(EY(a)) * uy;
                const R geq = Ja * (Cr[k] - R(P.shift_c[k])) + R(0.5) * Cr[k] * eu;
                nbr(P, x, y, EX(a), EY(a), xn, yn);
                st<TG, R>(gout + ((long long)k * 5 + a) * N + (long long)yn * P.nx + xn, geq);
              }
            }
          }
        }
        tout[node] = t;
      } else {
        tout[node] = t;
      }
    }

    // ---- block max of rho_1 over fluid nodes (next step's threshold) and status
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mymax = fmax(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
    if ((tid & 31) == 0) s_max[tid >> 5] = mymax;
    if (status) atomicOr(&s_status, status);
    __syncthreads();
    if (tid == 0) {
      double m = s_max[0];
      for (int w = 1; w < NTHREADS / 32; ++w) m = fmax(m, s_max[w]);
      if (m > -1.0 / 0.0) atomicMax(&Ip->scal[S_MAX0 + (cur ^ 1)], ord_enc(m));
      if (s_status) atomicOr(&Ip->scal[S_STATUS], (unsigned long long)s_status);
    }
    __syncthreads();
  }
}

}  // namespace pslbm
