// Initialisation, field read-out and deterministic budget reduction.
#pragma once
#include "device.cuh"

namespace pslbm {

// Rest equilibrium (Eq. 8 at u = 0, Eq. 21 at u = 0) from initial fields.
template <class TF, class TG, class R, int NS>
__global__ void k_init(DevInst* __restrict__ Ip, const uint8_t* __restrict__ mask, const double* __restrict__ rho1,
                       const double* __restrict__ rho2, const double* __restrict__ conc) {
  const DevParams& P = Ip->P;
  const long long N = Ip->N;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < N;
       node += (long long)gridDim.x * blockDim.x) {
    const uint8_t t = mask[node] & T_MASK;
    Ip->type[0][node] = t;
    Ip->type[1][node] = t;
    TF* F = (TF*)Ip->f[0];
    TG* G = (TG*)Ip->g[0];
    const bool fl = is_fluid(t);
    const R r1 = fl ? R(rho1[node]) : R(0), r2 = fl ? R(rho2[node]) : R(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R w = w9<R>(a);
      st<TF, R>(F + a * N + node, fl ? w * r1 - w * fshift<R>(P, 0, t) : R(0));
      st<TF, R>(F + (9 + a) * N + node, fl ? w * r2 - w * fshift<R>(P, 1, t) : R(0));
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const R c = (t == T_LIQUID && conc) ? R(conc[k * N + node]) : R(0);
      const R J0 = rp<R>(P).J0[k], Ja = (R(1) - J0) / R(4);
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        const R ja = a == 0 ? J0 : Ja;
        gst<TG, R>(P, k, G + ((long long)k * 5 + a) * N + node, ja * c - ja * rp<R>(P).shift_c[k]);
      }
    }
  }
}

// Observable fields of the current state: rho_1, rho_2, u_r (Eq. 19) at fluid
// nodes, C_k at liquid nodes, node types.  Forces are recomputed from the
// neighbours' densities exactly as in the bulk kernel.
template <class TF, class TG, class R, int NS>
__global__ void k_fields(const DevInst* __restrict__ Ip, double* __restrict__ o_rho1, double* __restrict__ o_rho2,
                         double* __restrict__ o_ux, double* __restrict__ o_uy, double* __restrict__ o_conc,
                         uint8_t* __restrict__ o_type) {
  const DevParams& P = Ip->P;
  const long long N = Ip->N;
  const unsigned long long step = Ip->scal[S_STEP];
  const int cur = int(step & 1ULL);
  const TF* F = (const TF*)Ip->f[cur];
  const TG* G = (const TG*)Ip->g[cur];
  const uint8_t* T = Ip->type[cur];
  unsigned status = 0;
  for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < N;
       node += (long long)gridDim.x * blockDim.x) {
    const uint8_t t = T[node] & T_MASK;
    o_type[node] = t;
    double r1o = 0, r2o = 0, uxo = 0, uyo = 0;
    const int x = int(node % P.nx), y = int(node / P.nx);
    if (is_fluid(t)) {
      R f1[9], f2[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        f1[a] = ldc<R>(F + a * N + node);
        f2[a] = ldc<R>(F + (9 + a) * N + node);
      }
      R d1 = f1[0], d2 = f2[0];
#pragma unroll
      for (int a = 1; a < 9; ++a) { d1 += f1[a]; d2 += f2[a]; }
      const R rho1 = fshift<R>(P, 0, t) + d1, rho2 = fshift<R>(P, 1, t) + d2;
      const R j1x = (f1[1] - f1[3]) + (f1[5] - f1[6]) + (f1[8] - f1[7]);
      const R j1y = (f1[2] - f1[4]) + (f1[5] - f1[8]) + (f1[6] - f1[7]);
      const R j2x = (f2[1] - f2[3]) + (f2[5] - f2[6]) + (f2[8] - f2[7]);
      const R j2y = (f2[2] - f2[4]) + (f2[5] - f2[8]) + (f2[6] - f2[7]);
      R psc, p1c, p2c;
      potentials<R>(P, rho1, rho2, psc, p1c, p2c, status);
      // neighbours' potentials (live ones) first, then the stencils with a
      // solid neighbour replaced by its mirror image across the wall, as in
      // the bulk kernel
      R nps[9], nq1[9], nq2[9];
      bool nlv[9];
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        int xn, yn;
        const bool in = nbr(P, x, y, EX(a), EY(a), xn, yn);
        const long long nn = (long long)yn * P.nx + xn;
        const uint8_t tn = in ? (T[nn] & T_MASK) : T_WALL;
        nps[a] = psc;
        nq1[a] = p1c;
        nq2[a] = p2c;
        nlv[a] = is_live(tn);
        if (nlv[a]) {
          R a1, a2;
          if (is_fluid(tn)) {
            a1 = fshift<R>(P, 0, tn) + density_shifted<R>(F, N, nn);
            a2 = fshift<R>(P, 1, tn) + density_shifted<R>(F + 9 * N, N, nn);
          } else {
            double u, v;
            const R theta = theta_of<R>(Ip);
            reservoir_rho(P, tn, step, tn == T_OUTLET && outlet_up_liquid<R, TF>(P, T, F, (int)N, (int)nn, theta), u, v);
            a1 = R(u);
            a2 = R(v);
          }
          potentials<R>(P, a1, a2, nps[a], nq1[a], nq2[a], status);
        }
      }
      nps[0] = psc;
      nq1[0] = p1c;
      nq2[0] = p2c;
      nlv[0] = true;
      const Stencils<R> S = force_stencils<R>(nps, nq1, nq2, nlv);
      const R spx = S.psx, spy = S.psy, s2x = S.p2x, s2y = S.p2y, s1x = S.p1x, s1y = S.p1y, ssx = S.ssx,
              ssy = S.ssy;
      const R G11 = rp<R>(P).G11, G12 = rp<R>(P).G12, G21 = rp<R>(P).G21, w1 = rp<R>(P).w_adh[0], w2 = rp<R>(P).w_adh[1];
      const R F1x = force1<R>(G11, G12, w1, psc, p1c, spx, s2x, ssx, rho1, rp<R>(P).gx);
      const R F1y = force1<R>(G11, G12, w1, psc, p1c, spy, s2y, ssy, rho1, rp<R>(P).gy);
      const R F2x = force2<R>(G21, w2, p2c, s1x, ssx, rho2, rp<R>(P).gx);
      const R F2y = force2<R>(G21, w2, p2c, s1y, ssy, rho2, rp<R>(P).gy);
      const R rrt = rrcp<R>(radd<R>(rho1, rho2));
      r1o = double(rho1);
      r2o = double(rho2);
      uxo = double(u_phys<R>(j1x, j2x, F1x, F2x, rrt));
      uyo = double(u_phys<R>(j1y, j2y, F1y, F2y, rrt));
    }
    if (o_rho1) o_rho1[node] = r1o;
    if (o_rho2) o_rho2[node] = r2o;
    if (o_ux) o_ux[node] = uxo;
    if (o_uy) o_uy[node] = uyo;
    if (o_conc) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        double c = 0.0;
        if (t == T_LIQUID) {
          const TG* gk = G + (long long)k * 5 * N;
          R s = gldc<R>(P, k, gk + node);
#pragma unroll
          for (int a = 1; a < 5; ++a) s += gldc<R>(P, k, gk + a * N + node);
          c = double(rp<R>(P).shift_c[k] + s);
        }
        o_conc[k * N + node] = c;
      }
    }
  }
}

// Budget partials: per block [max rho1, sum rho1, sum rho2, sum C_k (k < NS), sum V_D, sum V_F].
// Each block covers a fixed contiguous range and reduces in a fixed tree, so
// the result is independent of scheduling.

template <class TF, class TG, class R, int NS>
__global__ void __launch_bounds__(BUD_THREADS) k_budget_partial(const DevInst* __restrict__ Ip,
                                                                 double* __restrict__ part) {
  const DevParams& P = Ip->P;
  const long long N = Ip->N;
  const int cur = int(Ip->scal[S_STEP] & 1ULL);
  const TF* F = (const TF*)Ip->f[cur];
  const TG* G = (const TG*)Ip->g[cur];
  const uint8_t* T = Ip->type[cur];
  const long long per = (N + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = min(N, lo + per);
  double acc[NBUD];
  acc[0] = -1.0 / 0.0;
#pragma unroll
  for (int i = 1; i < NBUD; ++i) acc[i] = 0.0;
  for (long long node = lo + threadIdx.x; node < hi; node += blockDim.x) {
    const uint8_t t = T[node] & T_MASK;
    if (is_fluid(t)) {
      const double r1 = double(fshift<R>(P, 0, t) + density_c<R>(F, N, node));
      const double r2 = double(fshift<R>(P, 1, t) + density_c<R>(F + 9 * N, N, node));
      acc[0] = fmax(acc[0], r1);
      acc[1] += r1;
      acc[2] += r2;
    }
    if (t == T_LIQUID) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const TG* gk = G + (long long)k * 5 * N;
        R s = gldc<R>(P, k, gk + node);
#pragma unroll
        for (int a = 1; a < 5; ++a) s += gldc<R>(P, k, gk + a * N + node);
        acc[3 + k] += double(rp<R>(P).shift_c[k] + s);
      }
    }
    acc[3 + MAXS] += Ip->V[node];
    acc[4 + MAXS] += Ip->V[N + node];
  }
  __shared__ double sh[BUD_THREADS];
  for (int i = 0; i < NBUD; ++i) {
    sh[threadIdx.x] = acc[i];
    __syncthreads();
    for (int s = BUD_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] = (i == 0) ? fmax(sh[threadIdx.x], sh[threadIdx.x + s])
                                                      : sh[threadIdx.x] + sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x * NBUD + i] = sh[0];
    __syncthreads();
  }
}

// Fixed-order reduction of the per-block budget rows (max for entry 0, sums
// for the rest): thread t folds rows t, t + BUD_FINAL_THREADS, ... in order,
// then a shared-memory tree combines the threads; the result depends only on
// the rows and their count.  Valid in v[] of thread 0.
constexpr int BUD_FINAL_THREADS = 256;
__device__ __forceinline__ void budget_reduce(const double* __restrict__ part, int nblocks, double* v) {
  __shared__ double sh[NBUD][BUD_FINAL_THREADS];
  const int t = threadIdx.x;
  double acc[NBUD];
  acc[0] = -1.0 / 0.0;
#pragma unroll
  for (int i = 1; i < NBUD; ++i) acc[i] = 0.0;
  for (int b = t; b < nblocks; b += BUD_FINAL_THREADS) {
    acc[0] = fmax(acc[0], part[b * NBUD]);
#pragma unroll
    for (int i = 1; i < NBUD; ++i) acc[i] += part[b * NBUD + i];
  }
#pragma unroll
  for (int i = 0; i < NBUD; ++i) sh[i][t] = acc[i];
  __syncthreads();
  for (int s = BUD_FINAL_THREADS / 2; s > 0; s >>= 1) {
    if (t < s) {
      sh[0][t] = fmax(sh[0][t], sh[0][t + s]);
#pragma unroll
      for (int i = 1; i < NBUD; ++i) sh[i][t] += sh[i][t + s];
    }
    __syncthreads();
  }
  if (t == 0)
#pragma unroll
    for (int i = 0; i < NBUD; ++i) v[i] = sh[i][0];
}

static __global__ void __launch_bounds__(BUD_FINAL_THREADS) k_budget_final(const double* __restrict__ part,
                                                                          int nblocks, double* __restrict__ out) {
  double v[NBUD];
  budget_reduce(part, nblocks, v);
  if (threadIdx.x == 0)
    for (int i = 0; i < NBUD; ++i) out[i] = v[i];
}

}  // namespace pslbm
