// Amendment kernel of one time step (Chen, Kang et al., arXiv 1410.3464):
// status changes and the amendment of Step 5 (Section 4.5) at nodes flipped
// by the volume-of-pixel kernel; one block per instance, idle unless the VOP
// kernel recorded events.  Every gather runs in the fixed order E, N, W, S, so
// the result does not depend on thread scheduling.
#pragma once
#include "device.cuh"

namespace pslbm {

__device__ __forceinline__ bool surv_fluid(uint8_t tf) { return (tf & (T_NEW | T_VANISH)) == 0 && is_fluid(tf & T_MASK); }
__device__ __forceinline__ bool surv_liquid(uint8_t tf) { return tf == T_LIQUID; }

template <class TF, class TG, class R, int NS>
__global__ void __launch_bounds__(NTHREADS) k_amend(const DevInst* __restrict__ insts) {
  const DevInst* Ip = insts + blockIdx.x;
  const unsigned long long nev_raw = Ip->scal[S_NEVENT];
  if (nev_raw == 0) return;
  const DevParams& P = Ip->P;
  const long long N = Ip->N;
  const int nev = (int)min(nev_raw, (unsigned long long)Ip->evcap);
  // the VOP kernel has advanced the step counter: buffer cur is the new state
  const int cur = int(Ip->scal[S_STEP] & 1ULL);
  TF* F = (TF*)Ip->f[cur];
  TG* G = (TG*)Ip->g[cur];
  uint8_t* T = Ip->type[cur];
  int* vlist = Ip->evlist + Ip->evcap;   // second half: vanishing nodes
  __shared__ int s_nv;
  if (threadIdx.x == 0) s_nv = 0;
  __syncthreads();

  // phase 1: new types; each overflow target sums the excess of its choosers
  for (int i = threadIdx.x; i < nev; i += blockDim.x) {
    const int node = Ip->evlist[i];
    const int code = Ip->evt[node];
    const int x = node % P.nx, y = node / P.nx;
    if ((code & 15) == EV_DISSOLVE) {
      T[node] = T_LIQUID | T_NEW;
    } else if ((code & 15) == EV_OVERFLOW) {
      const int d = code >> 4;
      int xt, yt;
      nbr(P, x, y, EX(d), EY(d), xt, yt);
      const int tgt = yt * P.nx + xt;
      if (atomicCAS(&Ip->claim[tgt], 0, 1) == 0) {
        double acc = 0.0;
#pragma unroll
        for (int b = 1; b < 5; ++b) {
          int xz, yz;
          if (!nbr(P, xt, yt, EX(b), EY(b), xz, yz)) continue;
          const int z = yz * P.nx + xz;
          const int cz = Ip->evt[z];
          if ((cz & 15) != EV_OVERFLOW) continue;
          int xc, yc;
          nbr(P, xz, yz, EX(cz >> 4), EY(cz >> 4), xc, yc);
          if (yc * P.nx + xc == tgt) acc += Ip->xs[z];
        }
        Ip->V[tgt] = 0.0;
        Ip->V[N + tgt] = acc;
        T[tgt] = T_SOLID_F | T_VANISH;
        const int k = atomicAdd(&s_nv, 1);
        vlist[k] = tgt;
      }
    }
  }
  __syncthreads();
  const int nv = s_nv;

  // phase 2: refill dissolved nodes at rest with the mean density of their
  // surviving fluid neighbours and the mean concentration of their surviving
  // liquid neighbours (post-streaming values)
  for (int i = threadIdx.x; i < nev; i += blockDim.x) {
    const int node = Ip->evlist[i];
    if ((Ip->evt[node] & 15) != EV_DISSOLVE) continue;
    const int x = node % P.nx, y = node / P.nx;
    R s1 = R(0), s2 = R(0), sc[NS > 0 ? NS : 1];
#pragma unroll
    for (int k = 0; k < NS; ++k) sc[k] = R(0);
    int nf = 0, nl = 0;
#pragma unroll
    for (int b = 1; b < 5; ++b) {
      int xn, yn;
      if (!nbr(P, x, y, EX(b), EY(b), xn, yn)) continue;
      const long long nn = (long long)yn * P.nx + xn;
      const uint8_t tf = T[nn];
      if (surv_fluid(tf)) {
        s1 += R(P.shift_f[0]) + density_c<R>(F, N, nn);
        s2 += R(P.shift_f[1]) + density_c<R>(F + 9 * N, N, nn);
        ++nf;
      }
      if (surv_liquid(tf)) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const TG* gk = G + (long long)k * 5 * N;
          R c = ldc<R>(gk + nn);
#pragma unroll
          for (int a = 1; a < 5; ++a) c += ldc<R>(gk + a * N + nn);
          sc[k] += R(P.shift_c[k]) + c;
        }
        ++nl;
      }
    }
    const R r1 = nf ? s1 / R(nf) : R(P.rho_fill[0]);
    const R r2 = nf ? s2 / R(nf) : R(P.rho_fill[1]);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R w = w9<R>(a);
      st<TF, R>(F + a * N + node, w * r1 - w * R(P.shift_f[0]));
      st<TF, R>(F + (9 + a) * N + node, w * r2 - w * R(P.shift_f[1]));
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const R c = nl ? sc[k] / R(nl) : R(0);
      const R J0 = R(P.J0[k]), Ja = (R(1) - J0) / R(4);
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        const R ja = a == 0 ? J0 : Ja;
        st<TG, R>(G + ((long long)k * 5 + a) * N + node, ja * c - ja * R(P.shift_c[k]));
      }
    }
  }
  __syncthreads();

  // phase 3: surviving neighbours of vanished nodes take equal shares of the
  // vanished node's fluid mass (added at rest) and solute
  for (int i = threadIdx.x; i < nv * 4; i += blockDim.x) {
    const int v = vlist[i >> 2];
    const int b0 = (i & 3) + 1;
    int xr, yr;
    if (!nbr(P, v % P.nx, v / P.nx, EX(b0), EY(b0), xr, yr)) continue;
    const int n = yr * P.nx + xr;
    if (!surv_fluid(T[n])) continue;
    if (atomicCAS(&Ip->claim[n], 0, 2) != 0) continue;
    R add1 = R(0), add2 = R(0), addc[NS > 0 ? NS : 1];
#pragma unroll
    for (int k = 0; k < NS; ++k) addc[k] = R(0);
    const bool nliq = surv_liquid(T[n]);
#pragma unroll
    for (int b = 1; b < 5; ++b) {
      int xv, yv;
      if (!nbr(P, xr, yr, EX(b), EY(b), xv, yv)) continue;
      const long long w = (long long)yv * P.nx + xv;
      if (!(T[w] & T_VANISH)) continue;
      int nf = 0, nl = 0;
#pragma unroll
      for (int c = 1; c < 5; ++c) {
        int xz, yz;
        if (!nbr(P, xv, yv, EX(c), EY(c), xz, yz)) continue;
        const uint8_t tz = T[(long long)yz * P.nx + xz];
        nf += surv_fluid(tz) ? 1 : 0;
        nl += surv_liquid(tz) ? 1 : 0;
      }
      add1 += (R(P.shift_f[0]) + density_c<R>(F, N, w)) / R(nf);
      add2 += (R(P.shift_f[1]) + density_c<R>(F + 9 * N, N, w)) / R(nf);
      if (nliq && nl) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const TG* gk = G + (long long)k * 5 * N;
          R c = ldc<R>(gk + w);
#pragma unroll
          for (int a = 1; a < 5; ++a) c += ldc<R>(gk + a * N + w);
          addc[k] += (R(P.shift_c[k]) + c) / R(nl);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R w = w9<R>(a);
      TF* p1 = F + a * N + n;
      TF* p2 = F + (9 + a) * N + n;
      st<TF, R>(p1, ldc<R>(p1) + w * add1);
      st<TF, R>(p2, ldc<R>(p2) + w * add2);
    }
    if (nliq) {
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const R J0 = R(P.J0[k]), Ja = (R(1) - J0) / R(4);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          TG* p = G + ((long long)k * 5 + a) * N + n;
          st<TG, R>(p, ldc<R>(p) + (a == 0 ? J0 : Ja) * addc[k]);
        }
      }
    }
  }
  __syncthreads();

  // phase 4: clear the scratch state used by this step
  for (int i = threadIdx.x; i < nv * 4; i += blockDim.x) {
    const int v = vlist[i >> 2];
    int xr, yr;
    if (nbr(P, v % P.nx, v / P.nx, EX((i & 3) + 1), EY((i & 3) + 1), xr, yr)) Ip->claim[yr * P.nx + xr] = 0;
  }
  for (int i = threadIdx.x; i < nv; i += blockDim.x) Ip->claim[vlist[i]] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nev; i += blockDim.x) Ip->evt[Ip->evlist[i]] = 0;
  if (threadIdx.x == 0) Ip->scal[S_NEVENT] = 0;
}

}  // namespace pslbm
