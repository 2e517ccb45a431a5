// Interface kernels of one time step (Chen, Kang et al., arXiv 1410.3464):
//   k_vop   -- heterogeneous reactions at liquid-mineral links (Eqs. 29-31)
//              and the volume-of-pixel update (Eqs. 32-35, Step 4) with the
//              status decisions (dissolution, precipitation overflow);
//   k_amend -- status changes and the amendment of Step 5 (Section 4.5) at
//              flipped nodes, one block per instance; it ends the step.
// Every gather runs in the fixed order E, N, W, S, so the result does not
// depend on thread scheduling.
#pragma once
#include "device.cuh"

namespace pslbm {

// The bulk kernel bounces every solute population that leaves a liquid node
// toward a mineral back into the node (halfway bounce-back).  At a reactive
// link this kernel replaces the bounced value by the reactive link rule: with
// the outgoing population `out`, J_w = (1 - J0)/4 and kappa = k / (2 J_w),
// the returning population is (out (1 - kappa) + k C_sat) / (1 + kappa) and the
// link flux q = out - back is the amount consumed (B by R2 at D(s), F by R4 at
// D(s) or F(s)); E gains the B consumed on the same link.  The flux is computed
// directly, q = out 2 kappa / (1 + kappa) - k C_sat / (1 + kappa), since out and
// back differ by a relative 2 kappa only.  Then V_D -= Vbar_D
// sum q_B, V_F += Vbar_F sum q_F, and the node dissolves, overflows or changes
// between D(s) and F(s).
//
// The bulk kernel sets a bit for every mineral node a liquid node touched in
// the step (the only nodes this kernel changes).  Each warp takes a chunk of
// VOP_CHUNK consecutive words of that bitmap, clears them, and deals the set
// bits of the chunk out to its lanes in node order (32 nodes per round), so
// that every lane of a round has a node to update.
template <class TF, class TG, class R, int NS>
__device__ __forceinline__ void vop_node(const DevInst* Ip, const DevParams& P, int N, int cur,
                                         unsigned long long step, int node) {
  uint8_t* __restrict__ tnew = Ip->type[cur ^ 1];
  double* __restrict__ V = Ip->V;
  // independent loads first: own type, volumes, the four neighbour types
  const uint8_t t = tnew[node] & T_MASK;
  double VD = V[node], VF = V[N + node];
  const int x = node % P.nx, y = node / P.nx;
  int nbx[4];
#pragma unroll
  for (int b = 1; b < 5; ++b) {
    int xn, yn;
    nbx[b - 1] = nbr(P, x, y, EX(b), EY(b), xn, yn) ? yn * P.nx + xn : -1;
  }
  uint8_t tn[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) tn[b] = nbx[b] >= 0 ? (tnew[nbx[b]] & T_MASK) : T_WALL;
  if (!is_mineral(t)) return;
  int nl = 0;
  int dirs[4];
#pragma unroll
  for (int b = 1; b < 5; ++b) {
    if (tn[b - 1] != T_LIQUID) nbx[b - 1] = -1;
    else dirs[nl++] = b;
  }
  if (nl == 0) return;
  R sB = R(0), sF = R(0);
  if constexpr (NS > 0) {
    TG* __restrict__ gout = (TG*)Ip->g[cur ^ 1];
    const bool useB = (t == T_SOLID_D) && P.useB;
    const bool useF = P.useF != 0;
    // the population that left neighbour nn toward this node was bounced into
    // slot b of nn; gather every slot before writing any
    R oB[4], oE[4], oF[4];
#pragma unroll
    for (int b = 1; b < 5; ++b) {
      const int nn = nbx[b - 1];
      oB[b - 1] = oE[b - 1] = oF[b - 1] = R(0);
      if (nn < 0) continue;
      if (useB) {
        oB[b - 1] = gldc<R>(P, P.iB, gout + (P.iB * 5 + b) * N + nn);
        if (P.iE >= 0) oE[b - 1] = gldc<R>(P, P.iE, gout + (P.iE * 5 + b) * N + nn);
      }
      if (useF) oF[b - 1] = gldc<R>(P, P.iF, gout + (P.iF * 5 + b) * N + nn);
    }
#pragma unroll
    for (int b = 1; b < 5; ++b) {
      const int nn = nbx[b - 1];
      if (nn < 0) continue;
      if (useB) {
        const int iB = P.iB;
        const R sh = rp<R>(P).vB_sh;
        const R out = oB[b - 1] + sh;
        const R q = out * rp<R>(P).vB_qa;
        const R bk = out - q;
        gst<TG, R>(P, iB, gout + (iB * 5 + b) * N + nn, bk - sh);
        sB += q;
        if (P.iE >= 0) gst<TG, R>(P, P.iE, gout + (P.iE * 5 + b) * N + nn, oE[b - 1] + q);
      }
      if (useF) {
        const int iF = P.iF;
        const R sh = rp<R>(P).vF_sh;
        const R out = oF[b - 1] + sh;
        const R q = out * rp<R>(P).vF_qa - rp<R>(P).vF_qc;
        gst<TG, R>(P, iF, gout + (iF * 5 + b) * N + nn, (out - q) - sh);
        sF += q;
      }
    }
  }
  // volumes accumulate in FP64: per-step increments are far below FP32 resolution of V
  if (t == T_SOLID_D) VD = VD - P.Vbar_D * double(sB);   // Eq. 33
  VF = VF + P.Vbar_F * double(sF);                        // Eq. 35 (precipitation adds volume)
  if (VD < 0.0) VD = 0.0;
  const double total = VD + VF;
  int code = EV_NONE;
  if (total <= 0.0) {
    VD = 0.0;
    VF = 0.0;
    code = EV_DISSOLVE;
  } else {
    tnew[node] = VD > 0.0 ? T_SOLID_D : T_SOLID_F;
    if (total >= P.V_split) {
      const double excess = total - 1.0;
      VF = VF - excess;
      const unsigned long long key = P.seed ^ (step << 40) ^ (unsigned long long)node;
      const int pick = int(splitmix64(key) % (unsigned long long)nl);
      code = EV_OVERFLOW | (dirs[pick] << 4);
      Ip->xs[node] = excess;
    }
  }
  V[node] = VD;
  V[N + node] = VF;
  if (code != EV_NONE) {
    Ip->evt[node] = (uint8_t)code;
    const unsigned long long slot = atomicAdd(&Ip->scal[S_NEVENT], 1ULL);
    if (slot < (unsigned long long)Ip->evcap)
      Ip->evlist[slot] = node;
    else
      atomicOr(&Ip->scal[S_STATUS], (unsigned long long)ST_EVOVERFLOW);
  }
}

// Blocks per SM the VOP kernel's register budget targets (its grid is one
// wave of resident blocks): five in FP32, four in FP64 (twice the registers
// per value).
template <class R>
constexpr int vop_min_blocks() {
  return sizeof(R) == 8 ? 4 : 5;
}

// chunk_map: (instance, chunk within it) of every chunk of a batch, in
// instance order, or null for one simulation (instance 0, chunk g); nchunks:
// the number of chunks.  Warps take chunks with a grid stride, so every
// member's chunks are spread over the whole grid.
template <class TF, class TG, class R, int NS>
__global__ void __launch_bounds__(NTHREADS, vop_min_blocks<R>())
    k_vop(const DevInst* __restrict__ insts, const int2* __restrict__ chunk_map, long long nchunks) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long c0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long cs = (gridDim.x * (long long)blockDim.x) >> 5;
  for (long long g = c0; g < nchunks; g += cs) {
    const int2 ic = chunk_map ? chunk_map[g] : make_int2(0, (int)g);
    const DevInst* Ip = insts + ic.x;
    const int c = ic.y;
    const unsigned long long step = Ip->scal[S_STEP];
    if (step >= Ip->scal[S_LIMIT]) continue;   // frozen instance
    const int N = (int)Ip->N;
    const int nw = (N + 31) >> 5;
    const int cur = int(step & 1ULL);
    unsigned* vmask = Ip->vmask;
    // lane j < VOP_CHUNK holds word c VOP_CHUNK + j, and the number of set
    // bits before it in the chunk
    const int wj = c * VOP_CHUNK + lane;
    const unsigned m = (lane < VOP_CHUNK && wj < nw) ? vmask[wj] : 0u;
    if (m) vmask[wj] = 0u;
    const int cnt = __popc(m);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < VOP_CHUNK; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, VOP_CHUNK - 1);
    const int excl = incl - cnt;
    for (int r = 0; r < total; r += 32) {
      // the k-th set bit of the chunk: its word j and its rank within it
      const int k = r + lane;
      int node = -1;
#pragma unroll
      for (int j = 0; j < VOP_CHUNK; ++j) {
        const int ej = __shfl_sync(FULL, excl, j);
        const int nj = __shfl_sync(FULL, cnt, j);
        const unsigned mj = __shfl_sync(FULL, m, j);
        if (k >= ej && k < ej + nj) {
          unsigned mm = mj;
          for (int i = k - ej; i > 0; --i) mm &= mm - 1u;   // drop the lower set bits
          node = (c * VOP_CHUNK + j) * 32 + (__ffs(mm) - 1);
        }
      }
      if (node >= 0) vop_node<TF, TG, R, NS>(Ip, Ip->P, N, cur, step, node);
    }
  }
}

__device__ __forceinline__ bool surv_fluid(uint8_t tf) { return (tf & (T_NEW | T_VANISH)) == 0 && is_fluid(tf & T_MASK); }
__device__ __forceinline__ bool surv_liquid(uint8_t tf) { return tf == T_LIQUID; }

// End of a step for one instance: decode the next step's liquid threshold
// (half the maximum the bulk kernel gathered this step) into both precisions,
// free the slot this step read (it receives the maximum two steps later) and
// advance the step counter.  mx: the encoded maximum of this step's slot,
// S_MAX0 + ((step + 1) & 1).
__device__ __forceinline__ void finish_step(const DevInst* Ip, unsigned long long step, unsigned long long mx) {
  const double th = 0.5 * ord_dec(mx);
  Ip->scal[S_THETA] = (unsigned long long)__double_as_longlong(th);
  Ip->scal[S_THETAF] = (unsigned long long)(unsigned)__float_as_int(float(th));
  Ip->scal[S_MAX0 + int(step & 1ULL)] = 0ULL;
  Ip->scal[S_NEVENT] = 0ULL;
  Ip->scal[S_STEP] = step + 1;
}

template <class TF, class TG, class R, int NS>
__global__ void __launch_bounds__(NTHREADS) k_amend(const DevInst* __restrict__ insts) {
  // the bulk kernel's tile claims start from zero at its next launch
  if (blockIdx.x == 0 && threadIdx.x == 0) insts[0].scal[S_TILES] = 0ULL;
  const DevInst* Ip = insts + blockIdx.x;
  // the counters this kernel reads, loaded together (one memory round trip)
  const volatile unsigned long long* sc = Ip->scal;
  const unsigned long long step = sc[S_STEP], limit = sc[S_LIMIT], nev_raw = sc[S_NEVENT], m0 = sc[S_MAX0],
                           m1 = sc[S_MAX1];
  if (step >= limit) return;   // frozen instance
  const unsigned long long mx = (step & 1ULL) ? m0 : m1;
  if (nev_raw == 0) {
    if (threadIdx.x == 0) finish_step(Ip, step, mx);
    return;
  }
  const DevParams& P = Ip->P;
  const long long N = Ip->N;
  const int nev = (int)min(nev_raw, (unsigned long long)Ip->evcap);
  // buffer cur is the state the bulk kernel just wrote
  const int cur = int(step & 1ULL) ^ 1;
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
        s1 += fshift<R>(P, 0, tf) + density_c<R>(F, N, nn);
        s2 += fshift<R>(P, 1, tf) + density_c<R>(F + 9 * N, N, nn);
        ++nf;
      }
      if (surv_liquid(tf)) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const TG* gk = G + (long long)k * 5 * N;
          R c = gldc<R>(P, k, gk + nn);
#pragma unroll
          for (int a = 1; a < 5; ++a) c += gldc<R>(P, k, gk + a * N + nn);
          sc[k] += rp<R>(P).shift_c[k] + c;
        }
        ++nl;
      }
    }
    const R r1 = nf ? s1 / R(nf) : rp<R>(P).rho_fill[0];
    const R r2 = nf ? s2 / R(nf) : rp<R>(P).rho_fill[1];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const R w = w9<R>(a);
      st<TF, R>(F + a * N + node, w * r1 - w * rp<R>(P).shift_f[0]);
      st<TF, R>(F + (9 + a) * N + node, w * r2 - w * rp<R>(P).shift_f[1]);
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const R c = nl ? sc[k] / R(nl) : R(0);
      const R J0 = rp<R>(P).J0[k], Ja = (R(1) - J0) / R(4);
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        const R ja = a == 0 ? J0 : Ja;
        gst<TG, R>(P, k, G + ((long long)k * 5 + a) * N + node, ja * c - ja * rp<R>(P).shift_c[k]);
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
      add1 += (fshift<R>(P, 0, T[w]) + density_c<R>(F, N, w)) / R(nf);
      add2 += (fshift<R>(P, 1, T[w]) + density_c<R>(F + 9 * N, N, w)) / R(nf);
      if (nliq && nl) {
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          const TG* gk = G + (long long)k * 5 * N;
          R c = gldc<R>(P, k, gk + w);
#pragma unroll
          for (int a = 1; a < 5; ++a) c += gldc<R>(P, k, gk + a * N + w);
          addc[k] += (rp<R>(P).shift_c[k] + c) / R(nl);
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
        const R J0 = rp<R>(P).J0[k], Ja = (R(1) - J0) / R(4);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
          TG* p = G + ((long long)k * 5 + a) * N + n;
          gst<TG, R>(P, k, p, gldc<R>(P, k, p) + (a == 0 ? J0 : Ja) * addc[k]);
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
  if (threadIdx.x == 0) finish_step(Ip, step, mx);
}

}  // namespace pslbm
