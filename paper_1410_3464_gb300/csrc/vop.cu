// Volume-of-pixel kernel of one time step (Chen, Kang et al., arXiv
// 1410.3464, Eqs. 32-35, Step 4 of Section 4.7): at every mineral node with a
// liquid axis neighbour, gather the link fluxes written by the bulk kernel in
// the fixed order E, N, W, S, update V_D and V_F in FP64, and record the status
// decisions (dissolution, precipitation overflow into a liquid neighbour picked
// by SplitMix64).  The last tile of each instance advances its step counter and
// frees the threshold slot the bulk kernel read.
#include "launch.h"

namespace pslbm {

__global__ void __launch_bounds__(NTHREADS) k_vop(const Tile* __restrict__ tiles, int ntiles,
                                                   const DevInst* __restrict__ insts) {
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const Tile tl = tiles[ti];
    const DevInst* Ip = insts + tl.inst;
    const DevParams& P = Ip->P;
    const long long N = Ip->N;
    const unsigned long long step = Ip->scal[S_STEP];
    const int cur = int(step & 1ULL);
    uint8_t* tnew = Ip->type[cur ^ 1];
    const int x = tl.x0 + tx, y = tl.y0 + ty;
    if (x < P.nx && y < P.ny) {
      const long long node = (long long)y * P.nx + x;
      const uint8_t t = tnew[node] & T_MASK;
      if (is_mineral(t)) {
        double sB = 0.0, sF = 0.0;
        int nl = 0;
        int dirs[4];
        const bool useB = (t == T_SOLID_D) && P.iB >= 0 && P.k2 != 0.0;
        const bool useF = P.iF >= 0 && P.k4 != 0.0;
#pragma unroll
        for (int b = 1; b < 5; ++b) {
          int xn, yn;
          if (!nbr(P, x, y, EX(b), EY(b), xn, yn)) continue;
          const long long nn = (long long)yn * P.nx + xn;
          if ((tnew[nn] & T_MASK) != T_LIQUID) continue;
          dirs[nl++] = b;
          const int link = OPP(b) - 1;   // direction from the neighbour toward this node
          if (useB) sB += Ip->q[(0LL * 4 + link) * N + nn];
          if (useF) sF += Ip->q[(1LL * 4 + link) * N + nn];
        }
        if (nl > 0) {
          double VD = Ip->V[node], VF = Ip->V[N + node];
          if (t == T_SOLID_D) VD = VD - P.Vbar_D * sB;   // Eq. 33
          VF = VF + P.Vbar_F * sF;                        // Eq. 35 (precipitation adds volume)
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
          Ip->V[node] = VD;
          Ip->V[N + node] = VF;
          if (code != EV_NONE) {
            Ip->evt[node] = (uint8_t)code;
            const unsigned long long slot = atomicAdd(&Ip->scal[S_NEVENT], 1ULL);
            if (slot < (unsigned long long)Ip->evcap)
              Ip->evlist[slot] = (int)node;
            else
              atomicOr(&Ip->scal[S_STATUS], (unsigned long long)ST_EVOVERFLOW);
          }
        }
      }
    }
    // last tile of this instance: advance the step counter, free the threshold slot
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned long long done = atomicAdd(&Ip->scal[S_DONE], 1ULL);
      if (done == (unsigned long long)(Ip->ntiles - 1)) {
        __threadfence();
        Ip->scal[S_DONE] = 0;
        Ip->scal[S_MAX0 + cur] = 0ULL;
        Ip->scal[S_STEP] = step + 1;
        __threadfence();
      }
    }
    __syncthreads();
  }
}

void launch_vop(cudaStream_t s, const Tile* tiles, int ntiles, const DevInst* insts) {
  if (ntiles <= 0) return;
  k_vop<<<ntiles, NTHREADS, 0, s>>>(tiles, ntiles, insts);
}

}  // namespace pslbm
