// MUSCL-Hancock (MHM, Sec. 2) for one patch group, streamed along z.
//
// Sec. 2: the half-step face values are obtained from the reconstructed face
// values with their physical fluxes (no Riemann solver), advanced by dt/2 with
// the flux differences of all three directions; Sec. 3.1: all six face values
// of a cell are evaluated before moving to the next cell, so the fluxes stay
// in registers.  Then 3 Riemann solves per cell and the update.
//
// In a uniform field the CTA streams through a chain of K groups stacked
// along z (planes 0..KN-1) without restarting.
//
// The planes -1-S..-1+S are loaded first; iteration t then runs two barrier
// intervals for the plane pB = t-1:
//   1  F  update of plane pB-2 (its fluxes are complete);
//      B  reconstruct + predict the 6 face states of the cells [-1,N]^2 of
//         plane pB;
//   2  A  global reads of the input plane pA = pB+S+1 issued into registers,
//      C  final fluxes: x/y faces of plane pB, z faces below it,
//      A  then converted to primitives and stored in the ring (in the slot
//         of plane pB-S, which B has finished with).
#pragma once
#include <cuda_pipeline.h>

#include "stages.cuh"

namespace hyd {

template <int N, int S> struct MhmLayout {
  static constexpr int L = N + 2;
  static constexpr int LW = N + 2 + 2 * S;
  using WR = PlaneRing<float, LW, 2 * S + 1>;
  using FRf = FaceRings<float, N, 1, 2>;
  static constexpr int OFF_FR = WR::ELEMS;
  static constexpr int TOTAL = OFF_FR + FRf::ELEMS;
};

// Physical flux along d of a global-frame face state (W primitive, U its
// conserved form; energy U[4]).
template <int D, class T> __device__ __forceinline__ void pflux_global(const T W[5], const T U[5], T F[5]) {
  T wl[5], fl[5];
  rot_in<D>(W, wl);
  pflux(wl, U[4], fl);
  rot_out<D>(fl, F);
}

// Reconstruction along D of the cell (jj, ii) of plane p (primitive
// variables, or with CH characteristic ones in the frame of D), its two face
// states (conserved) and their physical fluxes along D.
template <int D, int REC, bool CH, class T, class WRing>
__device__ __forceinline__ void mhm_faces(const WRing& Wr, int p, int jj, int ii, const Opts<T>& o, T Uf[2][5],
                                          T Ff[2][5]) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  T w[5][5], Wf[2][5], dW[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
#pragma unroll
    for (int o2 = -S_; o2 <= S_; ++o2) {
      if (D == 0) w[v][o2 + 2] = Wr(p, v, jj + S_, ii + S_ + o2);
      else if (D == 1) w[v][o2 + 2] = Wr(p, v, jj + S_ + o2, ii + S_);
      else w[v][o2 + 2] = Wr(p + o2, v, jj + S_, ii + S_);
    }
  }
  if constexpr (CH) {
    T wl[5][5], fl[2][5];
#pragma unroll
    for (int o2 = 2 - S_; o2 <= 2 + S_; ++o2) {
      T g[5], l[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) g[v] = w[v][o2];
      rot_in<D>(g, l);
#pragma unroll
      for (int v = 0; v < 5; ++v) wl[v][o2] = l[v];
    }
    recon5c<REC>(wl, o, fl[0], fl[1], dW);
    rot_out<D>(fl[0], Wf[0]);
    rot_out<D>(fl[1], Wf[1]);
  } else {
    recon5<REC>(w, o, Wf[0], Wf[1], dW);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    cons(Wf[s], Uf[s], o.gas);
    pflux_global<D>(Wf[s], Uf[s], Ff[s]);
  }
}

template <class T, class S, bool MIXED, int RS, int REC, bool CH, int N, bool GCH>
__device__ void mhm_group(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, T* ring, int K, unsigned* sts) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  using Lay = MhmLayout<N, S_>;
  constexpr int L = Lay::L, LL = L * L, LW = Lay::LW;
  PlaneRing<T, LW, 2 * S_ + 1> Wr{ring};
  FaceRings<T, N, 1, 2> R{ring + Lay::OFF_FR};
  const T h0 = C.hdtdx[0], h1 = C.hdtdx[1], h2 = C.hdtdx[2];
  const int NP = K * N;
  const int tid = threadIdx.x, nthr = blockDim.x;

  for (int p = -1 - S_; p <= -1 + S_; ++p) stage_load<true, T, S, MIXED, N, LW, 2 * S_ + 1>(C, o, p, 1 + S_, Wr);
  __syncthreads();

  const int T_ITERS = NP + 3;
  for (int t = 0; t < T_ITERS; ++t) {
    const int pB = t - 1;
    const int pF = pB - 2;
    const int pA = pB + S_ + 1;
    // ---- 1: F (update of plane pF) and B (prediction of plane pB) ---------
    // the update items (whose reads of U^n wait on global memory) go to the
    // whole warps after the prediction items when there are at least two
    // such warps, so no warp does both; else to all threads
    {
      const int fw0 = (LL + 31) & ~31;
      const int t0 = (pB <= NP && nthr - fw0 >= 64) ? fw0 : 0;
      if (pF >= 0 && pF < NP) stage_update<T, S, MIXED, N>(C, o, R, pF, K, sts, t0);
    }
    if (pB <= NP) {
      for (int idx = tid; idx < LL; idx += nthr) {
        int jj = idx / L, ii = idx - jj * L;
        T Uf[3][2][5], Ff[3][2][5];
        mhm_faces<0, REC, CH>(Wr, pB, jj, ii, o, Uf[0], Ff[0]);
        mhm_faces<1, REC, CH>(Wr, pB, jj, ii, o, Uf[1], Ff[1]);
        mhm_faces<2, REC, CH>(Wr, pB, jj, ii, o, Uf[2], Ff[2]);
        // S = dt/(2dx) (Fx(R) - Fx(L)) + dt/(2dy) (...) + dt/(2dz) (...)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          T Sv = h0 * (Ff[0][1][v] - Ff[0][0][v]) + h1 * (Ff[1][1][v] - Ff[1][0][v]) + h2 * (Ff[2][1][v] - Ff[2][0][v]);
          R.XY(pB, 0, 0, v, jj, ii) = Uf[0][0][v] - Sv;
          R.XY(pB, 0, 1, v, jj, ii) = Uf[0][1][v] - Sv;
          R.XY(pB, 1, 0, v, jj, ii) = Uf[1][0][v] - Sv;
          R.XY(pB, 1, 1, v, jj, ii) = Uf[1][1][v] - Sv;
          R.Zs(pB, 0, v, jj, ii) = Uf[2][0][v] - Sv;
          R.Zs(pB, 1, v, jj, ii) = Uf[2][1][v] - Sv;
        }
      }
    }
    __syncthreads();

    // ---- 2: A (next input plane) around C (3 Riemann solves per cell) -----
    {
      const int nx = (pB >= 0 && pB < NP) ? N * (N + 1) : 0;
      const int ne = (pB >= 0 && pB <= NP) ? 2 * nx + N * N : 0;
      const int na = (pA <= NP + S_) ? LW * LW : 0;
      // FP32 forms: the conserved values of plane pA go straight into its
      // ring slot (that of plane pB-S, which B has finished with) by
      // asynchronous global-to-shared copies, all in flight during C; each
      // thread converts the cells it copied, in place, after its own copies
      // have landed.  FP64 (ring in global memory): load items go to the
      // threads with the fewest face items (thread t has one face item more
      // than the others below ne % nthr).
      constexpr bool ASYNC = sizeof(T) == 4 && sizeof(S) == 4;
      // copies (and their conversions) go to the threads with the fewest
      // face items when there are enough of them, else to all threads
      const int cw0 = ASYNC && 4 * (nthr - ne % nthr) >= nthr ? ne % nthr : 0;
      if constexpr (ASYNC) {
        for (int k = tid - cw0; k >= 0 && k < na; k += nthr - cw0) {
          const int jj = k / LW, ii = k - jj * LW;
          long long vs;
          const S* src = C.src5(ii - 1 - S_, jj - 1 - S_, pA, vs);
#pragma unroll
          for (int v = 0; v < 5; ++v) __pipeline_memcpy_async(&Wr(pA, v, jj, ii), src + v * vs, sizeof(T));
        }
        __pipeline_commit();
      }
      const int aw0 = ne % nthr;
      const int naw = nthr - aw0;
      const int atid = ASYNC ? -1 : tid - aw0;
      T Ua0[5];
      if (atid >= 0 && atid < na) {
        int jj = atid / LW, ii = atid - jj * LW;
        C.load5(ii - 1 - S_, jj - 1 - S_, pA, Ua0);
      }
      if (ne) stage_flux2<T, S, MIXED, RS, N>(C, o, R, pB, K, sts);
      for (int k = atid; atid >= 0 && k < na; k += naw) {
        int jj = k / LW, ii = k - jj * LW;
        T U[5], W[5];
        if (k == atid) {
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = Ua0[v];
        } else {
          C.load5(ii - 1 - S_, jj - 1 - S_, pA, U);
        }
        prim<T, MIXED>(U, W, o.gas);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wr(pA, v, jj, ii) = W[v];
      }
      if constexpr (ASYNC) {
        __pipeline_wait_prior(0);
        for (int k = tid - cw0; k >= 0 && k < na; k += nthr - cw0) {
          const int jj = k / LW, ii = k - jj * LW;
          T U[5], W[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = Wr(pA, v, jj, ii);
          prim<T, MIXED>(U, W, o.gas);
#pragma unroll
          for (int v = 0; v < 5; ++v) Wr(pA, v, jj, ii) = W[v];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace hyd
