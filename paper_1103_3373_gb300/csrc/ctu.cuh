// Simplified 6-solve CTU (Sec. 2, steps (1)-(5); Gardiner & Stone 2008) for
// one patch group, streamed plane by plane along z.
//
// The paper's GPU solver keeps whole-group face values and fluxes in global
// memory (Sec. 3.1).  Here each CTA walks its group along z and keeps only the
// planes still needed in small ring buffers (shared memory for FP32, a
// per-CTA slice of an L2-resident workspace for FP64).  At iteration t the CTA
//   A  loads plane pA = t-1-S and converts it to primitives        (W ring)
//   B  reconstructs + traces the cells of plane pB = pA-S to t+dt/2 in all
//      three directions (step (1))                         (face-state rings)
//   C  solves the stage-1 Riemann problems on the x/y faces of plane pB and
//      the z faces between pB-1 and pB (step (2))            (flux rings)
//   D  applies the transverse flux-gradient correction to the face states of
//      plane pD = pB-1 (step (3))
//   E  solves the stage-2 Riemann problems of plane pD (x/y) and of the z faces
//      below it, storing group-boundary fluxes at once (steps (3) and (5))
//   F  updates plane pD-1 (step (4)); it runs at the start of the next
//      iteration, in the same barrier interval as that iteration's A (the two
//      touch disjoint buffers)
// with S the reconstruction stencil (1 PLM, 2 PPM).  Every stage is a flat
// loop of the CTA's threads over the plane's work items (Sec. 3.1's
// index-flattening), separated by block barriers.
//
// Index ranges (interior coordinates, cells 0..N-1):
//   traced states on cells [-1,N]^3; stage-1 fluxes on the faces of those
//   cells; corrected states on cells [-1,N] along their normal and [0,N-1]
//   laterally; stage-2 fluxes on the faces of the interior cells.
#pragma once
#include "stages.cuh"

namespace hyd {

// Scratch of one CTA: W ring | face states + final fluxes | stage-1 fluxes.
template <int N, int S> struct CtuLayout {
  static constexpr int L = N + 2;           // traced cells [-1, N]
  static constexpr int LW = N + 2 + 2 * S;  // W plane [-1-S, N+S]
  static constexpr int LL = L * L;
  using WR = PlaneRing<float, LW, 2 * S + 1>;
  using FRf = FaceRings<float, N, 2, 3>;
  static constexpr int F1X = 5 * L * (N + 1);  // [var][L rows][N+1 faces]
  static constexpr int F1XYPL = 2 * F1X;       // x then y ([var][N+1 faces][L cols])
  static constexpr int F1ZPL = 5 * LL;
  static constexpr int OFF_FR = WR::ELEMS;
  static constexpr int OFF_F1XY = OFF_FR + FRf::ELEMS;
  static constexpr int OFF_F1Z = OFF_F1XY + 2 * F1XYPL;
  static constexpr int TOTAL = OFF_F1Z + 2 * F1ZPL;
};

template <class T, int N, int S> struct CtuF1 {
  using Lay = CtuLayout<N, S>;
  T* base;
  // stage-1 x flux: face f (between cells f-1 and f), row jj
  __device__ __forceinline__ T& x(int p, int v, int jj, int f) const {
    return base[slot<2>(p) * Lay::F1XYPL + (v * Lay::L + jj) * (N + 1) + f];
  }
  __device__ __forceinline__ T& y(int p, int v, int f, int ii) const {
    return base[slot<2>(p) * Lay::F1XYPL + Lay::F1X + (v * (N + 1) + f) * Lay::L + ii];
  }
  // stage-1 z flux of the face below plane p
  __device__ __forceinline__ T& z(int p, int v, int jj, int ii) const {
    return base[2 * Lay::F1XYPL + slot<2>(p) * Lay::F1ZPL + (v * Lay::L + jj) * Lay::L + ii];
  }
};

template <class T, class S, bool MIXED, int RS, int REC, int N>
__device__ void ctu_group(const GroupCtx<T, S, N>& C, const Opts<T>& o, T* ring, unsigned& st_sh) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  using Lay = CtuLayout<N, S_>;
  constexpr int L = Lay::L, LL = Lay::LL, LW = Lay::LW;
  PlaneRing<T, LW, 2 * S_ + 1> Wr{ring};
  FaceRings<T, N, 2, 3> R{ring + Lay::OFF_FR};
  CtuF1<T, N, S_> F1{ring + Lay::OFF_F1XY};
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  unsigned st = 0;

  // one extra iteration drains the last update
  constexpr int T_ITERS = N + 4 + 2 * S_;
  for (int t = 0; t < T_ITERS; ++t) {
    const int pA = t - 1 - S_;
    const int pB = pA - S_;
    const int pD = pB - 1;
    const int pF = pD - 2;  // the plane whose final fluxes the previous iteration completed

    // ---- F (update of plane pF) and A (load of plane pA) ----------------
    if (pF >= 0 && pF < N) st |= stage_update<T, S, MIXED, N>(C, o, R, pF);
    if (pA <= N + S_) stage_load<true, T, S, MIXED, N, LW, 2 * S_ + 1>(C, o, pA, 1 + S_, Wr);
    __syncthreads();

    // ---- B: reconstruction + characteristic tracing of plane pB ---------
    if (pB >= -1 && pB <= N) {
      for (int idx = tid; idx < 3 * LL; idx += nthr) {
        int d = idx / LL;
        int rem = idx - d * LL;
        int jj = rem / L, ii = rem - jj * L;
        T w[5][5], WLf[5], WRf[5], dW[5], W0[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
#pragma unroll
          for (int o2 = -S_; o2 <= S_; ++o2) {
            if (d == 0) w[v][o2 + 2] = Wr(pB, v, jj + S_, ii + S_ + o2);
            else if (d == 1) w[v][o2 + 2] = Wr(pB, v, jj + S_ + o2, ii + S_);
            else w[v][o2 + 2] = Wr(pB + o2, v, jj + S_, ii + S_);
          }
          W0[v] = w[v][2];
        }
        recon5<REC>(w, o, WLf, WRf, dW);
        T w0l[5], a[5], b[5], tl[5], tr[5];
        rot_in(W0, w0l, d);
        if (REC == PPM) {
          rot_in(WLf, a, d);
          rot_in(WRf, b, d);
          trace_ppm(w0l, a, b, C.dtdx[d], o.gas, tl, tr);
        } else {
          rot_in(dW, a, d);
          trace_plm(w0l, a, C.dtdx[d], o.gas, tl, tr);
        }
        T wg[5], U[5];
        rot_out(tl, wg, d);
        cons(wg, U, o.gas);
        if (d < 2) {
#pragma unroll
          for (int v = 0; v < 5; ++v) R.XY(pB, d, 0, v, jj, ii) = U[v];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) R.Zs(pB, 0, v, jj, ii) = U[v];
        }
        rot_out(tr, wg, d);
        cons(wg, U, o.gas);
        if (d < 2) {
#pragma unroll
          for (int v = 0; v < 5; ++v) R.XY(pB, d, 1, v, jj, ii) = U[v];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) R.Zs(pB, 1, v, jj, ii) = U[v];
        }
      }
    }
    __syncthreads();

    // ---- C: stage-1 fluxes (x/y faces of plane pB, z faces below it) ----
    if (pB >= -1 && pB <= N) {
      constexpr int NX = L * (N + 1);
      const int nz = pB >= 0 ? LL : 0;
      const int cnt = 2 * NX + nz;
      for (int idx = tid; idx < cnt; idx += nthr) {
        T UL[5], UR[5], F[5];
        if (idx < NX) {
          int jj = idx / (N + 1), f = idx - jj * (N + 1);
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            UL[v] = R.XY(pB, 0, 1, v, jj, f);
            UR[v] = R.XY(pB, 0, 0, v, jj, f + 1);
          }
          st |= riemann<T, MIXED, RS>(0, UL, UR, o, F);
#pragma unroll
          for (int v = 0; v < 5; ++v) F1.x(pB, v, jj, f) = F[v];
        } else if (idx < 2 * NX) {
          int k = idx - NX;
          int f = k / L, ii = k - f * L;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            UL[v] = R.XY(pB, 1, 1, v, f, ii);
            UR[v] = R.XY(pB, 1, 0, v, f + 1, ii);
          }
          st |= riemann<T, MIXED, RS>(1, UL, UR, o, F);
#pragma unroll
          for (int v = 0; v < 5; ++v) F1.y(pB, v, f, ii) = F[v];
        } else {
          int k = idx - 2 * NX;
          int jj = k / L, ii = k - jj * L;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            UL[v] = R.Zs(pB - 1, 1, v, jj, ii);
            UR[v] = R.Zs(pB, 0, v, jj, ii);
          }
          st |= riemann<T, MIXED, RS>(2, UL, UR, o, F);
#pragma unroll
          for (int v = 0; v < 5; ++v) F1.z(pB, v, jj, ii) = F[v];
        }
      }
    }
    __syncthreads();

    // ---- D: transverse flux-gradient correction of plane pD -------------
    //   U -= dt/(2 dx_e) (F1_e(+1/2) - F1_e(-1/2)) for the two e != d, in
    //   increasing e
    if (pD >= -1 && pD <= N) {
      const bool xy = pD >= 0 && pD < N;
      const int nx = xy ? L * N : 0;  // x states: rows j in [0,N), cells ii in [0,L)
      const int cnt = 2 * nx + N * N;
      const T h0 = C.hdtdx[0], h1 = C.hdtdx[1], h2 = C.hdtdx[2];
      for (int idx = tid; idx < cnt; idx += nthr) {
        if (idx < nx) {
          int j = idx / L, ii = idx - j * L, jj = j + 1;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            T gy = F1.y(pD, v, jj, ii) - F1.y(pD, v, jj - 1, ii);
            T gz = F1.z(pD + 1, v, jj, ii) - F1.z(pD, v, jj, ii);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              T u = R.XY(pD, 0, side, v, jj, ii);
              u = u - h1 * gy;
              u = u - h2 * gz;
              R.XY(pD, 0, side, v, jj, ii) = u;
            }
          }
        } else if (idx < 2 * nx) {
          int k = idx - nx;
          int jj = k / N, i = k - jj * N, ii = i + 1;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            T gx = F1.x(pD, v, jj, ii) - F1.x(pD, v, jj, ii - 1);
            T gz = F1.z(pD + 1, v, jj, ii) - F1.z(pD, v, jj, ii);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              T u = R.XY(pD, 1, side, v, jj, ii);
              u = u - h0 * gx;
              u = u - h2 * gz;
              R.XY(pD, 1, side, v, jj, ii) = u;
            }
          }
        } else {
          int k = idx - 2 * nx;
          int j = k / N, i = k - j * N, jj = j + 1, ii = i + 1;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            T gx = F1.x(pD, v, jj, ii) - F1.x(pD, v, jj, ii - 1);
            T gy = F1.y(pD, v, jj, ii) - F1.y(pD, v, jj - 1, ii);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
              T u = R.Zs(pD, side, v, jj, ii);
              u = u - h0 * gx;
              u = u - h1 * gy;
              R.Zs(pD, side, v, jj, ii) = u;
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- E: stage-2 fluxes of plane pD, group-boundary fluxes (step 5) --
    if (pD >= 0 && pD <= N) st |= stage_flux2<T, S, MIXED, RS, N>(C, o, R, pD);
    __syncthreads();
  }
  if (st) atomicOr(&st_sh, st);
}

}  // namespace hyd
