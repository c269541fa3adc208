// Van Leer variant of MUSCL-Hancock (VL, Sec. 2; Falle 1991) for one patch
// group, streamed along z.
//
// Sec. 2: the half-step solution comes from first-order fluxes computed with
// the Riemann solver on the cell-centred data before the reconstruction; the
// half-step state is then reconstructed (no characteristic tracing), three
// Riemann solves per cell give the fluxes of the full-step update from U^n.
//
// Iteration t:  F  update of plane pD-2 (completed by the previous iteration)
//               A  load plane pA = t-2-S of U^n (conserved)
//               B  first-order fluxes: x/y faces of plane pA, z faces below it
//               C  half step U^{n+1/2} of plane pC = pA-1 -> primitives
//               D  reconstruct plane pD = pC-S of the half-step state
//               E  final fluxes: x/y faces of plane pD, z faces below it
// The half-step state covers the cells [-1-S, N+S]^2 of each plane, the
// first-order fluxes the faces of those cells.  In a uniform field the CTA
// streams through a chain of K groups stacked along z (planes 0..KN-1)
// without restarting.
#pragma once
#include "stages.cuh"

namespace hyd {

template <int N, int S> struct VlLayout {
  static constexpr int L = N + 2;
  static constexpr int LH = N + 2 + 2 * S;  // half-step cells [-1-S, N+S]
  static constexpr int LU = N + 4 + 2 * S;  // U^n cells [-2-S, N+1+S]
  using UR = PlaneRing<float, LU, 2>;
  using WR = PlaneRing<float, LH, 2 * S + 1>;
  using FRf = FaceRings<float, N, 1, 2>;
  static constexpr int F1X = 5 * LH * (LH + 1);  // [var][LH rows][LH+1 faces]
  static constexpr int F1XYPL = 2 * F1X;
  static constexpr int F1ZPL = 5 * LH * LH;
  static constexpr int OFF_W = UR::ELEMS;
  static constexpr int OFF_FR = OFF_W + WR::ELEMS;
  static constexpr int OFF_F1 = OFF_FR + FRf::ELEMS;
  static constexpr int TOTAL = OFF_F1 + 2 * F1XYPL + 2 * F1ZPL;
};

template <class T, int N, int S> struct VlF1 {
  using Lay = VlLayout<N, S>;
  static constexpr int LH = Lay::LH;
  T* base;
  // face f lies between half-step-domain cells f-1 and f (U ring columns f and f+1)
  __device__ __forceinline__ T& x(int p, int v, int jj, int f) const {
    return base[slot<2>(p) * Lay::F1XYPL + (v * LH + jj) * (LH + 1) + f];
  }
  __device__ __forceinline__ T& y(int p, int v, int f, int ii) const {
    return base[slot<2>(p) * Lay::F1XYPL + Lay::F1X + (v * (LH + 1) + f) * LH + ii];
  }
  __device__ __forceinline__ T& z(int p, int v, int jj, int ii) const {
    return base[2 * Lay::F1XYPL + slot<2>(p) * Lay::F1ZPL + (v * LH + jj) * LH + ii];
  }
};

template <class T, class S, bool MIXED, int RS, int REC, bool CH, int N>
__device__ void vl_group(const GroupCtx<T, S, N>& C, const Opts<T>& o, T* ring, int K, unsigned* sts) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  using Lay = VlLayout<N, S_>;
  constexpr int L = Lay::L, LH = Lay::LH, LU = Lay::LU;
  PlaneRing<T, LU, 2> Ur{ring};
  PlaneRing<T, LH, 2 * S_ + 1> Wh{ring + Lay::OFF_W};
  FaceRings<T, N, 1, 2> R{ring + Lay::OFF_FR};
  VlF1<T, N, S_> F1{ring + Lay::OFF_F1};
  const int tid = threadIdx.x, nthr = blockDim.x;
  const T h0 = C.hdtdx[0], h1 = C.hdtdx[1], h2 = C.hdtdx[2];
  const int NP = K * N;

  const int T_ITERS = NP + 5 + 2 * S_;
  for (int t = 0; t < T_ITERS; ++t) {
    const int pA = t - 2 - S_;
    const int pC = pA - 1;
    const int pD = pC - S_;
    const int pF = pD - 2;
    if (pF >= 0 && pF < NP) stage_update<T, S, MIXED, N>(C, o, R, pF, K, sts);
    if (pA <= NP + 1 + S_) stage_load<false, T, S, MIXED, N, LU, 2>(C, o, pA, 2 + S_, Ur);
    __syncthreads();

    // B: first-order fluxes on the cell-centred data
    if (pA <= NP + 1 + S_) {
      const bool xy = pA >= -1 - S_ && pA <= NP + S_;
      const int nx = xy ? LH * (LH + 1) : 0;
      const int nz = pA >= -1 - S_ ? LH * LH : 0;
      const int cnt = 2 * nx + nz;
      constexpr int PLU = LU * LU;
      for (int idx = tid; idx < cnt; idx += nthr) {
        const T *pl, *pr;
        T* pf;
        int d, fs;
        if (idx < nx) {
          int jj = idx / (LH + 1), f = idx - jj * (LH + 1);
          d = 0;
          pl = &Ur(pA, 0, jj + 1, f);
          pr = &Ur(pA, 0, jj + 1, f + 1);
          pf = &F1.x(pA, 0, jj, f);
          fs = LH * (LH + 1);
        } else if (idx < 2 * nx) {
          int k = idx - nx;
          int f = k / LH, ii = k - f * LH;
          d = 1;
          pl = &Ur(pA, 0, f, ii + 1);
          pr = &Ur(pA, 0, f + 1, ii + 1);
          pf = &F1.y(pA, 0, f, ii);
          fs = (LH + 1) * LH;
        } else {
          int k = idx - 2 * nx;
          int jj = k / LH, ii = k - jj * LH;
          d = 2;
          pl = &Ur(pA - 1, 0, jj + 1, ii + 1);
          pr = &Ur(pA, 0, jj + 1, ii + 1);
          pf = &F1.z(pA, 0, jj, ii);
          fs = LH * LH;
        }
        const LocalComps lc(d);
        T UL[5], UR[5], F[5];
        load_local(pl, PLU, lc, UL);
        load_local(pr, PLU, lc, UR);
        const unsigned s = riemann_local<T, MIXED, RS>(UL, UR, o, F);
        store_local(pf, fs, lc, F);
        // a group's own first-order fluxes: x/y faces of its planes
        // [-1-S, N+S], z faces below its planes [-1-S, N+1+S]
        mark_status<N>(sts, K, pA, -1 - S_, d == 2 ? 2 + S_ : 1 + S_, s);
      }
    }
    __syncthreads();

    // C: unsplit half step of plane pC, U^{n+1/2} = U^n - S, then primitives
    if (pC >= -1 - S_ && pC <= NP + S_) {
      for (int idx = tid; idx < LH * LH; idx += nthr) {
        int jj = idx / LH, ii = idx - jj * LH;
        T Uh[5], W[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          T Sv = h0 * (F1.x(pC, v, jj, ii + 1) - F1.x(pC, v, jj, ii)) +
                 h1 * (F1.y(pC, v, jj + 1, ii) - F1.y(pC, v, jj, ii)) +
                 h2 * (F1.z(pC + 1, v, jj, ii) - F1.z(pC, v, jj, ii));
          Uh[v] = Ur(pC, v, jj + 1, ii + 1) - Sv;
        }
        prim<T, MIXED>(Uh, W, o.gas);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wh(pC, v, jj, ii) = W[v];
      }
    }
    __syncthreads();

    // D: reconstruction of the half-step state on plane pD (no tracing)
    if (pD >= -1 && pD <= NP) {
      const bool xy = pD >= 0 && pD < NP;
      const int nx = xy ? L * N : 0;
      const int cnt = 2 * nx + N * N;
      for (int idx = tid; idx < cnt; idx += nthr) {
        int d, jj, ii;  // face-ring coordinates of the cell
        if (idx < nx) {
          d = 0;
          int j = idx / L;
          ii = idx - j * L;
          jj = j + 1;
        } else if (idx < 2 * nx) {
          d = 1;
          int k = idx - nx;
          jj = k / N;
          ii = k - jj * N + 1;
        } else {
          d = 2;
          int k = idx - 2 * nx;
          int j = k / N;
          jj = j + 1;
          ii = k - j * N + 1;
        }
        T w[5][5], Wf[2][5], dW[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
#pragma unroll
          for (int o2 = -S_; o2 <= S_; ++o2) {
            if (d == 0) w[v][o2 + 2] = Wh(pD, v, jj + S_, ii + S_ + o2);
            else if (d == 1) w[v][o2 + 2] = Wh(pD, v, jj + S_ + o2, ii + S_);
            else w[v][o2 + 2] = Wh(pD + o2, v, jj + S_, ii + S_);
          }
        }
        if constexpr (CH) {
          // characteristic variables in the frame of d
          T wl[5][5], fl[2][5];
#pragma unroll
          for (int o2 = 2 - S_; o2 <= 2 + S_; ++o2) {
            T g[5], l[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) g[v] = w[v][o2];
            to_local_rt(d, g, l);
#pragma unroll
            for (int v = 0; v < 5; ++v) wl[v][o2] = l[v];
          }
          recon5c<REC>(wl, o, fl[0], fl[1], dW);
          to_global_rt(d, fl[0], Wf[0]);
          to_global_rt(d, fl[1], Wf[1]);
        } else {
          recon5<REC>(w, o, Wf[0], Wf[1], dW);
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          T U[5];
          cons(Wf[s], U, o.gas);
          if (d < 2) {
#pragma unroll
            for (int v = 0; v < 5; ++v) R.XY(pD, d, s, v, jj, ii) = U[v];
          } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) R.Zs(pD, s, v, jj, ii) = U[v];
          }
        }
      }
    }
    __syncthreads();

    // E: 3 Riemann solves per cell (x/y faces of plane pD, z faces below it)
    if (pD >= 0 && pD <= NP) stage_flux2<T, S, MIXED, RS, N>(C, o, R, pD, K, sts);
    __syncthreads();
  }
}

}  // namespace hyd
