// Van Leer variant of MUSCL-Hancock (VL, Sec. 2; Falle 1991) for one patch
// group, streamed along z.
//
// Sec. 2: the half-step solution comes from first-order fluxes computed with
// the Riemann solver on the cell-centred data before the reconstruction; the
// half-step state is then reconstructed (no characteristic tracing), three
// Riemann solves per cell give the fluxes of the full-step update from U^n.
//
// Each stage runs one plane behind the stage it reads, so that one iteration
// needs two barrier intervals.  With a = t-2-S (the U^n plane loaded by
// iteration t), b = a-1, c = a-2, d = a-3-S:
//   1  B  first-order fluxes: x/y faces of plane b, z faces below it;
//      D  reconstruct plane d of the half-step state (planes d-S..d+S, made
//         by earlier iterations);
//      F  update of plane d-2 (its fluxes are complete);
//   2  A  global reads of plane a issued into registers,
//      C  half step U^{n+1/2} of plane c -> primitives,
//      E  final fluxes: x/y faces of plane d, z faces below it,
//      A  then stored in the U^n ring (3 planes: a, and b, c still read).
// The half-step state covers the cells [-1-S, N+S]^2 of each plane, the
// first-order fluxes the faces of those cells.  In a uniform field the CTA
// streams through a chain of K groups stacked along z (planes 0..KN-1)
// without restarting.
#pragma once
#include <cuda_pipeline.h>

#include "stages.cuh"

namespace hyd {

template <int N, int S> struct VlLayout {
  static constexpr int L = N + 2;
  static constexpr int LH = N + 2 + 2 * S;  // half-step cells [-1-S, N+S]
  static constexpr int LU = N + 4 + 2 * S;  // U^n cells [-2-S, N+1+S]
  using UR = PlaneRing<float, LU, 3>;
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

// Reconstruction of the half-step state on plane pD for the face states of
// one cell (item idx of 2 nx + N^2: x, y, then z direction; nx = L N on the
// interior planes, else 0).
template <class T, int REC, bool CH, int N, class WRing, class FR>
__device__ __forceinline__ void vl_recon_item(const WRing& Wh, const FR& R, int pD, int idx, int nx, const Opts<T>& o) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  constexpr int L = N + 2;
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

template <class T, class S, bool MIXED, int RS, int REC, bool CH, int N, bool GCH>
__device__ void vl_group(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, T* ring, int K, unsigned* sts) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  using Lay = VlLayout<N, S_>;
  constexpr int L = Lay::L, LH = Lay::LH, LU = Lay::LU;
  constexpr int PLU = LU * LU;
  PlaneRing<T, LU, 3> Ur{ring};
  PlaneRing<T, LH, 2 * S_ + 1> Wh{ring + Lay::OFF_W};
  FaceRings<T, N, 1, 2> R{ring + Lay::OFF_FR};
  VlF1<T, N, S_> F1{ring + Lay::OFF_F1};
  const int tid = threadIdx.x, nthr = blockDim.x;
  const T h0 = C.hdtdx[0], h1 = C.hdtdx[1], h2 = C.hdtdx[2];
  const int NP = K * N;

  const int T_ITERS = NP + 7 + 2 * S_;
  for (int t = 0; t < T_ITERS; ++t) {
    const int a = t - 2 - S_;
    const int b = a - 1;
    const int c = a - 2;
    const int d = a - 3 - S_;
    const int f = d - 2;
    // ---- 1: B (first-order fluxes of plane b), D (reconstruction of plane
    //         d), F (update of plane f), one flat list of items ------------
    {
      const bool bz = b >= -1 - S_ && b <= NP + 1 + S_;
      const bool bxy = b >= -1 - S_ && b <= NP + S_;
      const int nxB = bxy ? LH * (LH + 1) : 0;
      const int cntB = bz ? 2 * nxB + LH * LH : 0;
      const bool dz = d >= -1 && d <= NP;
      const int nxD = (d >= 0 && d < NP) ? L * N : 0;
      const int cntD = dz ? 2 * nxD + N * N : 0;
      const int cntF = (f >= 0 && f < NP) ? N * N : 0;
      const int cnt = cntB + cntD + cntF;
      for (int idx = tid; idx < cnt; idx += nthr) {
        if (idx < cntB) {
          const T *pl, *pr;
          T* pf;
          int dd, fs;
          if (idx < nxB) {
            int jj = idx / (LH + 1), fc = idx - jj * (LH + 1);
            dd = 0;
            pl = &Ur(b, 0, jj + 1, fc);
            pr = &Ur(b, 0, jj + 1, fc + 1);
            pf = &F1.x(b, 0, jj, fc);
            fs = LH * (LH + 1);
          } else if (idx < 2 * nxB) {
            int k = idx - nxB;
            int fc = k / LH, ii = k - fc * LH;
            dd = 1;
            pl = &Ur(b, 0, fc, ii + 1);
            pr = &Ur(b, 0, fc + 1, ii + 1);
            pf = &F1.y(b, 0, fc, ii);
            fs = (LH + 1) * LH;
          } else {
            int k = idx - 2 * nxB;
            int jj = k / LH, ii = k - jj * LH;
            dd = 2;
            pl = &Ur(b - 1, 0, jj + 1, ii + 1);
            pr = &Ur(b, 0, jj + 1, ii + 1);
            pf = &F1.z(b, 0, jj, ii);
            fs = LH * LH;
          }
          const LocalComps lc(dd);
          T UL[5], UR[5], F[5];
          load_local(pl, PLU, lc, UL);
          load_local(pr, PLU, lc, UR);
          const unsigned s = riemann_local<T, MIXED, RS>(UL, UR, o, F);
          store_local(pf, fs, lc, F);
          // a group's own first-order fluxes: x/y faces of its planes
          // [-1-S, N+S], z faces below its planes [-1-S, N+1+S]
          mark_status<N>(sts, K, b, -1 - S_, dd == 2 ? 2 + S_ : 1 + S_, s);
        } else if (idx < cntB + cntD) {
          vl_recon_item<T, REC, CH, N>(Wh, R, d, idx - cntB, nxD, o);
        } else {
          update_item<T, S, MIXED, N>(C, o, R, f, K, sts, idx - cntB - cntD);
        }
      }
    }
    __syncthreads();

    // ---- 2: A (plane a) around C (half step of plane c) and E (final
    //         fluxes of plane d) -------------------------------------------
    {
      const int na = (a <= NP + 1 + S_) ? PLU : 0;
      const int cntC = (c >= -1 - S_ && c <= NP + S_) ? LH * LH : 0;
      const int nxE = (d >= 0 && d < NP) ? N * (N + 1) : 0;
      const int cntE = (d >= 0 && d <= NP) ? 2 * nxE + N * N : 0;
      const int ne = cntC + cntE;
      // FP32 forms: plane a goes straight into its ring slot (the slot of
      // plane a-3, which nothing reads any more) by asynchronous global-to-
      // shared copies, all in flight while C and E run.  FP64 (rings in
      // global memory): load items go to the threads with the fewest C/E
      // items, their first cell's reads issued before C and E.
      constexpr bool ASYNC = sizeof(T) == 4 && sizeof(S) == 4;
      if constexpr (ASYNC) {
        for (int k = tid; k < na; k += nthr) {
          const int jj = k / LU, ii = k - jj * LU;
          long long vs;
          const S* src = C.src5(ii - 2 - S_, jj - 2 - S_, a, vs);
#pragma unroll
          for (int v = 0; v < 5; ++v) __pipeline_memcpy_async(&Ur(a, v, jj, ii), src + v * vs, sizeof(T));
        }
        __pipeline_commit();
      }
      const int aw0 = ne % nthr;
      const int naw = nthr - aw0;
      const int atid = ASYNC ? -1 : tid - aw0;
      T Ua0[5];
      if (atid >= 0 && atid < na) {
        int jj = atid / LU, ii = atid - jj * LU;
        C.load5(ii - 2 - S_, jj - 2 - S_, a, Ua0);
      }
      // the final solves first, on all threads; the half-step items then go
      // to the threads with one solve fewer (from cntE % nthr on) when those
      // can take them at 3 a thread, else to all threads
      for (int idx = tid; idx < cntE; idx += nthr) flux2_item<T, S, MIXED, RS, N>(C, o, R, d, K, sts, idx, nxE);
      const int cw = 3 * (nthr - cntE % nthr) >= cntC ? cntE % nthr : 0;
      for (int idx = tid - cw; idx >= 0 && idx < cntC; idx += nthr - cw) {
        // unsplit half step of plane c, U^{n+1/2} = U^n - S, then primitives
        int jj = idx / LH, ii = idx - jj * LH;
        T Uh[5], W[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          T Sv = h0 * (F1.x(c, v, jj, ii + 1) - F1.x(c, v, jj, ii)) +
                 h1 * (F1.y(c, v, jj + 1, ii) - F1.y(c, v, jj, ii)) +
                 h2 * (F1.z(c + 1, v, jj, ii) - F1.z(c, v, jj, ii));
          Uh[v] = Ur(c, v, jj + 1, ii + 1) - Sv;
        }
        prim<T, MIXED>(Uh, W, o.gas);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wh(c, v, jj, ii) = W[v];
      }
      for (int k = atid; atid >= 0 && k < na; k += naw) {
        int jj = k / LU, ii = k - jj * LU;
        T U[5];
        if (k == atid) {
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = Ua0[v];
        } else {
          C.load5(ii - 2 - S_, jj - 2 - S_, a, U);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) Ur(a, v, jj, ii) = U[v];
      }
      if constexpr (ASYNC) __pipeline_wait_prior(0);
    }
    __syncthreads();
  }
}

}  // namespace hyd
