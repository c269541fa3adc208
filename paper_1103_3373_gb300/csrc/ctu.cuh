// Simplified 6-solve CTU (Sec. 2, steps (1)-(5); Gardiner & Stone 2008) for
// one patch group, streamed plane by plane along z.
//
// The paper's GPU solver keeps whole-group face values and fluxes in global
// memory (Sec. 3.1).  Here each CTA walks its group along z and keeps only the
// planes still needed in ring buffers (shared memory for FP32, a per-CTA
// slice of an L2-resident workspace for FP64).  Iteration t works on three
// planes, q = t-1 (tracing), q-1 (final fluxes) and q-3 (update), in three
// barrier intervals:
//   S1  B: reconstruct + trace the cells of plane q to t+dt/2 in all three
//          directions (step (1));
//       F: conservative update of plane q-3 (step (4));
//   S2  C: stage-1 Riemann problems on the x/y faces of plane q and the z
//          faces between q-1 and q (step (2));
//   S3  E: stage-2 Riemann problems of plane q-1 (x/y faces) and of the z
//          faces below it; each face first applies the transverse
//          flux-gradient correction (step (3)) to its two states, and fluxes
//          on the group boundary are stored at once (step (5));
//       A: load of the next input plane (primitives).
// Every corrected state feeds exactly one face, so correcting inside the face
// item recomputes nothing.  In a uniform field the CTA streams through a
// chain of K groups stacked along z (planes 0..KN-1) without restarting, so
// the planes between two groups are traced and solved once.  The stages are flat loops of the CTA's threads
// over the plane's work items (Sec. 3.1's index flattening).
//
// Index ranges (interior coordinates, cells 0..N-1): traced states on the
// cells [-1,N]^3; stage-1 fluxes on the faces of those cells; corrected
// states on the cells [-1,N] along their normal and [0,N-1] laterally;
// stage-2 fluxes on the faces of the interior cells.
#pragma once
#include <cuda_pipeline.h>

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
  static constexpr int D1XY = 3;               // stage-1 x/y flux planes kept
  static constexpr int OFF_FR = WR::ELEMS;
  static constexpr int OFF_F1XY = OFF_FR + FRf::ELEMS;
  static constexpr int OFF_F1Z = OFF_F1XY + D1XY * F1XYPL;
  static constexpr int TOTAL = OFF_F1Z + 2 * F1ZPL;
};

template <class T, int N, int S> struct CtuF1 {
  using Lay = CtuLayout<N, S>;
  T* base;
  // stage-1 x flux: face f (between cells f-1 and f), row jj
  __device__ __forceinline__ T& x(int p, int v, int jj, int f) const {
    return base[slot<Lay::D1XY>(p) * Lay::F1XYPL + (v * Lay::L + jj) * (N + 1) + f];
  }
  __device__ __forceinline__ T& y(int p, int v, int f, int ii) const {
    return base[slot<Lay::D1XY>(p) * Lay::F1XYPL + Lay::F1X + (v * (N + 1) + f) * Lay::L + ii];
  }
  // stage-1 z flux of the face below plane p
  __device__ __forceinline__ T& z(int p, int v, int jj, int ii) const {
    return base[Lay::D1XY * Lay::F1XYPL + slot<2>(p) * Lay::F1ZPL + (v * Lay::L + jj) * Lay::L + ii];
  }
};

// Step (1) for one cell along direction d (known at run time; one inlined
// copy serves all three): reconstruction (of primitive or, with CH, of
// characteristic variables) of the primitive ring around
// (jj, ii) of plane p, characteristic tracing to t + dt/2.  The
// rotation into the local frame is folded into the shared-memory addressing;
// the traced states come back in the local frame (Ul, Ur conserved, normal
// momentum first).
template <int REC, int LIM, bool CH, class T, class WRing>
__device__ __forceinline__ void trace_cell_rt(const WRing& Wr, int p, int jj, int ii, int d, const LocalComps& lc,
                                              const Opts<T>& o, T dtdx, T Ul[5], T Ur[5]) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  constexpr int VS = WRing::PL / 5;  // variable stride of a W plane
  const int sx = d == 0, sy = d == 1, sz = d == 2;
  T w[5][5], WLf[5], WRf[5], dW[5], W0[5];
#pragma unroll
  for (int o2 = -S_; o2 <= S_; ++o2) {
    const T* base = &Wr(p + sz * o2, 0, jj + S_ + sy * o2, ii + S_ + sx * o2);
    T a[5];
    load_local(base, VS, lc, a);
#pragma unroll
    for (int v = 0; v < 5; ++v) w[v][o2 + 2] = a[v];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) W0[v] = w[v][2];
  recon5_local<REC, LIM, CH>(w, o, WLf, WRf, dW);
  T tl[5], tr[5];
  if (REC == PPM)
    trace_ppm(W0, WLf, WRf, dtdx, o.gas, tl, tr);
  else
    trace_plm(W0, dW, dtdx, o.gas, tl, tr);
  cons_local(tl, d, o.gas, Ul);
  cons_local(tr, d, o.gas, Ur);
}

// Transverse flux-gradient correction (step (3)) of one face state:
//   u = (u - h1 (G1+ - G1-)) - h2 (G2+ - G2-), the two other directions in
//   increasing order.
template <class T> __device__ __forceinline__ T correct(T u, T h1, T a1p, T a1m, T h2, T a2p, T a2m) {
  u = u - h1 * (a1p - a1m);
  u = u - h2 * (a2p - a2m);
  return u;
}

template <class T, class S, bool MIXED, int RS, int REC, int LIM, bool CH, int N, bool GCH>
__device__ __forceinline__ void ctu_group_impl(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, T* ring, int K,
                                               unsigned* sts) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  using Lay = CtuLayout<N, S_>;
  constexpr int L = Lay::L, LL = Lay::LL, LW = Lay::LW;
  PlaneRing<T, LW, 2 * S_ + 1> Wr{ring};
  FaceRings<T, N, 2, 3> R{ring + Lay::OFF_FR};
  CtuF1<T, N, S_> F1{ring + Lay::OFF_F1XY};
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const T h0 = C.hdtdx[0], h1 = C.hdtdx[1], h2 = C.hdtdx[2];
  const int NP = K * N;

  // prologue: the planes the first tracing needs
  for (int p = -1 - S_; p <= -1 + S_; ++p) stage_load<true, T, S, MIXED, N, LW, 2 * S_ + 1>(C, o, p, 1 + S_, Wr);
  __syncthreads();

  const int T_ITERS = NP + 4;
  for (int t = 0; t < T_ITERS; ++t) {
    const int q = t - 1;  // plane traced and given stage-1 fluxes
    const int r = q - 1;  // plane given stage-2 fluxes
    const int u = q - 3;  // plane updated
    // ---- S1: B (trace plane q) and F (update plane u) --------------------
    {
      // the update's reads of U^n are issued first and consumed after the
      // tracing, so their latency hides behind it
      const int nf = (u >= 0 && u < NP) ? N * N : 0;
      T Un0[5];
      const bool pre_f = tid < nf;
      if (pre_f) {
        int j = tid / N, i = tid - j * N;
#pragma unroll
        for (int v = 0; v < 5; ++v) Un0[v] = (T)C.load_raw(v, i, j, u);
      }
      if (q <= NP) {
        for (int k = tid; k < 3 * LL; k += nthr) {
          int d = k / LL;
          int rem = k - d * LL;
          int jj = rem / L, ii = rem - jj * L;
          T Ul[5], Ur[5];
          const LocalComps lc(d);
          trace_cell_rt<REC, LIM, CH>(Wr, q, jj, ii, d, lc, o, d == 0 ? C.dtdx[0] : (d == 1 ? C.dtdx[1] : C.dtdx[2]),
                                  Ul, Ur);
          T* dl = d < 2 ? &R.XY(q, d, 0, 0, jj, ii) : &R.Zs(q, 0, 0, jj, ii);
          T* dr = d < 2 ? &R.XY(q, d, 1, 0, jj, ii) : &R.Zs(q, 1, 0, jj, ii);
          store_local(dl, LL, lc, Ul);
          store_local(dr, LL, lc, Ur);
        }
      }
      for (int k = tid; k < nf; k += nthr) {
        int j = k / N, i = k - j * N;
        T Uc[5], dF[3][5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          Uc[v] = k == tid ? Un0[v] : (T)C.load_raw(v, i, j, u);
          dF[0][v] = R.F2x(u, v, j, i + 1) - R.F2x(u, v, j, i);
          dF[1][v] = R.F2y(u, v, j + 1, i) - R.F2y(u, v, j, i);
          dF[2][v] = R.F2z(u + 1, v, j, i) - R.F2z(u, v, j, i);
        }
        mark_status<N>(sts, K, u, 0, 0, update_cell_from<T, S, MIXED, N>(C, i, j, u, Uc, dF, o.gas));
      }
    }
    __syncthreads();

    // ---- S2: C, stage-1 fluxes (x/y faces of plane q, z faces below it) --
    if (q <= NP) {
      constexpr int NX = L * (N + 1);
      const int nz = q >= 0 ? LL : 0;
      const int cnt = 2 * NX + nz;
      for (int idx = tid; idx < cnt; idx += nthr) {
        // the two states (stride LL between variables) and the flux slot
        const T *pl, *pr;
        T* pf;
        int fs, d;
        if (idx < NX) {
          int jj = idx / (N + 1), f = idx - jj * (N + 1);
          d = 0;
          pl = &R.XY(q, 0, 1, 0, jj, f);
          pr = &R.XY(q, 0, 0, 0, jj, f + 1);
          pf = &F1.x(q, 0, jj, f);
          fs = L * (N + 1);
        } else if (idx < 2 * NX) {
          int k = idx - NX;
          int f = k / L, ii = k - f * L;
          d = 1;
          pl = &R.XY(q, 1, 1, 0, f, ii);
          pr = &R.XY(q, 1, 0, 0, f + 1, ii);
          pf = &F1.y(q, 0, f, ii);
          fs = (N + 1) * L;
        } else {
          int k = idx - 2 * NX;
          int jj = k / L, ii = k - jj * L;
          d = 2;
          pl = &R.Zs(q - 1, 1, 0, jj, ii);
          pr = &R.Zs(q, 0, 0, jj, ii);
          pf = &F1.z(q, 0, jj, ii);
          fs = LL;
        }
        const LocalComps lc(d);
        T UL[5], UR[5], F[5];
        load_local(pl, LL, lc, UL);
        load_local(pr, LL, lc, UR);
        const unsigned s = riemann_local<T, MIXED, RS>(UL, UR, o, F);
        store_local(pf, fs, lc, F);
        // a group's own stage-1 fluxes: x/y faces of its planes [-1, N], z
        // faces below its planes [0, N]
        mark_status<N>(sts, K, q, d == 2 ? 0 : -1, 1, s);
      }
    }
    __syncthreads();

    // ---- S3: E, corrected stage-2 fluxes of plane r; A, next input plane --
    {
      const int nx = (r >= 0 && r < NP) ? N * (N + 1) : 0;
      const int nz = (r >= 0 && r <= NP) ? N * N : 0;
      const int rk = r >= 0 ? r / N : 0;  // chain group of plane r
      const int ne = 2 * nx + nz;
      const int pa = q + 1 + S_;  // plane the next tracing needs last
      const int na = (pa <= NP + S_) ? LW * LW : 0;
      // the next plane's global loads are issued first and converted after
      // the Riemann work, so their latency hides behind it.  FP32 forms: as
      // asynchronous global-to-shared copies of the conserved values straight
      // into the plane's ring slot (that of plane q-S, which the tracing has
      // finished with), every copy in flight at once; each thread converts
      // the cells it copied, in place, once its own copies have landed.
      // FP64 (ring in global memory): the load items go to the threads with
      // the fewest face items (thread t has ceil((ne - t) / nthr) of them,
      // one more below ne % nthr), their first cell's reads issued first.
      constexpr bool ASYNC = sizeof(T) == 4 && sizeof(S) == 4;
      // copies (and their conversions) go to the threads with the fewest
      // face items when there are enough of them, else to all threads
      const int cw0 = ASYNC && 4 * (nthr - ne % nthr) >= nthr ? ne % nthr : 0;
      if constexpr (ASYNC) {
        for (int k = tid - cw0; k >= 0 && k < na; k += nthr - cw0) {
          const int jj = k / LW, ii = k - jj * LW;
          long long vs;
          const S* src = C.src5(ii - 1 - S_, jj - 1 - S_, pa, vs);
#pragma unroll
          for (int v = 0; v < 5; ++v) __pipeline_memcpy_async(&Wr(pa, v, jj, ii), src + v * vs, sizeof(T));
        }
        __pipeline_commit();
      }
      const int aw0 = ne % nthr;
      const int naw = nthr - aw0;
      const int atid = ASYNC ? -1 : tid - aw0;
      T Ua0[5];
      if (atid >= 0 && atid < na) {
        int jj = atid / LW, ii = atid - jj * LW;
        C.load5(ii - 1 - S_, jj - 1 - S_, pa, Ua0);
      }
      for (int idx = tid; idx < ne; idx += nthr) {
        // per item: the two face states, the four stage-1 flux pairs that
        // correct them (first transverse direction e1, second e2), the flux
        // slot and the boundary face it may belong to
        const T *sl, *sr, *a1p, *a1m, *a2p, *a2m, *b1p, *b1m, *b2p, *b2m;
        T* pf;
        T g1, g2;
        int d, fs, bface = -1, ba = 0, bb = 0;
        if (idx < nx) {
          // x face f of row j: R state of cell f-1 and L state of cell f
          int j = idx / (N + 1), f = idx - j * (N + 1), jj = j + 1;
          d = 0;
          g1 = h1;
          g2 = h2;
          sl = &R.XY(r, 0, 1, 0, jj, f);
          sr = &R.XY(r, 0, 0, 0, jj, f + 1);
          a1p = &F1.y(r, 0, jj, f);
          a1m = &F1.y(r, 0, jj - 1, f);
          a2p = &F1.z(r + 1, 0, jj, f);
          a2m = &F1.z(r, 0, jj, f);
          b1p = &F1.y(r, 0, jj, f + 1);
          b1m = &F1.y(r, 0, jj - 1, f + 1);
          b2p = &F1.z(r + 1, 0, jj, f + 1);
          b2m = &F1.z(r, 0, jj, f + 1);
          pf = &R.F2x(r, 0, j, f);
          fs = N * (N + 1);
          if (f == 0 || f == N) {
            bface = f == 0 ? 0 : 1;
            ba = r - rk * N;
            bb = j;
          }
        } else if (idx < 2 * nx) {
          // y face f of column i: R state of cell f-1 and L state of cell f
          int k = idx - nx;
          int f = k / N, i = k - f * N, ii = i + 1;
          d = 1;
          g1 = h0;
          g2 = h2;
          sl = &R.XY(r, 1, 1, 0, f, ii);
          sr = &R.XY(r, 1, 0, 0, f + 1, ii);
          a1p = &F1.x(r, 0, f, ii);
          a1m = &F1.x(r, 0, f, ii - 1);
          a2p = &F1.z(r + 1, 0, f, ii);
          a2m = &F1.z(r, 0, f, ii);
          b1p = &F1.x(r, 0, f + 1, ii);
          b1m = &F1.x(r, 0, f + 1, ii - 1);
          b2p = &F1.z(r + 1, 0, f + 1, ii);
          b2m = &F1.z(r, 0, f + 1, ii);
          pf = &R.F2y(r, 0, f, i);
          fs = (N + 1) * N;
          if (f == 0 || f == N) {
            bface = f == 0 ? 2 : 3;
            ba = r - rk * N;
            bb = i;
          }
        } else {
          // z face below plane r: R state of plane r-1 and L state of plane r
          int k = idx - 2 * nx;
          int j = k / N, i = k - j * N, jj = j + 1, ii = i + 1;
          d = 2;
          g1 = h0;
          g2 = h1;
          sl = &R.Zs(r - 1, 1, 0, jj, ii);
          sr = &R.Zs(r, 0, 0, jj, ii);
          a1p = &F1.x(r - 1, 0, jj, ii);
          a1m = &F1.x(r - 1, 0, jj, ii - 1);
          a2p = &F1.y(r - 1, 0, jj, ii);
          a2m = &F1.y(r - 1, 0, jj - 1, ii);
          b1p = &F1.x(r, 0, jj, ii);
          b1m = &F1.x(r, 0, jj, ii - 1);
          b2p = &F1.y(r, 0, jj, ii);
          b2m = &F1.y(r, 0, jj - 1, ii);
          pf = &R.F2z(r, 0, j, i);
          fs = N * N;
          if (r == rk * N) {
            bface = 4;  // -z face of group rk and +z face of group rk-1
            ba = j;
            bb = i;
          }
        }
        // variable strides of the stage-1 flux arrays used for e1 and e2
        const int s1 = d == 0 ? (N + 1) * L : L * (N + 1);
        const int s2 = d == 2 ? (N + 1) * L : LL;
        const LocalComps lc(d);
        const int gv[5] = {0, lc.c1, lc.c2, lc.c3, 4};  // global variable of each local slot
        T UL[5], UR[5], F[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int v = gv[k];
          UL[k] = correct(sl[v * LL], g1, a1p[v * s1], a1m[v * s1], g2, a2p[v * s2], a2m[v * s2]);
          UR[k] = correct(sr[v * LL], g1, b1p[v * s1], b1m[v * s1], g2, b2p[v * s2], b2m[v * s2]);
        }
        const unsigned s = riemann_local<T, MIXED, RS>(UL, UR, o, F);
        store_local(pf, fs, lc, F);
        mark_status<N>(sts, K, r, 0, d == 2 ? 1 : 0, s);
        if (bface >= 0) {
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            if (bface < 4) {
              C.store_flux(rk, bface, gv[k], ba, bb, F[k]);
            } else {
              if (rk < K) C.store_flux(rk, 4, gv[k], ba, bb, F[k]);
              if (rk > 0) C.store_flux(rk - 1, 5, gv[k], ba, bb, F[k]);
            }
          }
        }
      }
      for (int k = atid; atid >= 0 && k < na; k += naw) {
        int jj = k / LW, ii = k - jj * LW;
        T U[5], W[5];
        if (k == atid) {
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = Ua0[v];
        } else {
          C.load5(ii - 1 - S_, jj - 1 - S_, pa, U);
        }
        prim<T, MIXED>(U, W, o.gas);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wr(pa, v, jj, ii) = W[v];
      }
      if constexpr (ASYNC) {
        __pipeline_wait_prior(0);
        for (int k = tid - cw0; k >= 0 && k < na; k += nthr - cw0) {
          const int jj = k / LW, ii = k - jj * LW;
          T U[5], W[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) U[v] = Wr(pa, v, jj, ii);
          prim<T, MIXED>(U, W, o.gas);
#pragma unroll
          for (int v = 0; v < 5; ++v) Wr(pa, v, jj, ii) = W[v];
        }
      }
    }
    __syncthreads();
  }
}

template <class T, class S, bool MIXED, int RS, int REC, bool CH, int N, bool GCH>
__device__ void ctu_group(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, T* ring, int K, unsigned* sts) {
  if (o.limiter == LIM_MINMOD && o.theta == T(1))
    ctu_group_impl<T, S, MIXED, RS, REC, LIM_MINMOD1, CH, N>(C, o, ring, K, sts);
  else
    ctu_group_impl<T, S, MIXED, RS, REC, -1, CH, N>(C, o, ring, K, sts);
}

}  // namespace hyd
