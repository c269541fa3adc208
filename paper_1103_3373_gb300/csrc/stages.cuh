// Stages shared by the three plane-streaming group kernels (MHM, VL, CTU):
// ring-buffer addressing of the face states and final fluxes, the final
// Riemann solves of one plane with the group-boundary flux store (Sec. 2
// steps (2)/(3) and (5)), the conservative update of one plane (step (4)),
// and the load of one input plane.
//
// Ring planes are addressed by their z index p; a ring of depth R keeps
// planes p, p-1, ..., p-R+1.  Within a plane the layout is [var][row][col]
// so that consecutive threads touch consecutive words.
#pragma once
#include "group.cuh"

namespace hyd {

// Face states (conserved, after prediction / tracing / correction) and the
// final fluxes of one group.
//   XY: [dir x|y][side L|R][var][L][L], cells [-1,N]^2 of the plane
//   Z : [side][var][L][L]
//   F2x: [var][N rows][N+1 faces]   (face f between cells f-1 and f)
//   F2y: [var][N+1 faces][N cols]
//   F2z: [var][N][N], the faces below plane p
template <class T, int N, int DXY, int DZ> struct FaceRings {
  static constexpr int L = N + 2, LL = L * L;
  static constexpr int XYPL = 2 * 2 * 5 * LL;
  static constexpr int ZPL = 2 * 5 * LL;
  static constexpr int F2X = 5 * N * (N + 1);
  static constexpr int F2XYPL = 2 * F2X;
  static constexpr int F2ZPL = 5 * N * N;
  static constexpr int ELEMS = DXY * XYPL + DZ * ZPL + 2 * F2XYPL + 2 * F2ZPL;
  T* base;
  __device__ __forceinline__ T& XY(int p, int dir, int side, int v, int jj, int ii) const {
    return base[slot<DXY>(p) * XYPL + (((dir * 2 + side) * 5 + v) * L + jj) * L + ii];
  }
  __device__ __forceinline__ T& Zs(int p, int side, int v, int jj, int ii) const {
    return base[DXY * XYPL + slot<DZ>(p) * ZPL + ((side * 5 + v) * L + jj) * L + ii];
  }
  __device__ __forceinline__ T& F2x(int p, int v, int j, int f) const {
    return base[DXY * XYPL + DZ * ZPL + slot<2>(p) * F2XYPL + (v * N + j) * (N + 1) + f];
  }
  __device__ __forceinline__ T& F2y(int p, int v, int f, int i) const {
    return base[DXY * XYPL + DZ * ZPL + slot<2>(p) * F2XYPL + F2X + (v * (N + 1) + f) * N + i];
  }
  __device__ __forceinline__ T& F2z(int p, int v, int j, int i) const {
    return base[DXY * XYPL + DZ * ZPL + 2 * F2XYPL + slot<2>(p) * F2ZPL + (v * N + j) * N + i];
  }
};

// One final Riemann solve of chain plane p (0 <= p <= NP, NP = K N), item
// idx of 2 nx + N^2 (nx = N (N+1) if p < NP, else 0): the x faces, then the
// y faces of the interior cells of plane p, then the z faces between planes
// p-1 and p.  Fluxes on a group boundary are stored at once (step (5)); a z
// face between two groups of a chain is the +z face of the lower and the -z
// face of the upper one.
template <class T, class S, bool MIXED, int RS, int N, class FR, bool GCH>
__device__ __forceinline__ void flux2_item(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, const FR& R, int p, int K,
                                           unsigned* sts, int idx, int nx) {
  constexpr int LL = FR::LL;
  const int pk = p / N;  // chain group of plane p (K for the top face)
  const T *pl, *pr;
  T* pf;
  int d, fs, bface = -1, ba = 0, bb = 0;
  if (idx < nx) {
    int j = idx / (N + 1), f = idx - j * (N + 1);
    d = 0;
    pl = &R.XY(p, 0, 1, 0, j + 1, f);
    pr = &R.XY(p, 0, 0, 0, j + 1, f + 1);
    pf = &R.F2x(p, 0, j, f);
    fs = N * (N + 1);
    if (f == 0 || f == N) {
      bface = f == 0 ? 0 : 1;
      ba = p - pk * N;
      bb = j;
    }
  } else if (idx < 2 * nx) {
    int k = idx - nx;
    int f = k / N, i = k - f * N;
    d = 1;
    pl = &R.XY(p, 1, 1, 0, f, i + 1);
    pr = &R.XY(p, 1, 0, 0, f + 1, i + 1);
    pf = &R.F2y(p, 0, f, i);
    fs = (N + 1) * N;
    if (f == 0 || f == N) {
      bface = f == 0 ? 2 : 3;
      ba = p - pk * N;
      bb = i;
    }
  } else {
    int k = idx - 2 * nx;
    int j = k / N, i = k - j * N;
    d = 2;
    pl = &R.Zs(p - 1, 1, 0, j + 1, i + 1);
    pr = &R.Zs(p, 0, 0, j + 1, i + 1);
    pf = &R.F2z(p, 0, j, i);
    fs = N * N;
    if (p == pk * N) {
      bface = 4;
      ba = j;
      bb = i;
    }
  }
  const LocalComps lc(d);
  T UL[5], UR[5], F[5];
  load_local(pl, LL, lc, UL);
  load_local(pr, LL, lc, UR);
  const unsigned s = riemann_local<T, MIXED, RS>(UL, UR, o, F);
  store_local(pf, fs, lc, F);
  mark_status<N>(sts, K, p, 0, d == 2 ? 1 : 0, s);
  if (bface >= 0) {
    const int gv[5] = {0, lc.c1, lc.c2, lc.c3, 4};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      if (bface < 4) {
        C.store_flux(pk, bface, gv[k], ba, bb, F[k]);
      } else {
        if (pk < K) C.store_flux(pk, 4, gv[k], ba, bb, F[k]);
        if (pk > 0) C.store_flux(pk - 1, 5, gv[k], ba, bb, F[k]);
      }
    }
  }
}

// All final Riemann solves of chain plane p, over the CTA's threads.
template <class T, class S, bool MIXED, int RS, int N, class FR, bool GCH>
__device__ __forceinline__ void stage_flux2(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, const FR& R, int p, int K,
                                            unsigned* sts) {
  const int nx = (p < K * N) ? N * (N + 1) : 0;
  const int cnt = 2 * nx + N * N;
  for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) flux2_item<T, S, MIXED, RS, N>(C, o, R, p, K, sts, idx, nx);
}

// Conservative update of cell idx (of N^2) of chain plane p from the final
// fluxes (step (4)).
template <class T, class S, bool MIXED, int N, class FR, bool GCH>
__device__ __forceinline__ void update_item(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, const FR& R, int p, int K,
                                            unsigned* sts, int idx) {
  int j = idx / N, i = idx - j * N;
  T dF[3][5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dF[0][v] = R.F2x(p, v, j, i + 1) - R.F2x(p, v, j, i);
    dF[1][v] = R.F2y(p, v, j + 1, i) - R.F2y(p, v, j, i);
    dF[2][v] = R.F2z(p + 1, v, j, i) - R.F2z(p, v, j, i);
  }
  mark_status<N>(sts, K, p, 0, 0, update_cell<T, S, MIXED, N>(C, i, j, p, dF, o.gas));
}

// Conservative update of chain plane p, over the CTA's threads.
template <class T, class S, bool MIXED, int N, class FR, bool GCH>
__device__ __forceinline__ void stage_update(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, const FR& R, int p, int K,
                                             unsigned* sts, int t0 = 0) {
  // on the threads t0 .. blockDim.x-1
  const int step = (int)blockDim.x - t0;
  for (int idx = (int)threadIdx.x - t0; idx >= 0 && idx < N * N; idx += step)
    update_item<T, S, MIXED, N>(C, o, R, p, K, sts, idx);
}

// Ring of LW x LW input planes; the plane's lateral index ii maps to the
// interior coordinate ii - off.
template <class T, int LW, int R> struct PlaneRing {
  static constexpr int PL = 5 * LW * LW;
  static constexpr int ELEMS = R * PL;
  T* base;
  __device__ __forceinline__ T& operator()(int p, int v, int jj, int ii) const {
    return base[slot<R>(p) * PL + (v * LW + jj) * LW + ii];
  }
};

// Load plane p into a ring, as primitives (PRIM) or conserved variables.
template <bool PRIM, class T, class S, bool MIXED, int N, int LW, int R, bool GCH>
__device__ __forceinline__ void stage_load(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, int p, int off,
                                           const PlaneRing<T, LW, R>& ring) {
  for (int idx = threadIdx.x; idx < LW * LW; idx += blockDim.x) {
    int jj = idx / LW, ii = idx - jj * LW;
    T U[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) U[v] = C.load(v, ii - off, jj - off, p);
    if (PRIM) {
      T W[5];
      prim<T, MIXED>(U, W, o.gas);
#pragma unroll
      for (int v = 0; v < 5; ++v) ring(p, v, jj, ii) = W[v];
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) ring(p, v, jj, ii) = U[v];
    }
  }
}

// Face values of one cell along d from a primitive ring (Sec. 2 step (1)):
// w[] = the 2S+1 stencil values per variable, centre at index 2.
template <int REC, int LIM = -1, class T>
__device__ __forceinline__ void recon5(const T w[5][5], const Opts<T>& o, T WLf[5], T WRf[5], T dW[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    if (REC == PPM)
      ppm<LIM>(w[v][0], w[v][1], w[v][2], w[v][3], w[v][4], o.limiter, o.theta, WLf[v], WRf[v]);
    else
      plm<LIM>(w[v][1], w[v][2], w[v][3], o.limiter, o.theta, WLf[v], WRf[v], dW[v]);
  }
}

// Face values of one cell from a LOCAL-frame primitive stencil, in
// characteristic variables (Sec. 2: the reconstruction may act on primitive
// or characteristic variables): every stencil value is projected on the
// left eigenvectors at the cell centre, alpha_a(j) = l_a(W_0) . W_j, each
// alpha_a goes through the scalar PLM / PPM with the limiter, and the faces
// (and PLM slope) return as sum_a alpha_a r_a(W_0), waves added in the order
// 1..5 starting from zero.  Outputs in the local frame.
template <int REC, int LIM = -1, class T>
__device__ __forceinline__ void recon5c(const T w[5][5], const Opts<T>& o, T WLf[5], T WRf[5], T dW[5]) {
  constexpr int S_ = REC == PPM ? 2 : 1;
  T W0[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) W0[v] = w[v][2];
  Eig<T> e;
  eig(W0, o.gas, e);
  T al[5][5];
#pragma unroll
  for (int j = 2 - S_; j <= 2 + S_; ++j) {
    T X[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) X[v] = w[v][j];
#pragma unroll
    for (int a = 0; a < 5; ++a) al[a][j] = lproj(e, a, X);
  }
  T aL[5], aR[5], ad[5];
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    if (REC == PPM) {
      ppm<LIM>(al[a][0], al[a][1], al[a][2], al[a][3], al[a][4], o.limiter, o.theta, aL[a], aR[a]);
      ad[a] = T(0);
    } else {
      plm<LIM>(al[a][1], al[a][2], al[a][3], o.limiter, o.theta, aL[a], aR[a], ad[a]);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    WLf[v] = T(0);
    WRf[v] = T(0);
    dW[v] = T(0);
  }
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    radd(e, a, aL[a], WLf);
    radd(e, a, aR[a], WRf);
    radd(e, a, ad[a], dW);
  }
}

// Primitive or characteristic reconstruction of a local-frame stencil.
template <int REC, int LIM, bool CH, class T>
__device__ __forceinline__ void recon5_local(const T w[5][5], const Opts<T>& o, T WLf[5], T WRf[5], T dW[5]) {
  if constexpr (CH)
    recon5c<REC, LIM>(w, o, WLf, WRf, dW);
  else
    recon5<REC, LIM>(w, o, WLf, WRf, dW);
}

}  // namespace hyd
