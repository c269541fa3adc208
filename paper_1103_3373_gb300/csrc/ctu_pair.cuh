// FP32 CTU group update with two work items per thread (Sec. 2 steps
// (1)-(5); the same stages, rings and index ranges as ctu_group_impl in
// ctu.cuh, which the FP64, mixed and characteristic forms keep).
//
// Each barrier interval's items are taken in blocks of 64 per warp: lane t of
// the warp takes items 64 b + t and 64 b + 32 + t, so every shared-memory
// access of the warp touches 32 consecutive items, and the FP32 arithmetic
// of the two items runs packed (phys_pair.cuh).  The intervals are arranged
// so that every warp has about one block in each:
//   S1  trace plane q in x, y, z (3 (N+2)^2 items); conservative update of
//       plane q-3 (its global reads issued before the tracing);
//   S2  stage-1 Riemann problems of plane q (x / y faces) and of the z faces
//       below it;
//   S3  corrected stage-2 Riemann problems of plane q-1 and the z faces
//       below it (boundary fluxes stored at once); the next input plane is
//       loaded by threads 0 .. (N+2S+2)^2-1, its global reads issued first.
#pragma once
#include "ctu.cuh"
#include "phys_pair.cuh"

namespace hyd {

// Items 64 b + lane and 64 b + 32 + lane of a block; lane 1 duplicates lane 0
// past the end (its results are dropped).
struct PairIdx {
  int i0, i1;
  bool v1;
};
__device__ __forceinline__ PairIdx pair_idx(int b, int lane, int n) {
  PairIdx p;
  p.i0 = 64 * b + lane;
  p.i1 = p.i0 + 32;
  p.v1 = p.i1 < n;
  if (!p.v1) p.i1 = p.i0;
  return p;
}

// Stencil of one lane for the tracing of cell (jj, ii) of plane p along d,
// in the local frame of d: w[v][o + S], o = -S..S.  pb[o + S] = offset of
// ring plane p + o.
template <int S_, int LW>
__device__ __forceinline__ void pair_stencil(const float* ring, const int pb[2 * S_ + 1], int jj, int ii, int d,
                                             float w[5][2 * S_ + 1]) {
  constexpr int VS = LW * LW;
  const LocalComps lc(d);
  const int rc = (jj + S_) * LW + ii + S_;
  const int st = d == 0 ? 1 : LW;
#pragma unroll
  for (int o = -S_; o <= S_; ++o) {
    const int off = d == 2 ? pb[o + S_] + rc : pb[S_] + rc + o * st;
    const float* b = ring + off;
    w[0][o + S_] = b[0];
    w[1][o + S_] = b[lc.c1 * VS];
    w[2][o + S_] = b[lc.c2 * VS];
    w[3][o + S_] = b[lc.c3 * VS];
    w[4][o + S_] = b[4 * VS];
  }
}

template <int RS, int REC, int LIM, int N>
__device__ __forceinline__ void ctu_pair_impl(const GroupCtx<float, float, N>& C, const Opts<float>& o, float* ring,
                                              int K, unsigned* sts) {
  using T = float;
  constexpr int S_ = REC == PPM ? 2 : 1;
  using Lay = CtuLayout<N, S_>;
  constexpr int L = Lay::L, LL = Lay::LL, LW = Lay::LW;
  constexpr int RW = 2 * S_ + 1;  // W ring depth
  PlaneRing<T, LW, RW> Wr{ring};
  FaceRings<T, N, 2, 3> R{ring + Lay::OFF_FR};
  CtuF1<T, N, S_> F1{ring + Lay::OFF_F1XY};
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const T h0 = C.hdtdx[0], h1 = C.hdtdx[1], h2 = C.hdtdx[2];
  const int NP = K * N;

  for (int p = -1 - S_; p <= -1 + S_; ++p) stage_load<true, T, T, false, N, LW, RW>(C, o, p, 1 + S_, Wr);
  __syncthreads();

  const int T_ITERS = NP + 4;
  for (int t = 0; t < T_ITERS; ++t) {
    const int q = t - 1;  // plane traced and given stage-1 fluxes
    const int r = q - 1;  // plane given stage-2 fluxes
    const int u = q - 3;  // plane updated

    // ---- S1: trace plane q in the three directions; update plane u -------
    // the update's reads of U^n are issued first and consumed after the
    // tracing, so their latency hides behind it
    const int nf = (u >= 0 && u < NP) ? N * N : 0;
    T Un0[5];
    if (tid < nf) {
      const int j = tid / N, i = tid - j * N;
#pragma unroll
      for (int v = 0; v < 5; ++v) Un0[v] = C.load_raw(v, i, j, u);
    }
    if (q <= NP) {
      int pb[2 * S_ + 1];
#pragma unroll
      for (int k = 0; k < 2 * S_ + 1; ++k) pb[k] = slot<RW>(q - S_ + k) * PlaneRing<T, LW, RW>::PL;
      const int n = 3 * LL;
      for (int b = warp; 64 * b < n; b += nwarp) {
        const PairIdx P = pair_idx(b, lane, n);
        if (P.i0 >= n) continue;
        int dd[2], jq[2], iq[2];
        float w0[5][2 * S_ + 1], w1[5][2 * S_ + 1];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int k = l ? P.i1 : P.i0;
          const int d = k / LL;
          const int rem = k - d * LL;
          dd[l] = d;
          jq[l] = rem / L;
          iq[l] = rem - jq[l] * L;
        }
        pair_stencil<S_, LW>(ring, pb, jq[0], iq[0], dd[0], w0);
        pair_stencil<S_, LW>(ring, pb, jq[1], iq[1], dd[1], w1);
        V2 W0[5], Wl[5], Wr[5];
        const V2 dtdx = mk2(dd[0] == 0 ? C.dtdx[0] : (dd[0] == 1 ? C.dtdx[1] : C.dtdx[2]),
                            dd[1] == 0 ? C.dtdx[0] : (dd[1] == 1 ? C.dtdx[1] : C.dtdx[2]));
        if constexpr (REC == PPM) {
          V2 WLf[5], WRf[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            W0[v] = mk2(w0[v][2], w1[v][2]);
            pp::ppm<LIM>(mk2(w0[v][0], w1[v][0]), mk2(w0[v][1], w1[v][1]), W0[v], mk2(w0[v][3], w1[v][3]),
                         mk2(w0[v][4], w1[v][4]), o, WLf[v], WRf[v]);
          }
          pp::trace_ppm(W0, WLf, WRf, dtdx, o.gas, Wl, Wr);
        } else {
          V2 dW[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            W0[v] = mk2(w0[v][1], w1[v][1]);
            dW[v] = pp::slope<LIM>(o, W0[v] - mk2(w0[v][0], w1[v][0]), mk2(w0[v][2], w1[v][2]) - W0[v]);
          }
          pp::trace_plm(W0, dW, dtdx, o.gas, Wl, Wr);
        }
        V2 Ul[5], Ur[5];
        pp::cons(Wl, Ul, o.gas);
        pp::cons(Wr, Ur, o.gas);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          if (l == 1 && !P.v1) break;
          const int d = dd[l];
          const LocalComps lc(d);
          T* dl = d < 2 ? &R.XY(q, d, 0, 0, jq[l], iq[l]) : &R.Zs(q, 0, 0, jq[l], iq[l]);
          T* dr = d < 2 ? &R.XY(q, d, 1, 0, jq[l], iq[l]) : &R.Zs(q, 1, 0, jq[l], iq[l]);
          float a[5], c[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            a[v] = lane_of(Ul[v], l);
            c[v] = lane_of(Ur[v], l);
          }
          store_local(dl, LL, lc, a);
          store_local(dr, LL, lc, c);
        }
      }
    }
    for (int k = tid; k < nf; k += blockDim.x) {
      const int j = k / N, i = k - j * N;
      T Uc[5], dF[3][5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        Uc[v] = k == tid ? Un0[v] : C.load_raw(v, i, j, u);
        dF[0][v] = R.F2x(u, v, j, i + 1) - R.F2x(u, v, j, i);
        dF[1][v] = R.F2y(u, v, j + 1, i) - R.F2y(u, v, j, i);
        dF[2][v] = R.F2z(u + 1, v, j, i) - R.F2z(u, v, j, i);
      }
      mark_status<N>(sts, K, u, 0, 0, update_cell_from<T, T, false, N>(C, i, j, u, Uc, dF, o.gas));
    }
    __syncthreads();

    // ---- S2: stage-1 fluxes of plane q (x / y faces, z faces below it) ---
    {
      constexpr int NX = L * (N + 1);
      const int nz = q >= 0 ? LL : 0;
      const int cnt = q <= NP ? 2 * NX + nz : 0;
      const int nb1 = (cnt + 63) / 64;
      for (int b = warp; b < nb1; b += nwarp) {
        {
          const PairIdx P = pair_idx(b, lane, cnt);
          if (P.i0 >= cnt) continue;
          int pl[2], pr[2], pf[2], fs[2], dd[2];
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            const int idx = l ? P.i1 : P.i0;
            if (idx < NX) {
              int jj = idx / (N + 1), f = idx - jj * (N + 1);
              dd[l] = 0;
              pl[l] = &R.XY(q, 0, 1, 0, jj, f) - ring;
              pr[l] = &R.XY(q, 0, 0, 0, jj, f + 1) - ring;
              pf[l] = &F1.x(q, 0, jj, f) - ring;
              fs[l] = L * (N + 1);
            } else if (idx < 2 * NX) {
              int k = idx - NX;
              int f = k / L, ii = k - f * L;
              dd[l] = 1;
              pl[l] = &R.XY(q, 1, 1, 0, f, ii) - ring;
              pr[l] = &R.XY(q, 1, 0, 0, f + 1, ii) - ring;
              pf[l] = &F1.y(q, 0, f, ii) - ring;
              fs[l] = (N + 1) * L;
            } else {
              int k = idx - 2 * NX;
              int jj = k / L, ii = k - jj * L;
              dd[l] = 2;
              pl[l] = &R.Zs(q - 1, 1, 0, jj, ii) - ring;
              pr[l] = &R.Zs(q, 0, 0, jj, ii) - ring;
              pf[l] = &F1.z(q, 0, jj, ii) - ring;
              fs[l] = LL;
            }
          }
          V2 UL[5], UR[5], F[5];
          {
            const LocalComps c0(dd[0]), c1(dd[1]);
            float a0[5], a1[5], b0[5], b1[5];
            load_local(ring + pl[0], LL, c0, a0);
            load_local(ring + pl[1], LL, c1, a1);
            load_local(ring + pr[0], LL, c0, b0);
            load_local(ring + pr[1], LL, c1, b1);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              UL[v] = mk2(a0[v], a1[v]);
              UR[v] = mk2(b0[v], b1[v]);
            }
          }
          unsigned s[2];
          pp::riemann<RS>(UL, UR, o, F, s);
#pragma unroll
          for (int l = 0; l < 2; ++l) {
            if (l == 1 && !P.v1) break;
            const LocalComps lc(dd[l]);
            float f[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) f[v] = lane_of(F[v], l);
            store_local(ring + pf[l], fs[l], lc, f);
            mark_status<N>(sts, K, q, dd[l] == 2 ? 0 : -1, 1, s[l]);
          }
        }
      }
    }
    __syncthreads();

    // ---- S3: corrected stage-2 fluxes of plane r; next input plane --------
    {
      const int nx = (r >= 0 && r < NP) ? N * (N + 1) : 0;
      const int nz = (r >= 0 && r <= NP) ? N * N : 0;
      const int rk = r >= 0 ? r / N : 0;
      const int ne = 2 * nx + nz;
      const int pa = q + 1 + S_;
      const int na = (pa <= NP + S_) ? LW * LW : 0;
      T Ua[5];
      const bool do_load = tid < na;
      if (do_load) {
        const int jj = tid / LW, ii = tid - jj * LW;
        C.load5(ii - 1 - S_, jj - 1 - S_, pa, Ua);
      }
      for (int b = warp; 64 * b < ne; b += nwarp) {
        const PairIdx P = pair_idx(b, lane, ne);
        if (P.i0 >= ne) continue;
        V2 UL[5], UR[5];
        int dd[2], pf[2], fs[2], bface[2], ba[2], bb[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          const int idx = l ? P.i1 : P.i0;
          // the two face states, the stage-1 flux pairs of the two
          // transverse directions that correct them, the flux slot
          int sl, sr, a1p, a1m, a2p, a2m, b1p, b1m, b2p, b2m, d, s1, s2;
          T g1, g2;
          bface[l] = -1;
          ba[l] = bb[l] = 0;
          if (idx < nx) {
            int j = idx / (N + 1), f = idx - j * (N + 1), jj = j + 1;
            d = 0;
            g1 = h1;
            g2 = h2;
            sl = &R.XY(r, 0, 1, 0, jj, f) - ring;
            sr = &R.XY(r, 0, 0, 0, jj, f + 1) - ring;
            a1p = &F1.y(r, 0, jj, f) - ring;
            a1m = &F1.y(r, 0, jj - 1, f) - ring;
            a2p = &F1.z(r + 1, 0, jj, f) - ring;
            a2m = &F1.z(r, 0, jj, f) - ring;
            b1p = a1p + 1;
            b1m = a1m + 1;
            b2p = a2p + 1;
            b2m = a2m + 1;
            pf[l] = &R.F2x(r, 0, j, f) - ring;
            fs[l] = N * (N + 1);
            if (f == 0 || f == N) {
              bface[l] = f == 0 ? 0 : 1;
              ba[l] = r - rk * N;
              bb[l] = j;
            }
          } else if (idx < 2 * nx) {
            int k = idx - nx;
            int f = k / N, i = k - f * N, ii = i + 1;
            d = 1;
            g1 = h0;
            g2 = h2;
            sl = &R.XY(r, 1, 1, 0, f, ii) - ring;
            sr = &R.XY(r, 1, 0, 0, f + 1, ii) - ring;
            a1p = &F1.x(r, 0, f, ii) - ring;
            a1m = &F1.x(r, 0, f, ii - 1) - ring;
            a2p = &F1.z(r + 1, 0, f, ii) - ring;
            a2m = &F1.z(r, 0, f, ii) - ring;
            b1p = a1p + (N + 1);
            b1m = a1m + (N + 1);
            b2p = a2p + L;
            b2m = a2m + L;
            pf[l] = &R.F2y(r, 0, f, i) - ring;
            fs[l] = (N + 1) * N;
            if (f == 0 || f == N) {
              bface[l] = f == 0 ? 2 : 3;
              ba[l] = r - rk * N;
              bb[l] = i;
            }
          } else {
            int k = idx - 2 * nx;
            int j = k / N, i = k - j * N, jj = j + 1, ii = i + 1;
            d = 2;
            g1 = h0;
            g2 = h1;
            sl = &R.Zs(r - 1, 1, 0, jj, ii) - ring;
            sr = &R.Zs(r, 0, 0, jj, ii) - ring;
            a1p = &F1.x(r - 1, 0, jj, ii) - ring;
            a1m = &F1.x(r - 1, 0, jj, ii - 1) - ring;
            a2p = &F1.y(r - 1, 0, jj, ii) - ring;
            a2m = &F1.y(r - 1, 0, jj - 1, ii) - ring;
            b1p = &F1.x(r, 0, jj, ii) - ring;
            b1m = &F1.x(r, 0, jj, ii - 1) - ring;
            b2p = &F1.y(r, 0, jj, ii) - ring;
            b2m = &F1.y(r, 0, jj - 1, ii) - ring;
            pf[l] = &R.F2z(r, 0, j, i) - ring;
            fs[l] = N * N;
            if (r == rk * N) {
              bface[l] = 4;
              ba[l] = j;
              bb[l] = i;
            }
          }
          dd[l] = d;
          s1 = d == 0 ? (N + 1) * L : L * (N + 1);
          s2 = d == 2 ? (N + 1) * L : LL;
          const LocalComps lc(d);
          const int gv[5] = {0, lc.c1, lc.c2, lc.c3, 4};
          // step (3): u = (u - g1 (G1+ - G1-)) - g2 (G2+ - G2-)
#pragma unroll
          for (int k = 0; k < 5; ++k) {
            const int v = gv[k];
            const T* q0 = ring;
            const T ul = correct(q0[sl + v * LL], g1, q0[a1p + v * s1], q0[a1m + v * s1], g2, q0[a2p + v * s2],
                                 q0[a2m + v * s2]);
            const T ur = correct(q0[sr + v * LL], g1, q0[b1p + v * s1], q0[b1m + v * s1], g2, q0[b2p + v * s2],
                                 q0[b2m + v * s2]);
            UL[k] = l ? mk2(UL[k].v.x, ul) : mk2(ul, ul);
            UR[k] = l ? mk2(UR[k].v.x, ur) : mk2(ur, ur);
          }
        }
        V2 F[5];
        unsigned s[2];
        pp::riemann<RS>(UL, UR, o, F, s);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          if (l == 1 && !P.v1) break;
          const LocalComps lc(dd[l]);
          const int gv[5] = {0, lc.c1, lc.c2, lc.c3, 4};
          float f[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) f[v] = lane_of(F[v], l);
          store_local(ring + pf[l], fs[l], lc, f);
          mark_status<N>(sts, K, r, 0, dd[l] == 2 ? 1 : 0, s[l]);
          if (bface[l] >= 0) {
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              if (bface[l] < 4) {
                C.store_flux(rk, bface[l], gv[k], ba[l], bb[l], f[k]);
              } else {
                if (rk < K) C.store_flux(rk, 4, gv[k], ba[l], bb[l], f[k]);
                if (rk > 0) C.store_flux(rk - 1, 5, gv[k], ba[l], bb[l], f[k]);
              }
            }
          }
        }
      }
      if (do_load) {
        const int jj = tid / LW, ii = tid - jj * LW;
        T W[5];
        prim<T, false>(Ua, W, o.gas);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wr(pa, v, jj, ii) = W[v];
      }
      // planes wider than one pass of the CTA's threads
      for (int k = tid + blockDim.x; k < na; k += blockDim.x) {
        const int jj = k / LW, ii = k - jj * LW;
        T U[5], W[5];
        C.load5(ii - 1 - S_, jj - 1 - S_, pa, U);
        prim<T, false>(U, W, o.gas);
#pragma unroll
        for (int v = 0; v < 5; ++v) Wr(pa, v, jj, ii) = W[v];
      }
    }
    __syncthreads();
  }
}

template <int RS, int REC, int N>
__device__ void ctu_pair_group(const GroupCtx<float, float, N>& C, const Opts<float>& o, float* ring, int K,
                               unsigned* sts) {
  if (o.limiter == LIM_MINMOD && o.theta == 1.0f)
    ctu_pair_impl<RS, REC, LIM_MINMOD1, N>(C, o, ring, K, sts);
  else
    ctu_pair_impl<RS, REC, -1, N>(C, o, ring, K, sts);
}

}  // namespace hyd
