// The directionally split schemes measured beside the unsplit ones in
// Sec. 3.2 (RTVD and WAF) for one patch group: three 1D sweeps per step,
// x, y, z (split_order 0) or z, y, x (1), each with the full dt.
//
// The whole padded group (M = N + 2G cells per edge, G the schemes' stencil)
// is held as conserved variables in the CTA's ring (shared memory for FP32,
// a slice of the workspace for FP64).  Sec. 3.1 notes that the split schemes
// need 1D stencils only; here each thread owns one row of a sweep and walks
// along it, keeping a few cells of state in registers and writing each cell
// back in place once no later stencil of its row reads it.  The first sweep
// updates every row whose transverse coordinates lie in [-G, N+G), the second
// [0, N) along the first sweep's axis, the last [0, N)^2; the fluxes through
// the group faces of each sweep's update are the boundary fluxes (step (5)).
#pragma once
#include <cuda_pipeline.h>

#include "stages.cuh"

namespace hyd {

enum { SCH_RTVD = 3, SCH_WAF = 4 };

template <int SCH> struct SplitGhost {
  static constexpr int value = SCH == SCH_RTVD ? 3 : 2;
};

// RTVD (relaxing TVD in the flux-split form of Trac & Pen 2003): freezing
// speed c = |u_n| + c_s, FR = (c U + F)/2, FL = (c U - F)/2.
template <class T, bool MIXED>
__device__ __forceinline__ void rtvd_split(const T U[5], const Gas<T>& g, T FR[5], T FL[5]) {
  T W[5], F[5];
  prim<T, MIXED>(U, W, g);
  const T c = absv(W[1]) + csound(W[0], W[4], g);
  pflux(W, U[4], F);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    FR[v] = T(0.5) * (c * U[v] + F[v]);
    FL[v] = T(0.5) * (c * U[v] - F[v]);
  }
}

// One RTVD row of M cells (local frame; var stride VS, cell stride sd),
// updated in place on [G, M-G):
//   half step  F1_{j+1/2} = FR_j - FL_{j+1},  Uh_j = U_j - (dt/2dx)(F1_{j+1/2} - F1_{j-1/2});
//   full step  FR_{i+1/2} = FRh_i + psi(FRh_i - FRh_{i-1}, FRh_{i+1} - FRh_i)/2,
//              FL_{i+1/2} = FLh_{i+1} - psi(FLh_{i+1} - FLh_i, FLh_{i+2} - FLh_{i+1})/2,
//              U_i <- U_i - (dt/dx)(F_{i+1/2} - F_{i-1/2}),  F = FR - FL.
// Walking j = 0..M-1: cell j's split fluxes, the first-order flux at
// j - 1/2, the half step of cell m = j-1, the limited flux at i + 1/2 with
// i = m-2 and the update of cell i.  Returns the fluxes through G - 1/2 and
// M-G - 1/2.
template <class T, bool MIXED, int LIM, int M, int VS>
__device__ __forceinline__ void rtvd_row(T* p, int sd, const LocalComps& lc, const Opts<T>& o, T dtdx, T hdtdx,
                                         T Flo[5], T Fhi[5]) {
  constexpr int G = 3, LO = G, HI = M - G;
  // every carried value starts defined (read before written only by the
  // window shifts of the first iterations, whose results are never used)
  T uprev[5], FRp[5], F1p[5], FTp[5];
  T FRw[3][5];  // right-moving split fluxes of the half-step cells m-3, m-2, m-1
  T FLw[3][5];  // left-moving ones of m-2, m-1, m
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    uprev[v] = FRp[v] = F1p[v] = FTp[v] = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) FRw[k][v] = FLw[k][v] = T(0);
  }
  for (int j = 0; j < M; ++j) {
    T u[5], FR[5], FL[5];
    load_local(p + j * sd, VS, lc, u);
    rtvd_split<T, MIXED>(u, o.gas, FR, FL);
    if (j >= 1) {
      T F1[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) F1[v] = FRp[v] - FL[v];  // face (j-1) + 1/2
      if (j >= 2) {
        const int m = j - 1;
        T uh[5], FRm[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) uh[v] = uprev[v] - hdtdx * (F1[v] - F1p[v]);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          FLw[0][v] = FLw[1][v];
          FLw[1][v] = FLw[2][v];
        }
        rtvd_split<T, MIXED>(uh, o.gas, FRm, FLw[2]);
        const int i = m - 2;
        if (i >= LO - 1 && i <= HI - 1 && m >= 4) {
          T FT[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            // FRw: cells i-1, i, i+1; FLw: cells i, i+1, i+2
            T fr = FRw[1][v] + T(0.5) * slope<LIM>(o.limiter, o.theta, FRw[1][v] - FRw[0][v],
                                                     FRw[2][v] - FRw[1][v]);
            T fl = FLw[1][v] - T(0.5) * slope<LIM>(o.limiter, o.theta, FLw[1][v] - FLw[0][v],
                                                     FLw[2][v] - FLw[1][v]);
            FT[v] = fr - fl;
          }
          if (i == LO - 1) {
#pragma unroll
            for (int v = 0; v < 5; ++v) Flo[v] = FT[v];
          }
          if (i == HI - 1) {
#pragma unroll
            for (int v = 0; v < 5; ++v) Fhi[v] = FT[v];
          }
          if (i >= LO) {
            T ui[5];
            load_local(p + i * sd, VS, lc, ui);
#pragma unroll
            for (int v = 0; v < 5; ++v) ui[v] = ui[v] - dtdx * (FT[v] - FTp[v]);
            store_local(p + i * sd, VS, lc, ui);
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) FTp[v] = FT[v];
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          FRw[0][v] = FRw[1][v];
          FRw[1][v] = FRw[2][v];
          FRw[2][v] = FRm[v];
        }
      }
#pragma unroll
      for (int v = 0; v < 5; ++v) F1p[v] = F1[v];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      uprev[v] = u[v];
      FRp[v] = FR[v];
    }
  }
}

// The HLLC fan of a face (the Einfeldt speeds and star states of hllc()):
// speeds (SL, S*, SR), the fluxes of the star states U*L, U*R (the outer
// two are the sides' own fluxes) and the density jumps across the waves.
template <class T> struct Fan {
  T S[3];
  T Fs[2][5];
  T drho[3];
};

template <class T> __device__ __forceinline__ void hllc_fan(const Side<T>& L, const Side<T>& R, const Gas<T>& g, Fan<T>& f) {
  T SL, SR;
  einfeldt(L, R, g, SL, SR);
  T mL = L.W[0] * (SL - L.W[1]);
  T mR = R.W[0] * (SR - R.W[1]);
  T Ss = (R.W[4] - L.W[4] + mL * L.W[1] - mR * R.W[1]) / (mL - mR);
  T fL = mL / (SL - Ss), fR = mR / (SR - Ss);
  T UsL[5] = {fL, fL * Ss, fL * L.W[2], fL * L.W[3], fL * (L.U[4] / L.W[0] + (Ss - L.W[1]) * (Ss + L.W[4] / mL))};
  T UsR[5] = {fR, fR * Ss, fR * R.W[2], fR * R.W[3], fR * (R.U[4] / R.W[0] + (Ss - R.W[1]) * (Ss + R.W[4] / mR))};
  f.S[0] = SL;
  f.S[1] = Ss;
  f.S[2] = SR;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    f.Fs[0][v] = L.F[v] + SL * (UsL[v] - L.U[v]);
    f.Fs[1][v] = R.F[v] + SR * (UsR[v] - R.U[v]);
  }
  f.drho[0] = UsL[0] - L.W[0];
  f.drho[1] = UsR[0] - UsL[0];
  f.drho[2] = R.W[0] - UsR[0];
}

// WAF flux of the face with fan f between sides of fluxes FL, FR, its
// upwind neighbours' density jumps dm (face - 1) and dp (face + 1):
//   F = (F1 + F4)/2 - sum_k (0.5 sign(c_k) A_k) (F_{k+1} - F_k),
//   (F1, F2, F3, F4) = (FL, F*L, F*R, FR),
//   A_k = 1 - (1 - |c_k|) psi(r_k),  c_k = (dt/dx) S_k,
//   r_k = drho_k(upwind face) / drho_k(this face), psi(r) = the limiter's
//   slope(r, 1); psi = 0 where this face's jump is 0.
template <class T, int LIM>
__device__ __forceinline__ void waf_flux(const Fan<T>& f, const T FL[5], const T FR[5], const T dm[3],
                                         const T dp[3], const Opts<T>& o, T dtdx, T F[5]) {
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = T(0.5) * (FL[v] + FR[v]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T c = dtdx * f.S[k];
    const T s = c > T(0) ? T(1) : (c < T(0) ? T(-1) : T(0));
    const T up = c > T(0) ? dm[k] : dp[k];
    const T r = up / f.drho[k];
    const T psi = f.drho[k] != T(0) ? slope<LIM>(o.limiter, o.theta, r, T(1)) : T(0);
    const T A = T(1) - (T(1) - absv(c)) * psi;
    const T w = T(0.5) * s * A;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const T hi = k == 0 ? f.Fs[0][v] : (k == 1 ? f.Fs[1][v] : FR[v]);
      const T lo = k == 0 ? FL[v] : (k == 1 ? f.Fs[0][v] : f.Fs[1][v]);
      F[v] = F[v] - w * (hi - lo);
    }
  }
}

// One WAF row of M cells updated in place on [G, M-G) (G = 2).  Walking
// j = 0..M-1: cell j's side, the fan of face (j-1) + 1/2, the WAF flux of
// face i + 1/2 with i = j-2 (its upwind neighbours are the faces on either
// side) and the update of cell i.
template <class T, bool MIXED, int LIM, int M, int VS>
__device__ __forceinline__ void waf_row(T* p, int sd, const LocalComps& lc, const Opts<T>& o, T dtdx, T Flo[5],
                                        T Fhi[5]) {
  constexpr int G = 2, LO = G, HI = M - G;
  Side<T> sp;        // cell j-1
  T Fpp[5];          // flux of cell j-2
  Fan<T> fmid;       // face (j-2) + 1/2
  T dprev[3], FWp[5];
  // every carried value starts defined (the first iterations copy some of
  // them before they are written; those copies are never used)
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    sp.U[v] = sp.W[v] = sp.F[v] = Fpp[v] = FWp[v] = fmid.Fs[0][v] = fmid.Fs[1][v] = T(0);
  }
  sp.c = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) dprev[k] = fmid.S[k] = fmid.drho[k] = T(0);
  for (int j = 0; j < M; ++j) {
    T u[5];
    load_local(p + j * sd, VS, lc, u);
    Side<T> sj;
    mkside<T, MIXED>(u, o.gas, sj);
    if (j >= 1) {
      Fan<T> fnew;
      hllc_fan(sp, sj, o.gas, fnew);  // face (j-1) + 1/2
      if (j >= 3) {
        const int i = j - 2;  // fmid is face i + 1/2 (cells i, i+1), dprev face i - 1/2, fnew face i + 3/2
        if (i >= LO - 1 && i <= HI - 1) {
          T FW[5];
          waf_flux<T, LIM>(fmid, Fpp, sp.F, dprev, fnew.drho, o, dtdx, FW);
          if (i == LO - 1) {
#pragma unroll
            for (int v = 0; v < 5; ++v) Flo[v] = FW[v];
          }
          if (i == HI - 1) {
#pragma unroll
            for (int v = 0; v < 5; ++v) Fhi[v] = FW[v];
          }
          if (i >= LO) {
            T ui[5];
            load_local(p + i * sd, VS, lc, ui);
#pragma unroll
            for (int v = 0; v < 5; ++v) ui[v] = ui[v] - dtdx * (FW[v] - FWp[v]);
            store_local(p + i * sd, VS, lc, ui);
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) FWp[v] = FW[v];
        }
      }
      if (j >= 2) {
#pragma unroll
        for (int k = 0; k < 3; ++k) dprev[k] = fmid.drho[k];
      }
      fmid = fnew;
#pragma unroll
      for (int v = 0; v < 5; ++v) Fpp[v] = sp.F[v];
    }
    sp = sj;
  }
}

// The padded group into a global-memory ring (FP64 forms): UB cells per
// thread are loaded before any of them is stored, so their global reads are
// in flight together.
template <class T, class S, bool MIXED, int G, int M, int N, bool GCH>
__device__ __forceinline__ void split_load_group(const GroupCtx<T, S, N, GCH>& C, T* ring) {
  constexpr int M2 = M * M, M3 = M * M * M;
  constexpr int UB = (sizeof(T) == 4 && !MIXED) ? 2 : 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int base = tid; base < M3; base += UB * nthr) {
    T U[UB][5];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = base + u * nthr;
      if (idx < M3) {
        const int z = idx / M2, r = idx - z * M2, y = r / M, x = r - y * M;
        C.load5(x - G, y - G, z - G, U[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      const int idx = base + u * nthr;
      if (idx < M3) {
#pragma unroll
        for (int v = 0; v < 5; ++v) ring[v * M3 + idx] = U[u][v];
      }
    }
  }
}

template <class T, class S, bool MIXED, int SCH, int LIM, int N, bool GCH>
__device__ __forceinline__ void split_group_impl(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, T* ring,
                                                 unsigned* sts) {
  constexpr int G = SplitGhost<SCH>::value;
  constexpr int M = N + 2 * G;
  constexpr int M2 = M * M, M3 = M * M * M;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if constexpr (sizeof(T) == 4 && sizeof(S) == 4) {
    // the padded group into the shared-memory ring with asynchronous
    // global-to-shared copies: every copy of the thread is in flight at
    // once, nothing is staged in registers
    for (int idx = tid; idx < M3; idx += nthr) {
      const int z = idx / M2, r = idx - z * M2, y = r / M, x = r - y * M;
      long long vs;
      const S* src = C.src5(x - G, y - G, z - G, vs);
#pragma unroll
      for (int v = 0; v < 5; ++v) __pipeline_memcpy_async(&ring[v * M3 + idx], src + v * vs, sizeof(T));
    }
    __pipeline_commit();
    __pipeline_wait_prior(0);
  } else {
    split_load_group<T, S, MIXED, G, M, N>(C, ring);
  }
  __syncthreads();
  const int first = o.split_order ? 2 : 0, last = o.split_order ? 0 : 2;
  for (int k = 0; k < 3; ++k) {
    const int d = k == 0 ? first : (k == 1 ? 1 : last);
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;  // transverse axes, e1 < e2
    // an axis swept later still needs its ghost rows updated
    const bool l1 = (k == 0) || (k == 1 && e1 == last);
    const bool l2 = (k == 0) || (k == 1 && e2 == last);
    const int n1 = l1 ? M : N, o1 = l1 ? 0 : G;
    const int n2 = l2 ? M : N, o2 = l2 ? 0 : G;
    const int sd = d == 0 ? 1 : (d == 1 ? M : M2);
    const int s1 = e1 == 0 ? 1 : M;
    const int s2 = e2 == 1 ? M : M2;
    const LocalComps lc(d);
    // selects, not an index: a run-time index would put the context in local memory
    const T dtdx = d == 0 ? C.dtdx[0] : (d == 1 ? C.dtdx[1] : C.dtdx[2]);
    const T hdtdx = d == 0 ? C.hdtdx[0] : (d == 1 ? C.hdtdx[1] : C.hdtdx[2]);
    for (int r = tid; r < n1 * n2; r += nthr) {
      const int q2 = r / n1, q1 = r - q2 * n1;
      const int c1 = q1 + o1, c2 = q2 + o2;  // padded coordinates
      T* p = ring + c1 * s1 + c2 * s2;
      T Flo[5], Fhi[5];
      if (SCH == SCH_RTVD)
        rtvd_row<T, MIXED, LIM, M, M3>(p, sd, lc, o, dtdx, hdtdx, Flo, Fhi);
      else
        waf_row<T, MIXED, LIM, M, M3>(p, sd, lc, o, dtdx, Flo, Fhi);
      const int a = c2 - G, b = c1 - G;  // [a][b]: larger transverse axis first
      if (a >= 0 && a < N && b >= 0 && b < N) {
        const int gv[5] = {0, lc.c1, lc.c2, lc.c3, 4};
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          C.store_flux(0, 2 * d, gv[v], a, b, Flo[v]);
          C.store_flux(0, 2 * d + 1, gv[v], a, b, Fhi[v]);
        }
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < N * N * N; idx += nthr) {
    const int z = idx / (N * N), r = idx - z * N * N, y = r / N, x = r - y * N;
    const int pi = ((z + G) * M + (y + G)) * M + (x + G);
    T Un[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      Un[v] = ring[v * M3 + pi];
      C.store(v, x, y, z, (S)Un[v]);
    }
    mark_status<N>(sts, 1, z, 0, 0, state_status(Un, o.gas));
  }
}

template <class T, class S, bool MIXED, int SCH, int N, bool GCH>
__device__ void split_group(const GroupCtx<T, S, N, GCH>& C, const Opts<T>& o, T* ring, unsigned* sts) {
  if (o.limiter == LIM_MINMOD && o.theta == T(1))
    split_group_impl<T, S, MIXED, SCH, LIM_MINMOD1, N>(C, o, ring, sts);
  else
    split_group_impl<T, S, MIXED, SCH, -1, N>(C, o, ring, sts);
}

}  // namespace hyd
