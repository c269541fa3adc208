// Device-side numerics of the unsplit schemes (Sec. 2 of Schive, Zhang &
// Chiueh 2011): equation of state, limiters, PLM/PPM, CTU characteristic
// tracing, and the exact / HLLE / HLLC / Roe Riemann solvers with the Roe
// failure fallback.
//
// Every formula is evaluated in a fixed operation order (stated next to it)
// so that the FP64 build, compiled without FMA contraction, rounds exactly
// like a plain sequential evaluation of the same formula.  The FP32 builds
// use the same code with fast division / square root.
//
// Frames: "global" 5-vectors are (rho, m_x, m_y, m_z, E) or (rho, u, v, w, p);
// "local" ones for a sweep along d put the normal component first,
// (n, t1, t2) = (x, y, z), (y, z, x), (z, x, y) for d = 0, 1, 2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hyd {

// ---------------------------------------------------------------- options
enum { MHM = 0, VL = 1, CTU = 2 };
enum { PLM = 0, PPM = 1 };
enum { LIM_MINMOD = 0, LIM_VANLEER = 1, LIM_VANALBADA = 2, LIM_HYBRID = 3 };
// Internal: generalized minmod with theta = 1, i.e. sign(dL) min(|dL|, |dR|)
// (equal, value for value, to the three-term form: |dC| >= min(|dL|, |dR|)
// when dL dR > 0, also after rounding).
constexpr int LIM_MINMOD1 = 4;
enum { RS_EXACT = 0, RS_HLLE = 1, RS_HLLC = 2, RS_ROE = 3 };
enum { P_FP64 = 0, P_FP32 = 1, P_MIXED = 2 };

enum : unsigned { ST_ROE_FALLBACK = 1u, ST_NEG_DENS = 2u, ST_NEG_PRES = 4u, ST_NAN = 8u, ST_EXACT_FAIL = 16u };

// Precision forms: T = arithmetic type, S = storage type, MIXED = FP64
// internal-energy recovery where E - |m|^2/2rho cancels (the FP64 totals and
// the FP64 dt reduction are separate kernels).
template <int P> struct Prec;
template <> struct Prec<P_FP64> { using T = double; using S = double; static constexpr bool MIXED = false; };
template <> struct Prec<P_FP32> { using T = float; using S = float; static constexpr bool MIXED = false; };
template <> struct Prec<P_MIXED> { using T = float; using S = float; static constexpr bool MIXED = true; };

template <class T> struct Gas {
  T gamma;       // ratio of specific heats
  T gm1;         // gamma - 1
  T dens_floor;  // floors, applied as max(q, floor)
  T pres_floor;
  T igm1;        // 1 / (gamma - 1)
};

// FP32 forms: a denominator used more than once (rho, c^2, gamma - 1) is
// inverted once and multiplied by; the FP64 form divides at every use, in the
// operation order its bit-for-bit parity with the FP64 oracle rests on.
template <class T> struct FastRcp {
  static constexpr bool on = false;
};
template <> struct FastRcp<float> {
  static constexpr bool on = true;
};

// Options a kernel reads at run time (uniform over the launch).
template <class T> struct Opts {
  Gas<T> gas;
  T theta;
  int limiter;
  int fallback;
  int split_order;  // split schemes: sweeps x, y, z (0) or z, y, x (1)
};

template <class T> __device__ __forceinline__ T absv(T a) { return a < T(0) ? -a : a; }
__device__ __forceinline__ double sqrtv(double a) { return sqrt(a); }
__device__ __forceinline__ float sqrtv(float a) { return sqrtf(a); }
__device__ __forceinline__ double powv(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float powv(float a, float b) { return powf(a, b); }
__device__ __forceinline__ bool isnanv(double a) { return isnan(a); }
// a / b.  FP64 divides (IEEE).  The FP32 forms use the fast division
// intrinsic (2 ulp for 2^-126 <= |b| <= 2^126), which covers every
// denominator it is used on: densities, sound speeds, Roe-averaged c^2,
// wave-speed differences, limiter sums and constants.  It is not used in
// the exact solver's Newton iteration.
__device__ __forceinline__ double divv(double a, double b) { return a / b; }
__device__ __forceinline__ float divv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ bool isnanv(float a) { return isnan(a); }

// Directions are compile-time constants everywhere so that the 5-vectors stay
// in registers.
template <int D> struct Dir {
  static constexpr int n = 1 + D;
  static constexpr int t1 = 1 + (D == 2 ? 0 : D + 1);
  static constexpr int t2 = 1 + (D == 0 ? 2 : D - 1);
};

template <int D, class T> __device__ __forceinline__ void rot_in(const T a[5], T b[5]) {
  b[0] = a[0];
  b[1] = a[Dir<D>::n];
  b[2] = a[Dir<D>::t1];
  b[3] = a[Dir<D>::t2];
  b[4] = a[4];
}
template <int D, class T> __device__ __forceinline__ void rot_out(const T b[5], T a[5]) {
  a[0] = b[0];
  a[Dir<D>::n] = b[1];
  a[Dir<D>::t1] = b[2];
  a[Dir<D>::t2] = b[3];
  a[4] = b[4];
}

// ------------------------------------------------------------- EOS
// U -> W in the frame U is given in:
//   rho = max(U0, floor); kin = (0.5 * ((U1*U1 + U2*U2) + U3*U3)) / rho;
//   p = max((gamma-1) * (U4 - kin), floor); velocities U_k / rho.
// MIXED: when U4 - kin has lost more than 10 bits to cancellation, the
// internal energy is recomputed in FP64.
template <class T, bool MIXED>
__device__ __forceinline__ void prim(const T U[5], T W[5], const Gas<T>& g, T* irho = nullptr) {
  T rho = U[0];
  if (rho < g.dens_floor) rho = g.dens_floor;
  T ir = T(0);
  T kin;
  if constexpr (FastRcp<T>::on) {
    ir = divv(T(1), rho);
    kin = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ir;
  } else {
    kin = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;
  }
  T eint = U[4] - kin;
  if (MIXED) {
    if (eint < T(1.0 / 1024.0) * U[4]) {
      double r = (double)rho;
      double k = 0.5 * ((double)U[1] * (double)U[1] + (double)U[2] * (double)U[2] + (double)U[3] * (double)U[3]) / r;
      eint = (T)((double)U[4] - k);
    }
  }
  T p = g.gm1 * eint;
  if (p < g.pres_floor) p = g.pres_floor;
  W[0] = rho;
  if constexpr (FastRcp<T>::on) {
    W[1] = U[1] * ir;
    W[2] = U[2] * ir;
    W[3] = U[3] * ir;
    if (irho) *irho = ir;
  } else {
    W[1] = U[1] / rho;
    W[2] = U[2] / rho;
    W[3] = U[3] / rho;
  }
  W[4] = p;
}

// W -> U:  E = p / (gamma-1) + (0.5 * rho) * ((u*u + v*v) + w*w).
template <class T> __device__ __forceinline__ void cons(const T W[5], T U[5], const Gas<T>& g) {
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  const T ke = T(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  if constexpr (FastRcp<T>::on)
    U[4] = W[4] * g.igm1 + ke;
  else
    U[4] = divv(W[4], g.gm1) + ke;
}

// Physical flux along the local normal of local primitives W with energy E.
template <class T> __device__ __forceinline__ void pflux(const T W[5], T E, T F[5]) {
  T mn = W[0] * W[1];
  F[0] = mn;
  F[1] = mn * W[1] + W[4];
  F[2] = mn * W[2];
  F[3] = mn * W[3];
  F[4] = (E + W[4]) * W[1];
}

template <class T> __device__ __forceinline__ T csound(T rho, T p, const Gas<T>& g) {
  return sqrtv(divv(g.gamma * p, rho));
}

// ------------------------------------------------------------- limiters
// dL = w_i - w_{i-1}, dR = w_{i+1} - w_i; 0 unless dL*dR > 0;
//   generalized minmod: sign(dC) min(|theta dL|, |theta dR|, |dC|), dC = 0.5 (dL + dR)
//   van Leer:   (2 dL dR) / (dL + dR)
//   van Albada: (dL dR (dL + dR)) / (dL dL + dR dR)
//   hybrid:     sign(dC) min(|theta dL|, |theta dR|, |dC|, |van Leer|)
// LIM >= 0 fixes the limiter at compile time; LIM = -1 reads `lim` at run time.
// Evaluated without branches on the data (selects), so neighbouring cells of
// a warp never diverge; the selected values are those of the formulas above.
template <int LIM = -1, class T> __device__ __forceinline__ T slope(int lim, T theta, T dL, T dR) {
  if (LIM == LIM_MINMOD1) {
    T prod = dL * dR;
    if constexpr (FastRcp<T>::on) {
      // the same values for finite data (prod > 0 leaves dL != 0): one min
      // and one sign copy instead of compares and selects
      const T r = copysignf(fminf(fabsf(dL), fabsf(dR)), dL);
      return prod > T(0) ? r : T(0);
    }
    T a = absv(dL), b = absv(dR);
    T m = b < a ? b : a;
    T r = dL > T(0) ? m : -m;
    return prod > T(0) ? r : T(0);
  }
  if (LIM >= 0) lim = LIM;
  T prod = dL * dR;
  T dC = T(0.5) * (dL + dR);
  T r;
  if (lim == LIM_VANLEER) {
    r = divv(T(2) * prod, dL + dR);
  } else if (lim == LIM_VANALBADA) {
    r = divv(prod * (dL + dR), dL * dL + dR * dR);
  } else {
    T m = absv(theta * dL);
    T b = absv(theta * dR);
    T c = absv(dC);
    m = b < m ? b : m;
    m = c < m ? c : m;
    if (lim == LIM_HYBRID) {
      T e = absv(divv(T(2) * prod, dL + dR));
      m = e < m ? e : m;
    }
    r = dC > T(0) ? m : -m;
  }
  return prod > T(0) ? r : T(0);
}

// PLM: wL = w0 - 0.5 d, wR = w0 + 0.5 d.
template <int LIM = -1, class T>
__device__ __forceinline__ void plm(T wm, T w0, T wp, int lim, T theta, T& wL, T& wR, T& d) {
  d = slope<LIM>(lim, theta, w0 - wm, wp - w0);
  wL = w0 - T(0.5) * d;
  wR = w0 + T(0.5) * d;
}

// PPM (Colella & Woodward 1984): edges from limited slopes, then the
// monotonicity constraints.
//   L = 0.5 (w_{-1} + w_0) - (d_0 - d_{-1}) / 6,  R = 0.5 (w_0 + w_1) - (d_1 - d_0) / 6
template <int LIM = -1, class T>
__device__ __forceinline__ void ppm(T wmm, T wm, T w0, T wp, T wpp, int lim, T theta, T& wL, T& wR) {
  T dm = slope<LIM>(lim, theta, wm - wmm, w0 - wm);
  T d0 = slope<LIM>(lim, theta, w0 - wm, wp - w0);
  T dp = slope<LIM>(lim, theta, wp - w0, wpp - wp);
  T L, R;
  if constexpr (FastRcp<T>::on) {
    L = T(0.5) * (wm + w0) - (d0 - dm) * T(1.0 / 6.0);
    R = T(0.5) * (w0 + wp) - (dp - d0) * T(1.0 / 6.0);
  } else {
    L = T(0.5) * (wm + w0) - divv(d0 - dm, T(6));
    R = T(0.5) * (w0 + wp) - divv(dp - d0, T(6));
  }
  // constraints as selects: local extremum -> flat; overshoot -> move one edge
  const bool ext = (R - w0) * (w0 - L) <= T(0);
  T dA = R - L;
  T a6 = T(6) * (w0 - T(0.5) * (L + R));
  const bool c1 = dA * a6 > dA * dA;
  const bool c2 = !c1 && (-(dA * dA) > dA * a6);
  T Ln = c1 ? T(3) * w0 - T(2) * R : L;
  T Rn = c2 ? T(3) * w0 - T(2) * L : R;
  wL = ext ? w0 : Ln;
  wR = ext ? w0 : Rn;
}

// ------------------------------------------------- CTU characteristic tracing
// Primitive eigen-system along the local normal at the cell centre:
// lambda = (u-c, u, u, u, u+c); projections l_a . X and additions coef * r_a
// with r_1 = (1, -c/rho, 0, 0, c^2), r_2 = e_0, r_3 = e_2, r_4 = e_3,
// r_5 = (1, c/rho, 0, 0, c^2), l_1 = (0, -rho/(2c), 0, 0, 1/(2c^2)),
// l_2 = (1, 0, 0, 0, -1/c^2), l_5 = (0, rho/(2c), 0, 0, 1/(2c^2)).
template <class T> struct Eig {
  T rho, c;
  T lam[5];
  T r2c;   // rho / (2 c)
  T i2cc;  // (2 c) c
  T cc;    // c c
  T cor;   // c / rho
  T icc;   // 1 / (c c)      (FP32 forms)
  T hicc;  // 1 / ((2 c) c)  (FP32 forms)
};

template <class T> __device__ __forceinline__ void eig(const T W[5], const Gas<T>& g, Eig<T>& e) {
  if constexpr (FastRcp<T>::on) {
    const T ir = divv(T(1), W[0]);
    const T c = sqrtv(g.gamma * W[4] * ir);
    const T ic = divv(T(1), c);
    e.rho = W[0];
    e.c = c;
    e.lam[0] = W[1] - c;
    e.lam[1] = W[1];
    e.lam[2] = W[1];
    e.lam[3] = W[1];
    e.lam[4] = W[1] + c;
    e.r2c = T(0.5) * W[0] * ic;
    e.cc = c * c;
    e.i2cc = T(2) * e.cc;
    e.cor = c * ir;
    e.icc = ic * ic;
    e.hicc = T(0.5) * e.icc;
    return;
  }
  T c = csound(W[0], W[4], g);
  e.rho = W[0];
  e.c = c;
  e.lam[0] = W[1] - c;
  e.lam[1] = W[1];
  e.lam[2] = W[1];
  e.lam[3] = W[1];
  e.lam[4] = W[1] + c;
  e.r2c = W[0] / (T(2) * c);
  e.i2cc = T(2) * c * c;
  e.cc = c * c;
  e.cor = c / W[0];
}

// l_a . X   (a = 0..4)
template <class T> __device__ __forceinline__ T lproj(const Eig<T>& e, int a, const T X[5]) {
  if constexpr (FastRcp<T>::on) {
    if (a == 0) return -e.r2c * X[1] + X[4] * e.hicc;
    if (a == 1) return X[0] - X[4] * e.icc;
    if (a == 2) return X[2];
    if (a == 3) return X[3];
    return e.r2c * X[1] + X[4] * e.hicc;
  }
  if (a == 0) return -e.r2c * X[1] + X[4] / e.i2cc;
  if (a == 1) return X[0] - X[4] / e.cc;
  if (a == 2) return X[2];
  if (a == 3) return X[3];
  return e.r2c * X[1] + X[4] / e.i2cc;
}
// Y += coef r_a
template <class T> __device__ __forceinline__ void radd(const Eig<T>& e, int a, T coef, T Y[5]) {
  if (a == 0) {
    Y[0] = Y[0] + coef;
    Y[1] = Y[1] - coef * e.cor;
    Y[4] = Y[4] + coef * e.cc;
  } else if (a == 1) {
    Y[0] = Y[0] + coef;
  } else if (a == 2) {
    Y[2] = Y[2] + coef;
  } else if (a == 3) {
    Y[3] = Y[3] + coef;
  } else {
    Y[0] = Y[0] + coef;
    Y[1] = Y[1] + coef * e.cor;
    Y[4] = Y[4] + coef * e.cc;
  }
}

// PLM tracing, "reference state" form (Colella 1990; Stone et al. 2008):
//   Wr = W0 + (0.5 (1 - lamM dtdx)) dW + sum_{lam_a>0} ((0.5 dtdx) (lamM - lam_a)) (l_a.dW) r_a
//   Wl = W0 - (0.5 (1 + lamm dtdx)) dW + sum_{lam_a<0} ((0.5 dtdx) (lamm - lam_a)) (l_a.dW) r_a
// lamM = max(lam_5, 0), lamm = min(lam_1, 0); local frame.  Each wave is
// evaluated once with the coefficients of the side it travels to; the other
// side receives an exact zero (no data-dependent branches).
template <class T>
__device__ __forceinline__ void trace_plm(const T W0[5], const T dW[5], T dtdx, const Gas<T>& g, T Wl[5], T Wr[5]) {
  Eig<T> e;
  eig(W0, g, e);
  T lamM, lamm;
  if constexpr (FastRcp<T>::on) {
    lamM = fmaxf(e.lam[4], 0.0f);
    lamm = fminf(e.lam[0], 0.0f);
  } else {
    lamM = e.lam[4] > T(0) ? e.lam[4] : T(0);
    lamm = e.lam[0] < T(0) ? e.lam[0] : T(0);
  }
  T fr = T(0.5) * (T(1) - lamM * dtdx);
  T fl = T(0.5) * (T(1) + lamm * dtdx);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Wr[v] = W0[v] + fr * dW[v];
    Wl[v] = W0[v] - fl * dW[v];
  }
  T hdt = T(0.5) * dtdx;
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    const T la = e.lam[a];
    const bool pos = la > T(0), neg = la < T(0);
    T coef = hdt * ((pos ? lamM : lamm) - la) * lproj(e, a, dW);
    radd(e, a, pos ? coef : T(0), Wr);
    radd(e, a, neg ? coef : T(0), Wl);
  }
}

// PPM tracing (Colella & Woodward 1984 parabola, averaged over each wave's
// domain of dependence; same reference-state form):
//   dA = WR - WL, W6 = 6 (W0 - 0.5 (WL + WR)), sM = lamM dtdx, sm = lamm dtdx
//   Wr = WR - (0.5 sM) (dA - (1 - (2/3) sM) W6)
//        + sum_{lam_a>0} l_a.[c1 (dA - W6) + c2 W6] r_a,
//          c1 = (0.5 dtdx) (lamM - lam_a), c2 = ((1/3) dtdx) dtdx (lamM^2 - lam_a^2)
//   Wl = WL - (0.5 sm) (dA + (1 + (2/3) sm) W6)
//        + sum_{lam_a<0} l_a.[c1 (dA + W6) + c2 W6] r_a   (lamm in place of lamM)
template <class T>
__device__ __forceinline__ void trace_ppm(const T W0[5], const T WL[5], const T WR[5], T dtdx, const Gas<T>& g, T Wl[5],
                                          T Wr[5]) {
  Eig<T> e;
  eig(W0, g, e);
  T lamM, lamm;
  if constexpr (FastRcp<T>::on) {
    lamM = fmaxf(e.lam[4], 0.0f);
    lamm = fminf(e.lam[0], 0.0f);
  } else {
    lamM = e.lam[4] > T(0) ? e.lam[4] : T(0);
    lamm = e.lam[0] < T(0) ? e.lam[0] : T(0);
  }
  T dA[5], W6[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dA[v] = WR[v] - WL[v];
    W6[v] = T(6) * (W0[v] - T(0.5) * (WL[v] + WR[v]));
  }
  T sM = lamM * dtdx;
  T sm = lamm * dtdx;
  T qr = T(0.5) * sM, qr2 = T(1) - T(2.0 / 3.0) * sM;
  T ql = T(0.5) * sm, ql2 = T(1) + T(2.0 / 3.0) * sm;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Wr[v] = WR[v] - qr * (dA[v] - qr2 * W6[v]);
    Wl[v] = WL[v] - ql * (dA[v] + ql2 * W6[v]);
  }
  T hdt = T(0.5) * dtdx;
  T tdt = T(1.0 / 3.0) * dtdx * dtdx;
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    const T la = e.lam[a];
    const bool pos = la > T(0), neg = la < T(0);
    const T lref = pos ? lamM : lamm;
    T c1 = hdt * (lref - la);
    T c2 = tdt * (lref * lref - la * la);
    T X[5];
    if constexpr (FastRcp<T>::on) {
      // c1 (dA -/+ W6) + c2 W6 = c1 dA + (c2 -/+ c1) W6: one coefficient per wave
      const T k = pos ? c2 - c1 : c2 + c1;
#pragma unroll
      for (int v = 0; v < 5; ++v) X[v] = fmaf(k, W6[v], c1 * dA[v]);
    } else {
#pragma unroll
      for (int v = 0; v < 5; ++v) X[v] = c1 * (pos ? dA[v] - W6[v] : dA[v] + W6[v]) + c2 * W6[v];
    }
    T coef = lproj(e, a, X);
    radd(e, a, pos ? coef : T(0), Wr);
    radd(e, a, neg ? coef : T(0), Wl);
  }
}

// ------------------------------------------------------------ Riemann
// One side of a face: local conserved U, local primitives W (floored), c,
// physical flux F.
template <class T> struct Side {
  T U[5], W[5], c, F[5];
  T ir;  // 1 / rho (FP32 forms)
};

template <class T, bool MIXED> __device__ __forceinline__ void mkside(const T U[5], const Gas<T>& g, Side<T>& s) {
#pragma unroll
  for (int v = 0; v < 5; ++v) s.U[v] = U[v];
  prim<T, MIXED>(U, s.W, g, &s.ir);
  if constexpr (FastRcp<T>::on)
    s.c = sqrtv(g.gamma * s.W[4] * s.ir);
  else
    s.c = csound(s.W[0], s.W[4], g);
  pflux(s.W, U[4], s.F);
}

// Roe averages with sqrt(rho) weights.
template <class T> struct RAvg {
  T u, v, w, H, q2, a2;
};
template <class T> __device__ __forceinline__ void ravg(const Side<T>& L, const Side<T>& R, const Gas<T>& g, RAvg<T>& A) {
  T sL = sqrtv(L.W[0]);
  T sR = sqrtv(R.W[0]);
  T inv = divv(T(1), sL + sR);
  A.u = (sL * L.W[1] + sR * R.W[1]) * inv;
  A.v = (sL * L.W[2] + sR * R.W[2]) * inv;
  A.w = (sL * L.W[3] + sR * R.W[3]) * inv;
  T HL, HR;
  if constexpr (FastRcp<T>::on) {
    HL = (L.U[4] + L.W[4]) * L.ir;
    HR = (R.U[4] + R.W[4]) * R.ir;
  } else {
    HL = (L.U[4] + L.W[4]) / L.W[0];
    HR = (R.U[4] + R.W[4]) / R.W[0];
  }
  A.H = (sL * HL + sR * HR) * inv;
  A.q2 = A.u * A.u + A.v * A.v + A.w * A.w;
  A.a2 = g.gm1 * (A.H - T(0.5) * A.q2);
}

// Einfeldt speeds SL = min(uL - cL, u~ - a~), SR = max(uR + cR, u~ + a~).
template <class T>
__device__ __forceinline__ void einfeldt(const Side<T>& L, const Side<T>& R, const Gas<T>& g, T& SL, T& SR) {
  RAvg<T> A;
  ravg(L, R, g, A);
  T a = A.a2 > T(0) ? sqrtv(A.a2) : T(0);
  if constexpr (FastRcp<T>::on) {
    SL = fminf(L.W[1] - L.c, A.u - a);
    SR = fmaxf(R.W[1] + R.c, A.u + a);
    return;
  }
  SL = L.W[1] - L.c;
  T t = A.u - a;
  if (t < SL) SL = t;
  SR = R.W[1] + R.c;
  t = A.u + a;
  if (t > SR) SR = t;
}

// HLLE: F = ((b+ FL - b- FR) + (b+ b-) (UR - UL)) * (1 / (b+ - b-)).
template <class T> __device__ __forceinline__ void hlle(const Side<T>& L, const Side<T>& R, const Gas<T>& g, T F[5]) {
  T SL, SR;
  einfeldt(L, R, g, SL, SR);
  T bp, bm;
  if constexpr (FastRcp<T>::on) {
    bp = fmaxf(SR, 0.0f);
    bm = fminf(SL, 0.0f);
  } else {
    bp = SR > T(0) ? SR : T(0);
    bm = SL < T(0) ? SL : T(0);
  }
  T inv = divv(T(1), bp - bm);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = (bp * L.F[v] - bm * R.F[v] + bp * bm * (R.U[v] - L.U[v])) * inv;
}

// HLLC with the Einfeldt speeds and
//   S* = (((pR - pL) + mL uL) - mR uR) / (mL - mR),  mK = rhoK (SK - uK),
//   U*K = f (1, S*, vK, wK, EK/rhoK + (S* - uK)(S* + pK/mK)),  f = mK / (SK - S*),
//   F = FK + SK (U*K - UK) in the star region of side K.
template <class T> __device__ __forceinline__ void hllc(const Side<T>& L, const Side<T>& R, const Gas<T>& g, T F[5]) {
  T SL, SR;
  einfeldt(L, R, g, SL, SR);
  T mL = L.W[0] * (SL - L.W[1]);
  T mR = R.W[0] * (SR - R.W[1]);
  T Ss = divv(R.W[4] - L.W[4] + mL * L.W[1] - mR * R.W[1], mL - mR);
  // region: SL >= 0 -> FL; S* >= 0 -> left star; SR > 0 -> right star; else FR
  const bool useL = SL >= T(0);
  const bool left = Ss >= T(0);
  const bool useR = !useL && !left && !(SR > T(0));
  T SK = left ? SL : SR;
  T mK = left ? mL : mR;
  T uK = left ? L.W[1] : R.W[1];
  T vK = left ? L.W[2] : R.W[2];
  T wK = left ? L.W[3] : R.W[3];
  T rK = left ? L.W[0] : R.W[0];
  T pK = left ? L.W[4] : R.W[4];
  T f = divv(mK, SK - Ss);
  T Us[5], UK[5], FK[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    UK[v] = left ? L.U[v] : R.U[v];
    FK[v] = left ? L.F[v] : R.F[v];
  }
  Us[0] = f;
  Us[1] = f * Ss;
  Us[2] = f * vK;
  Us[3] = f * wK;
  Us[4] = f * (divv(UK[4], rK) + (Ss - uK) * (Ss + divv(pK, mK)));
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T Fs = FK[v] + SK * (Us[v] - UK[v]);
    F[v] = useL ? L.F[v] : (useR ? R.F[v] : Fs);
  }
}

// Exact solver (Toro 2009 ch. 4): Newton on fL(p) + fR(p) + (uR - uL) = 0
// from the PVRS guess floored at 1e-8 of the mean pressure; stop when
// 2|p_new - p|/(p_new + p) < tol (1e-14 FP64, 1e-6 FP32) or after 64 steps.
template <class T> __device__ __forceinline__ T exact_tol();
template <> __device__ __forceinline__ double exact_tol<double>() { return 1.0e-14; }
template <> __device__ __forceinline__ float exact_tol<float>() { return 1.0e-6f; }

template <class T>
__device__ __forceinline__ void exact_fk(T p, T rk, T pk, T ck, const Gas<T>& g, T& f, T& df) {
  T gam = g.gamma;
  if (p > pk) {
    T A = T(2) / ((gam + T(1)) * rk);
    T B = (gam - T(1)) / (gam + T(1)) * pk;
    T q = sqrtv(A / (p + B));
    f = (p - pk) * q;
    df = q * (T(1) - (p - pk) / (T(2) * (B + p)));
  } else {
    T pr = p / pk;
    f = T(2) * ck / (gam - T(1)) * (powv(pr, (gam - T(1)) / (T(2) * gam)) - T(1));
    df = T(1) / (rk * ck) * powv(pr, -(gam + T(1)) / (T(2) * gam));
  }
}

// Result of the out-of-line exact solver: flux and status bits.
template <class T> struct Flux5 {
  T F[5];
  unsigned st;
};
template <class T> struct V5 {
  T v[5];
};

// Exact flux from local primitives (W), sound speeds and total energies of
// both sides.  On vacuum generation (no star state) the status gets
// ST_EXACT_FAIL and the flux is the HLLE flux; on no convergence the status
// gets ST_EXACT_FAIL and the last iterate is sampled.  Kept out of line and
// fed by value: it is the slow reference solver (Sec. 2) and the rare
// fallback path.
template <class T>
__device__ __noinline__ Flux5<T> exact_flux(V5<T> WLv, V5<T> WRv, T cL, T cR, T EL, T ER, Gas<T> g) {
  Flux5<T> out;
  out.st = 0;
  Side<T> L, R;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    L.W[v] = WLv.v[v];
    R.W[v] = WRv.v[v];
  }
  L.c = cL;
  R.c = cR;
  L.ir = T(1) / L.W[0];
  R.ir = T(1) / R.W[0];
  L.U[0] = L.W[0]; L.U[1] = L.W[0] * L.W[1]; L.U[2] = L.W[0] * L.W[2]; L.U[3] = L.W[0] * L.W[3]; L.U[4] = EL;
  R.U[0] = R.W[0]; R.U[1] = R.W[0] * R.W[1]; R.U[2] = R.W[0] * R.W[2]; R.U[3] = R.W[0] * R.W[3]; R.U[4] = ER;
  T gam = g.gamma;
  T du = R.W[1] - L.W[1];
  if (T(2) / (gam - T(1)) * (L.c + R.c) <= du) {
    // vacuum: the HLLE flux of the (unchanged) conserved states
    pflux(L.W, EL, L.F);
    pflux(R.W, ER, R.F);
    out.st = ST_EXACT_FAIL;
    hlle(L, R, g, out.F);
    return out;
  }
  T ppv = T(0.5) * (L.W[4] + R.W[4]) - T(0.125) * du * (L.W[0] + R.W[0]) * (L.c + R.c);
  T pmin = T(1.0e-8) * T(0.5) * (L.W[4] + R.W[4]);
  T p = ppv > pmin ? ppv : pmin;
  bool conv = false;
  for (int it = 0; it < 64; ++it) {
    T fL, dfL, fR, dfR;
    exact_fk(p, L.W[0], L.W[4], L.c, g, fL, dfL);
    exact_fk(p, R.W[0], R.W[4], R.c, g, fR, dfR);
    T pn = p - (fL + fR + du) / (dfL + dfR);
    if (pn < pmin) pn = pmin;
    T change = T(2) * absv(pn - p) / (pn + p);
    p = pn;
    if (change < exact_tol<T>()) {
      conv = true;
      break;
    }
  }
  if (!conv) out.st = ST_EXACT_FAIL;
  T fL, dfL, fR, dfR;
  exact_fk(p, L.W[0], L.W[4], L.c, g, fL, dfL);
  exact_fk(p, R.W[0], R.W[4], R.c, g, fR, dfR);
  T ps = p;
  T us = T(0.5) * (L.W[1] + R.W[1]) + T(0.5) * (fR - fL);
  // sample at x/t = 0 (a point on a wave takes its left state)
  T g5 = T(2) / (gam + T(1));
  T g6 = (gam - T(1)) / (gam + T(1));
  T g7 = T(0.5) * (gam - T(1));
  T W[5];
  const bool left = T(0) <= us;
  const Side<T>& K = left ? L : R;
  W[2] = K.W[2];
  W[3] = K.W[3];
  T sgn = left ? T(1) : T(-1);  // mirror the right side onto the left-side formulas
  T uK = sgn * K.W[1];
  if (ps > K.W[4]) {  // shock
    T pr = ps / K.W[4];
    T SK = uK - K.c * sqrtv((gam + T(1)) / (T(2) * gam) * pr + (gam - T(1)) / (T(2) * gam));
    if (T(0) <= SK) {
      W[0] = K.W[0];
      W[1] = K.W[1];
      W[4] = K.W[4];
    } else {
      W[0] = K.W[0] * (pr + g6) / (g6 * pr + T(1));
      W[1] = us;
      W[4] = ps;
    }
  } else {  // rarefaction
    T SH = uK - K.c;
    if (T(0) <= SH) {
      W[0] = K.W[0];
      W[1] = K.W[1];
      W[4] = K.W[4];
    } else {
      T pr = ps / K.W[4];
      T ST = sgn * us - K.c * powv(pr, (gam - T(1)) / (T(2) * gam));
      if (T(0) > ST) {
        W[0] = K.W[0] * powv(pr, T(1) / gam);
        W[1] = us;
        W[4] = ps;
      } else {
        T c = g5 * (K.c + g7 * uK);
        W[1] = sgn * c;
        W[0] = K.W[0] * powv(c / K.c, T(2) / (gam - T(1)));
        W[4] = K.W[4] * powv(c / K.c, T(2) * gam / (gam - T(1)));
      }
    }
  }
  T E = W[4] / (gam - T(1)) + T(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  pflux(W, E, out.F);
  return out;
}

template <class T> __device__ __forceinline__ unsigned exact_call(const Side<T>& L, const Side<T>& R, const Gas<T>& g,
                                                                  T F[5]) {
  V5<T> a, b;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    a.v[v] = L.W[v];
    b.v[v] = R.W[v];
  }
  Flux5<T> r = exact_flux(a, b, L.c, R.c, L.U[4], R.U[4], g);
#pragma unroll
  for (int v = 0; v < 5; ++v) F[v] = r.F[v];
  return r.st;
}

// Roe (1981) with the 3D wave strengths (Toro 2009 sec. 11.3); see the
// header comment of roe() for the evaluation order.  Returns false when the
// linearisation fails (a~^2 <= 0, or an intermediate state with rho <= 0 or
// p <= 0).
template <class T> __device__ __forceinline__ bool roe(const Side<T>& L, const Side<T>& R, const Gas<T>& g, T F[5]) {
  RAvg<T> A;
  ravg(L, R, g, A);
  if (!(A.a2 > T(0))) return false;
  // FP32: a, (gamma-1)/a^2 and 1/(2a) from one reciprocal square root
  T a, gma2, i2a;
  if constexpr (FastRcp<T>::on) {
    const T ia = rsqrtf(A.a2);
    a = A.a2 * ia;
    gma2 = g.gm1 * (ia * ia);
    i2a = T(0.5) * ia;
  } else {
    a = sqrtv(A.a2);
  }
  T d0 = R.U[0] - L.U[0], d1 = R.U[1] - L.U[1], d2 = R.U[2] - L.U[2], d3 = R.U[3] - L.U[3],
    d4 = R.U[4] - L.U[4];
  T a3 = d2 - A.v * d0;
  T a4 = d3 - A.w * d0;
  T d4b = d4 - a3 * A.v - a4 * A.w;
  T a2, a1;
  if constexpr (FastRcp<T>::on) {
    a2 = gma2 * (d0 * (A.H - A.u * A.u) + A.u * d1 - d4b);
    a1 = (d0 * (A.u + a) - d1 - a * a2) * i2a;
  } else {
    a2 = divv(g.gm1, A.a2) * (d0 * (A.H - A.u * A.u) + A.u * d1 - d4b);
    a1 = divv(d0 * (A.u + a) - d1 - a * a2, T(2) * a);
  }
  T a5 = d0 - (a1 + a2);
  T K11 = A.u - a, K14 = A.H - A.u * a;
  T K51 = A.u + a, K54 = A.H + A.u * a;
  T K24 = T(0.5) * A.q2;
  // intermediate states U*1 = UL + a1 K1, U*2 = U*1 + a2 K2 + a3 K3 + a4 K4
  T s0 = L.U[0] + a1, s1 = L.U[1] + a1 * K11, s2 = L.U[2] + a1 * A.v, s3 = L.U[3] + a1 * A.w, s4 = L.U[4] + a1 * K14;
  if (!(s0 > T(0))) return false;
  if constexpr (FastRcp<T>::on) {
    // p > 0  <=>  2 E rho > |m|^2 for rho > 0 (and gamma > 1)
    if (!(T(2) * s4 * s0 > s1 * s1 + s2 * s2 + s3 * s3)) return false;
  } else {
    T p1 = g.gm1 * (s4 - divv(T(0.5) * (s1 * s1 + s2 * s2 + s3 * s3), s0));
    if (!(p1 > T(0))) return false;
  }
  s0 = s0 + a2;
  s1 = s1 + a2 * A.u;
  s2 = s2 + a2 * A.v + a3;
  s3 = s3 + a2 * A.w + a4;
  s4 = s4 + a2 * K24 + a3 * A.v + a4 * A.w;
  if (!(s0 > T(0))) return false;
  if constexpr (FastRcp<T>::on) {
    if (!(T(2) * s4 * s0 > s1 * s1 + s2 * s2 + s3 * s3)) return false;
  } else {
    T p2 = g.gm1 * (s4 - divv(T(0.5) * (s1 * s1 + s2 * s2 + s3 * s3), s0));
    if (!(p2 > T(0))) return false;
  }
  T c1 = absv(A.u - a) * a1;
  T c2 = absv(A.u) * a2;
  T c3 = absv(A.u) * a3;
  T c4 = absv(A.u) * a4;
  T c5 = absv(A.u + a) * a5;
  T D0 = c1 + c2 + c5;
  T D1 = c1 * K11 + c2 * A.u + c5 * K51;
  T D2 = c1 * A.v + c2 * A.v + c3 + c5 * A.v;
  T D3 = c1 * A.w + c2 * A.w + c4 + c5 * A.w;
  T D4 = c1 * K14 + c2 * K24 + c3 * A.v + c4 * A.w + c5 * K54;
  F[0] = T(0.5) * (L.F[0] + R.F[0]) - T(0.5) * D0;
  F[1] = T(0.5) * (L.F[1] + R.F[1]) - T(0.5) * D1;
  F[2] = T(0.5) * (L.F[2] + R.F[2]) - T(0.5) * D2;
  F[3] = T(0.5) * (L.F[3] + R.F[3]) - T(0.5) * D3;
  F[4] = T(0.5) * (L.F[4] + R.F[4]) - T(0.5) * D4;
  return true;
}

// Riemann flux in the local frame (states and flux already ordered normal
// first); returns status bits.
template <class T, bool MIXED, int RS>
__device__ __forceinline__ unsigned riemann_local(const T ul[5], const T ur[5], const Opts<T>& o, T F[5]) {
  Side<T> L, R;
  mkside<T, MIXED>(ul, o.gas, L);
  mkside<T, MIXED>(ur, o.gas, R);
  unsigned st = 0;
  if (RS == RS_ROE) {
    if (!roe(L, R, o.gas, F)) {
      st = ST_ROE_FALLBACK;
      if (o.fallback == RS_HLLC)
        hllc(L, R, o.gas, F);
      else if (o.fallback == RS_EXACT)
        st |= exact_call(L, R, o.gas, F);
      else
        hlle(L, R, o.gas, F);
    }
  } else if (RS == RS_HLLC) {
    hllc(L, R, o.gas, F);
  } else if (RS == RS_HLLE) {
    hlle(L, R, o.gas, F);
  } else {
    st = exact_call(L, R, o.gas, F);
  }
  return st;
}

// Global component of the local momentum components for direction d:
// local 1, 2, 3 = global 1 + d, 1 + (d+1)%3, 1 + (d+2)%3.
struct LocalComps {
  int c1, c2, c3;
  __device__ __forceinline__ explicit LocalComps(int d)
      : c1(1 + d), c2(d == 2 ? 1 : d + 2), c3(d == 0 ? 3 : d) {}
};

// Global <-> local frame of a run-time direction d, by selects (no dynamic
// register indexing): local (n, t1, t2) = (x, y, z), (y, z, x), (z, x, y).
template <class T> __device__ __forceinline__ void to_local_rt(int d, const T g[5], T l[5]) {
  l[0] = g[0];
  l[1] = d == 0 ? g[1] : (d == 1 ? g[2] : g[3]);
  l[2] = d == 0 ? g[2] : (d == 1 ? g[3] : g[1]);
  l[3] = d == 0 ? g[3] : (d == 1 ? g[1] : g[2]);
  l[4] = g[4];
}
template <class T> __device__ __forceinline__ void to_global_rt(int d, const T l[5], T g[5]) {
  g[0] = l[0];
  g[1] = d == 0 ? l[1] : (d == 1 ? l[3] : l[2]);
  g[2] = d == 0 ? l[2] : (d == 1 ? l[1] : l[3]);
  g[3] = d == 0 ? l[3] : (d == 1 ? l[2] : l[1]);
  g[4] = l[4];
}

// Load / store a 5-vector in the local frame of direction d from / to memory
// holding it in the global frame with element stride s.
template <class T>
__device__ __forceinline__ void load_local(const T* p, int s, const LocalComps& lc, T a[5]) {
  a[0] = p[0];
  a[1] = p[lc.c1 * s];
  a[2] = p[lc.c2 * s];
  a[3] = p[lc.c3 * s];
  a[4] = p[4 * s];
}
template <class T>
__device__ __forceinline__ void store_local(T* p, int s, const LocalComps& lc, const T a[5]) {
  p[0] = a[0];
  p[lc.c1 * s] = a[1];
  p[lc.c2 * s] = a[2];
  p[lc.c3 * s] = a[3];
  p[4 * s] = a[4];
}

// W -> U for a state given in the local frame of direction d, with the
// kinetic sum taken in the GLOBAL component order (u^2 + v^2) + w^2, so the
// result equals cons() of the rotated-back state value for value.
template <class T> __device__ __forceinline__ void cons_local(const T W[5], int d, const Gas<T>& g, T U[5]) {
  T a = W[1] * W[1], b = W[2] * W[2], c = W[3] * W[3];
  // global (u, v, w) = (n, t1, t2) for x, (t2, n, t1) for y, (t1, t2, n) for z;
  // the FP32 forms take one order for every direction
  T ke;
  if constexpr (FastRcp<T>::on)
    ke = a + b + c;
  else
    ke = d == 0 ? a + b + c : (d == 1 ? c + a + b : b + c + a);
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  if constexpr (FastRcp<T>::on)
    U[4] = W[4] * g.igm1 + T(0.5) * W[0] * ke;
  else
    U[4] = divv(W[4], g.gm1) + T(0.5) * W[0] * ke;
}

}  // namespace hyd
