// ORACLE — test infrastructure only (see real.hpp).
//
// Spatial data reconstruction of step (1) of Sec. 2: PLM and PPM on primitive
// variables, the four slope limiters named in Sec. 2 (generalized minmod,
// van Leer type, van Albada type and the hybrid of generalized minmod and
// van Leer), and the CTU characteristic tracing to t + dt/2 (Sec. 2 step (1),
// after Colella 1990 and Stone et al. 2008 to which Sec. 2 refers).
#pragma once
#include "euler.hpp"

namespace orc {

enum Limiter { LIM_MINMOD = 0, LIM_VANLEER = 1, LIM_VANALBADA = 2, LIM_HYBRID = 3 };

// Limited slope from the left and right differences dL = w_i - w_{i-1},
// dR = w_{i+1} - w_i (Sec. 2; definitions per Toro 2009 ch. 13-14):
//   generalized minmod : minmod(theta dL, theta dR, (dL + dR)/2)
//   van Leer type      : 2 dL dR / (dL + dR)                 if dL dR > 0
//   van Albada type    : dL dR (dL + dR) / (dL^2 + dR^2)      if dL dR > 0
//   hybrid             : sign(dC) min(theta|dL|, theta|dR|, |dC|, |vanLeer|)
// and 0 whenever dL dR <= 0.  theta (1 <= theta <= 2) is the generalized
// minmod parameter; the hybrid reads "combines generalized minmod and van
// Leer" as the smaller in magnitude of the two.
template <class R> inline R limited_slope(int limiter, R theta, R dL, R dR) {
  R prod = dL * dR;
  if (!(prod > R(0.0))) return R(0.0);
  R dC = R(0.5) * (dL + dR);
  switch (limiter) {
    case LIM_MINMOD: {
      R a = fabs(theta * dL), b = fabs(theta * dR), c = fabs(dC);
      R m = a;
      if (b < m) m = b;
      if (c < m) m = c;
      return dC > R(0.0) ? m : -m;
    }
    case LIM_VANLEER:
      return R(2.0) * prod / (dL + dR);
    case LIM_VANALBADA:
      return prod * (dL + dR) / (dL * dL + dR * dR);
    default: {  // LIM_HYBRID
      R vl = R(2.0) * prod / (dL + dR);
      R a = fabs(theta * dL), b = fabs(theta * dR), c = fabs(dC), e = fabs(vl);
      R m = a;
      if (b < m) m = b;
      if (c < m) m = c;
      if (e < m) m = e;
      return dC > R(0.0) ? m : -m;
    }
  }
}

// PLM face values of one cell from the stencil w[-1..1] (pointer to w_i,
// element stride st):  wL = w_i - delta/2 (left face), wR = w_i + delta/2.
template <class R>
inline void plm_faces(const R* w, long st, int limiter, R theta, R* wL, R* wR, R* delta) {
  Sec<R> sec(SEC_RECON);
  R d = limited_slope(limiter, theta, w[0] - w[-st], w[st] - w[0]);
  *wL = w[0] - R(0.5) * d;
  *wR = w[0] + R(0.5) * d;
  if (delta) *delta = d;
}

// PPM face values of one cell from the stencil w[-2..2] (Colella & Woodward
// 1984, "PPM" of Sec. 2):
//   edge value w_{i+1/2} = (w_i + w_{i+1})/2 - (delta_{i+1} - delta_i)/6 with
//   delta the limited PLM slope (same limiter), then the monotonicity
//   constraints: flatten at a local extremum, and move one edge value so the
//   parabola's extremum sits on the cell edge when it would overshoot.
template <class R>
inline void ppm_faces(const R* w, long st, int limiter, R theta, R* wL, R* wR) {
  Sec<R> sec(SEC_RECON);
  R dm = limited_slope(limiter, theta, w[-st] - w[-2 * st], w[0] - w[-st]);   // delta_{i-1}
  R d0 = limited_slope(limiter, theta, w[0] - w[-st], w[st] - w[0]);          // delta_i
  R dp = limited_slope(limiter, theta, w[st] - w[0], w[2 * st] - w[st]);      // delta_{i+1}
  R L = R(0.5) * (w[-st] + w[0]) - (d0 - dm) / R(6.0);
  R Rr = R(0.5) * (w[0] + w[st]) - (dp - d0) / R(6.0);
  R a = w[0];
  if ((Rr - a) * (a - L) <= R(0.0)) {
    L = a;
    Rr = a;
  } else {
    R dA = Rr - L;
    R a6 = R(6.0) * (a - R(0.5) * (L + Rr));
    if (dA * a6 > dA * dA) {
      L = R(3.0) * a - R(2.0) * Rr;
    } else if (-(dA * dA) > dA * a6) {
      Rr = R(3.0) * a - R(2.0) * L;
    }
  }
  *wL = L;
  *wR = Rr;
}

// ---------------------------------------------------------------------------
// CTU characteristic tracing (Sec. 2 step (1)).
//
// Eigen-system of the primitive-variable Jacobian along the local normal,
// W = (rho, u_n, u_t1, u_t2, p), evaluated at the cell-centred state:
//   lambda = (u - c, u, u, u, u + c)
//   r_1 = (1, -c/rho, 0, 0, c^2)     l_1 = (0, -rho/(2c), 0, 0, 1/(2c^2))
//   r_2 = (1, 0, 0, 0, 0)            l_2 = (1, 0, 0, 0, -1/c^2)
//   r_3 = (0, 0, 1, 0, 0)            l_3 = (0, 0, 1, 0, 0)
//   r_4 = (0, 0, 0, 1, 0)            l_4 = (0, 0, 0, 1, 0)
//   r_5 = (1,  c/rho, 0, 0, c^2)     l_5 = (0,  rho/(2c), 0, 0, 1/(2c^2))
// ---------------------------------------------------------------------------
template <class R> struct Eigen {
  R lam[5];
  R rho, c;
};

template <class R> inline void eigen_prim(const R W[5], const Gas<R>& gas, Eigen<R>& e) {
  R c = sound_speed(W[0], W[4], gas);
  e.rho = W[0];
  e.c = c;
  e.lam[0] = W[1] - c;
  e.lam[1] = W[1];
  e.lam[2] = W[1];
  e.lam[3] = W[1];
  e.lam[4] = W[1] + c;
}

// Project X onto wave a (l_a . X) and add coef * r_a to Y.
template <class R> inline R left_proj(const Eigen<R>& e, int a, const R X[5]) {
  switch (a) {
    case 0: return -(e.rho / (R(2.0) * e.c)) * X[1] + X[4] / (R(2.0) * e.c * e.c);
    case 1: return X[0] - X[4] / (e.c * e.c);
    case 2: return X[2];
    case 3: return X[3];
    default: return (e.rho / (R(2.0) * e.c)) * X[1] + X[4] / (R(2.0) * e.c * e.c);
  }
}
template <class R> inline void add_right(const Eigen<R>& e, int a, R coef, R Y[5]) {
  switch (a) {
    case 0:
      Y[0] += coef;
      Y[1] -= coef * (e.c / e.rho);
      Y[4] += coef * (e.c * e.c);
      break;
    case 1: Y[0] += coef; break;
    case 2: Y[2] += coef; break;
    case 3: Y[3] += coef; break;
    default:
      Y[0] += coef;
      Y[1] += coef * (e.c / e.rho);
      Y[4] += coef * (e.c * e.c);
      break;
  }
}

// PLM tracing ("reference state" form, Colella 1990 / Stone et al. 2008):
//   state on the left of face i+1/2 (right edge of cell i):
//     W = W_i + (1 - lamM dtdx)/2 dW + dtdx/2 sum_{lam_a > 0} (lamM - lam_a)(l_a.dW) r_a,
//     lamM = max(lam_max, 0);
//   state on the right of face i-1/2 (left edge of cell i):
//     W = W_i - (1 + lamm dtdx)/2 dW + dtdx/2 sum_{lam_a < 0} (lamm - lam_a)(l_a.dW) r_a,
//     lamm = min(lam_min, 0).
// All arrays are in the local frame.
template <class R>
inline void trace_plm(const R W0[5], const R dW[5], R dtdx, const Gas<R>& gas, R Wl[5], R Wr[5]) {
  Sec<R> sec(SEC_TRACE);
  Eigen<R> e;
  eigen_prim(W0, gas, e);
  R lamM = e.lam[4] > R(0.0) ? e.lam[4] : R(0.0);
  R lamm = e.lam[0] < R(0.0) ? e.lam[0] : R(0.0);
  for (int v = 0; v < 5; ++v) {
    Wr[v] = W0[v] + R(0.5) * (R(1.0) - lamM * dtdx) * dW[v];
    Wl[v] = W0[v] - R(0.5) * (R(1.0) + lamm * dtdx) * dW[v];
  }
  for (int a = 0; a < 5; ++a) {
    if (e.lam[a] > R(0.0)) {
      R coef = R(0.5) * dtdx * (lamM - e.lam[a]) * left_proj(e, a, dW);
      add_right(e, a, coef, Wr);
    }
    if (e.lam[a] < R(0.0)) {
      R coef = R(0.5) * dtdx * (lamm - e.lam[a]) * left_proj(e, a, dW);
      add_right(e, a, coef, Wl);
    }
  }
}

// PPM tracing: the parabola of cell i, W(xi) = WL + xi (dA + W6 (1 - xi)) with
// dA = WR - WL and W6 = 6 (W_i - (WL + WR)/2), averaged over each wave's
// domain of dependence (Colella & Woodward 1984; Stone et al. 2008), in the
// same reference-state form as the PLM tracing:
//   left of face i+1/2:
//     W = WR - lamM dtdx/2 (dA - (1 - 2/3 lamM dtdx) W6)
//       + sum_{lam_a > 0} l_a.[dtdx/2 (lamM - lam_a)(dA - W6)
//                              + dtdx^2/3 (lamM^2 - lam_a^2) W6] r_a
//   right of face i-1/2:
//     W = WL - lamm dtdx/2 (dA + (1 + 2/3 lamm dtdx) W6)
//       + sum_{lam_a < 0} l_a.[dtdx/2 (lamm - lam_a)(dA + W6)
//                              + dtdx^2/3 (lamm^2 - lam_a^2) W6] r_a
// (the second line uses sigma = -lamm dtdx > 0 as the fraction of the cell
// swept by the fastest left-moving wave).
template <class R>
inline void trace_ppm(const R W0[5], const R WLc[5], const R WRc[5], R dtdx, const Gas<R>& gas,
                      R Wl[5], R Wr[5]) {
  Sec<R> sec(SEC_TRACE);
  Eigen<R> e;
  eigen_prim(W0, gas, e);
  R lamM = e.lam[4] > R(0.0) ? e.lam[4] : R(0.0);
  R lamm = e.lam[0] < R(0.0) ? e.lam[0] : R(0.0);
  R dA[5], W6[5];
  for (int v = 0; v < 5; ++v) {
    dA[v] = WRc[v] - WLc[v];
    W6[v] = R(6.0) * (W0[v] - R(0.5) * (WLc[v] + WRc[v]));
  }
  R sM = lamM * dtdx;  // fraction of the cell swept by the fastest right-mover
  R sm = lamm * dtdx;  // (negative) same for the fastest left-mover
  for (int v = 0; v < 5; ++v) {
    Wr[v] = WRc[v] - R(0.5) * sM * (dA[v] - (R(1.0) - R(2.0 / 3.0) * sM) * W6[v]);
    Wl[v] = WLc[v] - R(0.5) * sm * (dA[v] + (R(1.0) + R(2.0 / 3.0) * sm) * W6[v]);
  }
  for (int a = 0; a < 5; ++a) {
    if (e.lam[a] > R(0.0)) {
      R la = e.lam[a];
      R X[5];
      R c1 = R(0.5) * dtdx * (lamM - la);
      R c2 = R(1.0 / 3.0) * dtdx * dtdx * (lamM * lamM - la * la);
      for (int v = 0; v < 5; ++v) X[v] = c1 * (dA[v] - W6[v]) + c2 * W6[v];
      add_right(e, a, left_proj(e, a, X), Wr);
    }
    if (e.lam[a] < R(0.0)) {
      R la = e.lam[a];
      R X[5];
      R c1 = R(0.5) * dtdx * (lamm - la);
      R c2 = R(1.0 / 3.0) * dtdx * dtdx * (lamm * lamm - la * la);
      for (int v = 0; v < 5; ++v) X[v] = c1 * (dA[v] + W6[v]) + c2 * W6[v];
      add_right(e, a, left_proj(e, a, X), Wl);
    }
  }
}

}  // namespace orc
