// ORACLE — test infrastructure only (see real.hpp).
//
// Riemann solvers of Sec. 2: exact (Toro 2009 ch. 4), HLLE (Einfeldt 1991),
// HLLC (Toro 2009 ch. 10) and Roe (Roe 1981; 3D wave strengths per Toro 2009
// ch. 11), with the Roe failure fallback of Sec. 2: where the linearised
// solution has a non-positive density or pressure in an intermediate state,
// the face flux is recomputed with HLLE, HLLC or the exact solver.
//
// All solvers work in the local frame (normal component first) on conserved
// states; primitives are recovered with the floors of Gas.  Ties in the
// upwind choice (a wave speed exactly 0) take the left-hand state.
#pragma once
#include "euler.hpp"

namespace orc {

enum Riemann { RS_EXACT = 0, RS_HLLE = 1, RS_HLLC = 2, RS_ROE = 3 };

// Status bits (per group, OR-ed).
enum Status : unsigned {
  ST_ROE_FALLBACK = 1u,   // informational: Roe failed somewhere, fallback used
  ST_NEG_DENS = 2u,       // updated density <= 0
  ST_NEG_PRES = 4u,       // updated pressure <= 0
  ST_NAN = 8u,            // NaN in the updated state
  ST_EXACT_FAIL = 16u,    // exact solver: vacuum generated or no convergence
};

// Primitive state and derived quantities of one side of a face.
template <class R> struct Side {
  R U[5];   // local conserved
  R W[5];   // local primitive (floored)
  R E;      // total energy used in the physical flux (= U[4])
  R c;      // sound speed
  R F[5];   // physical flux
};

template <class R> inline void make_side(const R U[5], const Gas<R>& gas, Side<R>& s) {
  for (int v = 0; v < 5; ++v) s.U[v] = U[v];
  prim_from_cons(U, s.W, gas);  // the rotation does not change the formulas
  s.E = U[4];
  s.c = sound_speed(s.W[0], s.W[4], gas);
  phys_flux_local(s.W, s.E, s.F);
}

// Roe averages (sqrt(rho) weights): velocity, enthalpy H = (E + p)/rho, and
// the averaged sound speed squared a2 = (gamma - 1)(H - |u|^2/2).
template <class R> struct RoeAvg {
  R u, v, w, H, q2, a2;
};

template <class R> inline void roe_average(const Side<R>& L, const Side<R>& Rs, const Gas<R>& gas, RoeAvg<R>& A) {
  R sL = sqrt(L.W[0]);
  R sR = sqrt(Rs.W[0]);
  R inv = R(1.0) / (sL + sR);
  A.u = (sL * L.W[1] + sR * Rs.W[1]) * inv;
  A.v = (sL * L.W[2] + sR * Rs.W[2]) * inv;
  A.w = (sL * L.W[3] + sR * Rs.W[3]) * inv;
  R HL = (L.E + L.W[4]) / L.W[0];
  R HR = (Rs.E + Rs.W[4]) / Rs.W[0];
  A.H = (sL * HL + sR * HR) * inv;
  A.q2 = A.u * A.u + A.v * A.v + A.w * A.w;
  A.a2 = (gas.gamma - R(1.0)) * (A.H - R(0.5) * A.q2);
}

// HLLE with Einfeldt's wave-speed estimates
//   SL = min(uL - cL, u~ - a~),  SR = max(uR + cR, u~ + a~),
//   F = (b+ FL - b- FR + b+ b- (UR - UL)) / (b+ - b-),  b+ = max(SR,0), b- = min(SL,0).
template <class R> inline void hlle_flux(const Side<R>& L, const Side<R>& Rs, const Gas<R>& gas, R F[5]) {
  RoeAvg<R> A;
  roe_average(L, Rs, gas, A);
  R a = A.a2 > R(0.0) ? sqrt(A.a2) : R(0.0);
  R SL = L.W[1] - L.c;
  R t = A.u - a;
  if (t < SL) SL = t;
  R SR = Rs.W[1] + Rs.c;
  t = A.u + a;
  if (t > SR) SR = t;
  R bp = SR > R(0.0) ? SR : R(0.0);
  R bm = SL < R(0.0) ? SL : R(0.0);
  R inv = R(1.0) / (bp - bm);
  for (int v = 0; v < 5; ++v)
    F[v] = (bp * L.F[v] - bm * Rs.F[v] + bp * bm * (Rs.U[v] - L.U[v])) * inv;
}

// HLLC (Toro 2009 ch. 10) with the same Einfeldt speeds SL, SR as HLLE and the
// contact speed
//   S* = (pR - pL + rhoL uL (SL - uL) - rhoR uR (SR - uR))
//        / (rhoL (SL - uL) - rhoR (SR - uR)),
// star states U*K = rhoK (SK - uK)/(SK - S*) (1, S*, vK, wK,
//   EK/rhoK + (S* - uK)(S* + pK/(rhoK (SK - uK)))),  F*K = FK + SK (U*K - UK).
template <class R> inline void hllc_flux(const Side<R>& L, const Side<R>& Rs, const Gas<R>& gas, R F[5]) {
  RoeAvg<R> A;
  roe_average(L, Rs, gas, A);
  R a = A.a2 > R(0.0) ? sqrt(A.a2) : R(0.0);
  R SL = L.W[1] - L.c;
  R t = A.u - a;
  if (t < SL) SL = t;
  R SR = Rs.W[1] + Rs.c;
  t = A.u + a;
  if (t > SR) SR = t;
  R mL = L.W[0] * (SL - L.W[1]);   // rhoL (SL - uL)
  R mR = Rs.W[0] * (SR - Rs.W[1]); // rhoR (SR - uR)
  R Ss = (Rs.W[4] - L.W[4] + mL * L.W[1] - mR * Rs.W[1]) / (mL - mR);
  if (SL >= R(0.0)) {
    for (int v = 0; v < 5; ++v) F[v] = L.F[v];
  } else if (Ss >= R(0.0)) {
    R f = mL / (SL - Ss);
    R Us[5];
    Us[0] = f;
    Us[1] = f * Ss;
    Us[2] = f * L.W[2];
    Us[3] = f * L.W[3];
    Us[4] = f * (L.E / L.W[0] + (Ss - L.W[1]) * (Ss + L.W[4] / mL));
    for (int v = 0; v < 5; ++v) F[v] = L.F[v] + SL * (Us[v] - L.U[v]);
  } else if (SR > R(0.0)) {
    R f = mR / (SR - Ss);
    R Us[5];
    Us[0] = f;
    Us[1] = f * Ss;
    Us[2] = f * Rs.W[2];
    Us[3] = f * Rs.W[3];
    Us[4] = f * (Rs.E / Rs.W[0] + (Ss - Rs.W[1]) * (Ss + Rs.W[4] / mR));
    for (int v = 0; v < 5; ++v) F[v] = Rs.F[v] + SR * (Us[v] - Rs.U[v]);
  } else {
    for (int v = 0; v < 5; ++v) F[v] = Rs.F[v];
  }
}

// ---------------------------------------------------------------------------
// Exact solver (Toro 2009 ch. 4): Newton iteration for p* on
//   f(p) = fL(p) + fR(p) + (uR - uL) = 0,
//   fK(p) = (p - pK) sqrt(AK / (p + BK))                    p > pK (shock)
//         = 2 cK/(gamma-1) ((p/pK)^((gamma-1)/(2 gamma)) - 1)  p <= pK (rarefaction)
//   AK = 2/((gamma+1) rhoK), BK = (gamma-1)/(gamma+1) pK,
// from the primitive-variable (PVRS) guess, then sampling at x/t = 0.
// ---------------------------------------------------------------------------
template <class R> struct ExactResult {
  R pstar, ustar;
  int iters;
  bool ok;
};

template <class R> inline void exact_fK(R p, R rhoK, R pK, R cK, const Gas<R>& gas, R* f, R* df) {
  R g = gas.gamma;
  if (p > pK) {
    R A = R(2.0) / ((g + R(1.0)) * rhoK);
    R B = (g - R(1.0)) / (g + R(1.0)) * pK;
    R q = sqrt(A / (p + B));
    *f = (p - pK) * q;
    *df = q * (R(1.0) - (p - pK) / (R(2.0) * (B + p)));
  } else {
    R pr = p / pK;
    *f = R(2.0) * cK / (g - R(1.0)) * (pow(pr, (g - R(1.0)) / (R(2.0) * g)) - R(1.0));
    *df = R(1.0) / (rhoK * cK) * pow(pr, -(g + R(1.0)) / (R(2.0) * g));
  }
}

// Tolerance on the relative change 2|p_new - p|/(p_new + p) and iteration cap.
static const double EXACT_TOL = 1.0e-14;
static const int EXACT_MAXIT = 64;

template <class R>
inline ExactResult<R> exact_star(const R WL[5], R cL, const R WR[5], R cR, const Gas<R>& gas) {
  ExactResult<R> res;
  res.iters = 0;
  res.ok = true;
  R g = gas.gamma;
  R du = WR[1] - WL[1];
  // vacuum generated: the two rarefactions cannot meet
  if (R(2.0) / (g - R(1.0)) * (cL + cR) <= du) {
    res.ok = false;
    res.pstar = R(0.0);
    res.ustar = R(0.5) * (WL[1] + WR[1]);
    return res;
  }
  R ppv = R(0.5) * (WL[4] + WR[4]) - R(0.125) * du * (WL[0] + WR[0]) * (cL + cR);
  R pmin = R(1.0e-8) * R(0.5) * (WL[4] + WR[4]);  // guess floor, relative to the mean pressure
  R p = ppv > pmin ? ppv : pmin;
  bool conv = false;
  for (int it = 0; it < EXACT_MAXIT; ++it) {
    R fL, dfL, fR, dfR;
    exact_fK(p, WL[0], WL[4], cL, gas, &fL, &dfL);
    exact_fK(p, WR[0], WR[4], cR, gas, &fR, &dfR);
    R pn = p - (fL + fR + du) / (dfL + dfR);
    if (pn < pmin) pn = pmin;
    R change = R(2.0) * fabs(pn - p) / (pn + p);
    p = pn;
    res.iters = it + 1;
    if (change < R(EXACT_TOL)) {
      conv = true;
      break;
    }
  }
  R fL, dfL, fR, dfR;
  exact_fK(p, WL[0], WL[4], cL, gas, &fL, &dfL);
  exact_fK(p, WR[0], WR[4], cR, gas, &fR, &dfR);
  res.pstar = p;
  res.ustar = R(0.5) * (WL[1] + WR[1]) + R(0.5) * (fR - fL);
  res.ok = conv;
  return res;
}

// Sample the exact self-similar solution at x/t = S (Toro 2009 sec. 4.5); the
// face flux uses S = 0.  W local.  A point exactly on a wave takes the state
// on its left.
template <class R>
inline void exact_sample(const R WL[5], R cL, const R WR[5], R cR, R ps, R us, R S, const Gas<R>& gas, R W[5]) {
  R g = gas.gamma;
  R g5 = R(2.0) / (g + R(1.0));
  R g6 = (g - R(1.0)) / (g + R(1.0));
  R g7 = R(0.5) * (g - R(1.0));
  if (S <= us) {  // left of the contact
    W[2] = WL[2];
    W[3] = WL[3];
    if (ps > WL[4]) {  // left shock
      R pr = ps / WL[4];
      R SL = WL[1] - cL * sqrt((g + R(1.0)) / (R(2.0) * g) * pr + (g - R(1.0)) / (R(2.0) * g));
      if (S <= SL) {
        W[0] = WL[0]; W[1] = WL[1]; W[4] = WL[4];
      } else {
        W[0] = WL[0] * (pr + g6) / (g6 * pr + R(1.0)); W[1] = us; W[4] = ps;
      }
    } else {  // left rarefaction
      R SHL = WL[1] - cL;
      if (S <= SHL) {
        W[0] = WL[0]; W[1] = WL[1]; W[4] = WL[4];
      } else {
        R pr = ps / WL[4];
        R STL = us - cL * pow(pr, (g - R(1.0)) / (R(2.0) * g));
        if (S > STL) {
          W[0] = WL[0] * pow(pr, R(1.0) / g); W[1] = us; W[4] = ps;
        } else {  // inside the fan
          R c = g5 * (cL + g7 * (WL[1] - S));
          W[1] = g5 * (cL + g7 * WL[1] + S);
          W[0] = WL[0] * pow(c / cL, R(2.0) / (g - R(1.0)));
          W[4] = WL[4] * pow(c / cL, R(2.0) * g / (g - R(1.0)));
        }
      }
    }
  } else {  // right of the contact
    W[2] = WR[2];
    W[3] = WR[3];
    if (ps > WR[4]) {  // right shock
      R pr = ps / WR[4];
      R SR = WR[1] + cR * sqrt((g + R(1.0)) / (R(2.0) * g) * pr + (g - R(1.0)) / (R(2.0) * g));
      if (S >= SR) {
        W[0] = WR[0]; W[1] = WR[1]; W[4] = WR[4];
      } else {
        W[0] = WR[0] * (pr + g6) / (g6 * pr + R(1.0)); W[1] = us; W[4] = ps;
      }
    } else {  // right rarefaction
      R SHR = WR[1] + cR;
      if (S >= SHR) {
        W[0] = WR[0]; W[1] = WR[1]; W[4] = WR[4];
      } else {
        R pr = ps / WR[4];
        R STR = us + cR * pow(pr, (g - R(1.0)) / (R(2.0) * g));
        if (S < STR) {
          W[0] = WR[0] * pow(pr, R(1.0) / g); W[1] = us; W[4] = ps;
        } else {  // inside the fan
          R c = g5 * (cR - g7 * (WR[1] - S));
          W[1] = g5 * (-cR + g7 * WR[1] + S);
          W[0] = WR[0] * pow(c / cR, R(2.0) / (g - R(1.0)));
          W[4] = WR[4] * pow(c / cR, R(2.0) * g / (g - R(1.0)));
        }
      }
    }
  }
}

template <class R>
inline void exact_flux(const Side<R>& L, const Side<R>& Rs, const Gas<R>& gas, R F[5], unsigned* status) {
  ExactResult<R> r = exact_star(L.W, L.c, Rs.W, Rs.c, gas);
  if (!r.ok) {
    *status |= ST_EXACT_FAIL;
    if (r.pstar <= R(0.0)) {  // vacuum: no star state to sample
      hlle_flux(L, Rs, gas, F);
      return;
    }
  }
  R W[5];
  exact_sample(L.W, L.c, Rs.W, Rs.c, r.pstar, r.ustar, R(0.0), gas, W);
  R E = energy_local(W, gas);
  phys_flux_local(W, E, F);
}

// ---------------------------------------------------------------------------
// Roe (1981) with the 3D wave strengths of Toro 2009 sec. 11.3:
//   a3 = dU2 - v~ dU0,  a4 = dU3 - w~ dU0,   (dU = UR - UL, local frame)
//   dU4' = dU4 - a3 v~ - a4 w~,
//   a2 = (gamma-1)/a~^2 (dU0 (H~ - u~^2) + u~ dU1 - dU4'),
//   a1 = (dU0 (u~ + a~) - dU1 - a~ a2) / (2 a~),  a5 = dU0 - (a1 + a2),
// (wave order: a1 for u~-a~, a2 entropy, a3/a4 shear, a5 for u~+a~)
//   K1 = (1, u~-a~, v~, w~, H~-u~a~)   K2 = (1, u~, v~, w~, q~^2/2)
//   K3 = (0, 0, 1, 0, v~)              K4 = (0, 0, 0, 1, w~)
//   K5 = (1, u~+a~, v~, w~, H~+u~a~)
//   F = (FL + FR)/2 - 1/2 sum_k |lambda_k| a_k K_k.
// Failure: a~^2 <= 0, or density or pressure <= 0 in either intermediate state
//   U*1 = UL + a1 K1,  U*2 = U*1 + a2 K2 + a3 K3 + a4 K4.
// Returns false on failure (F is then not set).
// ---------------------------------------------------------------------------
template <class R> inline bool roe_flux(const Side<R>& L, const Side<R>& Rs, const Gas<R>& gas, R F[5]) {
  RoeAvg<R> A;
  roe_average(L, Rs, gas, A);
  if (!(A.a2 > R(0.0))) return false;
  R a = sqrt(A.a2);
  R d[5];
  for (int v = 0; v < 5; ++v) d[v] = Rs.U[v] - L.U[v];
  R a3 = d[2] - A.v * d[0];
  R a4 = d[3] - A.w * d[0];
  R d4 = d[4] - a3 * A.v - a4 * A.w;
  R a2 = (gas.gamma - R(1.0)) / A.a2 * (d[0] * (A.H - A.u * A.u) + A.u * d[1] - d4);
  R a1 = (d[0] * (A.u + a) - d[1] - a * a2) / (R(2.0) * a);
  R a5 = d[0] - (a1 + a2);
  R K1_1 = A.u - a, K1_4 = A.H - A.u * a;   // the non-trivial entries of K1
  R K5_1 = A.u + a, K5_4 = A.H + A.u * a;   // ... and of K5
  R K2_4 = R(0.5) * A.q2;
  // intermediate states U*1 = UL + a1 K1 and U*2 = U*1 + a2 K2 + a3 K3 + a4 K4
  R s1[5], s2[5];
  s1[0] = L.U[0] + a1;
  s1[1] = L.U[1] + a1 * K1_1;
  s1[2] = L.U[2] + a1 * A.v;
  s1[3] = L.U[3] + a1 * A.w;
  s1[4] = L.U[4] + a1 * K1_4;
  s2[0] = s1[0] + a2;
  s2[1] = s1[1] + a2 * A.u;
  s2[2] = s1[2] + a2 * A.v + a3;
  s2[3] = s1[3] + a2 * A.w + a4;
  s2[4] = s1[4] + a2 * K2_4 + a3 * A.v + a4 * A.w;
  const R* st[2] = {s1, s2};
  for (int k = 0; k < 2; ++k) {
    const R* s = st[k];
    if (!(s[0] > R(0.0))) return false;
    R p = (gas.gamma - R(1.0)) * (s[4] - R(0.5) * (s[1] * s[1] + s[2] * s[2] + s[3] * s[3]) / s[0]);
    if (!(p > R(0.0))) return false;
  }
  // |lambda_k| a_k, lambda = (u~ - a~, u~, u~, u~, u~ + a~)
  R c1 = fabs(A.u - a) * a1;
  R c2 = fabs(A.u) * a2;
  R c3 = fabs(A.u) * a3;
  R c4 = fabs(A.u) * a4;
  R c5 = fabs(A.u + a) * a5;
  R diss[5];
  diss[0] = c1 + c2 + c5;
  diss[1] = c1 * K1_1 + c2 * A.u + c5 * K5_1;
  diss[2] = c1 * A.v + c2 * A.v + c3 + c5 * A.v;
  diss[3] = c1 * A.w + c2 * A.w + c4 + c5 * A.w;
  diss[4] = c1 * K1_4 + c2 * K2_4 + c3 * A.v + c4 * A.w + c5 * K5_4;
  for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (L.F[v] + Rs.F[v]) - R(0.5) * diss[v];
  return true;
}

// Riemann solve at one face along direction d, global-frame conserved states.
// solver: RS_*; fallback: solver used where Roe fails (RS_HLLE/RS_HLLC/RS_EXACT).
template <class R>
inline void riemann(int solver, int fallback, int d, const R ULg[5], const R URg[5], const Gas<R>& gas, R Fg[5],
                    unsigned* status) {
  Sec<R> sec(SEC_RIEMANN);
  R ul[5], ur[5], F[5];
  to_local(ULg, ul, d);
  to_local(URg, ur, d);
  Side<R> L, Rs;
  make_side(ul, gas, L);
  make_side(ur, gas, Rs);
  int s = solver;
  if (s == RS_ROE) {
    if (roe_flux(L, Rs, gas, F)) {
      to_global(F, Fg, d);
      return;
    }
    *status |= ST_ROE_FALLBACK;
    s = fallback;
  }
  switch (s) {
    case RS_EXACT: exact_flux(L, Rs, gas, F, status); break;
    case RS_HLLC: hllc_flux(L, Rs, gas, F); break;
    default: hlle_flux(L, Rs, gas, F); break;
  }
  to_global(F, Fg, d);
}

}  // namespace orc
