// Paired FP32 numerics of the CTU group kernel (Sec. 2 steps (1)-(3)): the
// same formulas as the scalar FP32 forms (phys.cuh), evaluated for two work
// items at once with packed arithmetic (pair.cuh).  Every value is a pair
// (lane 0, lane 1) of independent items; nothing mixes the lanes.
//
// Operation order differs from the FP64 form (which follows the oracle bit
// for bit); like the scalar FP32 forms these change values only in the last
// bits of FP32:
//   * a * b + c is one fused multiply-add wherever the formula has that shape;
//   * one reciprocal per repeated denominator (rho, sqrt(rho_L) +
//     sqrt(rho_R), c), divisions by the fast intrinsic, a, (gamma-1)/a^2 and
//     1/(2a) of the Roe solver from one reciprocal square root;
//   * the Roe solver keeps F_L + F_R and U_R - U_L instead of the two sides'
//     fluxes and states, and its positivity checks compare 2 E rho with |m|^2.
// Floors keep compare-and-select, so a NaN state still reaches the status
// bits.  Where Roe's linearisation fails in a lane, that lane is recomputed
// by the scalar fallback solver (phys.cuh) from the same two states.
#pragma once
#include "pair.cuh"
#include "phys.cuh"

namespace hyd {
namespace pp {

// ------------------------------------------------------------------ EOS
// U -> W with the floors; ir = 1 / rho.
__device__ __forceinline__ void prim(const V2 U[5], V2 W[5], const Gas<float>& g, V2& ir) {
  const V2 df = sp2(g.dens_floor), pf = sp2(g.pres_floor);
  const V2 rho = sel2(lt2(U[0], df), df, U[0]);
  ir = rcp2(rho);
  V2 s = U[1] * U[1];
  s = fma2(U[2], U[2], s);
  s = fma2(U[3], U[3], s);
  const V2 kin = (s * 0.5f) * ir;
  V2 p = (U[4] - kin) * g.gm1;
  p = sel2(lt2(p, pf), pf, p);
  W[0] = rho;
  W[1] = U[1] * ir;
  W[2] = U[2] * ir;
  W[3] = U[3] * ir;
  W[4] = p;
}

// W -> U:  E = p / (gamma-1) + (rho / 2) |v|^2.
__device__ __forceinline__ void cons(const V2 W[5], V2 U[5], const Gas<float>& g) {
  V2 ke = W[1] * W[1];
  ke = fma2(W[2], W[2], ke);
  ke = fma2(W[3], W[3], ke);
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  U[4] = fma2(W[4], sp2(g.igm1), (W[0] * 0.5f) * ke);
}

// Physical flux along the local normal of primitives W with energy E.
__device__ __forceinline__ void pflux(const V2 W[5], V2 E, V2 F[5]) {
  const V2 mn = W[0] * W[1];
  F[0] = mn;
  F[1] = fma2(mn, W[1], W[4]);
  F[2] = mn * W[2];
  F[3] = mn * W[3];
  F[4] = (E + W[4]) * W[1];
}

// ------------------------------------------------------------------ Roe
// Roe (1981) flux with the 3D wave strengths (Toro 2009 sec. 11.3) in the
// local frame: F = (F_L + F_R)/2 - (1/2) sum |lambda_k| alpha_k K_k.
// Returns, per lane, whether the linearisation held (a~^2 > 0 and both
// intermediate states U_L + a1 K1 and U_L + a1 K1 + a2 K2 + a3 K3 + a4 K4
// with rho > 0 and p > 0); a failed lane's flux is meaningless.
__device__ __forceinline__ M2 roe(const V2 UL[5], const V2 UR[5], const Gas<float>& g, V2 F[5]) {
  V2 WL[5], WR[5], irL, irR, Fs[5];
  prim(UL, WL, g, irL);
  prim(UR, WR, g, irR);
  {
    V2 FL[5], FR[5];
    pflux(WL, UL[4], FL);
    pflux(WR, UR[4], FR);
#pragma unroll
    for (int k = 0; k < 5; ++k) Fs[k] = FL[k] + FR[k];
  }
  // Roe averages with sqrt(rho) weights
  const V2 sL = sqrt2(WL[0]), sR = sqrt2(WR[0]);
  const V2 inv = rcp2(sL + sR);
  const V2 u = fma2(sL, WL[1], sR * WR[1]) * inv;
  const V2 v = fma2(sL, WL[2], sR * WR[2]) * inv;
  const V2 w = fma2(sL, WL[3], sR * WR[3]) * inv;
  const V2 HL = (UL[4] + WL[4]) * irL;
  const V2 HR = (UR[4] + WR[4]) * irR;
  const V2 H = fma2(sL, HL, sR * HR) * inv;
  V2 q2 = u * u;
  q2 = fma2(v, v, q2);
  q2 = fma2(w, w, q2);
  const V2 K24 = q2 * 0.5f;
  const V2 a2 = (H - K24) * g.gm1;
  M2 ok = gt2(a2, sp2(0.0f));
  const V2 ia = rsqrt2(a2);
  const V2 a = a2 * ia;
  const V2 gma2 = (ia * ia) * g.gm1;
  const V2 i2a = ia * 0.5f;
  const V2 d0 = UR[0] - UL[0], d1 = UR[1] - UL[1], d2 = UR[2] - UL[2], d3 = UR[3] - UL[3], d4 = UR[4] - UL[4];
  const V2 a3 = d2 - v * d0;
  const V2 a4 = d3 - w * d0;
  const V2 d4b = d4 - fma2(a3, v, a4 * w);
  const V2 uu = u * u;
  const V2 al2 = (fma2(d0, H - uu, u * d1) - d4b) * gma2;
  const V2 upa = u + a;
  const V2 al1 = ((d0 * upa - d1) - a * al2) * i2a;
  const V2 al5 = d0 - (al1 + al2);
  const V2 K11 = u - a;
  const V2 ua = u * a;
  const V2 K14 = H - ua;
  const V2 K54 = H + ua;
  // intermediate states
  V2 s0 = UL[0] + al1, s1 = fma2(al1, K11, UL[1]), s2 = fma2(al1, v, UL[2]), s3 = fma2(al1, w, UL[3]),
     s4 = fma2(al1, K14, UL[4]);
  const V2 zero = sp2(0.0f);
  {
    V2 m2 = s1 * s1;
    m2 = fma2(s2, s2, m2);
    m2 = fma2(s3, s3, m2);
    ok = and2(ok, and2(gt2(s0, zero), gt2((s4 + s4) * s0, m2)));
  }
  s0 = s0 + al2;
  s1 = fma2(al2, u, s1);
  s2 = fma2(al2, v, s2) + a3;
  s3 = fma2(al2, w, s3) + a4;
  s4 = fma2(al2, K24, s4) + fma2(a3, v, a4 * w);
  {
    V2 m2 = s1 * s1;
    m2 = fma2(s2, s2, m2);
    m2 = fma2(s3, s3, m2);
    ok = and2(ok, and2(gt2(s0, zero), gt2((s4 + s4) * s0, m2)));
  }
  const V2 au = abs2(u);
  const V2 c1 = abs2(K11) * al1;
  const V2 c2 = au * al2;
  const V2 c3 = au * a3;
  const V2 c4 = au * a4;
  const V2 c5 = abs2(upa) * al5;
  const V2 D0 = (c1 + c2) + c5;
  const V2 D1 = fma2(c1, K11, fma2(c2, u, c5 * upa));
  const V2 D2 = fma2(D0, v, c3);
  const V2 D3 = fma2(D0, w, c4);
  const V2 D4 = fma2(c1, K14, fma2(c2, K24, fma2(c3, v, fma2(c4, w, c5 * K54))));
  F[0] = (Fs[0] - D0) * 0.5f;
  F[1] = (Fs[1] - D1) * 0.5f;
  F[2] = (Fs[2] - D2) * 0.5f;
  F[3] = (Fs[3] - D3) * 0.5f;
  F[4] = (Fs[4] - D4) * 0.5f;
  return ok;
}

// Fallback of one lane where Roe's linearisation failed: the flux of the
// fallback solver (HLLE, HLLC or exact; scalar forms of phys.cuh) and the
// status bits.  Out of line: it is rare, and inlined it would hold registers
// across the packed path.
static __device__ __noinline__ Flux5<float> roe_fallback_lane(V5<float> ul, V5<float> ur, Gas<float> g, int fallback) {
  Side<float> L, R;
  mkside<float, false>(ul.v, g, L);
  mkside<float, false>(ur.v, g, R);
  Flux5<float> out;
  out.st = ST_ROE_FALLBACK;
  if (fallback == RS_HLLC)
    hllc(L, R, g, out.F);
  else if (fallback == RS_EXACT)
    out.st |= exact_call(L, R, g, out.F);
  else
    hlle(L, R, g, out.F);
  return out;
}

// One lane through a non-Roe solver (scalar forms of phys.cuh).
template <int RS>
__device__ __noinline__ Flux5<float> solve_lane(V5<float> ul, V5<float> ur, Opts<float> o) {
  Flux5<float> out;
  out.st = riemann_local<float, false, RS>(ul.v, ur.v, o, out.F);
  return out;
}

// Riemann flux of both lanes in the local frame; returns the status bits of
// each lane in st[2].  Roe runs packed; where its linearisation fails in a
// lane, that lane takes the fallback solver on the same two states.  The
// other solvers run lane by lane.
template <int RS>
__device__ __forceinline__ void riemann(const V2 UL[5], const V2 UR[5], const Opts<float>& o, V2 F[5],
                                        unsigned st[2]) {
  st[0] = st[1] = 0;
  M2 ok{false, false};
  if (RS == RS_ROE) ok = roe(UL, UR, o.gas, F);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const bool done = l ? ok.y : ok.x;
    if (!done) {
      V5<float> ul, ur;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        ul.v[k] = lane_of(UL[k], l);
        ur.v[k] = lane_of(UR[k], l);
      }
      const Flux5<float> r = RS == RS_ROE ? roe_fallback_lane(ul, ur, o.gas, o.fallback) : solve_lane<RS>(ul, ur, o);
      st[l] = r.st;
#pragma unroll
      for (int k = 0; k < 5; ++k) F[k] = l ? mk2(F[k].v.x, r.F[k]) : mk2(r.F[k], F[k].v.y);
    }
  }
}

// ------------------------------------------------------- reconstruction
// Limited slope of both lanes (generalized minmod with theta = 1 packed;
// the other limiters lane by lane with the scalar form).
template <int LIM>
__device__ __forceinline__ V2 slope(const Opts<float>& o, V2 dL, V2 dR) {
  if constexpr (LIM == LIM_MINMOD1) {
    const V2 r = copysign2(min2(abs2(dL), abs2(dR)), dL);
    return sel2(gt2(dL * dR, sp2(0.0f)), r, sp2(0.0f));
  } else {
    return mk2(hyd::slope<LIM>(o.limiter, o.theta, dL.v.x, dR.v.x),
               hyd::slope<LIM>(o.limiter, o.theta, dL.v.y, dR.v.y));
  }
}

// PPM (Colella & Woodward 1984) face values from a 5-point stencil, then the
// monotonicity constraints (local extremum -> flat, overshoot -> move one
// edge):  L = (w_-1 + w_0)/2 + (d_-1 - d_0)/6,  R = (w_0 + w_1)/2 + (d_0 - d_1)/6.
template <int LIM>
__device__ __forceinline__ void ppm(V2 wmm, V2 wm, V2 w0, V2 wp, V2 wpp, const Opts<float>& o, V2& wL, V2& wR) {
  const V2 D1 = wm - wmm, D2 = w0 - wm, D3 = wp - w0, D4 = wpp - wp;
  const V2 dm = slope<LIM>(o, D1, D2);
  const V2 d0 = slope<LIM>(o, D2, D3);
  const V2 dp = slope<LIM>(o, D3, D4);
  const V2 sixth = sp2(1.0f / 6.0f);
  const V2 L = fma2(dm - d0, sixth, (wm + w0) * 0.5f);
  const V2 R = fma2(d0 - dp, sixth, (w0 + wp) * 0.5f);
  const V2 zero = sp2(0.0f);
  const M2 ext = le2((R - w0) * (w0 - L), zero);
  const V2 dA = R - L;
  const V2 a6 = fma2(L + R, sp2(-3.0f), w0 * 6.0f);
  const V2 dAa6 = dA * a6, dA2 = dA * dA;
  const M2 c1 = gt2(dAa6, dA2);
  const M2 c2 = and2(not2(c1), gt2(-dA2, dAa6));
  const V2 w03 = w0 * 3.0f;
  const V2 Ln = sel2(c1, fma2(R, sp2(-2.0f), w03), L);
  const V2 Rn = sel2(c2, fma2(L, sp2(-2.0f), w03), R);
  wL = sel2(ext, w0, Ln);
  wR = sel2(ext, w0, Rn);
}

// ------------------------------------------------------ CTU tracing
// Primitive eigen-system along the local normal (see Eig in phys.cuh).
struct Eig2 {
  V2 lm, lu, lp;  // u - c, u, u + c
  V2 r2c, cc, cor, hicc, icc;
};
__device__ __forceinline__ void eig(const V2 W[5], const Gas<float>& g, Eig2& e) {
  const V2 ir = rcp2(W[0]);
  const V2 c = sqrt2((W[4] * g.gamma) * ir);
  const V2 ic = rcp2(c);
  e.lm = W[1] - c;
  e.lu = W[1];
  e.lp = W[1] + c;
  e.r2c = (W[0] * 0.5f) * ic;
  e.cc = c * c;
  e.cor = c * ir;
  e.icc = ic * ic;
  e.hicc = e.icc * 0.5f;
}

// Wave a's coefficient into the two traced states: Y += coef r_a, with
// coef zeroed for the side the wave does not reach.
__device__ __forceinline__ void radd2(const Eig2& e, int a, V2 cr, V2 cl, V2 Wr[5], V2 Wl[5]) {
  if (a == 0 || a == 4) {
    const V2 cor = a == 0 ? -e.cor : e.cor;
    Wr[0] = Wr[0] + cr;
    Wr[1] = fma2(cr, cor, Wr[1]);
    Wr[4] = fma2(cr, e.cc, Wr[4]);
    Wl[0] = Wl[0] + cl;
    Wl[1] = fma2(cl, cor, Wl[1]);
    Wl[4] = fma2(cl, e.cc, Wl[4]);
  } else {
    const int k = a == 1 ? 0 : a;  // r_2 = e_0, r_3 = e_2, r_4 = e_3
    Wr[k] = Wr[k] + cr;
    Wl[k] = Wl[k] + cl;
  }
}

// PPM tracing, reference-state form (phys.cuh trace_ppm): the parabola
// averaged over each wave's domain of dependence.
__device__ __forceinline__ void trace_ppm(const V2 W0[5], const V2 WL[5], const V2 WR[5], V2 dtdx,
                                          const Gas<float>& g, V2 Wl[5], V2 Wr[5]) {
  Eig2 e;
  eig(W0, g, e);
  const V2 zero = sp2(0.0f);
  const V2 lamM = max2(e.lp, zero), lamm = min2(e.lm, zero);
  V2 dA[5], W6[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dA[v] = WR[v] - WL[v];
    W6[v] = fma2(WL[v] + WR[v], sp2(-3.0f), W0[v] * 6.0f);
  }
  const V2 sM = lamM * dtdx, sm = lamm * dtdx;
  const V2 nqr = sM * -0.5f, nqr2 = fma2(sM, sp2(2.0f / 3.0f), sp2(-1.0f));
  const V2 nql = sm * -0.5f, ql2 = fma2(sm, sp2(2.0f / 3.0f), sp2(1.0f));
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Wr[v] = fma2(nqr, fma2(nqr2, W6[v], dA[v]), WR[v]);
    Wl[v] = fma2(nql, fma2(ql2, W6[v], dA[v]), WL[v]);
  }
  const V2 hdt = dtdx * 0.5f;
  const V2 tdt = (dtdx * dtdx) * (1.0f / 3.0f);
  // waves: 0 (u - c), 1..3 (u, shared coefficients), 4 (u + c)
#pragma unroll
  for (int wv = 0; wv < 3; ++wv) {
    const V2 la = wv == 0 ? e.lm : (wv == 1 ? e.lu : e.lp);
    const M2 pos = gt2(la, zero), neg = lt2(la, zero);
    const V2 lref = sel2(pos, lamM, lamm);
    const V2 dl = lref - la;
    const V2 c1 = hdt * dl;
    const V2 c2 = (tdt * dl) * (lref + la);
    const V2 k = sel2(pos, c2 - c1, c2 + c1);
    if (wv == 1) {
      // l_2 . X = X0 - X4 / c^2; l_3 . X = X2; l_4 . X = X3
      const V2 X0 = fma2(k, W6[0], c1 * dA[0]);
      const V2 X2 = fma2(k, W6[2], c1 * dA[2]);
      const V2 X3 = fma2(k, W6[3], c1 * dA[3]);
      const V2 X4 = fma2(k, W6[4], c1 * dA[4]);
      const V2 co[3] = {fma2(-X4, e.icc, X0), X2, X3};
#pragma unroll
      for (int a = 1; a <= 3; ++a) radd2(e, a, sel2(pos, co[a - 1], zero), sel2(neg, co[a - 1], zero), Wr, Wl);
    } else {
      const V2 X1 = fma2(k, W6[1], c1 * dA[1]);
      const V2 X4 = fma2(k, W6[4], c1 * dA[4]);
      const V2 r2c = wv == 0 ? -e.r2c : e.r2c;
      const V2 coef = fma2(r2c, X1, X4 * e.hicc);
      radd2(e, wv == 0 ? 0 : 4, sel2(pos, coef, zero), sel2(neg, coef, zero), Wr, Wl);
    }
  }
}

// PLM tracing, reference-state form (phys.cuh trace_plm).
__device__ __forceinline__ void trace_plm(const V2 W0[5], const V2 dW[5], V2 dtdx, const Gas<float>& g, V2 Wl[5],
                                          V2 Wr[5]) {
  Eig2 e;
  eig(W0, g, e);
  const V2 zero = sp2(0.0f);
  const V2 lamM = max2(e.lp, zero), lamm = min2(e.lm, zero);
  const V2 fr = fma2(lamM * dtdx, sp2(-0.5f), sp2(0.5f));
  const V2 nfl = fma2(lamm * dtdx, sp2(-0.5f), sp2(-0.5f));
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    Wr[v] = fma2(fr, dW[v], W0[v]);
    Wl[v] = fma2(nfl, dW[v], W0[v]);
  }
  const V2 hdt = dtdx * 0.5f;
#pragma unroll
  for (int wv = 0; wv < 3; ++wv) {
    const V2 la = wv == 0 ? e.lm : (wv == 1 ? e.lu : e.lp);
    const M2 pos = gt2(la, zero), neg = lt2(la, zero);
    const V2 c = hdt * (sel2(pos, lamM, lamm) - la);
    if (wv == 1) {
      const V2 co[3] = {c * fma2(-dW[4], e.icc, dW[0]), c * dW[2], c * dW[3]};
#pragma unroll
      for (int a = 1; a <= 3; ++a) radd2(e, a, sel2(pos, co[a - 1], zero), sel2(neg, co[a - 1], zero), Wr, Wl);
    } else {
      const V2 r2c = wv == 0 ? -e.r2c : e.r2c;
      const V2 coef = c * fma2(r2c, dW[1], dW[4] * e.hicc);
      radd2(e, wv == 0 ? 0 : 4, sel2(pos, coef, zero), sel2(neg, coef, zero), Wr, Wl);
    }
  }
}

}  // namespace pp
}  // namespace hyd
