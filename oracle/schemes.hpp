// ORACLE — test infrastructure only (see real.hpp).
//
// One time step of one patch group (Sec. 3.1: 2x2x2 patches of 8^3 cells, i.e.
// N^3 interior cells plus g ghost layers) with the three directionally
// unsplit schemes of Sec. 2:
//   MHM  - MUSCL-Hancock: reconstruct, advance all six face values by dt/2
//          with the physical fluxes of the face values in all three
//          directions (no Riemann solver), 3 Riemann solves, update.
//   VL   - van Leer variant (Falle 1991): first-order Riemann fluxes on the
//          cell-centred data, unsplit dt/2 update, reconstruct that half-step
//          state, 3 Riemann solves, update from U^n.  6 solves per cell.
//   CTU  - simplified 6-solve corner transport upwind (Gardiner & Stone 2008):
//          (1) reconstruct + characteristic tracing to dt/2, (2) Riemann,
//          (3) transverse flux-gradient correction of the face states, then
//          Riemann again, (4) conservative update, (5) store the fluxes on the
//          group boundary.
// Written as plain loops over whole 3D arrays of the padded group, each stage
// on the index range the next stage needs, in the order of Sec. 2.
//
// Layout (Sec. 3.1): [var][z][y][x], x fastest.  Input U_in: [5][M][M][M] with
// M = N + 2g; output U_out: [5][N][N][N]; boundary flux: [6][5][N][N] with
// faces (-x, +x, -y, +y, -z, +z), the two transverse coordinates in
// [z][y][x] order with the normal one removed, fluxes time-centred (not
// multiplied by dt), positive along +axis.
#pragma once
#include <array>
#include <vector>
#include "reconstruct.hpp"
#include "riemann.hpp"

namespace orc {

enum Scheme { SCH_MHM = 0, SCH_VL = 1, SCH_CTU = 2, SCH_RTVD = 3, SCH_WAF = 4 };
enum Recon { REC_PLM = 0, REC_PPM = 1 };

template <class R> struct Params {
  int scheme, recon, limiter, riemann, fallback;
  R theta;
  Gas<R> gas;
  R dt;
  R dx[3];
  int characteristic = 0;  // reconstruct characteristic (1) or primitive (0) variables
  int split_order = 0;     // split schemes: sweeps x, y, z (0) or z, y, x (1)
};

inline int recon_stencil(int recon) { return recon == REC_PPM ? 2 : 1; }

// Ghost layers a scheme needs: face states are required for the cells -1..N
// along the normal; CTU also needs the stage-1 fluxes of the cells -1..N in
// the lateral directions, which the same width provides.  VL reconstructs its
// half-step state, which itself needs one more layer.  The split schemes need
// their 1D stencil: RTVD 3 (first-order half step, then limited fluxes of
// the half-step state), WAF 2 (the limiter reads the neighbouring fans).
inline int required_ghost(int scheme, int recon) {
  if (scheme == SCH_RTVD) return 3;
  if (scheme == SCH_WAF) return 2;
  int s = recon_stencil(recon);
  return scheme == SCH_VL ? s + 2 : s + 1;
}

struct Box {
  int N, g, M;
  long M2, M3;
  long st[3];
  Box(int N_, int g_) : N(N_), g(g_), M(N_ + 2 * g_) {
    M2 = (long)M * M;
    M3 = M2 * M;
    st[0] = 1;
    st[1] = M;
    st[2] = M2;
  }
  // padded linear index of the cell with interior coordinates (x, y, z)
  long at(int x, int y, int z) const { return ((long)(z + g) * M + (y + g)) * M + (x + g); }
};

// Visit the cells with lo[a] <= coordinate a <= hi[a] (interior coordinates).
template <class F> inline void for_box(const int lo[3], const int hi[3], F f) {
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) f(x, y, z);
}

// Range helper: along direction d from a to b, the other two from c to e.
inline void range(int d, int a, int b, int c, int e, int lo[3], int hi[3]) {
  for (int k = 0; k < 3; ++k) {
    lo[k] = (k == d) ? a : c;
    hi[k] = (k == d) ? b : e;
  }
}

template <class R> struct Field5 {
  std::vector<R> a;
  long M3;
  explicit Field5(long m3) : a(5 * m3), M3(m3) {}
  R& operator()(int v, long i) { return a[v * M3 + i]; }
  const R& operator()(int v, long i) const { return a[v * M3 + i]; }
  void get(long i, R out[5]) const { for (int v = 0; v < 5; ++v) out[v] = a[v * M3 + i]; }
  void set(long i, const R in[5]) { for (int v = 0; v < 5; ++v) a[v * M3 + i] = in[v]; }
};

// Face values (global-frame primitives) of cell i along d from the primitive
// field W.  For PLM also returns the limited slopes.
//
// Sec. 2 lets the reconstruction act on primitive or on characteristic
// variables.  Characteristic form (P.characteristic), in the frame of d:
// every stencil value W_j is projected on the left eigenvectors of the
// primitive Jacobian at cell i, alpha_a(j) = l_a(W_i) . W_j; each of the 5
// fields alpha_a goes through the same scalar PLM / PPM with the same
// limiter; the face values (and PLM slope) come back as sum_a alpha_a r_a(W_i),
// waves added in the order 1..5 starting from zero.
template <class R>
inline void recon_cell(const Params<R>& P, const Box& B, const Field5<R>& W, long i, int d, R WLf[5], R WRf[5],
                       R slope[5]) {
  long st = B.st[d];
  if (!P.characteristic) {
    for (int v = 0; v < 5; ++v) {
      const R* w = &W.a[v * W.M3 + i];
      if (P.recon == REC_PPM)
        ppm_faces(w, st, P.limiter, P.theta, &WLf[v], &WRf[v]);
      else
        plm_faces(w, st, P.limiter, P.theta, &WLf[v], &WRf[v], &slope[v]);
    }
    return;
  }
  Sec<R> sec(SEC_RECON);
  const int S = recon_stencil(P.recon);
  R wg[5], wl[5];
  W.get(i, wg);
  to_local(wg, wl, d);
  Eigen<R> e;
  eigen_prim(wl, P.gas, e);
  R al[5][5];  // [wave][stencil offset + 2]
  for (int j = -S; j <= S; ++j) {
    W.get(i + j * st, wg);
    to_local(wg, wl, d);
    for (int a = 0; a < 5; ++a) al[a][j + 2] = left_proj(e, a, wl);
  }
  R aL[5], aR[5], ad[5];
  for (int a = 0; a < 5; ++a) {
    if (P.recon == REC_PPM) {
      ppm_faces(&al[a][2], 1, P.limiter, P.theta, &aL[a], &aR[a]);
      ad[a] = R(0.0);
    } else {
      plm_faces(&al[a][2], 1, P.limiter, P.theta, &aL[a], &aR[a], &ad[a]);
    }
  }
  R fl[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  R fr[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  R sl[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
  for (int a = 0; a < 5; ++a) {
    add_right(e, a, aL[a], fl);
    add_right(e, a, aR[a], fr);
    add_right(e, a, ad[a], sl);
  }
  to_global(fl, WLf, d);
  to_global(fr, WRf, d);
  to_global(sl, slope, d);
}

// Physical flux along d of a global-frame face state (W primitive, U its
// conserved form); the energy used is U[4].
template <class R> inline void phys_flux_global(const R W[5], const R U[5], int d, R F[5]) {
  R wl[5], fl[5];
  to_local(W, wl, d);
  phys_flux_local(wl, U[4], fl);
  to_global(fl, F, d);
}

template <class R> struct GroupOut {
  R* U_out;
  R* flux;  // may be null
  unsigned status;
};

// Conservative update (step (4)) of the interior from the face fluxes
// F[d](c) = flux through the face c - e_d/2, and the boundary-flux store
// (step (5)).  Also sets the status bits of the updated state.
template <class R>
inline void update_and_store(const Params<R>& P, const Box& B, const R* Uin, const Field5<R> F[3], GroupOut<R>& out) {
  int N = B.N;
  R dtdx[3];
  for (int d = 0; d < 3; ++d) dtdx[d] = P.dt / P.dx[d];
  {
    Sec<R> sec(SEC_UPDATE);
    for (int z = 0; z < N; ++z)
      for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
          long c = B.at(x, y, z);
          R Un[5];
          for (int v = 0; v < 5; ++v) {
            R dU = dtdx[0] * (F[0](v, c + B.st[0]) - F[0](v, c)) + dtdx[1] * (F[1](v, c + B.st[1]) - F[1](v, c)) +
                   dtdx[2] * (F[2](v, c + B.st[2]) - F[2](v, c));
            Un[v] = Uin[v * B.M3 + c] - dU;
          }
          long o = ((long)z * N + y) * N + x;
          for (int v = 0; v < 5; ++v) out.U_out[(long)v * N * N * N + o] = Un[v];
          bool nan = false;
          for (int v = 0; v < 5; ++v) nan = nan || isnan_r(Un[v]);
          if (nan) out.status |= ST_NAN;
          if (!(Un[0] > R(0.0))) {
            out.status |= ST_NEG_DENS;
          } else {
            R p = (P.gas.gamma - R(1.0)) * (Un[4] - R(0.5) * (Un[1] * Un[1] + Un[2] * Un[2] + Un[3] * Un[3]) / Un[0]);
            if (!(p > R(0.0))) out.status |= ST_NEG_PRES;
          }
        }
  }
  if (!out.flux) return;
  long NN = (long)N * N;
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      int f = 2 * d + side;
      int cn = side == 0 ? 0 : N;  // face -1/2 is the left face of cell 0, N-1/2 the left face of cell N
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
          int x, y, z;
          if (d == 0) { x = cn; y = b; z = a; }
          else if (d == 1) { x = b; y = cn; z = a; }
          else { x = b; y = a; z = cn; }
          long c = B.at(x, y, z);
          for (int v = 0; v < 5; ++v) out.flux[((long)f * 5 + v) * NN + (long)a * N + b] = F[d](v, c);
        }
    }
}

// ----------------------------------------------------------------- MHM ----
template <class R> void mhm_group(const Params<R>& P, const Box& B, const R* Uin, GroupOut<R>& out) {
  int N = B.N;
  Field5<R> W(B.M3);
  for (long i = 0; i < B.M3; ++i) {
    R U[5], w[5];
    for (int v = 0; v < 5; ++v) U[v] = Uin[v * B.M3 + i];
    prim_from_cons(U, w, P.gas);
    W.set(i, w);
  }
  R hdtdx[3];
  for (int d = 0; d < 3; ++d) hdtdx[d] = R(0.5) * P.dt / P.dx[d];
  // step (1) + half-step prediction: face states FS[d][side], side 0 = left
  // face of the cell, side 1 = right face, conserved, advanced by dt/2
  std::vector<Field5<R>> FS(6, Field5<R>(B.M3));
  int lo[3] = {-1, -1, -1}, hi[3] = {N, N, N};
  for_box(lo, hi, [&](int x, int y, int z) {
    long c = B.at(x, y, z);
    R Wf[3][2][5], Uf[3][2][5], Ff[3][2][5], slope[5];
    for (int d = 0; d < 3; ++d) {
      recon_cell(P, B, W, c, d, Wf[d][0], Wf[d][1], slope);
      for (int s = 0; s < 2; ++s) {
        cons_from_prim(Wf[d][s], Uf[d][s], P.gas);
        phys_flux_global(Wf[d][s], Uf[d][s], d, Ff[d][s]);
      }
    }
    Sec<R> sec(SEC_PREDICT);
    for (int v = 0; v < 5; ++v) {
      R S = hdtdx[0] * (Ff[0][1][v] - Ff[0][0][v]) + hdtdx[1] * (Ff[1][1][v] - Ff[1][0][v]) +
            hdtdx[2] * (Ff[2][1][v] - Ff[2][0][v]);
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) FS[2 * d + s](v, c) = Uf[d][s][v] - S;
    }
  });
  // 3 Riemann solves per cell
  Field5<R> F[3] = {Field5<R>(B.M3), Field5<R>(B.M3), Field5<R>(B.M3)};
  for (int d = 0; d < 3; ++d) {
    range(d, 0, N, 0, N - 1, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R UL[5], UR[5], f[5];
      FS[2 * d + 1].get(c - B.st[d], UL);
      FS[2 * d + 0].get(c, UR);
      riemann(P.riemann, P.fallback, d, UL, UR, P.gas, f, &out.status);
      F[d].set(c, f);
    });
  }
  update_and_store(P, B, Uin, F, out);
}

// ------------------------------------------------------------------ VL ----
template <class R> void vl_group(const Params<R>& P, const Box& B, const R* Uin, GroupOut<R>& out) {
  int N = B.N;
  int s = recon_stencil(P.recon);
  R hdtdx[3];
  for (int d = 0; d < 3; ++d) hdtdx[d] = R(0.5) * P.dt / P.dx[d];
  // first-order fluxes on the cell-centred data
  Field5<R> F1[3] = {Field5<R>(B.M3), Field5<R>(B.M3), Field5<R>(B.M3)};
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    range(d, -1 - s, N + s + 1, -1 - s, N + s, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R UL[5], UR[5], f[5];
      for (int v = 0; v < 5; ++v) {
        UL[v] = Uin[v * B.M3 + c - B.st[d]];
        UR[v] = Uin[v * B.M3 + c];
      }
      riemann(P.riemann, P.fallback, d, UL, UR, P.gas, f, &out.status);
      F1[d].set(c, f);
    });
  }
  // unsplit half step U^{n+1/2} and its primitives
  Field5<R> Wh(B.M3);
  for (int k = 0; k < 3; ++k) { lo[k] = -1 - s; hi[k] = N + s; }
  for_box(lo, hi, [&](int x, int y, int z) {
    long c = B.at(x, y, z);
    R Uh[5], w[5];
    {
      Sec<R> sec(SEC_PREDICT);
      for (int v = 0; v < 5; ++v) {
        R S = hdtdx[0] * (F1[0](v, c + B.st[0]) - F1[0](v, c)) + hdtdx[1] * (F1[1](v, c + B.st[1]) - F1[1](v, c)) +
              hdtdx[2] * (F1[2](v, c + B.st[2]) - F1[2](v, c));
        Uh[v] = Uin[v * B.M3 + c] - S;
      }
    }
    prim_from_cons(Uh, w, P.gas);
    Wh.set(c, w);
  });
  // reconstruct the half-step state (no tracing), 3 Riemann solves, update
  std::vector<Field5<R>> FS(6, Field5<R>(B.M3));
  for (int d = 0; d < 3; ++d) {
    range(d, -1, N, 0, N - 1, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R Wf[2][5], Uf[5], slope[5];
      recon_cell(P, B, Wh, c, d, Wf[0], Wf[1], slope);
      for (int sd = 0; sd < 2; ++sd) {
        cons_from_prim(Wf[sd], Uf, P.gas);
        FS[2 * d + sd].set(c, Uf);
      }
    });
  }
  Field5<R> F[3] = {Field5<R>(B.M3), Field5<R>(B.M3), Field5<R>(B.M3)};
  for (int d = 0; d < 3; ++d) {
    range(d, 0, N, 0, N - 1, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R UL[5], UR[5], f[5];
      FS[2 * d + 1].get(c - B.st[d], UL);
      FS[2 * d + 0].get(c, UR);
      riemann(P.riemann, P.fallback, d, UL, UR, P.gas, f, &out.status);
      F[d].set(c, f);
    });
  }
  update_and_store(P, B, Uin, F, out);
}

// ----------------------------------------------------------------- CTU ----
template <class R> void ctu_group(const Params<R>& P, const Box& B, const R* Uin, GroupOut<R>& out) {
  int N = B.N;
  Field5<R> W(B.M3);
  for (long i = 0; i < B.M3; ++i) {
    R U[5], w[5];
    for (int v = 0; v < 5; ++v) U[v] = Uin[v * B.M3 + i];
    prim_from_cons(U, w, P.gas);
    W.set(i, w);
  }
  R dtdx[3], hdtdx[3];
  for (int d = 0; d < 3; ++d) {
    dtdx[d] = P.dt / P.dx[d];
    hdtdx[d] = R(0.5) * P.dt / P.dx[d];
  }
  // step (1): reconstruction + characteristic tracing to t + dt/2 on the cells
  // [-1, N]^3, stored as conserved face states FS[2d + side]
  std::vector<Field5<R>> FS(6, Field5<R>(B.M3));
  int lo[3] = {-1, -1, -1}, hi[3] = {N, N, N};
  for (int d = 0; d < 3; ++d) {
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R WLf[5], WRf[5], slope[5], w0[5];
      recon_cell(P, B, W, c, d, WLf, WRf, slope);
      W.get(c, w0);
      R w0l[5], a[5], b[5], tl[5], tr[5];
      to_local(w0, w0l, d);
      if (P.recon == REC_PPM) {
        to_local(WLf, a, d);
        to_local(WRf, b, d);
        trace_ppm(w0l, a, b, dtdx[d], P.gas, tl, tr);
      } else {
        to_local(slope, a, d);
        trace_plm(w0l, a, dtdx[d], P.gas, tl, tr);
      }
      R wg[5], u[5];
      to_global(tl, wg, d);
      cons_from_prim(wg, u, P.gas);
      FS[2 * d + 0].set(c, u);
      to_global(tr, wg, d);
      cons_from_prim(wg, u, P.gas);
      FS[2 * d + 1].set(c, u);
    });
  }
  // step (2): stage-1 fluxes on the faces c_d in [0, N], lateral [-1, N]
  Field5<R> F1[3] = {Field5<R>(B.M3), Field5<R>(B.M3), Field5<R>(B.M3)};
  for (int d = 0; d < 3; ++d) {
    range(d, 0, N, -1, N, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R UL[5], UR[5], f[5];
      FS[2 * d + 1].get(c - B.st[d], UL);
      FS[2 * d + 0].get(c, UR);
      riemann(P.riemann, P.fallback, d, UL, UR, P.gas, f, &out.status);
      F1[d].set(c, f);
    });
  }
  // step (3): transverse flux-gradient correction of the face states of the
  // cells c_d in [-1, N], lateral [0, N-1]:
  //   U -= dt/(2 dx_e) (F1_e(c + e_e/2) - F1_e(c - e_e/2))  for both e != d
  for (int d = 0; d < 3; ++d) {
    int e1 = (d == 0) ? 1 : 0;
    int e2 = (d == 2) ? 1 : 2;
    range(d, -1, N, 0, N - 1, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      Sec<R> sec(SEC_CORRECT);
      long c = B.at(x, y, z);
      for (int side = 0; side < 2; ++side)
        for (int v = 0; v < 5; ++v) {
          R u = FS[2 * d + side](v, c);
          u = u - hdtdx[e1] * (F1[e1](v, c + B.st[e1]) - F1[e1](v, c));
          u = u - hdtdx[e2] * (F1[e2](v, c + B.st[e2]) - F1[e2](v, c));
          FS[2 * d + side](v, c) = u;
        }
    });
  }
  // ... and the Riemann problem again with the corrected states
  Field5<R> F[3] = {Field5<R>(B.M3), Field5<R>(B.M3), Field5<R>(B.M3)};
  for (int d = 0; d < 3; ++d) {
    range(d, 0, N, 0, N - 1, lo, hi);
    for_box(lo, hi, [&](int x, int y, int z) {
      long c = B.at(x, y, z);
      R UL[5], UR[5], f[5];
      FS[2 * d + 1].get(c - B.st[d], UL);
      FS[2 * d + 0].get(c, UR);
      riemann(P.riemann, P.fallback, d, UL, UR, P.gas, f, &out.status);
      F[d].set(c, f);
    });
  }
  // steps (4) and (5)
  update_and_store(P, B, Uin, F, out);
}

// ---------------------------------------------------------------------------
// The directionally split schemes Sec. 3.2 measures beside the unsplit ones
// (RTVD and WAF): three 1D sweeps per step, x, y, z (split_order 0) or z, y,
// x (1; the caller alternates them, Strang), each with the full dt, on the
// local-frame conserved states of the rows along the sweep.  Each sweep
// updates the cells [0, N) along its direction in the rows the later sweeps
// still read: the first sweep every row whose transverse coordinates lie in
// [-g, N+g), the second [0, N) along the first sweep's direction and
// [-g, N+g) along the last's, the last [0, N)^2.  The fluxes of each sweep's
// update through the group faces are the boundary fluxes of step (5).
// ---------------------------------------------------------------------------

// RTVD (relaxing TVD, Jin & Xin 1995, in the flux-split form of Trac & Pen
// 2003).  Per cell the freezing speed c = |u_n| + c_s and the flux F;
// right- and left-moving parts FR = (c U + F)/2, FL = (c U - F)/2.
template <class R> inline void rtvd_split(const R U[5], const Gas<R>& gas, R FR[5], R FL[5]) {
  R W[5], F[5];
  prim_from_cons(U, W, gas);
  R c = fabs(W[1]) + sound_speed(W[0], W[4], gas);
  phys_flux_local(W, U[4], F);
  for (int v = 0; v < 5; ++v) {
    FR[v] = R(0.5) * (c * U[v] + F[v]);
    FL[v] = R(0.5) * (c * U[v] - F[v]);
  }
}

// One RTVD row u[0..n) (local frame; updated in place on [lo, hi), which
// needs lo >= 3 and hi <= n - 3):
//   half step, first-order upwind:  F1_{j+1/2} = FR_j - FL_{j+1},
//     Uh_j = U_j - (dt/2dx) (F1_{j+1/2} - F1_{j-1/2});
//   full step, limited fluxes of Uh (psi = limited slope of the limiter):
//     FR_{i+1/2} = FR_i + psi(FR_i - FR_{i-1}, FR_{i+1} - FR_i) / 2,
//     FL_{i+1/2} = FL_{i+1} - psi(FL_{i+1} - FL_i, FL_{i+2} - FL_{i+1}) / 2,
//     U_i <- U_i - (dt/dx) (F_{i+1/2} - F_{i-1/2}),  F = FR - FL.
// Returns the fluxes through lo - 1/2 and hi - 1/2.
template <class R>
inline void rtvd_row(const Params<R>& P, std::vector<std::array<R, 5>>& u, int lo, int hi, R dtdx, R hdtdx,
                     R Flo[5], R Fhi[5]) {
  const int n = (int)u.size();
  std::vector<std::array<R, 5>> FR(n), FL(n), F1(n), FRh(n), FLh(n), FT(n);
  // (operation-count scopes: per cell two splittings, one first-order flux
  // difference, one half step, one limited flux, one update)
  for (int j = lo - 3; j < hi + 3; ++j) {
    Sec<R> sec(SEC_EOS);
    rtvd_split(u[j].data(), P.gas, FR[j].data(), FL[j].data());
  }
  for (int j = lo - 3; j < hi + 2; ++j) {
    Sec<R> sec(SEC_RIEMANN);
    for (int v = 0; v < 5; ++v) F1[j][v] = FR[j][v] - FL[j + 1][v];
  }
  for (int j = lo - 2; j < hi + 2; ++j) {
    R uh[5];
    {
      Sec<R> sec(SEC_PREDICT);
      for (int v = 0; v < 5; ++v) uh[v] = u[j][v] - hdtdx * (F1[j][v] - F1[j - 1][v]);
    }
    Sec<R> sec(SEC_EOS);
    rtvd_split(uh, P.gas, FRh[j].data(), FLh[j].data());
  }
  for (int i = lo - 1; i < hi; ++i) {
    Sec<R> sec(SEC_RECON);
    for (int v = 0; v < 5; ++v) {
      R fr = FRh[i][v] + R(0.5) * limited_slope(P.limiter, P.theta, FRh[i][v] - FRh[i - 1][v],
                                                FRh[i + 1][v] - FRh[i][v]);
      R fl = FLh[i + 1][v] - R(0.5) * limited_slope(P.limiter, P.theta, FLh[i + 1][v] - FLh[i][v],
                                                    FLh[i + 2][v] - FLh[i + 1][v]);
      FT[i][v] = fr - fl;
    }
  }
  for (int i = lo; i < hi; ++i) {
    Sec<R> sec(SEC_UPDATE);
    for (int v = 0; v < 5; ++v) u[i][v] = u[i][v] - dtdx * (FT[i][v] - FT[i - 1][v]);
  }
  for (int v = 0; v < 5; ++v) {
    Flo[v] = FT[lo - 1][v];
    Fhi[v] = FT[hi - 1][v];
  }
}

// The HLLC wave fan of one face (Toro 2009 ch. 10, with the Einfeldt speeds
// of hllc_flux): speeds S = (SL, S*, SR), the fluxes of the four states
// U_L, U*L, U*R, U_R (F*K = FK + SK (U*K - UK)), and the density jumps across
// the three waves.
template <class R> struct Fan {
  R S[3];
  R F[4][5];
  R drho[3];
};

template <class R> inline void hllc_fan(const Side<R>& L, const Side<R>& Rs, const Gas<R>& gas, Fan<R>& f) {
  RoeAvg<R> A;
  roe_average(L, Rs, gas, A);
  R a = A.a2 > R(0.0) ? sqrt(A.a2) : R(0.0);
  R SL = L.W[1] - L.c;
  R t = A.u - a;
  if (t < SL) SL = t;
  R SR = Rs.W[1] + Rs.c;
  t = A.u + a;
  if (t > SR) SR = t;
  R mL = L.W[0] * (SL - L.W[1]);
  R mR = Rs.W[0] * (SR - Rs.W[1]);
  R Ss = (Rs.W[4] - L.W[4] + mL * L.W[1] - mR * Rs.W[1]) / (mL - mR);
  R fL = mL / (SL - Ss), fR = mR / (SR - Ss);
  R UsL[5] = {fL, fL * Ss, fL * L.W[2], fL * L.W[3], fL * (L.E / L.W[0] + (Ss - L.W[1]) * (Ss + L.W[4] / mL))};
  R UsR[5] = {fR, fR * Ss, fR * Rs.W[2], fR * Rs.W[3],
              fR * (Rs.E / Rs.W[0] + (Ss - Rs.W[1]) * (Ss + Rs.W[4] / mR))};
  f.S[0] = SL;
  f.S[1] = Ss;
  f.S[2] = SR;
  for (int v = 0; v < 5; ++v) {
    f.F[0][v] = L.F[v];
    f.F[1][v] = L.F[v] + SL * (UsL[v] - L.U[v]);
    f.F[2][v] = Rs.F[v] + SR * (UsR[v] - Rs.U[v]);
    f.F[3][v] = Rs.F[v];
  }
  f.drho[0] = UsL[0] - L.W[0];
  f.drho[1] = UsR[0] - UsL[0];
  f.drho[2] = Rs.W[0] - UsR[0];
}

// One WAF row (Toro 2009 ch. 14, TVD version with the HLLC fan): with
// c_k = (dt/dx) S_k,
//   F_{i+1/2} = (F_1 + F_4)/2 - sum_k (sign(c_k) A_k / 2) (F_{k+1} - F_k),
//   A_k = 1 - (1 - |c_k|) psi(r_k),
// r_k the density jump across wave k at the upwind face (i-1/2 if c_k > 0,
// i+3/2 otherwise) over the jump at this face (psi = 0 where that is 0), and
// psi(r) = limited_slope(r, 1), the limiter of the unsplit schemes in ratio
// form (minmod -> minbee for theta = 1, van Leer, van Albada, hybrid).
// Updates [lo, hi) in place (lo >= 2, hi <= n - 2); returns the fluxes
// through lo - 1/2 and hi - 1/2.
template <class R>
inline void waf_row(const Params<R>& P, std::vector<std::array<R, 5>>& u, int lo, int hi, R dtdx, R Flo[5],
                    R Fhi[5]) {
  const int n = (int)u.size();
  std::vector<Side<R>> sd(n);
  std::vector<Fan<R>> fan(n);
  std::vector<std::array<R, 5>> FW(n);
  // (operation-count scopes: per cell one side state, one wave fan, one
  // weighted flux, one update)
  for (int j = lo - 2; j < hi + 2; ++j) {
    Sec<R> sec(SEC_EOS);
    make_side(u[j].data(), P.gas, sd[j]);
  }
  for (int j = lo - 2; j < hi + 1; ++j) {
    Sec<R> sec(SEC_RIEMANN);
    hllc_fan(sd[j], sd[j + 1], P.gas, fan[j]);  // face j + 1/2
  }
  for (int i = lo - 1; i < hi; ++i) {
    Sec<R> sec(SEC_RECON);
    const Fan<R>& f = fan[i];
    R F[5];
    for (int v = 0; v < 5; ++v) F[v] = R(0.5) * (f.F[0][v] + f.F[3][v]);
    for (int k = 0; k < 3; ++k) {
      R c = dtdx * f.S[k];
      R s = c > R(0.0) ? R(1.0) : (c < R(0.0) ? R(-1.0) : R(0.0));
      const Fan<R>& up = c > R(0.0) ? fan[i - 1] : fan[i + 1];
      R psi = R(0.0);
      if (f.drho[k] != R(0.0)) psi = limited_slope(P.limiter, P.theta, up.drho[k] / f.drho[k], R(1.0));
      R A = R(1.0) - (R(1.0) - fabs(c)) * psi;
      R w = R(0.5) * s * A;
      for (int v = 0; v < 5; ++v) F[v] = F[v] - w * (f.F[k + 1][v] - f.F[k][v]);
    }
    for (int v = 0; v < 5; ++v) FW[i][v] = F[v];
  }
  for (int i = lo; i < hi; ++i) {
    Sec<R> sec(SEC_UPDATE);
    for (int v = 0; v < 5; ++v) u[i][v] = u[i][v] - dtdx * (FW[i][v] - FW[i - 1][v]);
  }
  for (int v = 0; v < 5; ++v) {
    Flo[v] = FW[lo - 1][v];
    Fhi[v] = FW[hi - 1][v];
  }
}

template <class R> inline void split_group(const Params<R>& P, const Box& B, const R* Uin, GroupOut<R>& out) {
  const int N = B.N, g = B.g, M = B.M;
  const int s = required_ghost(P.scheme, 0);
  Field5<R> U(B.M3);
  for (long i = 0; i < B.M3; ++i)
    for (int v = 0; v < 5; ++v) U(v, i) = Uin[v * B.M3 + i];
  const int order[3] = {P.split_order ? 2 : 0, 1, P.split_order ? 0 : 2};
  std::vector<R> FB(out.flux ? 30L * N * N : 0);
  for (int k = 0; k < 3; ++k) {
    const int d = order[k];
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;  // transverse axes, e1 < e2
    // rows the later sweeps read: [-s, N+s) along the axes swept later, [0, N) otherwise
    auto later = [&](int e) {
      for (int m = k + 1; m < 3; ++m)
        if (order[m] == e) return true;
      return false;
    };
    const int a1 = later(e1) ? -s : 0, b1 = later(e1) ? N + s : N;
    const int a2 = later(e2) ? -s : 0, b2 = later(e2) ? N + s : N;
    const R dtdx = P.dt / P.dx[d];
    const R hdtdx = R(0.5) * P.dt / P.dx[d];
    for (int q2 = a2; q2 < b2; ++q2)
      for (int q1 = a1; q1 < b1; ++q1) {
        std::vector<std::array<R, 5>> row(M);
        int c[3];
        c[e1] = q1;
        c[e2] = q2;
        for (int j = 0; j < M; ++j) {
          c[d] = j - g;
          R gl[5];
          U.get(B.at(c[0], c[1], c[2]), gl);
          to_local(gl, row[j].data(), d);
        }
        R Flo[5], Fhi[5];
        if (P.scheme == SCH_RTVD)
          rtvd_row(P, row, g, g + N, dtdx, hdtdx, Flo, Fhi);
        else
          waf_row(P, row, g, g + N, dtdx, Flo, Fhi);
        for (int j = g; j < g + N; ++j) {
          c[d] = j - g;
          R gl[5];
          to_global(row[j].data(), gl, d);
          U.set(B.at(c[0], c[1], c[2]), gl);
        }
        if (out.flux && q1 >= 0 && q1 < N && q2 >= 0 && q2 < N) {
          R fl[5], fh[5];
          to_global(Flo, fl, d);
          to_global(Fhi, fh, d);
          // [a][b]: a the larger transverse axis (e2), b the smaller (e1)
          for (int v = 0; v < 5; ++v) {
            FB[((2 * d) * 5 + v) * N * N + (long)q2 * N + q1] = fl[v];
            FB[((2 * d + 1) * 5 + v) * N * N + (long)q2 * N + q1] = fh[v];
          }
        }
      }
    (void)s;
  }
  for (int z = 0; z < N; ++z)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        R Un[5];
        U.get(B.at(x, y, z), Un);
        long o = ((long)z * N + y) * N + x;
        for (int v = 0; v < 5; ++v) out.U_out[(long)v * N * N * N + o] = Un[v];
        bool nan = false;
        for (int v = 0; v < 5; ++v) nan = nan || isnan_r(Un[v]);
        if (nan) out.status |= ST_NAN;
        if (!(Un[0] > R(0.0))) {
          out.status |= ST_NEG_DENS;
        } else {
          R p = (P.gas.gamma - R(1.0)) * (Un[4] - R(0.5) * (Un[1] * Un[1] + Un[2] * Un[2] + Un[3] * Un[3]) / Un[0]);
          if (!(p > R(0.0))) out.status |= ST_NEG_PRES;
        }
      }
  if (out.flux)
    for (long i = 0; i < 30L * N * N; ++i) out.flux[i] = FB[i];
}

template <class R> inline void advance_group(const Params<R>& P, const Box& B, const R* Uin, GroupOut<R>& out) {
  switch (P.scheme) {
    case SCH_MHM: mhm_group(P, B, Uin, out); break;
    case SCH_VL: vl_group(P, B, Uin, out); break;
    case SCH_RTVD:
    case SCH_WAF: split_group(P, B, Uin, out); break;
    default: ctu_group(P, B, Uin, out); break;
  }
}

}  // namespace orc
