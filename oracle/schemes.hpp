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
#include <vector>
#include "reconstruct.hpp"
#include "riemann.hpp"

namespace orc {

enum Scheme { SCH_MHM = 0, SCH_VL = 1, SCH_CTU = 2 };
enum Recon { REC_PLM = 0, REC_PPM = 1 };

template <class R> struct Params {
  int scheme, recon, limiter, riemann, fallback;
  R theta;
  Gas<R> gas;
  R dt;
  R dx[3];
  int characteristic = 0;  // reconstruct characteristic (1) or primitive (0) variables
};

inline int recon_stencil(int recon) { return recon == REC_PPM ? 2 : 1; }

// Ghost layers a scheme needs: face states are required for the cells -1..N
// along the normal; CTU also needs the stage-1 fluxes of the cells -1..N in
// the lateral directions, which the same width provides.  VL reconstructs its
// half-step state, which itself needs one more layer.
inline int required_ghost(int scheme, int recon) {
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

template <class R> inline void advance_group(const Params<R>& P, const Box& B, const R* Uin, GroupOut<R>& out) {
  switch (P.scheme) {
    case SCH_MHM: mhm_group(P, B, Uin, out); break;
    case SCH_VL: vl_group(P, B, Uin, out); break;
    default: ctu_group(P, B, Uin, out); break;
  }
}

}  // namespace orc
