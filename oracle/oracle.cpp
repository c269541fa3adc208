// ORACLE — test infrastructure only.  A plain, slow FP64 CPU implementation
// of the unsplit patch-group fluid update of the paper (Sec. 2 and 3.1).  Only
// tests/, __graft_entry__.smoke() and bench.py (cpu_baseline and the
// reference arm) may load it; it shares no code with the CUDA path.
//
// C entry points for ctypes.  All arrays are float64, C order.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "schemes.hpp"

namespace orc {
thread_local OpTally g_tally;
thread_local int g_section = SEC_OTHER;
}  // namespace orc

using namespace orc;

extern "C" {

struct OrcParams {
  int scheme, recon, limiter, riemann, fallback;
  double theta, gamma, dens_floor, pres_floor, dt;
  double dx[3];
  int characteristic;
  int split_order;
};

static Params<double> to_params(const OrcParams* p) {
  Params<double> P;
  P.scheme = p->scheme;
  P.recon = p->recon;
  P.limiter = p->limiter;
  P.riemann = p->riemann;
  P.fallback = p->fallback;
  P.theta = p->theta;
  P.gas.gamma = p->gamma;
  P.gas.dens_floor = p->dens_floor;
  P.gas.pres_floor = p->pres_floor;
  P.dt = p->dt;
  for (int d = 0; d < 3; ++d) P.dx[d] = p->dx[d];
  P.characteristic = p->characteristic;
  P.split_order = p->split_order;
  return P;
}

int orc_required_ghost(int scheme, int recon) { return required_ghost(scheme, recon); }

// Advance G groups one step.  U_in [G][5][M^3], U_out [G][5][N^3],
// flux [G][6][5][N][N] or NULL, status [G].  nthreads <= 0: all cores.
// Returns 0, or -1 when the ghost width is too small.
int orc_advance(const OrcParams* p, const double* U_in, double* U_out, double* flux, int G, int N, int g,
                unsigned* status, int nthreads) {
  if (g < required_ghost(p->scheme, p->recon)) return -1;
  Params<double> P = to_params(p);
  Box B(N, g);
  long in_stride = 5 * B.M3, out_stride = 5L * N * N * N, fx_stride = 30L * N * N;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
  for (int gi = 0; gi < G; ++gi) {
    GroupOut<double> out;
    out.U_out = U_out + gi * out_stride;
    out.flux = flux ? flux + gi * fx_stride : nullptr;
    out.status = 0;
    advance_group(P, B, U_in + gi * in_stride, out);
    status[gi] = out.status;
  }
  return 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Ghost-zone gather (the "preparation step" of Sec. 4.2) for a uniform field
// [5][Z][Y][X]: group gi's interior starts at origin[gi] = (x0, y0, z0) and
// its g-deep halo is filled periodically (bc = 0) or by copying the nearest
// boundary cell (bc = 1, outflow / zero gradient).
int orc_gather(const double* field, int X, int Y, int Z, int bc, const int* origin, int G, int N, int g,
               double* out) {
  int M = N + 2 * g;
  long M3 = (long)M * M * M, XYZ = (long)X * Y * Z;
  for (int gi = 0; gi < G; ++gi) {
    const int* o = origin + 3 * gi;
    for (int v = 0; v < 5; ++v)
      for (int k = 0; k < M; ++k)
        for (int j = 0; j < M; ++j)
          for (int i = 0; i < M; ++i) {
            long sx = o[0] + i - g, sy = o[1] + j - g, sz = o[2] + k - g;
            if (bc == 0) {
              sx = ((sx % X) + X) % X;
              sy = ((sy % Y) + Y) % Y;
              sz = ((sz % Z) + Z) % Z;
            } else {
              sx = sx < 0 ? 0 : (sx >= X ? X - 1 : sx);
              sy = sy < 0 ? 0 : (sy >= Y ? Y - 1 : sy);
              sz = sz < 0 ? 0 : (sz >= Z ? Z - 1 : sz);
            }
            out[gi * 5 * M3 + v * M3 + ((long)k * M + j) * M + i] = field[v * XYZ + (sz * Y + sy) * X + sx];
          }
  }
  return 0;
}

// CFL time step (the evolution time-step of Sec. 4.3):
//   dt = cfl / max_cells max_d (|v_d| + c) / dx_d,   c = sqrt(gamma p / rho).
// U is addressed as U[g * group_stride + v * var_stride + i], i < cells.
double orc_cfl_dt(const double* U, int G, long group_stride, long var_stride, long cells, double gamma,
                  double dens_floor, double pres_floor, const double* dx, double cfl) {
  Gas<double> gas{gamma, dens_floor, pres_floor};
  double smax = 0.0;
  for (int gi = 0; gi < G; ++gi)
    for (long i = 0; i < cells; ++i) {
      double u[5], w[5];
      for (int v = 0; v < 5; ++v) u[v] = U[gi * group_stride + v * var_stride + i];
      prim_from_cons(u, w, gas);
      double c = sound_speed(w[0], w[4], gas);
      for (int d = 0; d < 3; ++d) {
        double s = (std::fabs(w[1 + d]) + c) / dx[d];
        if (s > smax) smax = s;
      }
    }
  return cfl / smax;
}

// ---- single-routine entry points for the pins in tests/ -------------------

double orc_limiter(int limiter, double theta, double dL, double dR) {
  return limited_slope<double>(limiter, theta, dL, dR);
}

// 1D reconstruction of w[0..n): faces of cells s..n-1-s (s = stencil).
// Face values (and PLM slopes) of the cells S..n-1-S of a line of n
// primitive states W [5][n] (global frame) laid along direction d, as the
// schemes reconstruct them (primitive or characteristic form per p); outputs
// [5][n], untouched outside that range.
void orc_recon_line(const OrcParams* p, int d, const double* W, int n, double* WL, double* WR, double* slope) {
  Params<double> P = to_params(p);
  Field5<double> F(n);
  for (int v = 0; v < 5; ++v)
    for (int i = 0; i < n; ++i) F(v, i) = W[v * n + i];
  Box B(1, 0);
  B.st[d] = 1;
  const int S = recon_stencil(P.recon);
  for (int i = S; i < n - S; ++i) {
    double l[5], r[5], s[5] = {0, 0, 0, 0, 0};
    recon_cell(P, B, F, i, d, l, r, s);
    for (int v = 0; v < 5; ++v) {
      WL[v * n + i] = l[v];
      WR[v * n + i] = r[v];
      slope[v * n + i] = s[v];
    }
  }
}

void orc_recon1d(int recon, int limiter, double theta, const double* w, int n, double* wL, double* wR) {
  int s = recon_stencil(recon);
  for (int i = s; i < n - s; ++i) {
    double d;
    if (recon == REC_PPM)
      ppm_faces<double>(w + i, 1, limiter, theta, wL + i, wR + i);
    else
      plm_faces<double>(w + i, 1, limiter, theta, wL + i, wR + i, &d);
  }
}

// One sweep of a split scheme (RTVD or WAF per p->scheme) along one row of n
// conserved states u [n][5] in the local frame of the sweep (normal momentum
// second), updated in place on the cells [lo, hi) with the full dt over dx;
// Flo / Fhi receive the fluxes through the faces lo - 1/2 and hi - 1/2.
void orc_split_row(const OrcParams* p, double* u, int n, int lo, int hi, double dx, double* Flo, double* Fhi) {
  Params<double> P = to_params(p);
  std::vector<std::array<double, 5>> row(n);
  for (int j = 0; j < n; ++j)
    for (int v = 0; v < 5; ++v) row[j][v] = u[j * 5 + v];
  const double dtdx = P.dt / dx, hdtdx = 0.5 * P.dt / dx;
  if (P.scheme == SCH_RTVD)
    rtvd_row(P, row, lo, hi, dtdx, hdtdx, Flo, Fhi);
  else
    waf_row(P, row, lo, hi, dtdx, Flo, Fhi);
  for (int j = 0; j < n; ++j)
    for (int v = 0; v < 5; ++v) u[j * 5 + v] = row[j][v];
}

// Characteristic tracing of one cell (local frame arrays).  For PLM, a = slope
// and b is ignored; for PPM, a / b are the left / right face values.
void orc_trace(int recon, double gamma, const double* W0, const double* a, const double* b, double dtdx,
               double* Wl, double* Wr) {
  Gas<double> gas{gamma, 0.0, 0.0};
  if (recon == REC_PPM)
    trace_ppm<double>(W0, a, b, dtdx, gas, Wl, Wr);
  else
    trace_plm<double>(W0, a, dtdx, gas, Wl, Wr);
}

// Riemann flux at one face along direction d (global-frame conserved states).
unsigned orc_riemann(int solver, int fallback, int d, double gamma, double dens_floor, double pres_floor,
                     const double* UL, const double* UR, double* F) {
  Gas<double> gas{gamma, dens_floor, pres_floor};
  unsigned st = 0;
  riemann<double>(solver, fallback, d, UL, UR, gas, F, &st);
  return st;
}

// Roe flux alone: returns 1 when the linearisation is accepted, 0 on failure.
int orc_roe_only(double gamma, const double* UL, const double* UR, double* F) {
  Gas<double> gas{gamma, 0.0, 0.0};
  Side<double> L, R;
  make_side<double>(UL, gas, L);
  make_side<double>(UR, gas, R);
  return roe_flux<double>(L, R, gas, F) ? 1 : 0;
}

// Exact solver star state for local primitive states WL, WR; returns the
// iteration count (negative on failure) and the solution sampled at the nxi
// points x/t = xi[k] into Wsample[k][5].
int orc_exact_star(double gamma, const double* WL, const double* WR, double* pstar, double* ustar,
                   const double* xi, int nxi, double* Wsample) {
  Gas<double> gas{gamma, 0.0, 0.0};
  double cL = sound_speed(WL[0], WL[4], gas), cR = sound_speed(WR[0], WR[4], gas);
  ExactResult<double> r = exact_star<double>(WL, cL, WR, cR, gas);
  *pstar = r.pstar;
  *ustar = r.ustar;
  if (r.ok)
    for (int k = 0; k < nxi; ++k) exact_sample<double>(WL, cL, WR, cR, r.pstar, r.ustar, xi[k], gas, Wsample + 5 * k);
  return r.ok ? r.iters : -1 - r.iters;
}

// ---- operation counts ------------------------------------------------------
// Runs one group through the Counted instantiation and returns the tally:
// out[sec * OP_NCLASS + cls] for sec < SEC_N, followed by calls[sec].
int orc_count_ops(const OrcParams* p, const double* U_in, int N, int g, long long* out) {
  if (g < required_ghost(p->scheme, p->recon)) return -1;
  Params<Counted> P;
  P.scheme = p->scheme;
  P.recon = p->recon;
  P.limiter = p->limiter;
  P.riemann = p->riemann;
  P.fallback = p->fallback;
  P.theta = p->theta;
  P.gas.gamma = p->gamma;
  P.gas.dens_floor = p->dens_floor;
  P.gas.pres_floor = p->pres_floor;
  P.dt = p->dt;
  for (int d = 0; d < 3; ++d) P.dx[d] = p->dx[d];
  P.characteristic = p->characteristic;
  P.split_order = p->split_order;
  Box B(N, g);
  std::vector<Counted> Uin(5 * B.M3), Uout(5L * N * N * N), fl(30L * N * N);
  for (long i = 0; i < 5 * B.M3; ++i) Uin[i] = Counted(U_in[i]);
  std::memset(&g_tally, 0, sizeof(g_tally));
  g_section = SEC_OTHER;
  GroupOut<Counted> o;
  o.U_out = Uout.data();
  o.flux = fl.data();
  o.status = 0;
  advance_group(P, B, Uin.data(), o);
  for (int s = 0; s < SEC_N; ++s)
    for (int c = 0; c < OP_NCLASS; ++c) out[s * OP_NCLASS + c] = g_tally.ops[s][c];
  for (int s = 0; s < SEC_N; ++s) out[SEC_N * OP_NCLASS + s] = g_tally.calls[s];
  return 0;
}

// Operation tally of a single Riemann solve (for per-primitive counts).
int orc_count_riemann(int solver, int fallback, int d, double gamma, const double* UL, const double* UR,
                      long long* out) {
  Gas<Counted> gas{Counted(gamma), Counted(0.0), Counted(0.0)};
  Counted ul[5], ur[5], F[5];
  for (int v = 0; v < 5; ++v) {
    ul[v] = UL[v];
    ur[v] = UR[v];
  }
  std::memset(&g_tally, 0, sizeof(g_tally));
  g_section = SEC_OTHER;
  unsigned st = 0;
  riemann<Counted>(solver, fallback, d, ul, ur, gas, F, &st);
  for (int s = 0; s < SEC_N; ++s)
    for (int c = 0; c < OP_NCLASS; ++c) out[s * OP_NCLASS + c] = g_tally.ops[s][c];
  for (int s = 0; s < SEC_N; ++s) out[SEC_N * OP_NCLASS + s] = g_tally.calls[s];
  return 0;
}

}  // extern "C"
