// ORACLE — test infrastructure only (see real.hpp).
//
// The adiabatic Euler equations of an ideal gas (Sec. 1 and Sec. 5.1 of the
// paper: "adiabatic hydrodynamic" tests; gamma is a free parameter).
//   conserved  U = (rho, rho u, rho v, rho w, E)
//   primitive  W = (rho, u, v, w, p),   p = (gamma - 1) (E - |m|^2 / (2 rho))
// Directional quantities are evaluated in a "local" frame in which the
// component normal to the face comes first: (rho, m_n, m_t1, m_t2, E), with
// (n, t1, t2) = (x, y, z), (y, z, x) or (z, x, y) for directions 0, 1, 2.
#pragma once
#include "real.hpp"

namespace orc {

// Equation of state and the density / pressure floors.  A floor of 0 leaves
// every positive value untouched (floors are applied as max(q, floor)).
template <class R> struct Gas {
  R gamma;
  R dens_floor;
  R pres_floor;
};

// Index of the normal and the two transverse momentum components in U for a
// sweep along direction d (0 = x, 1 = y, 2 = z).
inline int mom_n(int d) { return 1 + d; }
inline int mom_t1(int d) { return 1 + (d + 1) % 3; }
inline int mom_t2(int d) { return 1 + (d + 2) % 3; }

// U (global frame) -> W (global frame), with floors.
template <class R> inline void prim_from_cons(const R U[5], R W[5], const Gas<R>& gas) {
  Sec<R> sec(SEC_EOS);
  R rho = U[0];
  if (rho < gas.dens_floor) rho = gas.dens_floor;
  R kin = R(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;
  R p = (gas.gamma - R(1.0)) * (U[4] - kin);
  if (p < gas.pres_floor) p = gas.pres_floor;
  W[0] = rho;
  W[1] = U[1] / rho;
  W[2] = U[2] / rho;
  W[3] = U[3] / rho;
  W[4] = p;
}

// W -> U (same frame on both sides).
template <class R> inline void cons_from_prim(const R W[5], R U[5], const Gas<R>& gas) {
  Sec<R> sec(SEC_EOS);
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  U[4] = W[4] / (gas.gamma - R(1.0)) + R(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

// Rotate a 5-vector from the global frame into the local frame of direction d.
template <class R> inline void to_local(const R a[5], R b[5], int d) {
  b[0] = a[0];
  b[1] = a[mom_n(d)];
  b[2] = a[mom_t1(d)];
  b[3] = a[mom_t2(d)];
  b[4] = a[4];
}
template <class R> inline void to_global(const R b[5], R a[5], int d) {
  a[0] = b[0];
  a[mom_n(d)] = b[1];
  a[mom_t1(d)] = b[2];
  a[mom_t2(d)] = b[3];
  a[4] = b[4];
}

// Physical flux along the local normal of a local primitive state W with
// total energy E:  F = (rho u, rho u u + p, rho u v, rho u w, (E + p) u).
template <class R> inline void phys_flux_local(const R W[5], R E, R F[5]) {
  Sec<R> sec(SEC_EOS);
  R mn = W[0] * W[1];
  F[0] = mn;
  F[1] = mn * W[1] + W[4];
  F[2] = mn * W[2];
  F[3] = mn * W[3];
  F[4] = (E + W[4]) * W[1];
}

// Total energy of a local primitive state.
template <class R> inline R energy_local(const R W[5], const Gas<R>& gas) {
  Sec<R> sec(SEC_EOS);
  return W[4] / (gas.gamma - R(1.0)) + R(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}

// Sound speed c = sqrt(gamma p / rho).
template <class R> inline R sound_speed(R rho, R p, const Gas<R>& gas) {
  Sec<R> sec(SEC_EOS);
  return sqrt(gas.gamma * p / rho);
}

}  // namespace orc
