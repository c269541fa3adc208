// ORACLE — test infrastructure only.  Only tests/, __graft_entry__.smoke() and
// bench.py's cpu_baseline / reference legs may load this code; the product path
// (paper_1103_3373_gb300) never imports, links or calls it.
//
// Scalar types for the oracle.  The oracle is written once, templated on the
// scalar R, and instantiated twice:
//   * R = double : the FP64 reference the GPU path is compared with;
//   * R = Counted: a double that counts every arithmetic operation, used only
//     to measure the algorithmic operation count per cell update (the roofline
//     numerator).  It never changes a value.
#pragma once
#include <cmath>

namespace orc {

// Operation classes counted by Counted.  add covers + and -, mul covers *,
// div covers /, sqrt and pow are the library calls, cmp covers comparisons,
// min/max and fabs (not flops, reported separately).
enum OpClass { OP_ADD = 0, OP_MUL, OP_DIV, OP_SQRT, OP_POW, OP_CMP, OP_NCLASS };

// Program sections the counts are attributed to (Sec. 2 steps).
enum Section {
  SEC_EOS = 0,    // primitive <-> conserved conversions, physical fluxes
  SEC_RECON,      // PLM / PPM reconstruction incl. limiters (step (1))
  SEC_TRACE,      // CTU characteristic tracing (step (1), CTU only)
  SEC_PREDICT,    // MHM / VL half-step prediction
  SEC_RIEMANN,    // Riemann solvers (steps (2), (3))
  SEC_CORRECT,    // CTU transverse flux-gradient correction (step (3))
  SEC_UPDATE,     // conservative update (step (4))
  SEC_OTHER,
  SEC_N
};

struct OpTally {
  long long ops[SEC_N][OP_NCLASS];
  long long calls[SEC_N];
};

// Thread-local tally and current section (only the Counted instantiation
// touches them).
extern thread_local OpTally g_tally;
extern thread_local int g_section;

// Operations are attributed to the outermost open section (a Riemann solve
// owns the state conversions it makes), and a call is counted only when its
// section is entered from outside any other section.
struct SectionScope {
  int saved;
  explicit SectionScope(int s) : saved(g_section) {
    if (g_section == SEC_OTHER) {
      g_section = s;
      g_tally.calls[s]++;
    }
  }
  ~SectionScope() { g_section = saved; }
};

struct Counted {
  double v;
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}  // implicit: literals mix freely
};

inline void tick(int c) { g_tally.ops[g_section][c]++; }

inline Counted operator+(Counted a, Counted b) { tick(OP_ADD); return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { tick(OP_ADD); return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { tick(OP_MUL); return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { tick(OP_DIV); return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }  // sign flip: free
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline Counted& operator*=(Counted& a, Counted b) { a = a * b; return a; }
inline bool operator<(Counted a, Counted b) { tick(OP_CMP); return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { tick(OP_CMP); return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { tick(OP_CMP); return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { tick(OP_CMP); return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { tick(OP_CMP); return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { tick(OP_CMP); return a.v != b.v; }
inline Counted sqrt(Counted a) { tick(OP_SQRT); return Counted(std::sqrt(a.v)); }
inline Counted pow(Counted a, Counted b) { tick(OP_POW); return Counted(std::pow(a.v, b.v)); }
inline Counted fabs(Counted a) { tick(OP_CMP); return Counted(std::fabs(a.v)); }
inline Counted fmax(Counted a, Counted b) { tick(OP_CMP); return Counted(std::fmax(a.v, b.v)); }
inline Counted fmin(Counted a, Counted b) { tick(OP_CMP); return Counted(std::fmin(a.v, b.v)); }
inline bool isnan_r(Counted a) { return std::isnan(a.v); }
inline double value(Counted a) { return a.v; }

// Plain double: the same names resolve to the C library.
using std::sqrt;
using std::pow;
using std::fabs;
using std::fmax;
using std::fmin;
inline bool isnan_r(double a) { return std::isnan(a); }
inline double value(double a) { return a; }

// Section scopes only cost anything for the Counted instantiation.
template <class R> struct Sec { explicit Sec(int) {} };
template <> struct Sec<Counted> : SectionScope { explicit Sec(int s) : SectionScope(s) {} };

}  // namespace orc
