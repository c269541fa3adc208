// Per-group context of the persistent patch-group kernels (Sec. 3.1: one
// thread block per patch group; here a persistent loop of each CTA over a
// flat list of groups that may span several AMR levels or boxes).
#pragma once
#include "phys.cuh"

namespace hyd {

constexpr int MAX_SEG = 32;  // == HYDRO_MAX_LEVELS

// One entry of the work list (a level, a box or a plain group batch).
struct SegDesc {
  const void* in;       // mode 0: groups [G][5][M^3]; mode 1: field [5][Z][Y][X]
  void* out;            // mode 0: groups [G][5][N^3]; mode 1: field
  void* flux;           // [G][6][5][N][N] or null
  unsigned* status;     // [G] or null
  const double* dt_dev; // optional device dt
  double dt;
  double dx[3];
  int G, mode, bc, X, Y, Z, GX, GY, GZ;
  int gz0;              // mode 1: first group layer of the entry (its GZ layers follow)
  int lc;               // mode 1: z-segment length of the work order; mode 0: longest chain (1..CHAIN_MAX)
  const int* zrun;      // mode 0: [G] groups from g on that continue one another along z, or null
  int first;            // flat index of this entry's first group
};

// Position of work item gi of a mode-1 entry.  Order: z-segments of lc
// group layers (the last one GZ % lc layers if that is not 0), all columns'
// segment s before any segment s+1; within a segment column by column, z
// fastest.  col = gx + GX gy; gz relative to the entry; left = items to the
// end of the segment (the longest chain that may start at gi).
struct SegPos {
  int col, gz, left;
};
__device__ __forceinline__ SegPos seg_pos(const SegDesc& sg, int gi) {
  const int ncol = sg.GX * sg.GY;
  const int lc = sg.lc;
  const int full = sg.GZ / lc;
  const int nfull = full * ncol * lc;
  SegPos p;
  if (gi < nfull) {
    const int zs = gi / (ncol * lc);
    const int r = gi - zs * ncol * lc;
    p.col = r / lc;
    const int zi = r - p.col * lc;
    p.gz = zs * lc + zi;
    p.left = lc - zi;
  } else {
    const int rem = sg.GZ - full * lc;
    const int r = gi - nfull;
    p.col = r / rem;
    const int zi = r - p.col * rem;
    p.gz = full * lc + zi;
    p.left = rem - zi;
  }
  return p;
}

// Longest run of z-consecutive groups of a uniform field that one CTA streams
// through without restarting (the ring buffers carry over from one group to
// the next, so the ghost planes between them are traced once).
constexpr int CHAIN_MAX = 32;

struct WorkTable {
  int nseg;
  int total;
  SegDesc seg[MAX_SEG];
};

// Launch-wide constants.
struct KConst {
  double gamma, dens_floor, pres_floor, theta;
  int limiter, fallback, ghost, split_order;
  long long ring_elems;  // per-CTA scratch elements (global-memory rings)
};

// Addressing of one group's input / output and its step constants.  In a
// uniform field (mode 1) the context may cover a chain of groups stacked
// along z; plane z of the chain then belongs to group z / N of the chain.
//
// Work order: mode 0 entries in list order; mode 1 entries in z-segments
// (seg_pos), z fastest within a segment, so that consecutive work items are
// z-neighbours.  The user's group index (flux and status arrays) is
// x-fastest:
//   gu = gx + GX (gy + GY gz).
template <class T, class S, int N, bool GCH = false> struct GroupCtx {
  const S* in;
  S* out;
  S* flux;            // boundary fluxes of the chain's first group
  long long fstride;  // elements between the flux arrays of chain groups
  int gu, ustride;    // user index of the first group; step between chain groups
  int mode, bc, g, M;
  int kmax;  // mode 0: last group of the chain (K - 1)
  long long Mpl;  // M*M
  int X, Y, Z, ox, oy, oz;
  long long XYZ;
  T dtdx[3], hdtdx[3];

  // sc[0..2] = dt/dx_d, sc[3..5] = (0.5 dt)/dx_d, evaluated once per group
  // (group_consts) and shared by the CTA.
  __device__ __forceinline__ void init(const SegDesc& sg, int gi, const KConst& kc, const double* sc, int K = 1) {
    mode = sg.mode;
    kmax = K - 1;
    g = kc.ghost;
    M = N + 2 * g;
    Mpl = (long long)M * M;
    for (int d = 0; d < 3; ++d) {
      dtdx[d] = (T)sc[d];
      hdtdx[d] = (T)sc[3 + d];
    }
    if (mode == 0) {
      in = (const S*)sg.in + (long long)gi * 5 * Mpl * M;
      out = (S*)sg.out + (long long)gi * 5 * N * N * N;
      bc = 0;
      gu = gi;
      ustride = 1;
    } else {
      in = (const S*)sg.in;
      out = (S*)sg.out;
      bc = sg.bc;
      X = sg.X;
      Y = sg.Y;
      Z = sg.Z;
      XYZ = (long long)X * Y * Z;
      const SegPos sp = seg_pos(sg, gi);
      int gz = sg.gz0 + sp.gz;
      int col = sp.col;
      int gx = col % sg.GX;
      int gy = col / sg.GX;
      ox = gx * N;
      oy = gy * N;
      oz = gz * N;
      gu = gx + sg.GX * (gy + sg.GY * gz);
      ustride = sg.GX * sg.GY;
    }
    fstride = (long long)ustride * 30 * N * N;
    flux = sg.flux ? (S*)sg.flux + (long long)gu * 30 * N * N : nullptr;
  }
  // User index of group k of the chain.
  __device__ __forceinline__ int user_index(int k) const { return gu + k * ustride; }

  // Box-edge index map for -n <= a < 2n (ghost width <= box size): periodic
  // wrap or outflow clamp.
  __device__ __forceinline__ static int wrap(int a, int n, int bc) {
    if (bc == 0) {
      a = a < 0 ? a + n : a;
      return a >= n ? a - n : a;
    }
    return a < 0 ? 0 : (a >= n ? n - 1 : a);
  }

  // Mode 0 chains (GCH: kernels that stream gathered groups as chains): plane
  // z of a chain of K gathered groups (z-consecutive, ghost zones agreeing
  // with each other's interiors) is read from group k = clamp(floor(z / N),
  // 0, K-1) at its local plane z - kN, so the planes between two groups come
  // from interiors and the ghost planes only from the first group's bottom
  // and the last group's top.  The group's input array starts at
  // in + 5 M^3 k; on return z is the local plane.  Without GCH every chain
  // is one group and the array is in.
  __device__ __forceinline__ const S* gin(int& z) const {
    if constexpr (!GCH) return in;
    int k = z < 0 ? 0 : z / N;
    k = k < kmax ? k : kmax;
    z -= k * N;
    return in + (long long)k * 5 * Mpl * M;
  }

  // Input value of variable v at interior coordinates (x, y, z), which may lie
  // in the ghost zone (-g <= x < N + g).
  __device__ __forceinline__ T load(int v, int x, int y, int z) const {
    if (mode == 0) {
      const S* b = gin(z);
      return (T)b[v * Mpl * M + ((long long)(z + g) * M + (y + g)) * M + (x + g)];
    }
    int sx = wrap(ox + x, X, bc), sy = wrap(oy + y, Y, bc), sz = wrap(oz + z, Z, bc);
    return (T)in[v * XYZ + ((long long)sz * Y + sy) * X + sx];
  }
  // All five variables at (x, y, z) (ghost zone allowed).
  __device__ __forceinline__ void load5(int x, int y, int z, T U[5]) const {
    if (mode == 0) {
      const S* p = gin(z);
      p += ((long long)(z + g) * M + (y + g)) * M + (x + g);
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = (T)p[v * Mpl * M];
    } else {
      int sx = wrap(ox + x, X, bc), sy = wrap(oy + y, Y, bc), sz = wrap(oz + z, Z, bc);
      const S* p = in + ((long long)sz * Y + sy) * X + sx;
#pragma unroll
      for (int v = 0; v < 5; ++v) U[v] = (T)p[v * XYZ];
    }
  }
  // Address of variable 0 at (x, y, z) (ghost zone allowed, box edges
  // wrapped or clamped as in load5) and the stride between variables.
  __device__ __forceinline__ const S* src5(int x, int y, int z, long long& vstride) const {
    if (mode == 0) {
      vstride = Mpl * M;
      const S* b = gin(z);
      return b + ((long long)(z + g) * M + (y + g)) * M + (x + g);
    }
    int sx = wrap(ox + x, X, bc), sy = wrap(oy + y, Y, bc), sz = wrap(oz + z, Z, bc);
    vstride = XYZ;
    return in + ((long long)sz * Y + sy) * X + sx;
  }
  // Interior values (0 <= z < K N).
  __device__ __forceinline__ S load_raw(int v, int x, int y, int z) const {
    if (mode == 0) {
      const S* b = gin(z);
      return b[v * Mpl * M + ((long long)(z + g) * M + (y + g)) * M + (x + g)];
    }
    return in[v * XYZ + ((long long)(oz + z) * Y + (oy + y)) * X + (ox + x)];
  }
  __device__ __forceinline__ void store(int v, int x, int y, int z, S val) const {
    if (mode == 0) {
      const int k = GCH ? z / N : 0;
      z -= k * N;
      out[(long long)(5 * k + v) * N * N * N + (z * N + y) * N + x] = val;
    } else {
      out[v * XYZ + ((long long)(oz + z) * Y + (oy + y)) * X + (ox + x)] = val;
    }
  }
  // Boundary flux of face f (0..5) of chain group k at transverse indices
  // (a, b).
  __device__ __forceinline__ void store_flux(int k, int f, int v, int a, int b, T val) const {
    if (flux) flux[k * fstride + ((f * 5 + v) * N + a) * N + b] = (S)val;
  }
};

// Step constants of one group, computed by one thread.
__device__ __forceinline__ void group_consts(const SegDesc& sg, double* sc) {
  double dt = sg.dt_dev ? *sg.dt_dev : sg.dt;
  for (int d = 0; d < 3; ++d) {
    sc[d] = dt / sg.dx[d];
    sc[3 + d] = 0.5 * dt / sg.dx[d];
  }
}

// ORs the status bits s into every group k < K of a chain whose own
// (unchained) computation covers plane p, i.e. kN + lo <= p <= kN + N-1 + hi
// (the caller guarantees p >= lo).  A group's status thus holds the same bits
// whether it is advanced alone or inside a chain.
template <int N>
__device__ __forceinline__ void mark_status(unsigned* sts, int K, int p, int lo, int hi, unsigned s) {
  if (!s) return;
  int k = (p - lo) / N;
  if (k > K - 1) k = K - 1;
  for (; k >= 0 && p <= k * N + N - 1 + hi; --k) atomicOr(&sts[k], s);
}

// Slot of plane p in a ring of R planes (p >= -8).
template <int R> __device__ __forceinline__ int slot(int p) { return (p + 8 * R) % R; }

// Conservative update of one interior cell (step (4)) from the face flux
// differences dF[d][v] = F(c + e_d/2) - F(c - e_d/2):
//   U_new = U - ((dtdx0 dF0 + dtdx1 dF1) + dtdx2 dF2);
// sets the status bits of the new state.
template <class T> __device__ __forceinline__ unsigned state_status(const T Un[5], const Gas<T>& gas);

// U0 holds U^n of the cell (already read from the input).  The sum is
// evaluated in the arithmetic type for every form: the result is rounded to
// the storage type, so an FP64 sum would change the stored FP32 value by less
// than one unit in the last place.
template <class T, class S, bool MIXED, int N, bool GCH>
__device__ __forceinline__ unsigned update_cell_from(const GroupCtx<T, S, N, GCH>& C, int x, int y, int z, const T U0[5],
                                                     const T dF[3][5], const Gas<T>& gas) {
  T Un[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T dU = C.dtdx[0] * dF[0][v] + C.dtdx[1] * dF[1][v] + C.dtdx[2] * dF[2][v];
    Un[v] = U0[v] - dU;
    C.store(v, x, y, z, (S)Un[v]);
  }
  return state_status(Un, gas);
}

// Status bits of an updated state: NaN, density <= 0, pressure <= 0.
template <class T> __device__ __forceinline__ unsigned state_status(const T Un[5], const Gas<T>& gas) {
  unsigned st = 0;
  bool nan = false;
#pragma unroll
  for (int v = 0; v < 5; ++v) nan = nan || isnanv(Un[v]);
  if (nan) st |= ST_NAN;
  if (!(Un[0] > T(0))) {
    st |= ST_NEG_DENS;
  } else {
    T p = gas.gm1 * (Un[4] - divv(T(0.5) * (Un[1] * Un[1] + Un[2] * Un[2] + Un[3] * Un[3]), Un[0]));
    if (!(p > T(0))) st |= ST_NEG_PRES;
  }
  return st;
}

template <class T, class S, bool MIXED, int N, bool GCH>
__device__ __forceinline__ unsigned update_cell(const GroupCtx<T, S, N, GCH>& C, int x, int y, int z, const T dF[3][5],
                                                const Gas<T>& gas) {
  T U0[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) U0[v] = (T)C.load_raw(v, x, y, z);
  return update_cell_from<T, S, MIXED, N>(C, x, y, z, U0, dF, gas);
}

}  // namespace hyd
