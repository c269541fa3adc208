// AMR level operations on the device (declared in include/hydro_amr.h):
// group maps, ghost-zone preparation by copy or spatial + temporal
// interpolation (Sec. 4.2), coarse-grid correction by the stored boundary
// fluxes (Sec. 2 step (5), Sec. 4.3) and restriction.
//
// All three data kernels are bound by memory traffic, not arithmetic:
//   prepare   one CTA per group, one thread per (x, y) column of the padded
//             group walking along z: per cell a map lookup, then 5 loads
//             (copy) or 7 x 5 (x2 with time interpolation) loads of parent
//             cells that neighbouring threads share through L1/L2;
//   reflux    one CTA per coarse group; only groups next to a refined one do
//             any work, one thread per cell of their boundary shell;
//   restrict  one thread per coarse cell under a fine group: 8 x 5 loads,
//             5 stores.
// The arithmetic follows the operation order stated in the header, in the
// storage type; this unit is built with -fmad=false, so FP64 results equal
// a plain FP64 evaluation of the same expressions.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/hydro_amr.h"

namespace hyd {
int record_cuda_error(cudaError_t e);
}

namespace {

constexpr int AN = 16;  // group edge (the only size built)
constexpr int AMR_THREADS = 256;
constexpr int AMR_PREP_THREADS = 512;  // >= (N + 2 ghost)^2 for ghost <= 3

struct LevelView {
  const void* U;
  const int* origin;
  const int* map;
  int G, X, Y, Z;
};

LevelView view(const hydro_amr_level* l) {
  LevelView v;
  v.U = l ? l->U : nullptr;
  v.origin = l ? l->origin : nullptr;
  v.map = l ? l->map : nullptr;
  v.G = l ? l->G : 0;
  v.X = l ? l->X : 0;
  v.Y = l ? l->Y : 0;
  v.Z = l ? l->Z : 0;
  return v;
}

__device__ __forceinline__ void raise_err(unsigned* err, unsigned bit) {
  if (err) atomicOr(err, bit);
}

// Box-edge map of a cell coordinate within one box length of the box.
__device__ __forceinline__ int amr_cell(int a, int n, int bc) {
  if (bc == HYDRO_BC_PERIODIC) {
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
  }
  return a < 0 ? 0 : (a >= n ? n - 1 : a);
}

// Group index of the level at in-box cell (x, y, z), -1 if none (a map
// entry outside [0, G) counts as none).
__device__ __forceinline__ int group_at(const LevelView& L, int x, int y, int z) {
  const int g = L.map[((long long)(z / AN) * (L.Y / AN) + y / AN) * (L.X / AN) + x / AN];
  return g < L.G ? g : -1;
}

// Origin of group k is a multiple of AN inside the level's box.
__device__ __forceinline__ bool origin_ok(const LevelView& L, int k) {
  const int x = L.origin[3 * k], y = L.origin[3 * k + 1], z = L.origin[3 * k + 2];
  return x >= 0 && y >= 0 && z >= 0 && x <= L.X - AN && y <= L.Y - AN && z <= L.Z - AN && x % AN == 0 &&
         y % AN == 0 && z % AN == 0;
}

template <class S> __device__ __forceinline__ S minmod(S a, S b) {
  return a * b > S(0) ? copysign(fmin(fabs(a), fabs(b)), a) : S(0);
}

// Parent state at in-box coarse cell (x, y, z) at time theta of its step.
template <class S>
__device__ __forceinline__ bool parent_at(const LevelView& C, const S* cnew, S theta, int x, int y, int z, S u[5]) {
  const int q = group_at(C, x, y, z);
  if (q < 0) return false;
  constexpr long long N3 = (long long)AN * AN * AN;
  const long long o = (long long)q * 5 * N3 + ((z % AN) * AN + y % AN) * AN + x % AN;
  const S* U0 = (const S*)C.U;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    S u0 = U0[o + v * N3];
    if (cnew) {
      S u1 = cnew[o + v * N3];
      u0 = u0 + theta * (u1 - u0);
    }
    u[v] = u0;
  }
  return true;
}

__global__ void amr_map_kernel(const int* __restrict__ origin, int G, int X, int Y, int Z, int* map,
                               unsigned* err) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < G; k += gridDim.x * blockDim.x) {
    int x = origin[3 * k], y = origin[3 * k + 1], z = origin[3 * k + 2];
    if (x < 0 || y < 0 || z < 0 || x >= X || y >= Y || z >= Z || x % AN || y % AN || z % AN) {
      raise_err(err, HYDRO_AMR_ENESTING);
      continue;
    }
    int prev = atomicExch(&map[((long long)(z / AN) * (Y / AN) + y / AN) * (X / AN) + x / AN], k);
    if (prev != -1) raise_err(err, HYDRO_AMR_EDUPLICATE);
  }
}

// One padded cell (a, b, c) of group k of F: a copy from F's group at that
// fine cell, else the prolongation ((Uc + qx) + qy) + qz from the parent C
// at time theta; NaN and HYDRO_AMR_ENESTING where neither level has it.
template <class S>
__device__ __forceinline__ void prepare_cell(const LevelView& F, const LevelView& C, const S* __restrict__ cnew,
                                             S theta, int bc, int ghost, int k, int a, int b, int c,
                                             S* __restrict__ o, long long M3, unsigned* err) {
  constexpr long long N3 = (long long)AN * AN * AN;
  const int fx = amr_cell(F.origin[3 * k] + a - ghost, F.X, bc);
  const int fy = amr_cell(F.origin[3 * k + 1] + b - ghost, F.Y, bc);
  const int fz = amr_cell(F.origin[3 * k + 2] + c - ghost, F.Z, bc);
  const int g = group_at(F, fx, fy, fz);
  if (g >= 0) {
    const S* s = (const S*)F.U + (long long)g * 5 * N3 + ((fz % AN) * AN + fy % AN) * AN + fx % AN;
#pragma unroll
    for (int v = 0; v < 5; ++v) o[v * M3] = s[v * N3];
    return;
  }
  S uc[5], acc[5];
  bool ok = C.U != nullptr && parent_at(C, cnew, theta, fx >> 1, fy >> 1, fz >> 1, uc);
  if (ok) {
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = uc[v];
    const int cc[3] = {fx >> 1, fy >> 1, fz >> 1};
    const int fc[3] = {fx, fy, fz};
    const int nc[3] = {F.X / 2, F.Y / 2, F.Z / 2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int up[3] = {cc[0], cc[1], cc[2]}, dn[3] = {cc[0], cc[1], cc[2]};
      up[d] = amr_cell(cc[d] + 1, nc[d], bc);
      dn[d] = amr_cell(cc[d] - 1, nc[d], bc);
      S uu[5], ud[5];
      ok = ok && parent_at(C, cnew, theta, up[0], up[1], up[2], uu) &&
           parent_at(C, cnew, theta, dn[0], dn[1], dn[2], ud);
      if (!ok) break;
      const S q = (fc[d] & 1) ? S(0.25) : S(-0.25);
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = acc[v] + q * minmod(uu[v] - uc[v], uc[v] - ud[v]);
    }
  }
  if (!ok) {
    raise_err(err, HYDRO_AMR_ENESTING);
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] = S(NAN);
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) o[v * M3] = acc[v];
}

// Halo-padded input of every group of F.  CTA k fills group k; each thread
// owns one (x, y) column of the padded group and walks it along z (MG = N + 2
// ghost known at compile time, so the index arithmetic is by constants; MG = 0
// reads the ghost width at run time).
template <class S, int MG>
__global__ void __launch_bounds__(AMR_PREP_THREADS)
    amr_prepare_kernel(LevelView F, LevelView C, const S* __restrict__ cnew, S theta, int bc, int ghost,
                       S* __restrict__ out, unsigned* err) {
  const int M = MG ? MG : AN + 2 * ghost;
  const int g = MG ? (MG - AN) / 2 : ghost;
  const long long M3 = (long long)M * M * M;
  for (int k = blockIdx.x; k < F.G; k += gridDim.x) {
    S* base = out + (long long)k * 5 * M3;
    if (!origin_ok(F, k)) {
      if (threadIdx.x == 0) raise_err(err, HYDRO_AMR_ENESTING);
      for (long long r = threadIdx.x; r < M3; r += blockDim.x)
#pragma unroll
        for (int v = 0; v < 5; ++v) base[v * M3 + r] = S(NAN);
      continue;
    }
    for (int r = threadIdx.x; r < M * M; r += blockDim.x) {
      const int b = r / M, a = r - b * M;
      for (int c = 0; c < M; ++c)
        prepare_cell<S>(F, C, cnew, theta, bc, g, k, a, b, c, base + (long long)c * M * M + r, M3, err);
    }
  }
}

// Coarse window a fine group's padded region (ghost G) and its
// interpolation stencil need: cells o/2 - LO_OFF + [0, CB) per axis.
template <int G> struct StageBox {
  static constexpr int LO_OFF = (G + 1) / 2 + 1;
  static constexpr int CB = AN / 2 + (G - 1) / 2 + (G + 1) / 2 + 3;
  static constexpr int CB3 = CB * CB * CB;
};

// Halo-padded input of every group of F, parents staged in shared memory.
// CTA k fills group k.  If every padded cell lies in a group of F (the 26
// neighbour slots are all present) the group is copied; otherwise the
// parent cells of its padded region and their stencil (the StageBox window,
// at time theta) are first staged in shared memory, each from its wrapped /
// clamped coarse cell, and the cells outside F interpolate from there:
// ((Uc + qx) + qy) + qz with the same operations and order as prepare_cell.
// Indexing the window by the unwrapped fine coordinate gives the same parent
// and neighbours as the wrapped one (periodic); at an outflow edge both give
// a zero slope along the clamped axis.
template <class S, int G>
__global__ void __launch_bounds__(AMR_PREP_THREADS, 2)
    amr_prepare_staged(LevelView F, LevelView C, const S* __restrict__ cnew, S theta, int bc, S* __restrict__ out,
                       unsigned* err) {
  constexpr int M = AN + 2 * G;
  constexpr long long M3 = (long long)M * M * M;
  constexpr long long N3 = (long long)AN * AN * AN;
  constexpr int CB = StageBox<G>::CB, CB3 = StageBox<G>::CB3, LO = StageBox<G>::LO_OFF;
  extern __shared__ __align__(16) unsigned char smraw[];
  S* cs = reinterpret_cast<S*>(smraw);  // [5][CB3] parent values at time theta
  unsigned char* okp = smraw + (size_t)5 * CB3 * sizeof(S);
  __shared__ int need;
  const S* Uf = (const S*)F.U;
  for (int k = blockIdx.x; k < F.G; k += gridDim.x) {
    S* base = out + (long long)k * 5 * M3;
    if (!origin_ok(F, k)) {  // uniform across the CTA
      if (threadIdx.x == 0) raise_err(err, HYDRO_AMR_ENESTING);
      for (long long r = threadIdx.x; r < M3; r += blockDim.x)
#pragma unroll
        for (int v = 0; v < 5; ++v) base[v * M3 + r] = S(NAN);
      continue;
    }
    const int ox = F.origin[3 * k], oy = F.origin[3 * k + 1], oz = F.origin[3 * k + 2];
    if (threadIdx.x == 0) need = 0;
    __syncthreads();
    if (threadIdx.x < 27) {
      const int sx = threadIdx.x % 3 - 1, sy = (threadIdx.x / 3) % 3 - 1, sz = threadIdx.x / 9 - 1;
      const int fx = amr_cell(ox + (sx < 0 ? -1 : (sx > 0 ? AN : 0)), F.X, bc);
      const int fy = amr_cell(oy + (sy < 0 ? -1 : (sy > 0 ? AN : 0)), F.Y, bc);
      const int fz = amr_cell(oz + (sz < 0 ? -1 : (sz > 0 ? AN : 0)), F.Z, bc);
      if (group_at(F, fx, fy, fz) < 0) atomicOr(&need, 1);
    }
    __syncthreads();
    const int cx0 = (ox >> 1) - LO, cy0 = (oy >> 1) - LO, cz0 = (oz >> 1) - LO;
    if (need) {
      for (int idx = threadIdx.x; idx < CB3; idx += blockDim.x) {
        const int i = idx % CB, j = (idx / CB) % CB, l = idx / (CB * CB);
        S u[5];
        const bool present = C.U != nullptr && parent_at(C, cnew, theta, amr_cell(cx0 + i, F.X / 2, bc),
                                                         amr_cell(cy0 + j, F.Y / 2, bc),
                                                         amr_cell(cz0 + l, F.Z / 2, bc), u);
        okp[idx] = present ? 1 : 0;
#pragma unroll
        for (int v = 0; v < 5; ++v) cs[v * CB3 + idx] = present ? u[v] : S(0);
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < M * M; r += blockDim.x) {
      const int b = r / M, a = r - b * M;
      const int fu = ox + a - G, fv = oy + b - G;  // unwrapped fine x, y
      const int fx = amr_cell(fu, F.X, bc), fy = amr_cell(fv, F.Y, bc);
      // the column's fine cells lie in at most three groups of the level:
      // below the group (c < G), beside it (G <= c < G + AN), above it
      int gseg[3];
#pragma unroll
      for (int s = 0; s < 3; ++s)
        gseg[s] = group_at(F, fx, fy, amr_cell(oz + (s == 0 ? -1 : (s == 1 ? 0 : AN)), F.Z, bc));
      const long long xy = (long long)(fy % AN) * AN + fx % AN;
      // CU cells at a time: every load of the batch is issued before its stores
      constexpr int CU = sizeof(S) == 4 ? 4 : 2;
      for (int c0 = 0; c0 < M; c0 += CU) {
        S val[CU][5];
#pragma unroll
        for (int q = 0; q < CU; ++q) {
          const int c = c0 + q;
          if (c >= M) break;
          const int fw = oz + c - G;
          const int fz = amr_cell(fw, F.Z, bc);
          const int g = gseg[c < G ? 0 : (c < G + AN ? 1 : 2)];
          if (g >= 0) {
            const S* s = Uf + (long long)g * 5 * N3 + (long long)(fz % AN) * AN * AN + xy;
#pragma unroll
            for (int v = 0; v < 5; ++v) val[q][v] = s[v * N3];
            continue;
          }
          const int ci = (fu >> 1) - cx0, cj = (fv >> 1) - cy0, ck = (fw >> 1) - cz0;  // 1 .. CB-2
          const int idx = (ck * CB + cj) * CB + ci;
          const int st[3] = {1, CB, CB * CB};
          bool ok = okp[idx] != 0;
#pragma unroll
          for (int d = 0; d < 3; ++d) ok = ok && okp[idx + st[d]] != 0 && okp[idx - st[d]] != 0;
          if (ok) {
            const int fc[3] = {fx, fy, fz};
#pragma unroll
            for (int v = 0; v < 5; ++v) val[q][v] = cs[v * CB3 + idx];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const S h = (fc[d] & 1) ? S(0.25) : S(-0.25);
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                const S uc = cs[v * CB3 + idx];
                const S uu = cs[v * CB3 + idx + st[d]];
                const S ud = cs[v * CB3 + idx - st[d]];
                val[q][v] = val[q][v] + h * minmod(uu - uc, uc - ud);
              }
            }
          } else {
            raise_err(err, HYDRO_AMR_ENESTING);
#pragma unroll
            for (int v = 0; v < 5; ++v) val[q][v] = S(NAN);
          }
        }
#pragma unroll
        for (int q = 0; q < CU; ++q) {
          const int c = c0 + q;
          if (c >= M) break;
          S* o = base + (long long)c * M * M + r;
#pragma unroll
          for (int v = 0; v < 5; ++v) o[v * M3] = val[q][v];
        }
      }
    }
    __syncthreads();  // the window is reused by the CTA's next group
  }
}

template <class S, int G>
cudaError_t launch_staged(const LevelView& F, const LevelView& C, const S* cnew, S theta, int bc, S* out,
                          unsigned* err, cudaStream_t st) {
  const size_t smem = (size_t)5 * StageBox<G>::CB3 * sizeof(S) + StageBox<G>::CB3;
  cudaError_t e = cudaFuncSetAttribute(amr_prepare_staged<S, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = F.G < (1 << 20) ? F.G : (1 << 20);
  amr_prepare_staged<S, G><<<grid, AMR_PREP_THREADS, smem, st>>>(F, C, cnew, theta, bc, out, err);
  return cudaSuccess;
}

template <class S>
cudaError_t launch_prepare(const LevelView& F, const LevelView& C, const S* cnew, S theta, int bc, int ghost,
                           S* out, unsigned* err, cudaStream_t st) {
  switch (ghost) {
    case 1: return launch_staged<S, 1>(F, C, cnew, theta, bc, out, err, st);
    case 2: return launch_staged<S, 2>(F, C, cnew, theta, bc, out, err, st);
    case 3: return launch_staged<S, 3>(F, C, cnew, theta, bc, out, err, st);
    case 4: return launch_staged<S, 4>(F, C, cnew, theta, bc, out, err, st);
    default: {
      const int grid = F.G < (1 << 20) ? F.G : (1 << 20);
      amr_prepare_kernel<S, 0><<<grid, AMR_PREP_THREADS, 0, st>>>(F, C, cnew, theta, bc, ghost, out, err);
      return cudaSuccess;
    }
  }
}

// Coarse-grid correction: CTA q handles coarse group q of C (corrected in
// place in Uc); faces -x,+x,-y,+y,-z,+z in order per cell, one face of the
// group at a time.
template <class S>
__global__ void __launch_bounds__(AMR_THREADS)
    amr_reflux_kernel(LevelView C, S* __restrict__ Uc, const S* __restrict__ cflux, LevelView F,
                      const S* __restrict__ ff0, const S* __restrict__ ff1, S h0, S h1, S h2, int bc,
                      unsigned* err) {
  constexpr int NN = AN * AN;
  constexpr long long N3 = (long long)AN * AN * AN;
  __shared__ int on[6];
  __shared__ int nbs[6];  // neighbour slot along the face's axis
  const int GXc = C.X / AN, GYc = C.Y / AN, GZc = C.Z / AN;
  const int gn[3] = {GXc, GYc, GZc};
  for (int q = blockIdx.x; q < C.G; q += gridDim.x) {
    if (!origin_ok(C, q)) {  // uniform across the CTA
      if (threadIdx.x == 0) raise_err(err, HYDRO_AMR_ENESTING);
      continue;
    }
    const int o[3] = {C.origin[3 * q], C.origin[3 * q + 1], C.origin[3 * q + 2]};
    const int s[3] = {o[0] / AN, o[1] / AN, o[2] / AN};
    if (threadIdx.x == 0) {
      auto refined = [&](int sx, int sy, int sz) {
        return F.map[((long long)(2 * sz) * (F.Y / AN) + 2 * sy) * (F.X / AN) + 2 * sx] >= 0;
      };
      const bool self = refined(s[0], s[1], s[2]);
      for (int f = 0; f < 6; ++f) {
        const int d = f >> 1, side = f & 1;
        int nb[3] = {s[0], s[1], s[2]};
        nb[d] += side ? 1 : -1;
        bool valid = true;
        if (bc == HYDRO_BC_PERIODIC) {
          nb[d] = nb[d] < 0 ? nb[d] + gn[d] : (nb[d] >= gn[d] ? nb[d] - gn[d] : nb[d]);
        } else if (nb[d] < 0 || nb[d] >= gn[d]) {
          valid = false;
        }
        on[f] = !self && valid && refined(nb[0], nb[1], nb[2]);
        nbs[f] = nb[d];
      }
    }
    __syncthreads();
    const bool any = on[0] || on[1] || on[2] || on[3] || on[4] || on[5];
    if (any) {
      // one face at a time, -x,+x,-y,+y,-z,+z, its N^2 cells spread over the
      // CTA: a cell on an edge or a corner takes its faces' corrections in
      // that order, each read back from memory (same rounding as applying
      // them one after another in registers)
      for (int f = 0; f < 6; ++f) {
        if (!on[f]) continue;  // uniform across the CTA
        const int d = f >> 1, side = f & 1;
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        const int ffc = 2 * d + (side ? 0 : 1);
        const S sg = side ? S(-1) : S(1);
        const S h = d == 0 ? h0 : (d == 1 ? h1 : h2);
        for (int ab = threadIdx.x; ab < NN; ab += blockDim.x) {
          const int a = ab / AN, b = ab - a * AN;  // along t2, along t1
          int l[3];
          l[d] = side ? AN - 1 : 0;
          l[t2] = a;
          l[t1] = b;
          const long long cell = ((long long)l[2] * AN + l[1]) * AN + l[0];
          // fine cells across the face and their face toward this cell
          int fc[3];
          fc[d] = 2 * nbs[f] * AN + (side ? 0 : 2 * AN - 1);
          fc[t2] = 2 * (o[t2] + a);
          fc[t1] = 2 * (o[t1] + b);
          const int k = group_at(F, fc[0], fc[1], fc[2]);
          if (k < 0) {
            raise_err(err, HYDRO_AMR_EOCTET);
            continue;
          }
          const int a0 = fc[t2] % AN, b0 = fc[t1] % AN;
          S* uc = Uc + (long long)q * 5 * N3 + cell;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const S Fc = cflux[(((long long)q * 6 + f) * 5 + v) * NN + a * AN + b];
            const long long fb = (((long long)k * 6 + ffc) * 5 + v) * NN;
            const S* p0 = ff0 + fb;
            const S* p1 = ff1 + fb;
            S s0 = p0[a0 * AN + b0] + p0[a0 * AN + b0 + 1];
            s0 = s0 + p0[(a0 + 1) * AN + b0];
            s0 = s0 + p0[(a0 + 1) * AN + b0 + 1];
            S s1 = p1[a0 * AN + b0] + p1[a0 * AN + b0 + 1];
            s1 = s1 + p1[(a0 + 1) * AN + b0];
            s1 = s1 + p1[(a0 + 1) * AN + b0 + 1];
            const S Fbar = S(0.125) * (s0 + s1);
            uc[v * N3] = uc[v * N3] + sg * (h * (Fbar - Fc));
          }
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

// Restriction: one thread per coarse cell under a fine group.
template <class S>
__global__ void __launch_bounds__(AMR_THREADS)
    amr_restrict_kernel(LevelView F, LevelView C, S* __restrict__ Uc, unsigned* err) {
  constexpr int H = AN / 2;
  constexpr long long N3 = (long long)AN * AN * AN;
  const long long total = (long long)F.G * H * H * H;
  const S* Uf = (const S*)F.U;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / (H * H * H));
    const int r = (int)(e - (long long)k * H * H * H);
    const int i = r % H, j = (r / H) % H, l = r / (H * H);
    if (!origin_ok(F, k)) {
      raise_err(err, HYDRO_AMR_ENESTING);
      continue;
    }
    const int cx0 = F.origin[3 * k] / 2, cy0 = F.origin[3 * k + 1] / 2, cz0 = F.origin[3 * k + 2] / 2;
    const int q = group_at(C, cx0, cy0, cz0);
    if (q < 0) {
      raise_err(err, HYDRO_AMR_ENESTING);
      continue;
    }
    const int ox = cx0 - C.origin[3 * q], oy = cy0 - C.origin[3 * q + 1], oz = cz0 - C.origin[3 * q + 2];
    if (ox < 0 || oy < 0 || oz < 0 || ox > AN - H || oy > AN - H || oz > AN - H) {  // map and origins disagree
      raise_err(err, HYDRO_AMR_ENESTING);
      continue;
    }
    const S* f = Uf + (long long)k * 5 * N3 + ((2 * l) * AN + 2 * j) * AN + 2 * i;
    S* dst = Uc + (long long)q * 5 * N3 + ((oz + l) * AN + oy + j) * AN + ox + i;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const S* p = f + v * N3;
      S acc = p[0] + p[1];
      acc = acc + p[AN];
      acc = acc + p[AN + 1];
      acc = acc + p[AN * AN];
      acc = acc + p[AN * AN + 1];
      acc = acc + p[AN * AN + AN];
      acc = acc + p[AN * AN + AN + 1];
      dst[v * N3] = S(0.125) * acc;
    }
  }
}

bool box_ok(const hydro_amr_level* l) {
  return l && l->G >= 0 && l->X > 0 && l->Y > 0 && l->Z > 0 && l->X % AN == 0 && l->Y % AN == 0 &&
         l->Z % AN == 0 && (l->G == 0 || (l->U && l->origin && l->map));
}

int grid_for(long long work) {
  long long b = (work + AMR_THREADS - 1) / AMR_THREADS;
  if (b < 1) b = 1;
  return (int)(b > (1 << 20) ? (1 << 20) : b);
}

int launched() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HYDRO_OK : hyd::record_cuda_error(e);
}

bool pos_finite(double a) { return a > 0.0 && a < 1e300; }

}  // namespace

extern "C" {

int hydro_amr_map(const int* origin, int G, int X, int Y, int Z, int N, int* map, unsigned* dev_error,
                  void* stream) {
  if (N != AN) return HYDRO_EUNSUPPORTED;
  if (G < 0 || X <= 0 || Y <= 0 || Z <= 0 || X % N || Y % N || Z % N || !map || (G > 0 && !origin))
    return HYDRO_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  size_t slots = (size_t)(X / N) * (Y / N) * (Z / N);
  cudaError_t e = cudaMemsetAsync(map, 0xff, slots * sizeof(int), st);
  if (e != cudaSuccess) return hyd::record_cuda_error(e);
  if (G == 0) return HYDRO_OK;
  amr_map_kernel<<<grid_for(G), AMR_THREADS, 0, st>>>(origin, G, X, Y, Z, map, dev_error);
  return launched();
}

int hydro_amr_prepare(const hydro_amr_level* fine, const hydro_amr_level* coarse, const void* coarse_new,
                      double theta, int bc, int N, int ghost, int precision, void* U_out, unsigned* dev_error,
                      void* stream) {
  if (N != AN) return HYDRO_EUNSUPPORTED;
  if (!box_ok(fine) || (coarse && !box_ok(coarse))) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  if (precision < HYDRO_FP64 || precision > HYDRO_FP32_MIXED) return HYDRO_EINVAL;
  if (ghost < 0 || ghost > AN || !(theta >= 0.0 && theta <= 1.0)) return HYDRO_EINVAL;
  if (coarse && (coarse->X * 2 != fine->X || coarse->Y * 2 != fine->Y || coarse->Z * 2 != fine->Z))
    return HYDRO_EINVAL;
  if (coarse_new && !coarse) return HYDRO_EINVAL;
  if (fine->G == 0) return HYDRO_OK;
  if (!U_out) return HYDRO_EINVAL;
  LevelView F = view(fine), C = view(coarse);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e =
      precision == HYDRO_FP64
          ? launch_prepare<double>(F, C, (const double*)coarse_new, theta, bc, ghost, (double*)U_out, dev_error, st)
          : launch_prepare<float>(F, C, (const float*)coarse_new, (float)theta, bc, ghost, (float*)U_out, dev_error,
                                  st);
  if (e != cudaSuccess) return hyd::record_cuda_error(e);
  return launched();
}

int hydro_amr_reflux(const hydro_amr_level* coarse, const void* coarse_flux, const hydro_amr_level* fine,
                     const void* fine_flux0, const void* fine_flux1, double dt, const double* dx, int bc, int N,
                     int precision, unsigned* dev_error, void* stream) {
  if (N != AN) return HYDRO_EUNSUPPORTED;
  if (!box_ok(coarse) || !box_ok(fine) || !dx) return HYDRO_EINVAL;
  if (bc != HYDRO_BC_PERIODIC && bc != HYDRO_BC_OUTFLOW) return HYDRO_EINVAL;
  if (precision < HYDRO_FP64 || precision > HYDRO_FP32_MIXED) return HYDRO_EINVAL;
  if (coarse->X * 2 != fine->X || coarse->Y * 2 != fine->Y || coarse->Z * 2 != fine->Z) return HYDRO_EINVAL;
  if (!(dt >= 0.0)) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!pos_finite(dx[d])) return HYDRO_EINVAL;
  if (coarse->G == 0 || fine->G == 0) return HYDRO_OK;
  if (!coarse_flux || !fine_flux0 || !fine_flux1) return HYDRO_EINVAL;
  LevelView C = view(coarse), F = view(fine);
  cudaStream_t st = (cudaStream_t)stream;
  const double h0 = dt / dx[0], h1 = dt / dx[1], h2 = dt / dx[2];
  const int grid = coarse->G < 65535 ? coarse->G : 65535;
  if (precision == HYDRO_FP64)
    amr_reflux_kernel<double><<<grid, AMR_THREADS, 0, st>>>(
        C, (double*)coarse->U, (const double*)coarse_flux, F, (const double*)fine_flux0,
        (const double*)fine_flux1, h0, h1, h2, bc, dev_error);
  else
    amr_reflux_kernel<float><<<grid, AMR_THREADS, 0, st>>>(C, (float*)coarse->U, (const float*)coarse_flux, F,
                                                           (const float*)fine_flux0, (const float*)fine_flux1,
                                                           (float)h0, (float)h1, (float)h2, bc, dev_error);
  return launched();
}

int hydro_amr_restrict(const hydro_amr_level* fine, const hydro_amr_level* coarse, int N, int precision,
                       unsigned* dev_error, void* stream) {
  if (N != AN) return HYDRO_EUNSUPPORTED;
  if (!box_ok(coarse) || !box_ok(fine)) return HYDRO_EINVAL;
  if (precision < HYDRO_FP64 || precision > HYDRO_FP32_MIXED) return HYDRO_EINVAL;
  if (coarse->X * 2 != fine->X || coarse->Y * 2 != fine->Y || coarse->Z * 2 != fine->Z) return HYDRO_EINVAL;
  if (fine->G == 0) return HYDRO_OK;
  if (coarse->G == 0) return HYDRO_EINVAL;
  LevelView C = view(coarse), F = view(fine);
  cudaStream_t st = (cudaStream_t)stream;
  const long long total = (long long)fine->G * (N / 2) * (N / 2) * (N / 2);
  if (precision == HYDRO_FP64)
    amr_restrict_kernel<double><<<grid_for(total), AMR_THREADS, 0, st>>>(F, C, (double*)coarse->U, dev_error);
  else
    amr_restrict_kernel<float><<<grid_for(total), AMR_THREADS, 0, st>>>(F, C, (float*)coarse->U, dev_error);
  return launched();
}

}  // extern "C"
