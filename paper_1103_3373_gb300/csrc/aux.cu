// Auxiliary kernels of the hot path:
//   * ghost-zone gather of halo-padded groups from a uniform field (the
//     "preparation step" of Sec. 4.2, on the device);
//   * CFL time step (the evolution time step of Sec. 4.3) as a two-pass
//     max-reduction (per-cell speeds in the storage precision, maxima and the
//     final dt in FP64);
//   * FP64 totals of the conserved variables (conservation monitor).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hydro.h"
#include "phys.cuh"

namespace hyd {

// Gather: one thread per output element, written in output order (coalesced
// 128-bit-friendly stores; the reads hit mostly in L2 because neighbouring
// groups share their halos).
template <class S>
__global__ void gather_kernel(const S* __restrict__ field, int X, int Y, int Z, int bc,
                              const int* __restrict__ origin, int G, int N, int g, S* __restrict__ out) {
  const int M = N + 2 * g;
  const long long M3 = (long long)M * M * M;
  const long long per = 5 * M3;
  const long long total = per * G;
  const long long XYZ = (long long)X * Y * Z;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long gi = e / per;
    long long r = e - gi * per;
    int v = (int)(r / M3);
    r -= (long long)v * M3;
    int k = (int)(r / (M * M));
    int rem = (int)(r - (long long)k * M * M);
    int j = rem / M, i = rem - j * M;
    int sx = origin[3 * gi + 0] + i - g;
    int sy = origin[3 * gi + 1] + j - g;
    int sz = origin[3 * gi + 2] + k - g;
    if (bc == 0) {
      sx %= X; sx += sx < 0 ? X : 0;
      sy %= Y; sy += sy < 0 ? Y : 0;
      sz %= Z; sz += sz < 0 ? Z : 0;
    } else {
      sx = sx < 0 ? 0 : (sx >= X ? X - 1 : sx);
      sy = sy < 0 ? 0 : (sy >= Y ? Y - 1 : sy);
      sz = sz < 0 ? 0 : (sz >= Z ? Z - 1 : sz);
    }
    out[e] = field[v * XYZ + ((long long)sz * Y + sy) * X + sx];
  }
}

// Warp + block max of non-negative doubles.
__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Signal speed |v_d| + c of one cell (c = sqrt(gamma p / rho), primitives
// with floors) folded into the per-direction maxima m[d]; NaN sets bad.
template <class S>
__device__ __forceinline__ void fold_speed(const S u[5], const Gas<S>& gas, S m[3], bool& bad) {
  S w[5];
  prim<S, false>(u, w, gas);
  S c = sqrtv(gas.gamma * w[4] / w[0]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    S s = absv(w[1 + d]) + c;
    if (isnanv(s)) bad = true;
    m[d] = s > m[d] ? s : m[d];
  }
}

template <class S> struct Vec16;
template <> struct Vec16<float> {
  using V = float4;
  static constexpr int W = 4;
  __device__ __forceinline__ static void split(const V& a, float* o) {
    o[0] = a.x;
    o[1] = a.y;
    o[2] = a.z;
    o[3] = a.w;
  }
};
template <> struct Vec16<double> {
  using V = double2;
  static constexpr int W = 2;
  __device__ __forceinline__ static void split(const V& a, double* o) {
    o[0] = a.x;
    o[1] = a.y;
  }
};

// Pass 1: per CTA and direction d, the maximum over cells of |v_d| + c,
// evaluated in the storage precision and kept as FP64; part[d * gridDim.x + b].
// Division by dx_d comes once, in pass 2: max_cells((|v_d| + c) / dx_d) equals
// (max_cells(|v_d| + c)) / dx_d because rounded division by a positive number
// is monotone.  A NaN cell makes the CTA's partials NaN.  With VEC, each
// thread reads 16 bytes per variable (4 FP32 / 2 FP64 cells) per iteration,
// for more bytes in flight; the caller checks that cells, strides and base
// are multiples of that width.  The maxima do not depend on the grouping.
template <class S, bool VEC>
__global__ void cfl_partial_kernel(const S* __restrict__ U, int G, long long gstride, long long vstride,
                                   long long cells, double gamma, double dfloor, double pfloor,
                                   double* __restrict__ part) {
  __shared__ double sh[32];
  __shared__ int anybad;
  if (threadIdx.x == 0) anybad = 0;
  S m[3] = {S(0), S(0), S(0)};
  bool bad = false;
  Gas<S> gas{(S)gamma, (S)(gamma - 1.0), (S)dfloor, (S)pfloor, (S)(1.0 / (gamma - 1.0))};
  if constexpr (VEC) {
    using VT = Vec16<S>;
    constexpr int W = VT::W;
    const long long cpv = cells / W;
    const long long total = (long long)G * cpv;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
      long long gi = e / cpv, i = (e - gi * cpv) * W;
      const S* b = U + gi * gstride + i;
      S q[5][W];
#pragma unroll
      for (int v = 0; v < 5; ++v) VT::split(*reinterpret_cast<const typename VT::V*>(b + v * vstride), q[v]);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        S u[5] = {q[0][k], q[1][k], q[2][k], q[3][k], q[4][k]};
        fold_speed(u, gas, m, bad);
      }
    }
  } else {
    const long long total = (long long)G * cells;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
      long long gi = e / cells, i = e - gi * cells;
      const S* b = U + gi * gstride + i;
      S u[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) u[v] = b[v * vstride];
      fold_speed(u, gas, m, bad);
    }
  }
  __syncthreads();
  if (bad) anybad = 1;
  for (int d = 0; d < 3; ++d) {
    double r = block_max((double)m[d], sh);
    __syncthreads();
    if (threadIdx.x == 0) part[d * gridDim.x + blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000LL) : r;
  }
}

// Pass 2: one CTA reduces the partials of nseg pass-1 launches of n CTAs
// each (laid out [segment][direction][CTA]) and writes
//   smax = max_d (max speed_d) / dx_d,   dt = cfl / smax.
__global__ void cfl_final_kernel(const double* __restrict__ part, int nseg, int n, double dx0, double dx1,
                                 double dx2, double cfl, double* dt, double* smax) {
  __shared__ double sh[32];
  __shared__ int anybad;
  __shared__ double md[3];
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    double m = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < nseg * n; i += blockDim.x) {
      const int s = i / n, b = i - s * n;
      double v = part[((long long)s * 3 + d) * n + b];
      if (isnan(v)) bad = true;
      m = fmax(m, v);
    }
    if (bad) anybad = 1;
    m = block_max(m, sh);
    __syncthreads();
    if (threadIdx.x == 0) md[d] = m;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double s = md[0] / dx0;
    double s1 = md[1] / dx1;
    double s2 = md[2] / dx2;
    s = s1 > s ? s1 : s;
    s = s2 > s ? s2 : s;
    double mm = anybad ? __longlong_as_double(0x7ff8000000000000LL) : s;
    *dt = cfl / mm;
    if (smax) *smax = mm;
  }
}

// ---- CFL time step of many boxes in one pass (continuous batching, AMR
// levels): the table of boxes is a kernel argument; box b owns the pass-1
// CTAs [first_b, first_b + nblk_b), each reducing one contiguous chunk of the
// box's G * cells cells exactly as cfl_partial_kernel does (a box of
// halo-padded groups numbers only their interior cells, x fastest, and maps
// each to its place in the padded cube); pass 2 runs one
// CTA per box; an optional pass 3 takes min_b scale_b dt_b.  A box's dt
// equals hydro_cfl_dt's on the same data bit for bit: both are maxima of the
// same per-cell FP64 values, divided and inverted the same way.
struct CflBoxDev {
  const void* U;
  long long gstride, vstride, cells;
  int G, first, nblk, n, gh, pad;  // n, gh: interior edge and ghost width (gh = 0: contiguous cells)
  double dx[3];
  double* dt;
  double* smax;
  double scale;
};
constexpr int CFL_MAX_BOXES = HYDRO_CFL_MAX_BOXES;
struct CflBoxTable {
  int n, total;
  CflBoxDev box[CFL_MAX_BOXES];
};

template <class S>
__global__ void __launch_bounds__(256) cfl_boxes_partial_kernel(const __grid_constant__ CflBoxTable tab, double gamma,
                                                                double dfloor, double pfloor,
                                                                double* __restrict__ part) {
  __shared__ double sh[32];
  __shared__ int anybad;
  // the box of this CTA: the last one whose first CTA is <= blockIdx.x
  int lo = 0, hi = tab.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab.box[mid].first <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const CflBoxDev& bx = tab.box[lo];
  const S* U = (const S*)bx.U;
  const long long total = (long long)bx.G * bx.cells;
  const int k = blockIdx.x - bx.first;
  const long long chunk = (total + bx.nblk - 1) / bx.nblk;
  const long long begin = (long long)k * chunk;
  const long long end = begin + chunk < total ? begin + chunk : total;
  if (threadIdx.x == 0) anybad = 0;
  S m[3] = {S(0), S(0), S(0)};
  bool bad = false;
  Gas<S> gas{(S)gamma, (S)(gamma - 1.0), (S)dfloor, (S)pfloor, (S)(1.0 / (gamma - 1.0))};
  for (long long e = begin + threadIdx.x; e < end; e += blockDim.x) {
    const long long gi = e / bx.cells, i = e - gi * bx.cells;
    long long off = i;
    if (bx.gh > 0) {
      const int n = bx.n, M = n + 2 * bx.gh;
      const int z = (int)(i / ((long long)n * n));
      const int r = (int)(i - (long long)z * n * n);
      const int y = r / n, x = r - y * n;
      off = ((long long)(z + bx.gh) * M + (y + bx.gh)) * M + (x + bx.gh);
    }
    const S* b = U + gi * bx.gstride + off;
    S u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = b[v * bx.vstride];
    fold_speed(u, gas, m, bad);
  }
  __syncthreads();
  if (bad) anybad = 1;
  for (int d = 0; d < 3; ++d) {
    double r = block_max((double)m[d], sh);
    __syncthreads();
    if (threadIdx.x == 0)
      part[(long long)d * tab.total + blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000LL) : r;
  }
}

// One CTA per box: dt_b = cfl / max_d (max speed_d / dx_d); sdt[b] = scale_b dt_b.
__global__ void __launch_bounds__(256) cfl_boxes_final_kernel(const __grid_constant__ CflBoxTable tab, double cfl,
                                                              const double* __restrict__ part, double* sdt) {
  __shared__ double sh[32];
  __shared__ int anybad;
  __shared__ double md[3];
  const CflBoxDev& bx = tab.box[blockIdx.x];
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    double m = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < bx.nblk; i += blockDim.x) {
      const double v = part[(long long)d * tab.total + bx.first + i];
      if (isnan(v)) bad = true;
      m = fmax(m, v);
    }
    if (bad) anybad = 1;
    m = block_max(m, sh);
    __syncthreads();
    if (threadIdx.x == 0) md[d] = m;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double s = md[0] / bx.dx[0];
    double s1 = md[1] / bx.dx[1];
    double s2 = md[2] / bx.dx[2];
    s = s1 > s ? s1 : s;
    s = s2 > s ? s2 : s;
    const double mm = anybad ? __longlong_as_double(0x7ff8000000000000LL) : s;
    const double dt = cfl / mm;
    *bx.dt = dt;
    if (bx.smax) *bx.smax = mm;
    sdt[blockIdx.x] = bx.scale * dt;
  }
}

// min over boxes of scale_b dt_b; NaN if any is NaN.
__global__ void __launch_bounds__(256) cfl_boxes_min_kernel(const double* __restrict__ sdt, int n, double* out) {
  __shared__ double sh[32];
  __shared__ int anybad;
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  double m = -__longlong_as_double(0x7ff0000000000000LL);  // max of -dt
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = sdt[i];
    if (isnan(v)) bad = true;
    m = fmax(m, -v);
  }
  if (bad) anybad = 1;
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    *out = anybad ? __longlong_as_double(0x7ff8000000000000LL) : -r;
  }
}

// Totals: per-CTA FP64 partial sums of the five variables, then one CTA.
template <class S>
__global__ void totals_partial_kernel(const S* __restrict__ U, int G, long long gstride, long long vstride,
                                      long long cells, double* __restrict__ part) {
  __shared__ double sh[32];
  const long long total = (long long)G * cells;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long gi = e / cells, i = e - gi * cells;
    const S* b = U + gi * gstride + i;
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += (double)b[v * vstride];
  }
  for (int v = 0; v < 5; ++v) {
    double s = block_sum(acc[v], sh);
    if (threadIdx.x == 0) part[v * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void totals_final_kernel(const double* __restrict__ part, int n, double* __restrict__ out) {
  __shared__ double sh[32];
  for (int v = 0; v < 5; ++v) {
    double a = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[v * n + i];
    a = block_sum(a, sh);
    if (threadIdx.x == 0) out[v] = a;
  }
}

}  // namespace hyd

// ---- launchers used by the C-ABI (hydro_api.cu) ---------------------------
namespace hyd {

cudaError_t launch_gather(const void* field, int X, int Y, int Z, int bc, const int* origin, int G, int N, int g,
                          int dbl, void* out, cudaStream_t st, int nsm) {
  long long total = 5LL * (N + 2 * g) * (N + 2 * g) * (N + 2 * g) * G;
  if (total == 0) return cudaSuccess;
  int threads = 256;
  long long want = (total + threads - 1) / threads;
  int grid = (int)(want < 8LL * nsm * 4 ? want : 8LL * nsm * 4);
  if (dbl)
    gather_kernel<double><<<grid, threads, 0, st>>>((const double*)field, X, Y, Z, bc, origin, G, N, g, (double*)out);
  else
    gather_kernel<float><<<grid, threads, 0, st>>>((const float*)field, X, Y, Z, bc, origin, G, N, g, (float*)out);
  return cudaGetLastError();
}

constexpr int RED_MAX_CTAS = 2048;

// CTAs of one pass-1 launch over `total` cells.
int cfl_grid(long long total, int nsm) {
  const int threads = 256;
  long long want = (total + threads - 1) / threads;
  int grid = (int)(want < 4LL * nsm ? want : 4LL * nsm);
  if (grid < 1) grid = 1;
  if (grid > RED_MAX_CTAS) grid = RED_MAX_CTAS;
  return grid;
}

// Pass 1 into part[3][grid].
cudaError_t launch_cfl_partial(const void* U, int G, long long gs, long long vs, long long cells, int dbl,
                               double gamma, double dfl, double pfl, double* ws, int grid, cudaStream_t st) {
  const int threads = 256;
  // 16-byte loads when every group's variables start on a 16-byte boundary
  const int w = dbl ? 2 : 4;
  const bool vec = ((uintptr_t)U % 16 == 0) && cells % w == 0 && gs % w == 0 && vs % w == 0;
  if (dbl) {
    if (vec)
      cfl_partial_kernel<double, true><<<grid, threads, 0, st>>>((const double*)U, G, gs, vs, cells, gamma, dfl,
                                                                 pfl, ws);
    else
      cfl_partial_kernel<double, false><<<grid, threads, 0, st>>>((const double*)U, G, gs, vs, cells, gamma, dfl,
                                                                  pfl, ws);
  } else {
    if (vec)
      cfl_partial_kernel<float, true><<<grid, threads, 0, st>>>((const float*)U, G, gs, vs, cells, gamma, dfl, pfl,
                                                                ws);
    else
      cfl_partial_kernel<float, false><<<grid, threads, 0, st>>>((const float*)U, G, gs, vs, cells, gamma, dfl, pfl,
                                                                 ws);
  }
  return cudaGetLastError();
}

// Pass 2 over nseg pass-1 launches of `grid` CTAs each.
cudaError_t launch_cfl_final(const double* ws, int nseg, int grid, const double* dx, double cfl, double* dt,
                             double* smax, cudaStream_t st) {
  cfl_final_kernel<<<1, 1024, 0, st>>>(ws, nseg, grid, dx[0], dx[1], dx[2], cfl, dt, smax);
  return cudaGetLastError();
}

cudaError_t launch_cfl(const void* U, int G, long long gs, long long vs, long long cells, int dbl, double gamma,
                       double dfl, double pfl, const double* dx, double cfl, double* dt, double* smax, double* ws,
                       cudaStream_t st, int nsm) {
  const int grid = cfl_grid((long long)G * cells, nsm);
  cudaError_t e = launch_cfl_partial(U, G, gs, vs, cells, dbl, gamma, dfl, pfl, ws, grid, st);
  if (e != cudaSuccess) return e;
  return launch_cfl_final(ws, 1, grid, dx, cfl, dt, smax, st);
}

// Workspace of the many-box reduction: 3 partials per pass-1 CTA (at most
// RED_MAX_CTAS + CFL_MAX_BOXES CTAs) and one scaled dt per box.
size_t cfl_boxes_workspace_bytes() { return sizeof(double) * (3 * (RED_MAX_CTAS + CFL_MAX_BOXES) + CFL_MAX_BOXES); }

// Pass-1 CTAs shared out in proportion to the boxes' cells, at least one per
// box, at most RED_MAX_CTAS + n in all.
cudaError_t launch_cfl_boxes(const hydro_cfl_box* boxes, int n, int dbl, double gamma, double dfl, double pfl,
                             double cfl, double* dt_min, double* ws, cudaStream_t st) {
  CflBoxTable tab;
  tab.n = n;
  long long all = 0;
  for (int b = 0; b < n; ++b) all += (long long)boxes[b].G * boxes[b].cells;
  // cells per pass-1 CTA: 64 per thread of a 256-thread CTA, more when the
  // boxes together would need more than RED_MAX_CTAS CTAs
  long long per = 256LL * 64;
  if ((all + per - 1) / per > RED_MAX_CTAS) per = (all + RED_MAX_CTAS - 1) / RED_MAX_CTAS;
  int first = 0;
  for (int b = 0; b < n; ++b) {
    CflBoxDev& t = tab.box[b];
    t.U = boxes[b].U;
    t.gstride = boxes[b].group_stride;
    t.vstride = boxes[b].var_stride;
    t.cells = boxes[b].cells;
    t.G = boxes[b].G;
    t.n = boxes[b].interior_n;
    t.gh = boxes[b].ghost;
    t.pad = 0;
    for (int d = 0; d < 3; ++d) t.dx[d] = boxes[b].dx[d];
    t.dt = boxes[b].dt_dev;
    t.smax = boxes[b].smax_dev;
    t.scale = boxes[b].dt_scale;
    const long long cb = (long long)boxes[b].G * boxes[b].cells;
    long long nb = (cb + per - 1) / per;
    if (nb < 1) nb = 1;
    tab.box[b].first = first;
    tab.box[b].nblk = (int)nb;
    first += (int)nb;
  }
  tab.total = first;
  double* part = ws;
  double* sdt = ws + 3 * (RED_MAX_CTAS + CFL_MAX_BOXES);
  if (dbl)
    cfl_boxes_partial_kernel<double><<<first, 256, 0, st>>>(tab, gamma, dfl, pfl, part);
  else
    cfl_boxes_partial_kernel<float><<<first, 256, 0, st>>>(tab, gamma, dfl, pfl, part);
  cfl_boxes_final_kernel<<<n, 256, 0, st>>>(tab, cfl, part, sdt);
  if (dt_min) cfl_boxes_min_kernel<<<1, 256, 0, st>>>(sdt, n, dt_min);
  return cudaGetLastError();
}

cudaError_t launch_totals(const void* U, int G, long long gs, long long vs, long long cells, int dbl, double* out,
                          double* ws, cudaStream_t st, int nsm) {
  long long total = (long long)G * cells;
  int threads = 256;
  long long want = (total + threads - 1) / threads;
  int grid = (int)(want < 4LL * nsm ? want : 4LL * nsm);
  if (grid < 1) grid = 1;
  if (grid > RED_MAX_CTAS) grid = RED_MAX_CTAS;
  if (dbl)
    totals_partial_kernel<double><<<grid, threads, 0, st>>>((const double*)U, G, gs, vs, cells, ws);
  else
    totals_partial_kernel<float><<<grid, threads, 0, st>>>((const float*)U, G, gs, vs, cells, ws);
  totals_final_kernel<<<1, 1024, 0, st>>>(ws, grid, out);
  return cudaGetLastError();
}

}  // namespace hyd
