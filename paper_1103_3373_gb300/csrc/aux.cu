// Auxiliary kernels of the hot path:
//   * ghost-zone gather of halo-padded groups from a uniform field (the
//     "preparation step" of Sec. 4.2, on the device);
//   * CFL time step (the evolution time step of Sec. 4.3) as a two-pass
//     FP64 max-reduction;
//   * FP64 totals of the conserved variables (conservation monitor).
#include <cuda_runtime.h>
#include <stdint.h>

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

// Pass 1: per-CTA maximum of max_d (|v_d| + c) / dx_d, evaluated in FP64.
// A NaN cell makes the maximum NaN (so dt becomes NaN and is noticed).
template <class S>
__global__ void cfl_partial_kernel(const S* __restrict__ U, int G, long long gstride, long long vstride,
                                   long long cells, double gamma, double dfloor, double pfloor, double dx0,
                                   double dx1, double dx2, double* __restrict__ part) {
  __shared__ double sh[32];
  const long long total = (long long)G * cells;
  double m = 0.0;
  bool bad = false;
  Gas<double> gas{gamma, gamma - 1.0, dfloor, pfloor};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long gi = e / cells, i = e - gi * cells;
    const S* b = U + gi * gstride + i;
    double u[5], w[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = (double)b[v * vstride];
    prim<double, false>(u, w, gas);
    double c = sqrt(gamma * w[4] / w[0]);
    double s0 = (fabs(w[1]) + c) / dx0;
    double s1 = (fabs(w[2]) + c) / dx1;
    double s2 = (fabs(w[3]) + c) / dx2;
    double s = fmax(s0, fmax(s1, s2));
    if (isnan(s)) bad = true;
    m = fmax(m, s);
  }
  m = block_max(m, sh);
  __syncthreads();
  __shared__ int anybad;
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  if (bad) anybad = 1;
  __syncthreads();
  if (threadIdx.x == 0) part[blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000LL) : m;
}

// Pass 2: one CTA reduces the partials and writes dt = cfl / max.
__global__ void cfl_final_kernel(const double* __restrict__ part, int n, double cfl, double* dt, double* smax) {
  __shared__ double sh[32];
  double m = 0.0;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = part[i];
    if (isnan(v)) bad = true;
    m = fmax(m, v);
  }
  m = block_max(m, sh);
  __shared__ int anybad;
  __syncthreads();
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  if (bad) anybad = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = anybad ? __longlong_as_double(0x7ff8000000000000LL) : m;
    *dt = cfl / mm;
    if (smax) *smax = mm;
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

cudaError_t launch_cfl(const void* U, int G, long long gs, long long vs, long long cells, int dbl, double gamma,
                       double dfl, double pfl, const double* dx, double cfl, double* dt, double* smax, double* ws,
                       cudaStream_t st, int nsm) {
  long long total = (long long)G * cells;
  int threads = 256;
  long long want = (total + threads - 1) / threads;
  int grid = (int)(want < 4LL * nsm ? want : 4LL * nsm);
  if (grid < 1) grid = 1;
  if (grid > RED_MAX_CTAS) grid = RED_MAX_CTAS;
  if (dbl)
    cfl_partial_kernel<double><<<grid, threads, 0, st>>>((const double*)U, G, gs, vs, cells, gamma, dfl, pfl,
                                                         dx[0], dx[1], dx[2], ws);
  else
    cfl_partial_kernel<float><<<grid, threads, 0, st>>>((const float*)U, G, gs, vs, cells, gamma, dfl, pfl,
                                                        dx[0], dx[1], dx[2], ws);
  cfl_final_kernel<<<1, 1024, 0, st>>>(ws, grid, cfl, dt, smax);
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
