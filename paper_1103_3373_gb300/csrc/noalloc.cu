// hydro_cfl_dt_noalloc: the CFL time-step reduction for callers that cannot
// allocate device memory (a kernel plug-in running inside someone else's
// CUDA graph capture, or a host framework whose allocator is unavailable in
// the calling context).  It has no counterpart in the paper.
//
// Scratch: three FP64 partial maxima (one per direction) per CTA, in a
// file-scope static device array of NOALLOC_MAX_PARTIALS doubles (64 KiB),
// which every GPU that loads the library keeps until the process exits.  Each
// CTA reduces a fixed chunk of NOALLOC_CELLS_PER_CTA cells, so one call
// handles at most (NOALLOC_MAX_PARTIALS / 3) * NOALLOC_CELLS_PER_CTA cells
// (1.79e8; a 512^3 box fits); larger inputs are rejected before anything is
// launched.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol, so its device address is looked up once per device, with that
// device current, by cudaGetSymbolAddress, and that address is what the
// kernels receive.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/hydro.h"
#include "phys.cuh"

namespace hyd {
int record_cuda_error(cudaError_t e);  // hydro_api.cu: keeps the text for hydro_last_cuda_error
}

namespace {

constexpr int NOALLOC_MAX_PARTIALS = HYDRO_NOALLOC_MAX_PARTIALS;
constexpr long long NOALLOC_CELLS_PER_CTA = HYDRO_NOALLOC_CELLS_PER_CTA;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEV = 64;

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_PARTIALS];

std::mutex g_mu;
double* g_partials_ptr[NOALLOC_MAX_DEV] = {nullptr};

// Pass 1 (variant of the CFL partial reduction): CTA b reduces the cells
// [b * NOALLOC_CELLS_PER_CTA, (b + 1) * NOALLOC_CELLS_PER_CTA) of the flat
// (group, cell) range and writes, per direction d, its maximum of
// |v_d| + c (storage precision per cell, kept as FP64) to
// part[d * nblk + b] (NaN if any of its cells gives NaN).
template <class S>
__global__ void __launch_bounds__(NOALLOC_THREADS)
    noalloc_cfl_partial(const S* __restrict__ U, int G, long long gstride, long long vstride, long long cells,
                        double gamma, double dfloor, double pfloor, double* __restrict__ part) {
  __shared__ double sh[3][NOALLOC_THREADS / 32];
  __shared__ int anybad;
  const long long total = (long long)G * cells;
  const long long begin = (long long)blockIdx.x * NOALLOC_CELLS_PER_CTA;
  long long end = begin + NOALLOC_CELLS_PER_CTA;
  if (end > total) end = total;
  if (threadIdx.x == 0) anybad = 0;
  hyd::Gas<S> gas{(S)gamma, (S)(gamma - 1.0), (S)dfloor, (S)pfloor, (S)(1.0 / (gamma - 1.0))};
  S m[3] = {S(0), S(0), S(0)};
  bool bad = false;
  for (long long e = begin + threadIdx.x; e < end; e += NOALLOC_THREADS) {
    long long gi = e / cells, i = e - gi * cells;
    const S* b = U + gi * gstride + i;
    S u[5], w[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = b[v * vstride];
    hyd::prim<S, false>(u, w, gas);
    S c = hyd::sqrtv(gas.gamma * w[4] / w[0]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      S s = hyd::absv(w[1 + d]) + c;
      if (hyd::isnanv(s)) bad = true;
      m[d] = s > m[d] ? s : m[d];
    }
  }
  double r[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    r[d] = (double)m[d];
    for (int o = 16; o > 0; o >>= 1) r[d] = fmax(r[d], __shfl_xor_sync(0xffffffffu, r[d], o));
  }
  __syncthreads();
  if (bad) anybad = 1;
  if ((threadIdx.x & 31) == 0)
    for (int d = 0; d < 3; ++d) sh[d][threadIdx.x >> 5] = r[d];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int d = 0; d < 3; ++d) {
      double x = sh[d][0];
      for (int k = 1; k < NOALLOC_THREADS / 32; ++k) x = fmax(x, sh[d][k]);
      part[d * gridDim.x + blockIdx.x] = anybad ? __longlong_as_double(0x7ff8000000000000LL) : x;
    }
  }
}

// Pass 2: one CTA reduces the 3 x n partials and writes
//   smax = max_d (max speed_d) / dx_d,  dt = cfl / smax.
__global__ void __launch_bounds__(1024) noalloc_cfl_final(const double* __restrict__ part, int n, double dx0,
                                                           double dx1, double dx2, double cfl, double* dt,
                                                           double* smax) {
  __shared__ double sh[3][32];
  __shared__ int anybad;
  if (threadIdx.x == 0) anybad = 0;
  __syncthreads();
  double m[3] = {0.0, 0.0, 0.0};
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int d = 0; d < 3; ++d) {
      double v = part[d * n + i];
      if (isnan(v)) bad = true;
      m[d] = fmax(m[d], v);
    }
  if (bad) anybad = 1;
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) m[d] = fmax(m[d], __shfl_xor_sync(0xffffffffu, m[d], o));
    if ((threadIdx.x & 31) == 0) sh[d][threadIdx.x >> 5] = m[d];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double md[3];
    for (int d = 0; d < 3; ++d) {
      md[d] = sh[d][0];
      for (int k = 1; k < (int)(blockDim.x >> 5); ++k) md[d] = fmax(md[d], sh[d][k]);
    }
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

// Device address of the static partials for the current device (looked up
// once per device, with that device current).  The cached address belongs
// to the device's primary context: it stays valid as long as that context
// lives, i.e. until the process exits unless the caller resets the device.
int partials_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hyd::record_cuda_error(e);
  if (dev < 0 || dev >= NOALLOC_MAX_DEV) return hyd::record_cuda_error(cudaErrorInvalidDevice);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return hyd::record_cuda_error(e);
    if (!p) return hyd::record_cuda_error(cudaErrorInvalidSymbol);
    g_partials_ptr[dev] = (double*)p;
  }
  *out = g_partials_ptr[dev];
  return HYDRO_OK;
}

bool pos_finite(double a) { return a > 0.0 && a < 1e300; }

}  // namespace

extern "C" int hydro_cfl_dt_noalloc(const void* U, int G, long long group_stride, long long var_stride,
                                    long long cells, int precision, double gamma, double dens_floor,
                                    double pres_floor, const double* dx, double cfl, double* dt_dev,
                                    double* smax_dev, void* stream) {
  if (!U || G < 0 || cells < 0 || !dx || !dt_dev || !(gamma > 1.0) || !(cfl > 0.0)) return HYDRO_EINVAL;
  if (precision < 0 || precision > 2) return HYDRO_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!pos_finite(dx[d])) return HYDRO_EINVAL;
  const long long total = (long long)G * cells;
  if ((G > 0 && total / G != cells) || total > (long long)(NOALLOC_MAX_PARTIALS / 3) * NOALLOC_CELLS_PER_CTA)
    return HYDRO_ETOOBIG;
  double* part = nullptr;
  int rc = partials_for_current_device(&part);
  if (rc != HYDRO_OK) return rc;
  // no cells (G == 0 or cells == 0): one CTA writes zero maxima and dt is
  // cfl / 0 = inf, as hydro_cfl_dt gives
  int nblk = (int)((total + NOALLOC_CELLS_PER_CTA - 1) / NOALLOC_CELLS_PER_CTA);
  if (nblk < 1) nblk = 1;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == HYDRO_FP64)
    noalloc_cfl_partial<double><<<nblk, NOALLOC_THREADS, 0, st>>>((const double*)U, G, group_stride, var_stride,
                                                                  cells, gamma, dens_floor, pres_floor, part);
  else
    noalloc_cfl_partial<float><<<nblk, NOALLOC_THREADS, 0, st>>>((const float*)U, G, group_stride, var_stride,
                                                                 cells, gamma, dens_floor, pres_floor, part);
  noalloc_cfl_final<<<1, 1024, 0, st>>>(part, nblk, dx[0], dx[1], dx[2], cfl, dt_dev, smax_dev);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HYDRO_OK : hyd::record_cuda_error(e);
}
