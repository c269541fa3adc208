// Peak arithmetic rate of the non-tensor pipes (the denominator of the
// roofline of the patch-group kernels, which are bound by FP32 / FP64
// arithmetic, not by a dense contraction).  Each thread runs CHAINS
// independent fused multiply-add chains a = a * b + c for `iters` iterations,
// so the pipe never waits on a result, and stores their sum so that nothing
// is eliminated.  b and c are launch arguments (no constant folding), chosen
// so that every chain converges to the fixed point c / (1 - b) = 1 and
// produces neither overflow nor subnormals.
//
// Kinds: FP32 scalar (one fma.rn.f32 per chain step), FP32 packed (one
// fma.rn.f32x2, two FP32 FMAs, per chain step) and FP64 (fma.rn.f64).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hydro_peaks.h"

namespace hyd {
int record_cuda_error(cudaError_t e);
}

namespace {

constexpr int CHAINS = 8;

__global__ void fma_fp32_kernel(float* out, float b, float c, int iters) {
  float a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = 0.5f + 0.01f * k + 1e-7f * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma_fp32x2_kernel(float* out, float b, float c, int iters) {
  uint64_t a[CHAINS];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  const uint64_t bb = *reinterpret_cast<const uint64_t*>(&b2);
  const uint64_t cc = *reinterpret_cast<const uint64_t*>(&c2);
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) {
    const float2 x = make_float2(0.5f + 0.01f * k, 0.25f + 1e-7f * threadIdx.x);
    a[k] = *reinterpret_cast<const uint64_t*>(&x);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) {
    const float2 x = *reinterpret_cast<const float2*>(&a[k]);
    s += x.x + x.y;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma_fp64_kernel(double* out, double b, double c, int iters) {
  double a[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) a[k] = 0.5 + 0.01 * k + 1e-9 * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int hydro_fma_peak(int kind, int ctas, int threads, int iters, void* out, void* stream,
                              double* flops_per_launch) {
  if (kind < HYDRO_PEAK_FP32 || kind > HYDRO_PEAK_FP64 || ctas < 1 || threads < 32 || threads > 1024 ||
      threads % 32 != 0 || iters < 1 || !out)
    return HYDRO_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const double lanes = (double)ctas * threads * iters * CHAINS;
  double flops = 2.0 * lanes;
  if (kind == HYDRO_PEAK_FP32) {
    fma_fp32_kernel<<<ctas, threads, 0, st>>>((float*)out, 0.999999f, 1e-6f, iters);
  } else if (kind == HYDRO_PEAK_FP32X2) {
    fma_fp32x2_kernel<<<ctas, threads, 0, st>>>((float*)out, 0.999999f, 1e-6f, iters);
    flops *= 2.0;
  } else {
    fma_fp64_kernel<<<ctas, threads, 0, st>>>((double*)out, 0.999999999, 1e-9, iters);
  }
  if (flops_per_launch) *flops_per_launch = flops;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HYDRO_OK : hyd::record_cuda_error(e);
}
