// Two FP32 lanes per thread: the paired arithmetic of the FP32 patch-group
// kernels.  Additions, subtractions, multiplications and fused multiply-adds
// of both lanes are one packed instruction (the f32x2 forms of sm_100 and
// later, through the compiler's float2 builtins), which halves the issue
// slots the arithmetic takes; comparisons, selects, min / max and the
// special functions act per lane.  Every operation rounds each lane as the
// scalar FP32 instruction does (round to nearest).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hyd {

struct V2 {
  float2 v;
};

struct M2 {
  bool x, y;
};

__device__ __forceinline__ V2 mk2(float a, float b) { return V2{make_float2(a, b)}; }
__device__ __forceinline__ V2 sp2(float a) { return V2{make_float2(a, a)}; }

// the compiler's packed builtins (one f32x2 instruction each)
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator-(V2 a) { return mk2(-a.v.x, -a.v.y); }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2{__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2{__fmul2_rn(a.v, b.v)}; }
// a * b + c, one rounding per lane
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return V2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ V2 operator*(float a, V2 b) { return sp2(a) * b; }
__device__ __forceinline__ V2 operator*(V2 a, float b) { return a * sp2(b); }
__device__ __forceinline__ V2 operator+(V2 a, float b) { return a + sp2(b); }
__device__ __forceinline__ V2 operator-(V2 a, float b) { return a - sp2(b); }
__device__ __forceinline__ V2 operator-(float a, V2 b) { return sp2(a) - b; }

// per lane
__device__ __forceinline__ V2 min2(V2 a, V2 b) { return mk2(fminf(a.v.x, b.v.x), fminf(a.v.y, b.v.y)); }
__device__ __forceinline__ V2 max2(V2 a, V2 b) { return mk2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
__device__ __forceinline__ V2 abs2(V2 a) { return mk2(fabsf(a.v.x), fabsf(a.v.y)); }
__device__ __forceinline__ V2 copysign2(V2 a, V2 s) { return mk2(copysignf(a.v.x, s.v.x), copysignf(a.v.y, s.v.y)); }
__device__ __forceinline__ V2 rcp2(V2 a) { return mk2(__fdividef(1.0f, a.v.x), __fdividef(1.0f, a.v.y)); }
__device__ __forceinline__ V2 sqrt2(V2 a) { return mk2(sqrtf(a.v.x), sqrtf(a.v.y)); }
__device__ __forceinline__ V2 rsqrt2(V2 a) { return mk2(rsqrtf(a.v.x), rsqrtf(a.v.y)); }
__device__ __forceinline__ M2 gt2(V2 a, V2 b) { return M2{a.v.x > b.v.x, a.v.y > b.v.y}; }
__device__ __forceinline__ M2 lt2(V2 a, V2 b) { return M2{a.v.x < b.v.x, a.v.y < b.v.y}; }
__device__ __forceinline__ M2 le2(V2 a, V2 b) { return M2{a.v.x <= b.v.x, a.v.y <= b.v.y}; }
__device__ __forceinline__ M2 ge2(V2 a, V2 b) { return M2{a.v.x >= b.v.x, a.v.y >= b.v.y}; }
__device__ __forceinline__ M2 and2(M2 a, M2 b) { return M2{a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ M2 or2(M2 a, M2 b) { return M2{a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ M2 not2(M2 a) { return M2{!a.x, !a.y}; }
__device__ __forceinline__ V2 sel2(M2 m, V2 a, V2 b) { return mk2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }
__device__ __forceinline__ float lane_of(V2 a, int l) { return l ? a.v.y : a.v.x; }

}  // namespace hyd
