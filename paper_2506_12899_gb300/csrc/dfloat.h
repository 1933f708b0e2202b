// Double-float numbers: x = hi + lo with |lo| <= ulp(hi)/2, both FP32 (Dekker 1971).  Sums use
// Knuth's two_sum and products the FMA-based two_prod, so every operation keeps about 48
// significant bits (relative error ~4e-15) while running on the FP32 pipes; on GB300 those issue
// 64 times as many operations per clock as the FP64 pipe.  The non-contracting intrinsics keep
// the compiler from fusing the steps of an error-free transformation.
#pragma once

#include <cuda_runtime.h>

namespace sbm {

struct __align__(8) dfl {
  float hi, lo;
  dfl() = default;                                              // trivial: usable in __shared__ arrays
  __host__ __device__ dfl(int x) : hi((float)x), lo(0.f) {}     // small integers (exact)
  __host__ __device__ dfl(float x) : hi(x), lo(0.f) {}
  __host__ __device__ dfl(float h, float l) : hi(h), lo(l) {}
  // Rounds an FP64 value to double-float (used on the host for constants).
  __host__ __device__ explicit dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDACC__
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float z = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.hi, z));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  return dfl(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float hi = __fadd_rn(p, e);
  return dfl(hi, __fsub_rn(e, __fsub_rn(hi, p)));
}

__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
__device__ __forceinline__ bool operator==(dfl a, dfl b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return !(a == b); }
#endif

}  // namespace sbm
