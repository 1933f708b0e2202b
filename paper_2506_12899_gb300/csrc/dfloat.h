// Double-float numbers: x = hi + lo with |lo| <= ulp(hi)/2, both FP32 (Dekker 1971).  Sums use
// Knuth's two_sum and products the FMA-based two_prod, so every operation keeps about 48
// significant bits (relative error ~4e-15) while running on the FP32 pipes; on GB300 those issue
// 64 times as many operations per clock as the FP64 pipe.  The non-contracting intrinsics keep
// the compiler from fusing the steps of an error-free transformation.
#pragma once

#include <cuda_runtime.h>

namespace sbm {

// A double-float product before renormalisation: p = fl(a.hi b.hi) and e = its exact rounding
// error plus the cross terms, value p + e.  Summing it into an accumulator (+=) skips the
// renormalisation of the product and of the sum; any other use converts it to dfl.
struct dfl_prod {
  float p, e;
};

struct __align__(8) dfl {
  float hi, lo;
  dfl() = default;                                              // trivial: usable in __shared__ arrays
  __host__ __device__ dfl(int x) : hi((float)x), lo(0.f) {}     // small integers (exact)
  __host__ __device__ dfl(float x) : hi(x), lo(0.f) {}
  __host__ __device__ dfl(float h, float l) : hi(h), lo(l) {}
  // Rounds an FP64 value to double-float (used on the host for constants).
  __host__ __device__ explicit dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
#ifdef __CUDACC__
  __device__ dfl(dfl_prod q) {                                  // renormalised (fast two_sum)
    hi = __fadd_rn(q.p, q.e);
    lo = __fsub_rn(q.e, __fsub_rn(hi, q.p));
  }
#endif
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

__device__ __forceinline__ dfl_prod operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dfl_prod{p, e};
}

// Product with an FP32 value (a double-float with a zero low part): the b.lo term drops out.
__device__ __forceinline__ dfl_prod operator*(dfl a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return dfl_prod{p, e};
}
__device__ __forceinline__ dfl_prod operator*(float a, dfl b) { return b * a; }

__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = dfl(a * b); }

// a += p + e: two_sum of the leading parts, every error term added into a.lo; a is left
// unrenormalised (|a.lo| may exceed half an ulp of a.hi by the accumulated errors, which keeps
// the represented value hi + lo exact to about 2^-48 of the largest term summed).
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl_prod b) {
  const float s = __fadd_rn(a.hi, b.p);
  const float z = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, z)), __fsub_rn(b.p, z));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(err, b.e));
  return a;
}
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl_prod b) { return a += dfl_prod{-b.p, -b.e}; }
__device__ __forceinline__ bool operator==(dfl a, dfl b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return !(a == b); }
#endif

}  // namespace sbm
