// FP64 building blocks of FGMRES (Sec. 3: GMRES preconditioned by one V-cycle): multi-vector
// dot products with a deterministic two-stage reduction (warp shuffles, then a fixed-order sum
// of per-block partials), multi-vector AXPY, scaling and precision casts.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <type_traits>

#include "ops.h"

namespace sbm {

namespace {

constexpr int kDotThreads = 256;
constexpr int kMaxVec = 32;
constexpr int kDotMaxBlocks = 152 * 4;     // grid cap of the multi-vector dot kernels (4 CTAs per SM)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block-level reduction of NV per-thread sums into partial[blockIdx][k].
template <int NV>
__device__ __forceinline__ void block_partials(const double (&acc)[NV], double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32][NV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double s = warp_sum(acc[k]);
    if (lane == 0) red[warp][k] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kDotThreads / 32; ++q) s += red[q][threadIdx.x];
    partial[(size_t)blockIdx.x * kMaxVec + threadIdx.x] = s;
  }
}

constexpr int kDotE = 4;                        // elements per thread per chunk
constexpr size_t kDotChunk = (size_t)kDotThreads * kDotE;

// partial[block][k] = this block's share of V_k . w, k < NV.  A block sweeps chunks of
// kDotChunk consecutive elements; within a chunk it reads each vector V_k as one contiguous
// 8 KB run (DRAM-friendly) while w stays in registers.  NV is a compile-time constant so that
// no predicated FP64 FMA is issued: the FP64 pipe (about 2 FMA per clock per SM on GB300) and
// HBM are the two limits of this kernel.
template <int NV>
__global__ void __launch_bounds__(kDotThreads) k_multi_dot(const double* __restrict__ V, size_t ldv,
                                                           const double* __restrict__ w, size_t N,
                                                           double* __restrict__ partial) {
  pdl_entry();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (size_t base = (size_t)blockIdx.x * kDotChunk; base < N; base += (size_t)gridDim.x * kDotChunk) {
    double wv[kDotE];
#pragma unroll
    for (int e = 0; e < kDotE; ++e) {
      const size_t i = base + (size_t)e * kDotThreads + threadIdx.x;
      wv[e] = i < N ? w[i] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const double* row = V + k * ldv;
      double sk = 0.0;
#pragma unroll
      for (int e = 0; e < kDotE; ++e) {
        const size_t i = base + (size_t)e * kDotThreads + threadIdx.x;
        sk = fma(i < N ? row[i] : 0.0, wv[e], sk);
      }
      acc[k] += sk;
    }
  }
  block_partials<NV>(acc, partial);
}

// Second Gram-Schmidt pass fused with the first update: w <- w - sum_k h[k] V_k, then
// partial sums of V_k . w (new w) for k < NV, and of |w|^2 when NORM (then NV = 0 dots).
template <int NV, bool NORM>
__global__ void __launch_bounds__(kDotThreads) k_axpy_dot(const double* __restrict__ V, size_t ldv,
                                                          const double* __restrict__ h, double* __restrict__ w,
                                                          size_t N, int nv, double* __restrict__ partial) {
  pdl_entry();
  constexpr int NA = NORM ? 1 : NV;            // accumulators
  __shared__ double hs[kMaxVec];
  if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  const size_t stride = (size_t)gridDim.x * kDotThreads;
  for (size_t i = (size_t)blockIdx.x * kDotThreads + threadIdx.x; i < N; i += stride) {
    if (NORM) {
      double wi = w[i];
      for (int k = 0; k < nv; ++k) wi = fma(-hs[k], V[k * ldv + i], wi);
      w[i] = wi;
      acc[0] = fma(wi, wi, acc[0]);
    } else {
      double v[NV > 0 ? NV : 1];
      double wi = w[i];
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        v[k] = V[k * ldv + i];
        wi = fma(-hs[k], v[k], wi);
      }
      w[i] = wi;
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = fma(v[k], wi, acc[k]);
    }
  }
  block_partials<NA>(acc, partial);
}

// out[k] = sum_b partial[b][k]: warp k sums a fixed lane-strided share and shuffles, so the
// order of the additions is fixed for a given number of blocks (deterministic results).
__global__ void __launch_bounds__(1024) k_reduce_partials(const double* __restrict__ partial, int nblk, int nv,
                                                          double* __restrict__ out, int take_sqrt) {
  pdl_entry();
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= nv) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[(size_t)b * kMaxVec + k];
  s = warp_sum(s);
  if (lane == 0) out[k] = take_sqrt ? sqrt(s) : s;
}

template <typename TZ>
__global__ void __launch_bounds__(256) k_multi_axpy(const TZ* __restrict__ Z, size_t ldz, int nv,
                                                    const double* __restrict__ coef, double sign,
                                                    double* __restrict__ w, size_t N) {
  pdl_entry();
  __shared__ double cf[kMaxVec];
  if (threadIdx.x < nv) cf[threadIdx.x] = sign * coef[threadIdx.x];
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    double s = w[i];
    for (int k = 0; k < nv; ++k) s += cf[k] * (double)Z[k * ldz + i];
    w[i] = s;
  }
}

// x += sum_k c_k Z_k for FP32 Z (the FP32 V-cycle's preconditioned vectors).  The increment is
// accumulated in double-float on the FP32 pipes (each product c_k Z_k[i] formed exactly in two
// FP32 parts, the sum to about 48 bits) and added to the FP64 x once: 27 dependent FP64 FMAs per
// entry made the plain form FP64-pipe bound (1/64 of the FP32 rate on this GPU).
__global__ void __launch_bounds__(256) k_multi_axpy_df(const float* __restrict__ Z, size_t ldz, int nv,
                                                       const double* __restrict__ coef, double sign,
                                                       double* __restrict__ w, size_t N) {
  pdl_entry();
  __shared__ dfl cf[kMaxVec];
  if (threadIdx.x < nv) cf[threadIdx.x] = dfl(sign * coef[threadIdx.x]);
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    dfl s(0.f);
    for (int k = 0; k < nv; ++k) s += cf[k] * dfl(Z[k * ldz + i]);
    w[i] += (double)s.hi + (double)s.lo;
  }
}

__global__ void k_div_scalar(const double* __restrict__ w, const double* __restrict__ s, double* __restrict__ v,
                             size_t N) {
  pdl_entry();
  const double inv = 1.0 / s[0];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) v[i] = w[i] * inv;
}

template <typename TI, typename TO>
__global__ void k_cast(const TI* __restrict__ x, TO* __restrict__ y, size_t N) {
  pdl_entry();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) y[i] = (TO)x[i];
}

// The norm sweep's reduction fused with the Hessenberg column: warp 0 sums the partial squares
// (same order as k_reduce_partials) into hn[0] = |w| and col[k]; threads i < k write
// col[i] = h1[i] + h2[i].
__global__ void __launch_bounds__(64) k_reduce_norm_column(const double* __restrict__ partial, int nblk,
                                                          double* __restrict__ hn, const double* __restrict__ h1,
                                                          const double* __restrict__ h2, int k, double* __restrict__ col) {
  pdl_entry();
  const int i = threadIdx.x;
  if (i < k) col[i] = h1[i] + h2[i];
  if (i < 32) {
    double s = 0.0;
    for (int b = i; b < nblk; b += 32) s += partial[(size_t)b * kMaxVec];
    s = warp_sum(s);
    if (i == 0) {
      const double r = sqrt(s);
      hn[0] = r;
      col[k] = r;
    }
  }
}

__global__ void k_hess_column(const double* h1, const double* h2, const double* hn, int k, double* col) {
  pdl_entry();
  const int i = threadIdx.x;
  if (i < k) col[i] = h1[i] + h2[i];
  if (i == k) col[k] = hn[0];
}

// ------------------------------------------------------------------------------------------
// Gram-Schmidt on a double-float Krylov basis.  A basis vector is stored as pairs (hi, lo) of
// FP32 values with v = hi + lo and |lo| <= ulp(hi)/2 (a double-float number, Dekker 1971), 8
// bytes per entry like FP64.  Products and sums use error-free transformations on the FP32
// pipes: two_prod (p = a*b, e = fma(a, b, -p), so a*b = p + e exactly) and Knuth's two_sum.
// Every operation carries about 48 significant bits (relative error ~4e-15), against FP64's
// 53; the FP64 pipe, which bounds the plain FP64 sweeps on GB300, is not used per entry.
// The non-contracting intrinsics (__fmul_rn, __fadd_rn, __fsub_rn) keep the compiler from
// fusing the steps of an error-free transformation into an FMA.
__device__ __forceinline__ float2 df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

// (s, c) += a * b: the exact product p + e of the high parts, the cross terms into e, the sum
// s + p by two_sum with its rounding error added to the compensation c.
__device__ __forceinline__ void df_dot_acc(float& s, float& c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// w - h * v in double-float, renormalised.
__device__ __forceinline__ float2 df_sub_prod(float2 w, float2 h, float2 v) {
  const float p = __fmul_rn(h.x, v.x);
  float e = fmaf(h.x, v.x, -p);
  e = fmaf(h.x, v.y, e);
  e = fmaf(h.y, v.x, e);
  const float t = __fsub_rn(w.x, p);
  const float z = __fsub_rn(t, w.x);
  const float err = __fadd_rn(__fsub_rn(w.x, __fsub_rn(t, z)), __fsub_rn(__fsub_rn(0.f, p), z));
  const float lo = __fsub_rn(__fadd_rn(w.y, err), e);
  const float hi = __fadd_rn(t, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t)));
}

// a + b in double-float, renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float t = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(t, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(b.x, z));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float hi = __fadd_rn(t, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, t)));
}

// (s, c) += (s2, c2) for double-float partial sums held as a leading value and a compensation.
__device__ __forceinline__ void df_acc_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), err);
}

// Block reduction of NV double-float per-thread sums into partial[blockIdx][k] (FP64): warp
// shuffles in double-float on the FP32 pipes, one FP64 value per warp and vector, then a
// fixed-order FP64 sum over the warps.
template <int NV>
__device__ __forceinline__ void block_partials_df(float (&s)[NV], float (&c)[NV], double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32][NV > 0 ? NV : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float s2 = __shfl_xor_sync(0xffffffffu, s[k], off);
      const float c2 = __shfl_xor_sync(0xffffffffu, c[k], off);
      df_acc_add(s[k], c[k], s2, c2);
    }
    if (lane == 0) red[warp][k] = (double)s[k] + (double)c[k];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kDotThreads / 32; ++q) t += red[q][threadIdx.x];
    partial[(size_t)blockIdx.x * kMaxVec + threadIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------------------------
// Gram-Schmidt sweeps staged by the Tensor Memory Accelerator.  A persistent grid (one CTA per
// SM) walks chunks of E consecutive entries.  One elected thread copies the chunk of every V_k and
// of w into shared memory with bulk asynchronous copies (cp.async.bulk), whose completion an
// mbarrier counts in bytes, S chunks ahead of the arithmetic; the double-float arithmetic then
// reads shared memory.  HBM therefore streams independently of the long dependent chains of the
// error-free transformations, and each V_k is read as one contiguous run of E * 8 bytes per chunk.
//
// Requirements (checked by the launchers): V, w and wdf 16-byte aligned, ldv even, and one entry
// of padding after the last one when N is odd (the copies move whole 16-byte units; the padding
// entry is never used in the arithmetic).
constexpr int kSweepThreads = 256;
constexpr int kSweepBudget = 216 * 1024;           // shared memory of the stages, bytes

// Set by a sweep whose staged copies did not complete within kAsyncSpin polls; the solve reads and
// clears it (sweep_fault_take) and reports SBM_ERR_CUDA.
__device__ int g_sweep_fault;

constexpr int kSweepBudgetNoW = 224 * 1024;        // stage budget when w is read directly

template <int NV>
struct SweepShape {
  static constexpr int SLOTW = NV + 1;             // V_0 .. V_{NV-1}, then w
  static constexpr int EW = 2 * SLOTW * 1024 * 8 <= kSweepBudget ? 1024 : (2 * SLOTW * 512 * 8 <= kSweepBudget ? 512 : 256);
  // when the w slot would force 256-entry chunks, w is read with plain coalesced loads instead and
  // the V rows alone fill two 512-entry stages (widths 26..28)
  static constexpr bool WIN = !(EW == 256 && 2 * NV * 512 * 8 <= kSweepBudgetNoW);
  static constexpr int SLOT = WIN ? SLOTW : NV;
  static constexpr int E = WIN ? EW : 512;
  static constexpr int S0 = (WIN ? kSweepBudget : kSweepBudgetNoW) / (SLOT * E * 8);
  static constexpr int S = S0 > 6 ? 6 : S0;        // stages in flight
  static constexpr size_t smem = (size_t)S * SLOT * E * sizeof(float2) + (size_t)S * sizeof(unsigned long long);
  static_assert(S >= 2, "two stages must fit");
};

// MODE 0: partial[block][k] = V_k . w, k < NV.  w is FP64 (TW = double; it is also written to
//         wdf as double-float for the next sweeps) or double-float (TW = float2).
// MODE 1: wdf <- wdf - sum_k h[k] V_k, then partial[block][k] = V_k . wdf.
// MODE 2: wdf <- wdf - sum_k h[k] V_k, then partial[block][0] = |wdf|^2.
template <int NV, int MODE, typename TW>
__global__ void __launch_bounds__(kSweepThreads) k_gs_sweep(const float2* __restrict__ V, size_t ldv, const TW* w_in,
                                                            const double* __restrict__ h, float2* wdf, size_t N,
                                                            double* __restrict__ partial) {
  using Sh = SweepShape<NV>;
  constexpr int E = Sh::E, S = Sh::S, SLOT = Sh::SLOT, EPT = E / kSweepThreads;
  constexpr int NA = MODE == 2 ? 1 : NV;
  extern __shared__ __align__(128) unsigned char sweep_smem[];
  float2* stage = reinterpret_cast<float2*>(sweep_smem);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(sweep_smem + (size_t)S * SLOT * E * sizeof(float2));
  __shared__ float2 hs[kMaxVec];
  const int tid = threadIdx.x;
  const size_t nchunk = (N + E - 1) / E;
  const size_t mine = nchunk > blockIdx.x ? (nchunk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  auto chunk = [&](size_t q, size_t& e0, unsigned& bytes) {   // local chunk q: first entry, bytes per row
    e0 = (blockIdx.x + q * gridDim.x) * (size_t)E;
    const size_t n = N - e0 < (size_t)E ? N - e0 : (size_t)E;
    bytes = (unsigned)(((n + 1) & ~(size_t)1) * sizeof(float2));
  };
  auto issue_v = [&](size_t q) {                     // arm stage q % S for all rows, copy the V rows
    size_t e0;
    unsigned bytes;
    chunk(q, e0, bytes);
    float2* dst = stage + (size_t)(q % S) * SLOT * E;
    unsigned long long* b = &bar[q % S];
    mbar_arrive_tx(b, bytes * SLOT);
#pragma unroll 1
    for (int k = 0; k < NV; ++k) bulk_load(dst + (size_t)k * E, V + (size_t)k * ldv + e0, bytes, b);
  };
  auto issue_w = [&](size_t q) {                     // (without a w slot, w is read from global memory)
    if constexpr (Sh::WIN) {
      size_t e0;
      unsigned bytes;
      chunk(q, e0, bytes);
      bulk_load(stage + (size_t)(q % S) * SLOT * E + (size_t)NV * E,
                reinterpret_cast<const unsigned char*>(w_in) + e0 * sizeof(float2), bytes, &bar[q % S]);
    }
  };
  // The first S chunks are copied before the dependency wait where that is safe: the V rows, and
  // w for the update sweeps, were written at least two launches back, and this grid starts only
  // after the kernel before it has passed its own griddepcontrol.wait, i.e. after everything
  // before that kernel has completed and become visible.  h, and w of the dot sweep (the operator
  // writes it just before), are read after the wait.
  if (tid == 0) {
    for (int q = 0; q < S; ++q) mbar_init(&bar[q], 1);
    mbar_fence_init();
    for (size_t q = 0; q < (size_t)S && q < mine; ++q) {
      issue_v(q);
      if (MODE != 0) issue_w(q);
    }
  }
  pdl_entry();
  if (tid == 0 && MODE == 0)
    for (size_t q = 0; q < (size_t)S && q < mine; ++q) issue_w(q);
  if (MODE != 0 && tid < NV) hs[tid] = df_from_double(h[tid]);
  __syncthreads();
  float s[NA], c[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) s[k] = c[k] = 0.f;
  for (size_t q = 0; q < mine; ++q) {
    const bool ok = mbar_wait(&bar[q % S], (unsigned)((q / S) & 1));
    const float2* sv = stage + (size_t)(q % S) * SLOT * E;
    const size_t e0 = (blockIdx.x + q * gridDim.x) * (size_t)E;
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int t = tid + r * kSweepThreads;
      const size_t e = e0 + t;
      if (!ok || e >= N) continue;
      float2 wi;
      if constexpr (!Sh::WIN) {
        if constexpr (std::is_same<TW, double>::value) wi = df_from_double(reinterpret_cast<const double*>(w_in)[e]);
        else wi = reinterpret_cast<const float2*>(w_in)[e];
      } else if constexpr (std::is_same<TW, double>::value) {
        wi = df_from_double(reinterpret_cast<const double*>(sv + NV * E)[t]);
      } else {
        wi = sv[NV * E + t];
      }
      if (MODE == 0) {
        if constexpr (std::is_same<TW, double>::value) wdf[e] = wi;
#pragma unroll
        for (int k = 0; k < NV; ++k) df_dot_acc(s[k], c[k], sv[k * E + t], wi);
      } else {
        float2 odd = make_float2(0.f, 0.f);          // two chains: even k into wi, odd k apart
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          if (k & 1) odd = df_sub_prod(odd, hs[k], sv[k * E + t]);
          else wi = df_sub_prod(wi, hs[k], sv[k * E + t]);
        }
        wi = df_add(wi, odd);
        wdf[e] = wi;
        if (MODE == 1) {
#pragma unroll
          for (int k = 0; k < NA; ++k) df_dot_acc(s[k], c[k], sv[k * E + t], wi);
        } else {
          df_dot_acc(s[0], c[0], wi, wi);
        }
      }
    }
    if (!__syncthreads_and(ok)) {                    // stage q % S is free again from here on
      if (tid == 0) {                                // record, then let the copies in flight land
        atomicExch(&g_sweep_fault, 1);
        for (size_t r = q; r < q + S && r < mine; ++r) mbar_wait(&bar[r % S], (unsigned)((r / S) & 1));
      }
      break;
    }
    if (tid == 0 && q + S < mine) {
      issue_v(q + S);
      issue_w(q + S);
    }
  }
  block_partials_df<NA>(s, c, partial);
}

// v = w / sc[0] as double-float (w FP64 or double-float), and, if out is not null, v rounded to
// TO (the next V-cycle's input).
template <typename TW, typename TO>
__global__ void k_gs_scale(const TW* __restrict__ w, const double* __restrict__ sc, float2* __restrict__ v,
                           TO* __restrict__ out, size_t N) {
  pdl_entry();
  const double inv = 1.0 / sc[0];
  const float2 g = df_from_double(inv);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    float2 r;
    if constexpr (sizeof(TW) == 8 && std::is_same<TW, double>::value) {
      r = df_from_double(w[i] * inv);
    } else {                                        // double-float product, renormalised
      const float2 a = w[i];
      const float p = __fmul_rn(a.x, g.x);
      float e = fmaf(a.x, g.x, -p);
      e = fmaf(a.x, g.y, e);
      e = fmaf(a.y, g.x, e);
      const float hi = __fadd_rn(p, e);
      r = make_float2(hi, __fsub_rn(e, __fsub_rn(hi, p)));
    }
    v[i] = r;
    if (out) {
      if constexpr (sizeof(TO) == 4) out[i] = __fadd_rn(r.x, r.y);
      else out[i] = df_to_double(r);
    }
  }
}

// y = v rounded to FP32 or to FP64.
template <typename TO>
__global__ void k_df_to(const float2* __restrict__ v, TO* __restrict__ y, size_t N) {
  pdl_entry();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    const float2 a = v[i];
    if constexpr (sizeof(TO) == 4) y[i] = __fadd_rn(a.x, a.y);
    else y[i] = df_to_double(a);
  }
}

// Scratch of sbm_dots_noalloc: room for the per-block partial sums of the largest grid the dot
// kernel uses (dot_blocks() caps its grid at kDotMaxBlocks) times 32 vectors: 152 KiB per device,
// held by every GPU that loads the library until the process exits.
constexpr int kNoAllocBlocks = kDotMaxBlocks;
static_assert(kNoAllocBlocks >= kDotMaxBlocks, "the static scratch must hold the largest dot grid");
static __device__ __align__(256) double g_dots_scratch[kNoAllocBlocks * kMaxVec];
std::mutex g_dots_scratch_mu;
double* g_dots_scratch_dev[256] = {};      // last resolved address of g_dots_scratch, per device ordinal

unsigned grid_for(size_t N) {
  size_t g = (N + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

}  // namespace

std::atomic<long long> g_kernel_launches{0};

bool& pdl_enabled() {
  thread_local bool on = true;
  return on;
}

int dot_blocks(size_t N) {
  size_t g = (N + kDotChunk - 1) / kDotChunk;
  if (g < 1) g = 1;
  if (g > kDotMaxBlocks) g = kDotMaxBlocks;
  return (int)g;
}

cudaError_t launch_multi_dot(const double* V, size_t ldv, int nv, const double* w, size_t N, double* partial,
                             double* out, int take_sqrt, cudaStream_t s) {
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  const int nblk = dot_blocks(N);
  switch (nv) {
#define SBM_DOT_CASE(K) \
  case K: SBM_PDL((k_multi_dot<K>), nblk, kDotThreads, 0, s, V, ldv, w, N, partial); break;
    SBM_DOT_CASE(1) SBM_DOT_CASE(2) SBM_DOT_CASE(3) SBM_DOT_CASE(4) SBM_DOT_CASE(5) SBM_DOT_CASE(6)
    SBM_DOT_CASE(7) SBM_DOT_CASE(8) SBM_DOT_CASE(9) SBM_DOT_CASE(10) SBM_DOT_CASE(11) SBM_DOT_CASE(12)
    SBM_DOT_CASE(13) SBM_DOT_CASE(14) SBM_DOT_CASE(15) SBM_DOT_CASE(16) SBM_DOT_CASE(17) SBM_DOT_CASE(18)
    SBM_DOT_CASE(19) SBM_DOT_CASE(20) SBM_DOT_CASE(21) SBM_DOT_CASE(22) SBM_DOT_CASE(23) SBM_DOT_CASE(24)
    SBM_DOT_CASE(25) SBM_DOT_CASE(26) SBM_DOT_CASE(27) SBM_DOT_CASE(28) SBM_DOT_CASE(29) SBM_DOT_CASE(30)
    SBM_DOT_CASE(31) SBM_DOT_CASE(32)
#undef SBM_DOT_CASE
  }
  SBM_PDL(k_reduce_partials, 1, 32 * nv, 0, s, partial, nblk, nv, out, take_sqrt);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_axpy_dot(const double* V, size_t ldv, int nv, const double* h, double* w, size_t N,
                            double* partial, double* out, cudaStream_t s) {
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  const int nblk = dot_blocks(N);
  switch (nv) {
#define SBM_AD_CASE(K) \
  case K: SBM_PDL((k_axpy_dot<K, false>), nblk, kDotThreads, 0, s, V, ldv, h, w, N, nv, partial); break;
    SBM_AD_CASE(1) SBM_AD_CASE(2) SBM_AD_CASE(3) SBM_AD_CASE(4) SBM_AD_CASE(5) SBM_AD_CASE(6)
    SBM_AD_CASE(7) SBM_AD_CASE(8) SBM_AD_CASE(9) SBM_AD_CASE(10) SBM_AD_CASE(11) SBM_AD_CASE(12)
    SBM_AD_CASE(13) SBM_AD_CASE(14) SBM_AD_CASE(15) SBM_AD_CASE(16) SBM_AD_CASE(17) SBM_AD_CASE(18)
    SBM_AD_CASE(19) SBM_AD_CASE(20) SBM_AD_CASE(21) SBM_AD_CASE(22) SBM_AD_CASE(23) SBM_AD_CASE(24)
    SBM_AD_CASE(25) SBM_AD_CASE(26) SBM_AD_CASE(27) SBM_AD_CASE(28) SBM_AD_CASE(29) SBM_AD_CASE(30)
    SBM_AD_CASE(31) SBM_AD_CASE(32)
#undef SBM_AD_CASE
  }
  SBM_PDL(k_reduce_partials, 1, 32 * nv, 0, s, partial, nblk, nv, out, 0);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_axpy_norm(const double* V, size_t ldv, int nv, const double* h, double* w, size_t N,
                             double* partial, double* out, cudaStream_t s) {
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  const int nblk = dot_blocks(N);
  SBM_PDL((k_axpy_dot<0, true>), nblk, kDotThreads, 0, s, V, ldv, h, w, N, nv, partial);
  SBM_PDL(k_reduce_partials, 1, 32, 0, s, partial, nblk, 1, out, 1);
  count_launches(2);
  return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_multi_axpy(const TZ* Z, size_t ldz, int nv, const double* coef, double sign, double* w,
                              size_t N, cudaStream_t s) {
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  if constexpr (std::is_same<TZ, float>::value)
    SBM_PDL(k_multi_axpy_df, grid_for(N), 256, 0, s, Z, ldz, nv, coef, sign, w, N);
  else
    SBM_PDL((k_multi_axpy<TZ>), grid_for(N), 256, 0, s, Z, ldz, nv, coef, sign, w, N);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_div_scalar(const double* w, const double* sc, double* v, size_t N, cudaStream_t s) {
  SBM_PDL(k_div_scalar, grid_for(N), 256, 0, s, w, sc, v, N);
  count_launches();
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_cast(const TI* x, TO* y, size_t N, cudaStream_t s) {
  SBM_PDL((k_cast<TI, TO>), grid_for(N), 256, 0, s, x, y, N);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_hess_column(const double* h1, const double* h2, const double* hn, int k, double* col,
                               cudaStream_t s) {
  SBM_PDL(k_hess_column, 1, 64, 0, s, h1, h2, hn, k, col);
  count_launches();
  return cudaGetLastError();
}

int gs_blocks(size_t N) {
  const size_t g = (N + kSweepThreads - 1) / kSweepThreads;
  return (int)(g < 1 ? 1 : (g > 152 ? 152 : g));
}

template <int K, int MODE, typename TW>
cudaError_t launch_sweep_k(const float2* V, size_t ldv, const TW* w, const double* h, float2* wdf, size_t N,
                           double* partial, int* nblk_out, cudaStream_t s) {
  using Sh = SweepShape<K>;
  auto kern = k_gs_sweep<K, MODE, TW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
  if (e != cudaSuccess) return e;
  const size_t nchunk = (N + Sh::E - 1) / Sh::E;
  const int nblk = (int)(nchunk < 1 ? 1 : (nchunk > 152 ? 152 : nchunk));
  *nblk_out = nblk;
  SBM_PDL(kern, nblk, kSweepThreads, Sh::smem, s, V, ldv, w, h, wdf, N, partial);
  return cudaSuccess;
}

// One staged sweep over nv basis vectors and the reduction of its per-block partial sums into out
// (nv values for MODE 0 and 1, the norm for MODE 2).
template <int MODE, typename TW>
cudaError_t launch_sweep(const float2* V, size_t ldv, int nv, const TW* w, const double* h, float2* wdf, size_t N,
                         double* partial, double* out, cudaStream_t s, const double* h1 = nullptr,
                         double* col = nullptr) {
  if (nv < 1 || nv > kMaxVec) return cudaErrorInvalidValue;
  const size_t padded = N + (N & 1);
  if (ldv % 2 != 0 || ldv < padded || reinterpret_cast<uintptr_t>(V) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(w) % 16 != 0 || reinterpret_cast<uintptr_t>(wdf) % 16 != 0)
    return cudaErrorInvalidValue;
  int nblk = 1;
  cudaError_t e = cudaSuccess;
  switch (nv) {
#define SBM_SW_CASE(K) \
  case K: e = launch_sweep_k<K, MODE, TW>(V, ldv, w, h, wdf, N, partial, &nblk, s); break;
    SBM_SW_CASE(1) SBM_SW_CASE(2) SBM_SW_CASE(3) SBM_SW_CASE(4) SBM_SW_CASE(5) SBM_SW_CASE(6)
    SBM_SW_CASE(7) SBM_SW_CASE(8) SBM_SW_CASE(9) SBM_SW_CASE(10) SBM_SW_CASE(11) SBM_SW_CASE(12)
    SBM_SW_CASE(13) SBM_SW_CASE(14) SBM_SW_CASE(15) SBM_SW_CASE(16) SBM_SW_CASE(17) SBM_SW_CASE(18)
    SBM_SW_CASE(19) SBM_SW_CASE(20) SBM_SW_CASE(21) SBM_SW_CASE(22) SBM_SW_CASE(23) SBM_SW_CASE(24)
    SBM_SW_CASE(25) SBM_SW_CASE(26) SBM_SW_CASE(27) SBM_SW_CASE(28) SBM_SW_CASE(29) SBM_SW_CASE(30)
    SBM_SW_CASE(31) SBM_SW_CASE(32)
#undef SBM_SW_CASE
  }
  if (e != cudaSuccess) return e;
  if (MODE == 2 && col) {                            // |w| and the Hessenberg column in one launch
    if (nv + 1 > 64) return cudaErrorInvalidValue;
    SBM_PDL(k_reduce_norm_column, 1, 64, 0, s, partial, nblk, out, h1, h, nv, col);
  } else {
    const int nout = MODE == 2 ? 1 : nv;
    SBM_PDL(k_reduce_partials, 1, 32 * nout, 0, s, partial, nblk, nout, out, MODE == 2 ? 1 : 0);
  }
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_gs_dot(const float2* V, size_t ldv, int nv, const double* w, float2* wdf, size_t N,
                          double* partial, double* out, cudaStream_t s) {
  return launch_sweep<0, double>(V, ldv, nv, w, nullptr, wdf, N, partial, out, s);
}

cudaError_t launch_gs_dot_df(const float2* V, size_t ldv, int nv, const float2* wdf, size_t N, double* partial,
                             double* out, cudaStream_t s) {
  return launch_sweep<0, float2>(V, ldv, nv, wdf, nullptr, const_cast<float2*>(wdf), N, partial, out, s);
}

cudaError_t launch_gs_axpy_dot(const float2* V, size_t ldv, int nv, const double* h, float2* wdf, size_t N,
                               double* partial, double* out, cudaStream_t s) {
  return launch_sweep<1, float2>(V, ldv, nv, wdf, h, wdf, N, partial, out, s);
}

cudaError_t launch_gs_axpy_norm(const float2* V, size_t ldv, int nv, const double* h, float2* wdf, size_t N,
                                double* partial, double* out, cudaStream_t s, const double* h1, double* col) {
  return launch_sweep<2, float2>(V, ldv, nv, wdf, h, wdf, N, partial, out, s, h1, col);
}

int sweep_fault_take() {
  int f = 0;
  if (cudaMemcpyFromSymbol(&f, g_sweep_fault, sizeof(int)) != cudaSuccess) return -1;
  if (f) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_sweep_fault, &zero, sizeof(int)) != cudaSuccess) return -1;
  }
  return f;
}

template <typename TW, typename TO>
cudaError_t launch_gs_scale(const TW* w, const double* sc, float2* v, TO* out, size_t N, cudaStream_t s) {
  SBM_PDL((k_gs_scale<TW, TO>), grid_for(N), 256, 0, s, w, sc, v, out, N);
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_gs_scale<double, float>(const double*, const double*, float2*, float*, size_t,
                                                    cudaStream_t);
template cudaError_t launch_gs_scale<double, double>(const double*, const double*, float2*, double*, size_t,
                                                     cudaStream_t);
template cudaError_t launch_gs_scale<float2, float>(const float2*, const double*, float2*, float*, size_t,
                                                    cudaStream_t);
template cudaError_t launch_gs_scale<float2, double>(const float2*, const double*, float2*, double*, size_t,
                                                     cudaStream_t);

template <typename TO>
cudaError_t launch_df_to(const float2* v, TO* y, size_t N, cudaStream_t s) {
  SBM_PDL((k_df_to<TO>), grid_for(N), 256, 0, s, v, y, N);
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_df_to<float>(const float2*, float*, size_t, cudaStream_t);
template cudaError_t launch_df_to<double>(const float2*, double*, size_t, cudaStream_t);

int dots_noalloc(const double* V, long long ldv, int nv, const double* w, long long n, double* out,
                 cudaStream_t stream) {
  if (!V || !w || !out || nv < 1 || nv > kMaxVec || n < 0 || ldv < n)
    return record_error(SBM_ERR_ARG, "sbm_dots_noalloc: need non-null pointers, 1 <= nv <= 32, 0 <= n <= ldv");
  if (dot_blocks((size_t)n) > kNoAllocBlocks)
    return record_error(SBM_ERR_ARG, "sbm_dots_noalloc: grid exceeds the static scratch");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_error(SBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 256) return record_error(SBM_ERR_ARG, "sbm_dots_noalloc: device ordinal out of range");
  // The array's device address belongs to the context current on this thread, and it changes when
  // that context is replaced (cudaDeviceReset, a primary-context reset, another driver context).
  // So it is looked up again on every call made outside stream capture, where the lookup is an
  // ordinary host call; only inside a capture, where a lookup that has to load the module could
  // break the capture, the address resolved by the last call outside capture is used.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess)
    return record_error(SBM_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_dots_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_dots_scratch);
      if (e != cudaSuccess)
        return record_error(SBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_dots_scratch_dev[dev] = static_cast<double*>(p);
    } else if (!g_dots_scratch_dev[dev]) {
      return record_error(SBM_ERR_ARG, "sbm_dots_noalloc: the first call on a device must come before any "
                                       "stream capture");
    }
    scratch = g_dots_scratch_dev[dev];
  }
  e = launch_multi_dot(V, (size_t)ldv, nv, w, (size_t)n, scratch, out, 0, stream);
  if (e != cudaSuccess) return record_error(SBM_ERR_CUDA, std::string("sbm_dots_noalloc: ") + cudaGetErrorString(e));
  return SBM_OK;
}

template cudaError_t launch_multi_axpy<double>(const double*, size_t, int, const double*, double, double*, size_t,
                                               cudaStream_t);
template cudaError_t launch_multi_axpy<float>(const float*, size_t, int, const double*, double, double*, size_t,
                                              cudaStream_t);
template cudaError_t launch_cast<double, float>(const double*, float*, size_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, size_t, cudaStream_t);

}  // namespace sbm

namespace sbm {
namespace {

__device__ __align__(16) float4 g_selftest_src;

// One bounded mbarrier wait: 16 bytes announced, then copied (starve = 0) or never copied
// (starve = 1, the phase cannot complete and the wait gives up after `spin` polls).
__global__ void k_async_selftest(int starve, unsigned spin) {
  __shared__ __align__(16) float4 dst;
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
    mbar_arrive_tx(&bar, 16);
    if (!starve) bulk_load(&dst, &g_selftest_src, 16, &bar);
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, spin);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicExch(&g_sweep_fault, 1);
}

}  // namespace
}  // namespace sbm

extern "C" int sbm_async_wait_selftest(int starve, void* stream) {
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (sbm::sweep_fault_take() < 0) return sbm::record_error(SBM_ERR_CUDA, "cannot read the fault flag");
  sbm::k_async_selftest<<<1, 32, 0, s>>>(starve ? 1 : 0, 1u << 12);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return sbm::record_error(SBM_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
  sbm::count_launches();
  const int f = sbm::sweep_fault_take();
  if (f < 0) return sbm::record_error(SBM_ERR_CUDA, "cannot read the fault flag");
  if (f) return sbm::record_error(SBM_ERR_CUDA, "bounded mbarrier wait gave up: the announced copy never completed");
  return SBM_OK;
}

extern "C" int sbm_dots_noalloc(const double* V_dev, long long ldv, int nv, const double* w_dev, long long n,
                                double* out_dev, void* stream) {
  return sbm::dots_noalloc(V_dev, ldv, nv, w_dev, n, out_dev, static_cast<cudaStream_t>(stream));
}
