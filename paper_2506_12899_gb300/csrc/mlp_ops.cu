// CUDA kernels of the learned boundary-cell correction (the learned variant of the V-cycle
// smoother; the paper has no learned component): feature gather, BF16 tensor-core GEMMs with
// FP32 accumulation for the MLP forward and backward passes, loss, Adam, correction scatter.
//
// Features of boundary cell K (row of X, BF16, padded with zeros to Fpad columns):
//   [ patch residual / s  (3^d cells x (p+1)^d, x fastest, zeros for missing cells),
//     d / h on every (face slot, face point, component), kappa(K), surrogate mask per slot ]
// with s = |patch residual|_2 (1 if zero).  The correction is u_K += s * MLP(x_K).
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "ops.h"

namespace sbm {
namespace {

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// One warp per boundary cell.
template <typename TI>
__global__ void __launch_bounds__(256) k_mlp_features(int n_bnd, int npatch, int np, int nstat, int Fpad,
                                                      const int* __restrict__ patch, const float* __restrict__ stat,
                                                      const TI* __restrict__ res, __nv_bfloat16* __restrict__ X,
                                                      float* __restrict__ s_out) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n_bnd) return;
  const int nv = npatch * np;
  float ss = 0.f;
  for (int k = lane; k < nv; k += 32) {
    const int c = patch[(size_t)b * npatch + k / np];
    const float v = c >= 0 ? (float)res[(size_t)c * np + k % np] : 0.f;
    ss += v * v;
  }
  ss = warp_sumf(ss);
  const float s = ss > 0.f ? sqrtf(ss) : 1.f;
  const float inv = 1.f / s;
  __nv_bfloat16* row = X + (size_t)b * Fpad;
  for (int k = lane; k < Fpad; k += 32) {
    float v = 0.f;
    if (k < nv) {
      const int c = patch[(size_t)b * npatch + k / np];
      v = c >= 0 ? (float)res[(size_t)c * np + k % np] * inv : 0.f;
    } else if (k < nv + nstat) {
      v = stat[(size_t)b * nstat + (k - nv)];
    }
    row[k] = __float2bfloat16_rn(v);
  }
  if (lane == 0) s_out[b] = s;
}

// Tensor-core GEMM, BF16 inputs, FP32 accumulation (mma.sync m16n8k16):
//   C[m][n] = sum_k opA(m,k) opB(k,n) (+ bias[n]) (relu)
//   opA(m,k) = A[m*lda + k] (TA = 0) or A[k*lda + m] (TA = 1)
//   opB(k,n) = B[k*ldb + n] (TB = 0) or B[n*ldb + k] (TB = 1)
// Outputs: Cf (FP32, ldc) and/or Cb (BF16, ldc), either may be null.
// Block tile 64 x 64, K step 32, 4 warps of 32 x 32 (2 x 4 mma tiles).
constexpr int GT = 64, GK = 32, GPAD = 8;

template <int TA, int TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int ldb,
                                                   const float* __restrict__ bias, int relu, float* __restrict__ Cf,
                                                   __nv_bfloat16* __restrict__ Cb, int ldc) {
  __shared__ __align__(16) __nv_bfloat16 As[GT][GK + GPAD];   // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[GT][GK + GPAD];   // [n][k]
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, tg = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
      const int r = TA ? e % GT : e / GK, kk = TA ? e / GT : e % GK;
      const int m = m0 + r, k = k0 + kk;
      As[r][kk] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : zero;
    }
    for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
      const int c = TB ? e / GK : e % GT, kk = TB ? e % GK : e / GT;
      const int n = n0 + c, k = k0 + kk;
      Bs[c][kk] = (n < N && k < K) ? (TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n]) : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GK; ks += 16) {
      unsigned af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + g;
        af[i][0] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * tg]);
        af[i][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * tg]);
        af[i][2] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * tg + 8]);
        af[i][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * tg + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + g;
        bf[j][0] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * tg]);
        bf[j][1] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * tg + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + 2 * tg + (q & 1);
        if (m < M && n < N) {
          float v = acc[i][j][q];
          if (bias) v += bias[n];
          if (relu) v = fmaxf(v, 0.f);
          if (Cf) Cf[(size_t)m * ldc + n] = v;
          if (Cb) Cb[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
        }
      }
}

// dY = 2 (Y - T) / count (FP32 and BF16 copies); loss partial sums per block.
__global__ void k_mse_grad(int rows, int O, const float* __restrict__ Y, const float* __restrict__ T,
                           float* __restrict__ dYf, __nv_bfloat16* __restrict__ dYb, float inv_count,
                           float* __restrict__ loss_partial) {
  __shared__ float red[8];
  float ls = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * O; e += gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    ls += d * d;
    const float g = 2.f * d * inv_count;
    dYf[e] = g;
    dYb[e] = __float2bfloat16_rn(g);
  }
  ls = warp_sumf(ls);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ls;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    loss_partial[blockIdx.x] = s;
  }
}

// dZ = dH * (H > 0) in place on the FP32 buffer, BF16 copy out.
__global__ void k_relu_mask(int n, float* __restrict__ dH, const __nv_bfloat16* __restrict__ H,
                            __nv_bfloat16* __restrict__ dZb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float v = __bfloat162float(H[e]) > 0.f ? dH[e] : 0.f;
    dH[e] = v;
    dZb[e] = __float2bfloat16_rn(v);
  }
}

// g[n] = sum_m D[m][n] (bias gradients), one block per column, fixed order.
__global__ void k_colsum(int rows, int cols, const float* __restrict__ D, float* __restrict__ g) {
  const int n = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < rows; m += blockDim.x) s += D[(size_t)m * cols + n];
  __shared__ float red[8];
  s = warp_sumf(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g[n] = t;
  }
}

// Adam (Kingma & Ba) on FP32 master parameters; writes the BF16 copy used by the forward pass.
__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float w = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = w;
    if (pb) pb[e] = __float2bfloat16_rn(w);
  }
}

__global__ void k_to_bf16(int n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    y[e] = __float2bfloat16_rn(x[e]);
}

// T[b][i] = -u[cell(b)][i] / s[b]  (training target: the error of u for the zero solution).
template <typename TU>
__global__ void k_mlp_targets(int n_bnd, int np, const int* __restrict__ cell, const TU* __restrict__ u,
                              const float* __restrict__ s, float hfac, float* __restrict__ T) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_bnd * np; e += gridDim.x * blockDim.x) {
    const int b = e / np, i = e % np;
    T[e] = -(float)u[(size_t)cell[b] * np + i] * hfac / s[b];
  }
}

// Sum of squares of x[0..n) in per-block FP64 partial sums, then one fixed-order sum (deterministic).
__global__ void __launch_bounds__(256) k_sumsq_partial(size_t n, const float* __restrict__ x, double* __restrict__ part) {
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    acc += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_sum_final(int nblk, const double* __restrict__ part, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[b];
    out[0] = s;
  }
}
__global__ void k_scale_f(size_t n, float a, float* __restrict__ x) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] *= a;
}

// z[cell(b)][i] += scale * s[b] * Y[b][i]
template <typename TZ>
__global__ void k_mlp_scatter(int n_bnd, int np, int ldy, const int* __restrict__ cell, const float* __restrict__ Y,
                              const float* __restrict__ s, float scale, TZ* __restrict__ z) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_bnd * np; e += gridDim.x * blockDim.x) {
    const int b = e / np, i = e % np;
    z[(size_t)cell[b] * np + i] += (TZ)(scale * s[b] * Y[(size_t)b * ldy + i]);
  }
}

// Minibatch rows: Xb[r] = X[idx[r]] (width bf16 values), Tb[r] = T[idx[r]] (owidth floats).
__global__ void k_rows_gather(int rows, int width, const int* __restrict__ idx, const __nv_bfloat16* __restrict__ X,
                              __nv_bfloat16* __restrict__ Xb, int owidth, const float* __restrict__ T,
                              float* __restrict__ Tb) {
  const int r = blockIdx.x;
  if (r >= rows) return;
  const size_t src = (size_t)idx[r];
  for (int k = threadIdx.x; k < width; k += blockDim.x) Xb[(size_t)r * width + k] = X[src * width + k];
  for (int k = threadIdx.x; k < owidth; k += blockDim.x) Tb[(size_t)r * owidth + k] = T[src * owidth + k];
}

__global__ void k_axpy_f(size_t n, float a, const float* __restrict__ x, float* __restrict__ y) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] += a * x[e];
}

// Xb[r][k] = bf16(X[r][k]) for k < F, 0 for F <= k < Fpad.
__global__ void k_pack_bf16(int rows, int F, int Fpad, const float* __restrict__ X, __nv_bfloat16* __restrict__ Xb) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)rows * Fpad;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / Fpad;
    const int k = (int)(e % Fpad);
    Xb[e] = __float2bfloat16_rn(k < F ? X[r * F + k] : 0.f);
  }
}

// X[r][k] = float(Xb[r][k]) for k < F.
__global__ void k_unpack_bf16(int rows, int F, int Fpad, const __nv_bfloat16* __restrict__ Xb, float* __restrict__ X) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)rows * F;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / F;
    const int k = (int)(e % F);
    X[e] = __bfloat162float(Xb[r * Fpad + k]);
  }
}

// y += x
template <typename R>
__global__ void k_add(size_t n, const R* __restrict__ x, R* __restrict__ y) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    y[e] += x[e];
}

unsigned g1(int n) { return (unsigned)((n + 255) / 256 > 152 * 8 ? 152 * 8 : (n + 255) / 256 < 1 ? 1 : (n + 255) / 256); }

}  // namespace

cudaError_t launch_rows_gather(int rows, int width, const int* idx, const __nv_bfloat16* X, __nv_bfloat16* Xb,
                               int owidth, const float* T, float* Tb, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  k_rows_gather<<<rows, 128, 0, s>>>(rows, width, idx, X, Xb, owidth, T, Tb);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_axpy_f(size_t n, float a, const float* x, float* y, cudaStream_t s) {
  k_axpy_f<<<g1((int)(n < 0x7fffffff ? n : 0x7fffffff)), 256, 0, s>>>(n, a, x, y);
  count_launches();
  return cudaGetLastError();
}

template <typename TI>
cudaError_t launch_mlp_features(int n_bnd, int npatch, int np, int nstat, int Fpad, const int* patch,
                                const float* stat, const TI* res, __nv_bfloat16* X, float* s, cudaStream_t st) {
  if (n_bnd == 0) return cudaSuccess;
  k_mlp_features<TI><<<(n_bnd + 7) / 8, 256, 0, st>>>(n_bnd, npatch, np, nstat, Fpad, patch, stat, res, X, s);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_gemm_bf16(int M, int N, int K, int ta, int tb, const __nv_bfloat16* A, int lda,
                             const __nv_bfloat16* B, int ldb, const float* bias, int relu, float* Cf,
                             __nv_bfloat16* Cb, int ldc, cudaStream_t s) {
  if (M == 0 || N == 0) return cudaSuccess;
  const dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  if (!ta && !tb) k_gemm_bf16<0, 0><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc);
  else if (!ta && tb) k_gemm_bf16<0, 1><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc);
  else if (ta && !tb) k_gemm_bf16<1, 0><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc);
  else k_gemm_bf16<1, 1><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_mse_grad(int rows, int O, const float* Y, const float* T, float* dYf, __nv_bfloat16* dYb,
                            float inv_count, float* loss_partial, int nblk, cudaStream_t s) {
  k_mse_grad<<<nblk, 256, 0, s>>>(rows, O, Y, T, dYf, dYb, inv_count, loss_partial);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(int n, float* dH, const __nv_bfloat16* H, __nv_bfloat16* dZb, cudaStream_t s) {
  k_relu_mask<<<g1(n), 256, 0, s>>>(n, dH, H, dZb);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_colsum(int rows, int cols, const float* D, float* g, cudaStream_t s) {
  k_colsum<<<cols, 256, 0, s>>>(rows, cols, D, g);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_adam(int n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<g1(n), 256, 0, s>>>(n, p, g, m, v, pb, lr, b1, b2, eps, c1, c2);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(int n, const float* x, __nv_bfloat16* y, cudaStream_t s) {
  k_to_bf16<<<g1(n), 256, 0, s>>>(n, x, y);
  count_launches();
  return cudaGetLastError();
}

template <typename TU>
cudaError_t launch_mlp_targets(int n_bnd, int np, const int* cell, const TU* u, const float* s, float hfac,
                               float* T, cudaStream_t st) {
  k_mlp_targets<TU><<<g1(n_bnd * np), 256, 0, st>>>(n_bnd, np, cell, u, s, hfac, T);
  count_launches();
  return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_mlp_scatter(int n_bnd, int np, int ldy, const int* cell, const float* Y, const float* s,
                               float scale, TZ* z, cudaStream_t st) {
  k_mlp_scatter<TZ><<<g1(n_bnd * np), 256, 0, st>>>(n_bnd, np, ldy, cell, Y, s, scale, z);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_pack_bf16(int rows, int F, int Fpad, const float* X, __nv_bfloat16* Xb, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  k_pack_bf16<<<g1((int)std::min<size_t>((size_t)rows * Fpad, 1u << 30)), 256, 0, s>>>(rows, F, Fpad, X, Xb);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_unpack_bf16(int rows, int F, int Fpad, const __nv_bfloat16* Xb, float* X, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  k_unpack_bf16<<<g1((int)std::min<size_t>((size_t)rows * F, 1u << 30)), 256, 0, s>>>(rows, F, Fpad, Xb, X);
  count_launches();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_add(size_t n, const R* x, R* y, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_add<R><<<g1((int)std::min<size_t>(n, 1u << 30)), 256, 0, s>>>(n, x, y);
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_add<float>(size_t, const float*, float*, cudaStream_t);
template cudaError_t launch_add<double>(size_t, const double*, double*, cudaStream_t);

template cudaError_t launch_mlp_features<float>(int, int, int, int, int, const int*, const float*, const float*,
                                                __nv_bfloat16*, float*, cudaStream_t);
template cudaError_t launch_mlp_features<double>(int, int, int, int, int, const int*, const float*, const double*,
                                                 __nv_bfloat16*, float*, cudaStream_t);
template cudaError_t launch_mlp_targets<float>(int, int, const int*, const float*, const float*, float, float*, cudaStream_t);
template cudaError_t launch_mlp_targets<double>(int, int, const int*, const double*, const float*, float, float*,
                                                cudaStream_t);
template cudaError_t launch_mlp_scatter<float>(int, int, int, const int*, const float*, const float*, float, float*,
                                               cudaStream_t);
template cudaError_t launch_mlp_scatter<double>(int, int, int, const int*, const float*, const float*, float, double*,
                                                cudaStream_t);

}  // namespace sbm

namespace sbm {
cudaError_t launch_sumsq(size_t n, const float* x, double* part, int nblk, double* out, cudaStream_t st) {
  k_sumsq_partial<<<nblk, 256, 0, st>>>(n, x, part);
  k_sum_final<<<1, 32, 0, st>>>(nblk, part, out);
  count_launches(2);
  return cudaGetLastError();
}
cudaError_t launch_scale_f(size_t n, float a, float* x, cudaStream_t st) {
  size_t g = (n + 255) / 256;
  k_scale_f<<<(unsigned)(g < 1 ? 1 : (g > 1216 ? 1216 : g)), 256, 0, st>>>(n, a, x);
  count_launches();
  return cudaGetLastError();
}
}  // namespace sbm
