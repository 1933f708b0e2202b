// L2 error of a discrete solution against the manufactured solution (the error measure of the
// paper's convergence studies, Sec. 5.1 and Sec. 5.4): ||u - u_h||_{L2} over the active cells of
// the finest level (the surrogate domain), with the (p+3)-point tensor Gauss-Legendre rule on each
// cell.  One thread per cell evaluates u_h at the quadrature points by sum factorisation of the
// 1D Lagrange values, forms the squared error against u, and the block sums in FP64; the partial
// sums are added in a fixed order by one block, so the result is deterministic.
#include <cuda_runtime.h>

#include "ops.h"

namespace sbm {
namespace {

constexpr int kErrThreads = 128;

// Manufactured solutions u (f = -Laplace u, g = u; Sec. 5.1, Eq. 23 for SBM_U_COSSIN, Sec. 5.4 for
// SBM_U_PHIP1 = phi + 1 of the complex domain).
__device__ double u_exact_dev(int kind, int dim, double x, double y, double z) {
  const double pi = 3.141592653589793238462643383279502884;
  switch (kind) {
    case SBM_U_SINPROD: {
      const double v = sin(pi * x) * sin(pi * y);
      return dim == 3 ? v * sin(pi * z) : v;
    }
    case SBM_U_EXPCOS: return exp(x) * cos(2.0 * y);
    case SBM_U_LINEAR: return 0.5 + x - 0.7 * y + 0.3 * z;
    case SBM_U_COSSIN: return 2.0 * cos(x) * sin(y);
    case SBM_U_QUADRATIC:
      return 0.5 + x - 0.7 * y + 0.3 * z + x * x - 0.5 * y * y + 0.25 * x * y - 0.4 * z * z + 0.2 * y * z;
    case SBM_U_PHIP1: {
      const double s = sin(pi * x);
      return (1.0 - 0.75 * s * s) * (x * x + y * y) + 0.8;
    }
  }
  return 0.0;
}

template <int D, int N1, int M1>
__global__ void __launch_bounds__(kErrThreads) k_l2_error(const __grid_constant__ L2ErrorParams E,
                                                          const int* __restrict__ cell, const double* __restrict__ x,
                                                          double* __restrict__ partial) {
  constexpr int NP = D == 2 ? N1 * N1 : N1 * N1 * N1;
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (a < E.n_act) {
    double u[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) u[i] = x[(size_t)a * NP + i];
    const int c0 = cell[3 * a], c1 = cell[3 * a + 1], c2 = cell[3 * a + 2];
#pragma unroll 1
    for (int q2 = 0; q2 < (D == 3 ? M1 : 1); ++q2) {
      // contract the z direction first (3D), then y, then x: u_h at quadrature point (q0, q1, q2)
      double s2[N1 * N1];
#pragma unroll
      for (int j = 0; j < N1 * N1; ++j) {
        double v = 0.0;
        if (D == 3) {
#pragma unroll
          for (int k = 0; k < N1; ++k) v += E.V[q2 * kMaxN1 + k] * u[j + N1 * N1 * k];
        } else {
          v = u[j];
        }
        s2[j] = v;
      }
      const double z = D == 3 ? E.lo[2] + E.h * (c2 + E.xq[q2]) : 0.0;
      const double wz = D == 3 ? E.wq[q2] : 1.0;
#pragma unroll 1
      for (int q1 = 0; q1 < M1; ++q1) {
        double s1[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          double v = 0.0;
#pragma unroll
          for (int k = 0; k < N1; ++k) v += E.V[q1 * kMaxN1 + k] * s2[i + N1 * k];
          s1[i] = v;
        }
        const double y = E.lo[1] + E.h * (c1 + E.xq[q1]);
#pragma unroll 1
        for (int q0 = 0; q0 < M1; ++q0) {
          double uh = 0.0;
#pragma unroll
          for (int k = 0; k < N1; ++k) uh += E.V[q0 * kMaxN1 + k] * s1[k];
          const double xx = E.lo[0] + E.h * (c0 + E.xq[q0]);
          const double e = u_exact_dev(E.kind, D, xx, y, z) - uh;
          acc += wz * E.wq[q1] * E.wq[q0] * e * e;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red[kErrThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kErrThreads / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

// out[0] = sqrt(h^d sum of the partial sums), summed in a fixed order.
__global__ void __launch_bounds__(256) k_l2_finish(const double* __restrict__ partial, int nblk, double hd,
                                                   double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += 256) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sqrt(hd * red[0]);
}

}  // namespace

int l2_error_blocks(int n_act) { return n_act < 1 ? 1 : (n_act + kErrThreads - 1) / kErrThreads; }

cudaError_t launch_l2_error(int dim, int p, const L2ErrorParams& E, const int* cell, const double* x,
                            double* partial, double* out, cudaStream_t s) {
  const int nblk = l2_error_blocks(E.n_act);
#define SBM_L2(D, N1) k_l2_error<D, N1, N1 + 2><<<nblk, kErrThreads, 0, s>>>(E, cell, x, partial)
  if (dim == 2 && p == 1) SBM_L2(2, 2);
  else if (dim == 2 && p == 2) SBM_L2(2, 3);
  else if (dim == 2 && p == 3) SBM_L2(2, 4);
  else if (dim == 3 && p == 1) SBM_L2(3, 2);
  else if (dim == 3 && p == 2) SBM_L2(3, 3);
  else if (dim == 3 && p == 3) SBM_L2(3, 4);
  else return cudaErrorInvalidValue;
#undef SBM_L2
  double hd = E.h * E.h * (dim == 3 ? E.h : 1.0);
  k_l2_finish<<<1, 256, 0, s>>>(partial, nblk, hd, out);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace sbm
