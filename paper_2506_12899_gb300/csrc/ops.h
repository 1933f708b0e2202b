// Host-side launchers of the libsbm CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include "sbm_internal.h"

#include <atomic>
#include <string>

namespace sbm {

// Number of kernel launches issued by the library since it was loaded.
extern std::atomic<long long> g_kernel_launches;
inline void count_launches(long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// Sets the calling thread's sbm_last_error() message and returns code.
int record_error(int code, const std::string& msg);

// Body of sbm_dots_noalloc (static scratch, no allocation).
int dots_noalloc(const double* V, long long ldv, int nv, const double* w, long long n, double* out,
                 cudaStream_t stream);

// Thread-per-cell kernels (cell_ops.cu) serve levels with (p+1)^d <= 16: 2D, and 3D with p = 1.
bool cell_kernels(int dim, int p);
template <typename TI, typename R>
cudaError_t launch_apply_cell(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                              cudaStream_t s);
template <typename R>
cudaError_t launch_smooth_cell(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f,
                               R* u, cudaStream_t s);
template <typename R>
cudaError_t launch_resid_restrict_p_cell(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T,
                                        const R* u, const R* f, R* rc, cudaStream_t s);
template <typename R>
cudaError_t launch_resid_restrict_h_cell(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                        const R* f, R* rc, cudaStream_t s);

// The V-cycle of levels 0..top (p = 1 h-levels) in one thread-block-cluster launch; z = M^{-1} r
// on level top.  cudaErrorNotSupported if no cluster of 8 or more CTAs fits.
template <typename R>
cudaError_t launch_vcycle_tail(int dim, const TailLevel<R>* TL, int top, const R* r, R* z, const double* coarse_inv,
                               int pre, int post, cudaStream_t s);
int tail_cluster_size(int dim, int prec);

// y = A x (mode 0) or y = f - A x (mode 1) on one level; TI is the input precision, R the
// compute / output precision.
template <typename TI, typename R>
cudaError_t launch_apply(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                         cudaStream_t s);

// One coloured block Gauss-Seidel sweep (all colours, forward or reverse).  zero_start (forward
// only): u holds zeros on entry and is not read or cleared beforehand.
template <typename R>
cudaError_t launch_smooth(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f, R* u,
                          cudaStream_t s);

// rc = P^T (f - A u) for a p-transfer (same mesh, degree pf -> pf - 1), residual not stored.
template <typename R>
cudaError_t launch_resid_restrict_p(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                   const R* f, R* rc, cudaStream_t s);
// rc = P^T (f - A u) for an h-transfer (p = 1, coarse cells gather their children).
template <typename R>
cudaError_t launch_resid_restrict_h(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                   const R* f, R* rc, cudaStream_t s);
// rc = P^T rf (restriction) and uf += P ec (prolongation) between level l-1 and l.
template <typename R>
cudaError_t launch_restrict(int dim, int pf, int pc, const TransferParams<R>& T, const R* rf, R* rc, cudaStream_t s);
template <typename R>
cudaError_t launch_prolong(int dim, int pf, int pc, const TransferParams<R>& T, const R* ec, R* uf, cudaStream_t s);

// e = Ainv r, dense FP64 matrix, N x N row-major.
template <typename T>
cudaError_t launch_coarse(const double* Ainv, int N, const T* r, T* e, cudaStream_t s);

// ---------------------------------------------------------------- FGMRES building blocks (FP64)
// Number of partial-sum blocks used for vectors of length N (fixed per N: deterministic sums).
int dot_blocks(size_t N);
// out[k] = sum_i V[k*ldv + i] w[i], k < nv (nv <= 32); partial holds dot_blocks(N)*32 doubles.
cudaError_t launch_multi_dot(const double* V, size_t ldv, int nv, const double* w, size_t N, double* partial,
                             double* out, int take_sqrt, cudaStream_t s);
// w <- w - sum_k h[k] V_k, then out[k] = V_k . w (k < nv): the second classical Gram-Schmidt
// pass fused with the update of the first.
cudaError_t launch_axpy_dot(const double* V, size_t ldv, int nv, const double* h, double* w, size_t N,
                            double* partial, double* out, cudaStream_t s);
// w <- w - sum_k h[k] V_k, then out[0] = |w|.
cudaError_t launch_axpy_norm(const double* V, size_t ldv, int nv, const double* h, double* w, size_t N,
                             double* partial, double* out, cudaStream_t s);
// w[i] += sign * sum_k coef[k] Z[k*ldz + i]
template <typename TZ>
cudaError_t launch_multi_axpy(const TZ* Z, size_t ldz, int nv, const double* coef, double sign, double* w,
                              size_t N, cudaStream_t s);
// v = w / (*s)
cudaError_t launch_div_scalar(const double* w, const double* s, double* v, size_t N, cudaStream_t st);
// y = (TO) x
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* x, TO* y, size_t N, cudaStream_t s);
// c = a + b (k <= 32 entries), c[k] = hn at index k
cudaError_t launch_hess_column(const double* h1, const double* h2, const double* hn, int k, double* col,
                               cudaStream_t s);

}  // namespace sbm
