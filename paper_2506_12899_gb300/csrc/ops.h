// Host-side launchers of the libsbm CUDA kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "dfloat.h"
#include "sbm_internal.h"

#include <atomic>
#include <string>

namespace sbm {

// Number of kernel launches issued by the library since it was loaded.
extern std::atomic<long long> g_kernel_launches;
inline void count_launches(long long n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// Programmatic dependent launch.  A kernel launched through SBM_PDL may be scheduled while the
// previous kernel of its stream is still running; it starts with pdl_entry(), which waits until
// that kernel has completed and its memory operations are visible (griddepcontrol.wait) and then
// lets the next kernel be scheduled (griddepcontrol.launch_dependents, which takes effect once
// every CTA of the grid has issued it or exited, so a waiting grid never holds back the blocks
// of the one before it).  This hides the launch latency between the many short kernels of a
// V-cycle.  pdl_enabled() is per calling thread and follows the context in use.
bool& pdl_enabled();

#ifdef __CUDACC__
// The two halves of pdl_entry, for kernels that first read data no earlier kernel writes (level
// tables, transfer maps, geometry: written once at set-up) and so overlap that latency with the
// end of the kernel before them.  Nothing a previous kernel writes may be read before pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_entry() {
  pdl_wait();
  pdl_trigger();
}

// Bulk asynchronous copies into shared memory (cp.async.bulk), completion counted in bytes on an
// mbarrier.  Every wait is bounded: mbar_wait gives up after kAsyncSpin polls and returns false,
// and the caller records the failure in a flag the host reads.
constexpr unsigned kAsyncSpin = 1u << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised mbarriers visible to the asynchronous proxy; call before the CTA syncs.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// One arrival that also announces `bytes` of asynchronous copies on the barrier's current phase.
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
      "r"(bytes)
      : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global memory to
// this CTA's shared memory.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Waits for the phase of parity `parity` to complete; false after `limit` unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned limit = kAsyncSpin) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Launches `kernel` (parenthesised if it has template arguments) with PDL; returns the error
// from the enclosing launcher on failure.
#define SBM_PDL(kernel, grid, block, smem, stream, ...)                                                \
  do {                                                                                                \
    const cudaError_t sbm_e_ = ::sbm::launch_pdl(kernel, dim3(grid), dim3(block), smem, stream, __VA_ARGS__); \
    if (sbm_e_ != cudaSuccess) return sbm_e_;                                                         \
  } while (0)
#endif

// Sets the calling thread's sbm_last_error() message and returns code.
int record_error(int code, const std::string& msg);

// Body of sbm_dots_noalloc (static scratch, no allocation).
int dots_noalloc(const double* V, long long ldv, int nv, const double* w, long long n, double* out,
                 cudaStream_t stream);

// Colour groups of the coloured smoother.  Colour c(K) = sum_k (i_k mod 2) 2^k; face neighbours
// differ in exactly one index parity, so a neighbour of colour c has colour c ^ 2^k: lower than c
// (visited earlier in the forward order 0, 1, ..., 2^d - 1) exactly when it has one odd bit less.
// Cells of colours with the same number g of odd bits therefore never neighbour one another, and
// the forward sweep over colours equals the sweep over groups g = 0..d (reverse: d..0) with all
// colours of a group updated by one launch: every cell reads the same neighbour values.
// With red-black ordering (LevelParams::ordering = 1) the groups are the two index-sum parities,
// popcount(c) mod 2: a face changes one index by one, so cells of equal parity never neighbour.
// smooth_segs lists the segments of group g with cpb cells per block.
template <typename R>
inline int colour_group(const LevelParams<R>& P, int c) {
  const int pc = __builtin_popcount((unsigned)c);
  return P.ordering == 1 ? (pc & 1) : pc;
}
template <typename R>
inline int n_colour_groups(const LevelParams<R>& P, int dim) {
  return P.ordering == 1 ? 2 : dim + 1;
}

// Modes of the smoother kernels' zero_start argument: which values of u a launch may treat as zero.
//   0: none (u holds the current iterate);
//   1: a forward colour-group sweep from u = 0: the cell's own u and its neighbours of later groups
//      (colour with one more odd bit) are zero;
//   2: every neighbour and the cell's own u are zero (the launch applies omega A_KK^-1 f);
//   3: the cell's own u is zero, every neighbour is current (later red-black group from u = 0).
enum { kZeroNone = 0, kZeroLater = 1, kZeroAll = 2, kZeroSelf = 3 };

template <typename R>
inline SmoothSegs smooth_segs(const LevelParams<R>& P, int dim, int g, int cpb) {
  SmoothSegs G{};
  G.n = 0;
  G.blk[0] = 0;
  for (int c = 0; c < (1 << dim); ++c) {
    if (colour_group(P, c) != g) continue;
    const int cs = P.colour_start[c], ce = P.colour_start[c + 1], nb = P.colour_nbnd[c];
    const int lo[2] = {cs, cs + nb}, hi[2] = {cs + nb, ce};
    for (int part = 0; part < 2; ++part) {
      if (hi[part] <= lo[part]) continue;
      const int k = G.n++;
      G.first[k] = lo[part];
      G.last[k] = hi[part];
      G.col[k] = c;
      G.cs[k] = cs;
      G.nbnd[k] = nb;
      G.b0[k] = P.bstart[c];
      G.blk[k + 1] = G.blk[k] + (hi[part] - lo[part] + cpb - 1) / cpb;
    }
  }
  return G;
}

// Cells of colour group g.
template <typename R>
inline int group_cells(const LevelParams<R>& P, int dim, int g) {
  int n = 0;
  for (int c = 0; c < (1 << dim); ++c)
    if (colour_group(P, c) == g) n += P.colour_start[c + 1] - P.colour_start[c];
  return n;
}

// Zero mode of the launch of group index q (0-based in sweep order) of a forward sweep started from
// u = 0: colour groups skip the later groups' neighbours; red-black treats every neighbour as zero
// in its first group and none in its second.
template <typename R>
inline int group_zero_mode(const LevelParams<R>& P, int zero_start, int q) {
  if (zero_start != kZeroLater) return zero_start;
  if (P.ordering == 1) return q == 0 ? kZeroAll : kZeroSelf;
  return kZeroLater;
}

// Thread-per-cell kernels (cell_ops.cu): cell_kernels covers the FP32 operator and the fused
// residual + restriction (2D, 3D p <= 2); cell_smoother the smoother and the double-float Arnoldi
// operator ((p+1)^d <= 16: 2D, 3D p = 1).  At 3D p = 2 one thread per cell is slower for those two
// (smoother 0.09 of HBM at 128^3 even with the 16-byte window loads; the double-float operator
// needs 255 registers per thread), and the thread-per-line kernels below take them.
bool cell_kernels(int dim, int p);
// Thread-per-line kernels (line_ops.cu), 3D p = 2 and 3: the operator (x FP32, arithmetic and y
// FP32 or double-float), the FP32 smoother, and (p = 3) the FP32 fused residual + restriction to
// p = 2; line_kernels, line_smoother and line_kernels_df say where each runs.  Vectors 16-byte
// aligned.
bool line_kernels(int dim, int p);      // FP32 operator, residual + restriction
bool line_smoother(int dim, int p);     // FP32 smoother
bool line_kernels_df(int dim, int p);   // double-float operator
template <typename R>
cudaError_t launch_apply_line(int p, const LevelParams<R>& P, const float* x, const R* f, R* y, int mode,
                              cudaStream_t s);
cudaError_t launch_resid_restrict_line(const LevelParams<float>& P, const TransferParams<float>& T, const float* u,
                                       const float* f, float* rc, cudaStream_t s, int early);
cudaError_t launch_smooth_line(int p, const LevelParams<float>& P, int reverse, int zero_start, const float* f,
                               float* u, cudaStream_t s, int early, int first_group);
bool cell_smoother(int dim, int p);
template <typename TI, typename R>
cudaError_t launch_apply_cell(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                              cudaStream_t s);
template <typename R>
cudaError_t launch_smooth_cell(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f,
                               R* u, cudaStream_t s, int early, int first_group = 0);
// Pc, zc non-null: the launch also performs the first colour group (colour 0) of the coarse level's
// first pre-smoothing sweep from zero, zc_K = omega A_KK^-1 rc_K (Pc: the coarse level's parameters).
template <typename R>
cudaError_t launch_resid_restrict_p_cell(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T,
                                        const R* u, const R* f, R* rc, cudaStream_t s, int early,
                                        const LevelParams<R>* Pc = nullptr, R* zc = nullptr);
template <typename R>
cudaError_t launch_resid_restrict_h_cell(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                        const R* f, R* rc, cudaStream_t s, int early,
                                        const LevelParams<R>* Pc = nullptr, R* zc = nullptr);

// Staged thread-per-cell kernels (staged_ops.cu), FP32 only: the CTA copies its cells and their
// face neighbours into shared memory with coalesced asynchronous copies before the per-cell
// arithmetic (2D p <= 3, 3D p <= 2).  Used for launches over >= LevelParams::staged_min cells.
bool staged_kernels(int dim, int p);
cudaError_t launch_apply_staged(int dim, int p, const LevelParams<float>& P, const float* x, const float* f,
                                float* y, int mode, cudaStream_t s);
cudaError_t launch_smooth_staged(int dim, int p, const LevelParams<float>& P, int reverse, int zero_start,
                                 const float* f, float* u, cudaStream_t s, int early);

// The V-cycle of levels 0..top (p = 1 h-levels) in one thread-block-cluster launch with the
// level vectors in shared memory; z = M^{-1} r on level top.  cudaErrorNotSupported if the plan
// has no cluster.
template <typename R>
cudaError_t launch_vcycle_tail(int dim, const TailLevel<R>* TL, int top, const R* r, R* z, const double* coarse_inv,
                               int pre, int post, int ssor, const TailPlan& plan, cudaStream_t s);
// Largest dynamic shared memory a tail CTA may use, and whether a cluster of `size` CTAs with
// `smem` bytes each can be resident (prec 0: FP64, 1: FP32).
size_t tail_smem_limit();
// The one-CTA tail (TailCta): whether `smem` bytes fit (sets the kernel's shared-memory limit),
// and the launch.  coarse_inv: the FP64 coarse inverse, row-major; coarse_invT: its transpose,
// FP64 for R = double and double-float (dfl) for R = float, staged when TP.cinv_off != 0.
bool tail_cta_fits(int dim, int prec, size_t smem, size_t param_bytes);
template <typename R>
cudaError_t launch_vcycle_tail_cta(int dim, const TailCta<R>& TP, const R* r, R* z, const double* coarse_inv,
                                   const void* coarse_invT, size_t smem, cudaStream_t s);
bool tail_cluster_fits(int dim, int prec, int size, size_t smem);

// y = A x (mode 0) or y = f - A x (mode 1) on one level; TI is the input precision, R the
// compute / output precision.
template <typename TI, typename R>
cudaError_t launch_apply(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                         cudaStream_t s);

// `early` (smoother, residual + restriction, prolongation): 1 when f, respectively uf, was written
// two or more launches before the call, so the kernels may read it before griddepcontrol.wait
// (the kernel before them has then passed its own wait, and everything earlier is complete).
// 0 (the default) is always safe.
//
// One coloured block Gauss-Seidel sweep (all colours, forward or reverse), one launch per colour
// group (smooth_segs).  zero_start (forward only): u holds zeros on entry and is not read or
// cleared beforehand.
// first_group > 0 (forward sweeps only): the sweep starts at that colour group, the earlier ones
// having been done by a fused kernel (launch_resid_restrict_*_cell with Pc, zc).
template <typename R>
cudaError_t launch_smooth(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f, R* u,
                          cudaStream_t s, int early = 0, int first_group = 0);

// Update step of the additive smoothers after y = D^-1 r (modes in level_ops.cu: z = b y, z += b y,
// and the Chebyshev d = a d + b y, z += d forms).
template <typename R>
cudaError_t launch_smoother_update(size_t n, R a, R b, const R* y, R* d, R* z, int mode, cudaStream_t s);

// rc = P^T (f - A u) for a p-transfer (same mesh, degree pf -> pf - 1), residual not stored.
template <typename R>
cudaError_t launch_resid_restrict_p(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                   const R* f, R* rc, cudaStream_t s, int early = 0, const LevelParams<R>* Pc = nullptr,
                                   R* zc = nullptr);
// rc = P^T (f - A u) for an h-transfer (p = 1, coarse cells gather their children).
template <typename R>
cudaError_t launch_resid_restrict_h(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                   const R* f, R* rc, cudaStream_t s, int early = 0, const LevelParams<R>* Pc = nullptr,
                                   R* zc = nullptr);
// Whether launch_resid_restrict_{p,h} can fuse the coarse level's first colour group (it takes the
// thread-per-cell path there and the coarse level's smoother would take it too).
template <typename R>
bool restrict_fuses_first_group(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T, int pc,
                                const LevelParams<R>& Pc);
// rc = P^T rf (restriction) and uf += P ec (prolongation) between level l-1 and l.
template <typename R>
cudaError_t launch_restrict(int dim, int pf, int pc, const TransferParams<R>& T, const R* rf, R* rc, cudaStream_t s);
template <typename R>
cudaError_t launch_prolong(int dim, int pf, int pc, const TransferParams<R>& T, const R* ec, R* uf, cudaStream_t s,
                           int early = 0);

// ||u - u_h||_L2 over the active cells of a level (error_ops.cu): per-block partial sums into
// partial (l2_error_blocks(n_act) doubles), then out[0] on the device.  cell: [n_act][3] background
// indices, x: FP64 solution in compact layout.
int l2_error_blocks(int n_act);
cudaError_t launch_l2_error(int dim, int p, const L2ErrorParams& E, const int* cell, const double* x,
                            double* partial, double* out, cudaStream_t s);

// e = Ainv r, dense FP64 matrix, N x N row-major.
template <typename T>
cudaError_t launch_coarse(const double* Ainv, int N, const T* r, T* e, cudaStream_t s);

// ---------------------------------------------------------------- FGMRES building blocks (FP64)
// Number of partial-sum blocks used for vectors of length N (fixed per N: deterministic sums).
int dot_blocks(size_t N);
// Upper bound on the blocks of the double-float Gram-Schmidt sweeps (rows of their partial sums).
int gs_blocks(size_t N);
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
// Gram-Schmidt on a double-float basis V (pairs hi, lo of FP32 per entry, Dekker 1971), with w
// carried between the sweeps as double-float in wdf:
//   gs_dot:        wdf = w (FP64 in), out = V^T w
//   gs_axpy_dot:   wdf -= V h, out = V^T wdf
//   gs_axpy_norm:  wdf -= V h, out = |wdf|
//   gs_scale:      v = w / s[0] (w FP64 or double-float), and out = v rounded to TO if non-null
// The first four stream V and w through shared memory with bulk asynchronous copies: V, w and
// wdf must be 16-byte aligned, ldv even and >= N rounded up to even, and w / wdf hold that many
// entries (cudaErrorInvalidValue otherwise).  A copy that does not complete in bounded time sets
// a flag that sweep_fault_take() returns (1) and clears; -1 if the flag cannot be read.
cudaError_t launch_gs_dot(const float2* V, size_t ldv, int nv, const double* w, float2* wdf, size_t N,
                          double* partial, double* out, cudaStream_t s);
// gs_dot with w already double-float (wdf, read only)
cudaError_t launch_gs_dot_df(const float2* V, size_t ldv, int nv, const float2* wdf, size_t N, double* partial,
                             double* out, cudaStream_t s);
cudaError_t launch_gs_axpy_dot(const float2* V, size_t ldv, int nv, const double* h, float2* wdf, size_t N,
                               double* partial, double* out, cudaStream_t s);
// With col: also col[i] = h1[i] + h[i] (i < nv) and col[nv] = |wdf| (the Hessenberg column), in
// the same reduction launch.
cudaError_t launch_gs_axpy_norm(const float2* V, size_t ldv, int nv, const double* h, float2* wdf, size_t N,
                                double* partial, double* out, cudaStream_t s, const double* h1 = nullptr,
                                double* col = nullptr);
template <typename TW, typename TO>
cudaError_t launch_gs_scale(const TW* w, const double* sc, float2* v, TO* out, size_t N, cudaStream_t s);
template <typename TO>
cudaError_t launch_df_to(const float2* v, TO* y, size_t N, cudaStream_t s);
cudaError_t launch_hess_column(const double* h1, const double* h2, const double* hn, int k, double* col,
                               cudaStream_t s);
int sweep_fault_take();
// 1 if a one-CTA tail's staging copies timed out since the last call (the tail then copied the data
// itself, so results stay valid), and clears the flag; -1 if it cannot be read.
int tail_fault_take();

// ---------------------------------------------------------------- learned boundary-cell correction
template <typename TI>
cudaError_t launch_mlp_features(int n_bnd, int npatch, int np, int nstat, int Fpad, const int* patch,
                                const float* stat, const TI* res, __nv_bfloat16* X, float* s, cudaStream_t st);
// C = opA(A) opB(B) (+ bias) (relu), BF16 in, FP32 accumulate; outputs FP32 Cf and/or BF16 Cb.
cudaError_t launch_gemm_bf16(int M, int N, int K, int ta, int tb, const __nv_bfloat16* A, int lda,
                             const __nv_bfloat16* B, int ldb, const float* bias, int relu, float* Cf,
                             __nv_bfloat16* Cb, int ldc, cudaStream_t s);
// The same GEMM on the tcgen05 tensor cores (tc_gemm.cu): 128 x 128 tiles, FP32 accumulators in
// tensor memory.  A commit that does not arrive in bounded time sets a flag that tc_fault_take()
// returns (1) and clears; -1 if it cannot be read.
cudaError_t launch_gemm_tc(int M, int N, int K, int ta, int tb, const __nv_bfloat16* A, int lda,
                           const __nv_bfloat16* B, int ldb, const float* bias, int relu, float* Cf,
                           __nv_bfloat16* Cb, int ldc, cudaStream_t s);
int tc_fault_take();
cudaError_t launch_mse_grad(int rows, int O, const float* Y, const float* T, float* dYf, __nv_bfloat16* dYb,
                            float inv_count, float* loss_partial, int nblk, cudaStream_t s);
cudaError_t launch_relu_mask(int n, float* dH, const __nv_bfloat16* H, __nv_bfloat16* dZb, cudaStream_t s);
cudaError_t launch_colsum(int rows, int cols, const float* D, float* g, cudaStream_t s);
cudaError_t launch_adam(int n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, float b1,
                        float b2, float eps, int t, cudaStream_t s);
cudaError_t launch_to_bf16(int n, const float* x, __nv_bfloat16* y, cudaStream_t s);
template <typename TU>
cudaError_t launch_mlp_targets(int n_bnd, int np, const int* cell, const TU* u, const float* s, float hfac, float* T,
                               cudaStream_t st);
// out[0] = sum of x[i]^2 (part: nblk doubles of per-block sums); x *= a.
cudaError_t launch_sumsq(size_t n, const float* x, double* part, int nblk, double* out, cudaStream_t st);
cudaError_t launch_scale_f(size_t n, float a, float* x, cudaStream_t st);
template <typename TZ>
cudaError_t launch_mlp_scatter(int n_bnd, int np, int ldy, const int* cell, const float* Y, const float* s,
                               float scale, TZ* z, cudaStream_t st);
cudaError_t launch_rows_gather(int rows, int width, const int* idx, const __nv_bfloat16* X, __nv_bfloat16* Xb,
                               int owidth, const float* T, float* Tb, cudaStream_t s);
cudaError_t launch_axpy_f(size_t n, float a, const float* x, float* y, cudaStream_t s);
// Xb = bf16(X) with rows padded from F to Fpad columns with zeros, and back.
cudaError_t launch_pack_bf16(int rows, int F, int Fpad, const float* X, __nv_bfloat16* Xb, cudaStream_t s);
cudaError_t launch_unpack_bf16(int rows, int F, int Fpad, const __nv_bfloat16* Xb, float* X, cudaStream_t s);
// y += x
template <typename R>
cudaError_t launch_add(size_t n, const R* x, R* y, cudaStream_t s);

}  // namespace sbm
