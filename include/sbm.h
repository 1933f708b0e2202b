/*
 * sbm.h - C ABI of the GB300 DG-SBM solver library (libsbm.so).
 *
 * The library solves the Poisson problem -Laplace(u) = f in Omega, u = g on Gamma
 * (arXiv 2506.12899, Sec. 2, Eq. 1) with the interior-penalty discontinuous Galerkin
 * discretisation of the Shifted Boundary Method (Sec. 2.2, Eqs. 7, 10, 11) on an unfitted
 * Cartesian background mesh, by flexible GMRES preconditioned with one hp-multigrid
 * V-cycle (Sec. 3).  Every step of the solve runs in the library's own CUDA kernels on one
 * GPU; the host computes only the one-time set-up (geometry, element matrices, block
 * factorisations, the coarse inverse, the right-hand side).
 *
 * Conventions for every call:
 *   - Return value: SBM_OK (0) or a negative SBM_ERR_* code.  sbm_last_error() returns a
 *     message for the last failure on the calling thread.  No C++ exception crosses the ABI.
 *   - "_dev" pointers are device pointers owned by the caller (e.g. torch CUDA tensors),
 *     contiguous, 16-byte aligned.  "_host" pointers are host memory owned by the caller.
 *   - All device work is enqueued on the stream given in sbm_setup_desc.stream (a
 *     cudaStream_t, NULL for the legacy default stream).  Calls return once the work is
 *     enqueued, except where a call says it synchronises.
 *   - Vector layout ("compact layout"): only active cells carry degrees of freedom.  On each
 *     level, active cells are ordered by colour c = sum_k (i_k mod 2) 2^k (c = 0 .. 2^d-1);
 *     within a colour, cells owning a surrogate face come first, then the others, each group
 *     in lexicographic background order (x index fastest).  The (p_l+1)^d degrees of freedom
 *     of a cell are contiguous, lexicographic (x fastest), and are the values of u at the
 *     tensor Gauss-Legendre nodes of the cell.  sbm_layout() returns the background index of
 *     every compact cell.
 *   - Levels are numbered 0 (coarsest) .. L (finest); level -1 means the finest.
 *   - dtype: SBM_F64 (double) or SBM_F32 (float) for the vectors of that call.
 */
#ifndef SBM_H
#define SBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SBM_OK = 0,
  SBM_ERR_ARG = -1,             /* invalid argument or descriptor                               */
  SBM_ERR_CUDA = -2,            /* a CUDA runtime call failed                                   */
  SBM_ERR_SINGULAR_BLOCK = -3,  /* a cell block or the coarse matrix has pivot ratio < 1e-13    */
  SBM_ERR_NOT_CONVERGED = -4,   /* FGMRES reached max_it without the requested tolerance        */
  SBM_ERR_NAN = -5,             /* a non-finite residual or Hessenberg entry was detected       */
  SBM_ERR_GEOMETRY = -6,        /* closest-point Newton failed or the finest level is empty     */
  SBM_ERR_ALLOC = -7            /* out of device or host memory                                 */
};

enum { SBM_F64 = 0, SBM_F32 = 1 };

/* Level-set shapes (Sec. 4.1: Omega = {phi < 0}). */
enum { SBM_SHAPE_DISK = 0, SBM_SHAPE_STAR = 1, SBM_SHAPE_ELLIPSOID = 2, SBM_SHAPE_BOX = 3,
       SBM_SHAPE_COMPLEX2D = 4 };
/* Manufactured solutions: f = -Laplace(u), g = u (Sec. 5.1, Eq. 23 for COSSIN). */
enum { SBM_U_SINPROD = 0, SBM_U_EXPCOS = 1, SBM_U_LINEAR = 2, SBM_U_COSSIN = 3, SBM_U_PHIP1 = 4,
       SBM_U_QUADRATIC = 5 };

typedef struct {
  int kind;              /* SBM_SHAPE_*                                                         */
  double center[3];
  double radius;         /* disk/sphere radius; star base radius r0; box half-width             */
  double amp, freq, phase; /* star: r(theta) = r0 (1 + amp sin(freq theta + phase))           */
  double semi[3];        /* ellipsoid semi-axes                                                 */
  double rot[9];         /* ellipsoid rotation R, row-major: phi = |S^-1 R^T (x - c)| - 1        */
} sbm_shape;

typedef struct {
  int dim;               /* 2 or 3                                                              */
  int n;                 /* background cells per direction on the finest level (even)          */
  int p;                 /* polynomial degree on the finest level, 1..3                          */
  double lo[3], hi[3];   /* background box; cells must be square: (hi-lo) equal in every dir     */
  sbm_shape shape;
  int exact;             /* SBM_U_*                                                             */
  double lambda;         /* volume-fraction threshold (Sec. 2.1)                                 */
  int lambda_inclusive;  /* 1: active iff kappa >= lambda; 0: kappa > lambda                      */
  double sigma_face_c;   /* sigma_F = c (p_l+1)^2 / h_l                                          */
  double sigma_bnd_c;    /* sigma_Gamma = c (p_l+1)^2 / h_l                                      */
  double alpha;          /* 1: quasi-symmetric Nitsche (Eq. 7); -1: penalty-free variant          */
  int extension;         /* 0: u(x~) + d.grad u(x~) (Eq. 6); 1: cell polynomial at x~ + d          */
  int coarsest_n;        /* h-coarsening stops at this many cells per direction                 */
  int pre_smooth, post_smooth;
  int ssor_each;         /* 0: a pre-smoothing step is one forward colour sweep and a post-       */
                         /* smoothing step one reverse sweep; 1: each step is a full SSOR step,   */
                         /* a forward then a reverse sweep, before and after the coarse correction */
  double omega;          /* block-smoother relaxation on levels with p_l <= 2                    */
  double omega_p3;       /* relaxation on levels with p_l = 3                                    */
  int vf_samples;        /* kappa sub-samples per direction; 0: 16 in 2D, 8 in 3D                 */
  int precision;         /* V-cycle precision inside sbm_solve: SBM_F64 or SBM_F32                */
  int tail_max_cells;    /* the coarse p = 1 h-levels with at most this many active cells run     */
                         /* their whole V-cycle in one launch with the level data in shared       */
                         /* memory (the largest such level that fits starts it); 0: library      */
                         /* default = every level that fits for FP32 V-cycles, none for FP64;    */
                         /* < 0: never                                                            */
  int tail_cluster_ctas; /* CTAs of that launch: 1 (one CTA, __syncthreads phases; the default    */
                         /* for 0) or 2, 4, 8, 16 (a thread-block cluster, vectors spread over    */
                         /* the CTAs' distributed shared memory)                                  */
  int launch_overlap;    /* > 0: the level and Krylov kernels use programmatic dependent launch,  */
                         /* so each may be scheduled while its predecessor finishes; < 0: plain   */
                         /* stream-ordered launches; 0: on with the FP32 V-cycle, off with FP64   */
  int krylov_basis;      /* FGMRES basis storage and Arnoldi arithmetic: 0 double-float pairs     */
                         /* (hi, lo) of FP32, Gram-Schmidt and (FP32 V-cycle) the operator A z on */
                         /* the FP32 pipes (~48-bit significands); 1 FP64; 2 double-float basis   */
                         /* with the FP64 operator                                                */
  int cell_kernel_min_cells; /* launches over at least this many cells use one thread per cell   */
                         /* when (p+1)^d <= 16 (and the FP32 operator at 3D p = 2), and one thread */
                         /* per line of a cell at 3D p = 3 (FP32; the double-float Arnoldi          */
                         /* operator at 3D p = 2 and 3); 0: always in FP32, never in FP64; < 0:     */
                         /* never (one thread per DoF everywhere)                                   */
  int staged_min_cells;  /* FP32 operator and smoother launches over at least this many cells     */
                         /* (2D p <= 3, 3D p <= 2) use the staged thread-per-cell kernels, whose  */
                         /* CTA copies its cells and their face neighbours into shared memory     */
                         /* first; 0: library default; < 0: never                                  */
  int smoother;          /* 0: coloured multiplicative block Gauss-Seidel (Eq. 16, the default);   */
                         /* 1: additive cell-wise block Jacobi u += omega_l D^-1 (f - A u) (the     */
                         /* additive form of Sec. 3.1); 2: block Jacobi inside a Chebyshev          */
                         /* iteration of cheb_degree steps on [b / cheb_ratio, b], b = 1.1 times a  */
                         /* power-iteration estimate of lambda_max(D^-1 A) (Sec. 5.3)               */
  int ordering;          /* Gauss-Seidel colours: 0 the 2^d colours c = sum (i_k mod 2) 2^k; 1     */
                         /* red-black, (sum_k i_k) mod 2 (even parity first in a forward sweep)     */
  int cheb_degree;       /* Chebyshev steps per smoothing step (smoother 2), 1..16                  */
  double cheb_ratio;     /* lambda_max / lambda_min of the Chebyshev interval (smoother 2), > 1      */
  int device_geometry;   /* sbm_setup: the volume fractions (s^d sub-cell samples of phi per cell)  */
                         /* and the closest-point Newton solves of the surrogate-face points run   */
                         /* as device kernels (0: default, on; < 0: on the host cores)              */
  void* stream;          /* cudaStream_t for every launch of this context                        */
} sbm_setup_desc;

typedef struct {
  int n;                 /* cells per direction                                                 */
  int p;                 /* degree                                                              */
  double h;              /* cell size                                                           */
  int n_active;          /* active cells                                                        */
  int n_dof;             /* n_active * (p+1)^dim                                                */
  int n_boundary;        /* active cells owning at least one surrogate face                     */
  int n_sface;           /* surrogate faces                                                     */
  int colour_start[9];   /* compact index of the first cell of each colour; [2^d] = n_active    */
  int colour_nbnd[8];    /* boundary cells at the start of each colour                          */
} sbm_level_info;

typedef struct {
  int converged;         /* 1 if ||b - A x|| <= tol ||b|| in FP64                                */
  int iterations;        /* Arnoldi steps (= V-cycle applications)                               */
  int restarts;          /* completed Arnoldi cycles                                             */
  double true_rel_residual; /* ||b - A x|| / ||b|| recomputed in FP64 at the end                  */
  double history[512];   /* |g_{j+1}| / ||b|| after each step (first 512)                        */
  double ms_total;       /* device time of the whole call (CUDA events)                          */
  int learned;           /* 1 if the solve started with the learned correction attached and on   */
  int learned_fallback;  /* 1 if the fallback rule switched it off during this solve             */
} sbm_solve_info;

/* Create a context: builds every level's geometry (Sec. 2.1, Sec. 4.2), element data, block
 * inverses (Eq. 14), transfer tables (Eqs. 17-18), the coarse inverse and the right-hand side,
 * and copies them to the device.  Synchronises.  *out is NULL on failure. */
int sbm_setup(const sbm_setup_desc* desc, void** out);

/* Host-only context for checking the set-up without a GPU: builds the same levels, element data
 * and right-hand side as sbm_setup but allocates no device memory.  Only sbm_num_levels,
 * sbm_info, sbm_layout, sbm_export_geometry, sbm_host_apply, sbm_host_rhs and sbm_destroy
 * accept it; the device calls return SBM_ERR_ARG. */
int sbm_setup_host(const sbm_setup_desc* desc, void** out);

/* Host FP64 evaluation of y = A_l x (Eq. 11) with the same element data the kernels use;
 * x_host, y_host hold n_dof doubles in compact layout. */
int sbm_host_apply(const void* ctx, int level, const double* x_host, double* y_host);

/* Right-hand side of Eq. 11 into a host buffer of n_dof doubles (compact layout). */
int sbm_host_rhs(const void* ctx, double* b_host);

/* Release the context and all device memory it owns.  Safe on NULL. */
void sbm_destroy(void* ctx);

/* Message of the last failing call on this thread (static storage, never NULL). */
const char* sbm_last_error(void);

/* Total number of CUDA kernel launches issued by this library since it was loaded (all
 * contexts; memsets and copies are not counted). */
long long sbm_kernel_launches(void);

/* Number of multigrid levels L+1. */
int sbm_num_levels(const void* ctx, int* out);

/* Sizes and colour ranges of one level. */
int sbm_info(const void* ctx, int level, sbm_level_info* out);

/* Background multi-index of every compact cell: coords_host[3*a + k] = i_k (i_2 = 0 in 2D). */
int sbm_layout(const void* ctx, int level, int* coords_host);

/* Surrogate faces of a level, in compact-cell order then face slot 2*direction + side:
 * cell_host[f], slot_host[f] and shifts d_host[f][(p+1)^(d-1)][3] (FP64, zero third component
 * in 2D).  Pass NULL to query the count through *n_faces only. */
int sbm_export_geometry(const void* ctx, int level, int* n_faces, int* cell_host, int* slot_host,
                        double* d_host);

/* Right-hand side b of Eq. 11 on the finest level, FP64, into the caller's device buffer. */
int sbm_rhs(void* ctx, double* b_dev);

/* y = A_l x: matrix-free operator of Eq. 11 on level l (volume, interior-penalty faces of
 * Eq. 10, Nitsche-SBM surrogate faces of Eq. 7).  x and y hold n_dof values of `dtype`;
 * x and y must not overlap. */
int sbm_apply(void* ctx, int level, int dtype, const void* x_dev, void* y_dev);

/* r = f - A_l u on level l (same operator as sbm_apply). */
int sbm_residual(void* ctx, int level, int dtype, const void* f_dev, const void* u_dev, void* r_dev);

/* One coloured block Gauss-Seidel sweep on level l (Eq. 16 with A_i of Eq. 14):
 * for c = 0 .. 2^d-1 (reverse = 1: 2^d-1 .. 0), for every cell K of colour c,
 * u_K <- u_K + omega_l A_KK^{-1} (f - A u)_K.  u is updated in place. */
int sbm_smooth(void* ctx, int level, int dtype, int reverse, const void* f_dev, void* u_dev);

/* Restriction (Eq. 18): rc = P^T rf from level l to level l-1 (l >= 1), masked to active cells. */
int sbm_restrict(void* ctx, int level, int dtype, const void* rf_dev, void* rc_dev);

/* Prolongation (Eq. 17): uf += P ec from level l-1 to level l (l >= 1), masked to active cells. */
int sbm_prolong_add(void* ctx, int level, int dtype, const void* ec_dev, void* uf_dev);

/* Coarse direct solve on level 0: e = A_0^{-1} r, always computed in FP64 (dense inverse of
 * the LU-factored coarse matrix); r and e are of `dtype`. */
int sbm_coarse_solve(void* ctx, int dtype, const void* r_dev, void* e_dev);

/* One V-cycle z = M^{-1} r on the finest level (Sec. 3): zero initial guess, pre-smoothing
 * (forward colours), residual, restriction, recursion, prolongation, post-smoothing (reverse
 * colours); coarse direct solve.  dtype selects the V-cycle precision (FP32: every level
 * operation in FP32 except the coarse solve, which applies the FP64 inverse; inside the one-CTA
 * tail of an FP32 V-cycle its products are formed exactly and summed in double-float, about 48
 * significant bits, on FP32 input and output). */
int sbm_vcycle(void* ctx, int dtype, const void* r_dev, void* z_dev);

/* Gram-Schmidt projections of the FGMRES Arnoldi step (Sec. 3): out[k] = sum_i V[k*ldv + i] w[i]
 * for k < nv (1 <= nv <= 32), FP64, with the deterministic two-stage reduction used inside
 * sbm_solve (warp shuffles, per-block partial sums in a context-owned buffer allocated on first
 * use, then a fixed-order sum).  V holds nv vectors of length n with leading dimension ldv >= n;
 * out_dev holds nv doubles. */
int sbm_dots(void* ctx, const double* V_dev, long long ldv, int nv, const double* w_dev, long long n,
             double* out_dev);

/* L2 error ||u - u_h||_{L2} over the active cells of the finest level (the surrogate domain), the
 * error measure of the paper's convergence studies (Sec. 5.1, Sec. 5.4): u is the manufactured
 * solution of sbm_setup_desc.exact, u_h the FP64 solution x_dev (compact layout, n_dof doubles),
 * integrated cell by cell with the (p+3)-point tensor Gauss-Legendre rule.  Runs on the device
 * (deterministic fixed-order sums), synchronises and writes the error to *err_host. */
int sbm_l2_error(void* ctx, const double* x_dev, double* err_host);

/* The three Gram-Schmidt sweeps of one FGMRES Arnoldi step (Sec. 3; two classical passes, CGS2)
 * on caller data, by the kernels sbm_solve uses:
 *   h1 = V w;  w1 = w - V^T h1;  h2 = V w1;  w2 = w1 - V^T h2;  norm = |w2|_2.
 * V_dev holds nv (1..32) FP64 vectors of the finest level's length N (row-major, [nv][N]), w_dev
 * one; outputs: h_dev[0..nv) = h1, h_dev[nv..2nv) = h2 (FP64), w_out_dev = w2 (N doubles),
 * norm_dev = |w2| (one double).  variant 0: the double-float basis of krylov_basis = 0/2 (V rounded
 * to FP32 pairs, ~48-bit significands, staged bulk-copy sweeps), w given in FP64 and converted by
 * the first sweep (FP64-V-cycle solves); 1: the same with w first rounded to double-float (the
 * path of FP32-V-cycle solves, where A z is formed in double-float); 2: the FP64 sweeps of
 * krylov_basis = 1.  The context keeps its own copy of the rows and of w (allocated on first use:
 * 32 padded rows of N double-floats) and does not touch the solve's workspace.  Synchronises.
 * Errors: SBM_ERR_ARG for null pointers, nv outside 1..32 or an unknown variant; SBM_ERR_CUDA if a
 * launch fails or a bounded wait of a staged sweep gave up. */
int sbm_gram_schmidt(void* ctx, int variant, const double* V_dev, int nv, const double* w_dev, double* h_dev,
                     double* w_out_dev, double* norm_dev);

/* sbm_dots without any allocation, for callers that cannot call cudaMalloc: for example a
 * process whose caching allocator has already reserved the device memory (a cudaMalloc would
 * fail), or a latency-critical loop that cannot accept the device-wide synchronisation a
 * cudaMalloc may cause.  It needs no context: out[k] = sum_i V[k*ldv + i] w[i] for k < nv,
 * computed by the same kernels and in the same order as sbm_dots, on `stream` (a cudaStream_t,
 * NULL for the legacy default stream, current device).  The per-block partial sums live in a
 * file-scope __device__ array of 608 x 32 doubles (152 KiB) that every GPU loading the library
 * holds until the process exits.  That array is created when the library's Krylov module is
 * loaded into a device's context.  Under CUDA's lazy module loading (the default) that happens on
 * the first use of the module there (this call, or any solve), and that one load allocates the
 * array: make the first call on each device at a point where 152 KiB can still be had, e.g.
 * before a caching allocator reserves the memory.  Later calls allocate nothing.  Every call
 * made outside stream capture looks the array's address up again in the current context
 * (cudaGetSymbolAddress), so a reset or replaced context is followed; inside a capture the
 * address of the last call outside capture on this device is used, so the first call on a
 * device must come before any stream capture.  Every call reuses the same array: each call
 * overwrites the partial sums it reads, so nothing carries over, but calls that overlap on the
 * GPU (other streams, other host threads) race on the array.
 * Errors: SBM_ERR_ARG for null pointers, nv outside 1..32, n < 0, ldv < n, or a first call
 * inside a capture; SBM_ERR_CUDA if the address lookup or the launch fails.  The paper has no
 * counterpart to this entry point. */
int sbm_dots_noalloc(const double* V_dev, long long ldv, int nv, const double* w_dev, long long n,
                     double* out_dev, void* stream);

/* Failure-path check of the bounded waits.  The staged kernels (Gram-Schmidt sweeps, V-cycle
 * tail) wait on mbarriers for bulk asynchronous copies; each wait gives up after a bounded number
 * of polls, records the failure in a device flag and lets its kernel finish, and sbm_solve then
 * returns SBM_ERR_CUDA.  This entry point runs one such wait in a one-block kernel on `stream`
 * (a cudaStream_t, NULL for the legacy default stream), synchronises and reads the flag:
 * starve = 0 announces 16 bytes and copies them (returns SBM_OK); starve = 1 announces 16 bytes
 * and copies nothing, so the wait runs out after 4096 polls and the call returns SBM_ERR_CUDA
 * with that reason.  The device context stays usable either way.  No counterpart in the paper. */
int sbm_async_wait_selftest(int starve, void* stream);

/* Solve A x = b by FGMRES(restart), right-preconditioned by one V-cycle in the precision of
 * sbm_setup_desc.precision (Sec. 3); the Hessenberg matrix, the Givens rotations, the update of x
 * and the true residual are FP64, and the basis, Gram-Schmidt (two classical passes) and the
 * Arnoldi operator are FP64 or double-float as sbm_setup_desc.krylov_basis selects.  x_dev holds
 * the initial guess on entry.  Stops when the Hessenberg residual estimate <= tol ||b|| and the
 * recomputed ||b - A x|| <= tol ||b||, or at max_it Arnoldi steps (SBM_ERR_NOT_CONVERGED).
 * The host reads each Hessenberg column; while the residual stays well above the tolerance the
 * next Arnoldi step is already queued behind the current one, and a step queued in vain is
 * discarded (the iterates do not depend on the queuing).  Synchronises; fills *info if non-NULL. */
int sbm_solve(void* ctx, const double* b_dev, double* x_dev, double tol, int restart, int max_it,
              sbm_solve_info* info);

/* sbm_solve with host buffers: copies b_host to the device, solves from x = 0, copies x back
 * into x_host.  The copies are part of the call. */
int sbm_solve_host(void* ctx, const double* b_host, double* x_host, double tol, int restart,
                   int max_it, sbm_solve_info* info);

/* ---------------------------------------------------------------------------------------------
 * Learned boundary-cell correction.  The paper has no learned component; this is a learned
 * variant of the V-cycle smoother built on its method (the p = 3 smoother weakens near the
 * surrogate boundary, Sec. 5.3).  After the finest level's post-smoothing every boundary cell K
 * (a cell owning a surrogate face) gets u_K += scale * s_K * h^(2-d) * MLP(x_K) (h^(2-d): the
 * operator scales like h^(d-2), so the network's outputs are mesh-independent), where
 *   x_K = [ patch residual / s_K, d / h at every face point, kappa(K), surrogate-face mask ],
 *   s_K = |patch residual|_2 (1 if zero),
 * the patch being the 3^d cells K + o, o in {-1,0,1}^d (x fastest), their residual r - A u with
 * zeros for inactive or missing cells; d / h is given per face slot s = 2 dir + side, face point
 * t (first tangential dimension fastest) and component, zero on slots that are not surrogate
 * faces.  F = 3^d (p+1)^d + 2d (p+1)^(d-1) d + 1 + 2d features.  The MLP is
 * y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 with hidden width H and O = (p+1)^d
 * outputs; FP32 master parameters, BF16 weights and activations on the tensor cores, FP32
 * accumulation.  Parameters travel packed as FP32 [W1 (F x H, input-major) | b1 | W2 (H x H) |
 * b2 | W3 (H x O) | b3].  An MLP handle is independent of a context and owned by the caller;
 * it must outlive every context it is attached to.  All MLP calls run on the stream given at
 * creation; the correction itself runs on the context's streams inside sbm_vcycle/sbm_solve.
 * ------------------------------------------------------------------------------------------- */

/* Create an MLP for dimension dim and degree p with hidden width `hidden` (8..1024): He-normal
 * weights from a splitmix64/Box-Muller stream seeded by `seed`, zero biases.  `stream` is a
 * cudaStream_t (NULL: legacy default stream).  SBM_ERR_ARG for a bad shape. */
int sbm_mlp_create(int dim, int p, int hidden, unsigned long long seed, void* stream, void** out);
void sbm_mlp_destroy(void* mlp);
/* F features, Fpad (F rounded up to 32, the device row length), H, O and the packed parameter
 * count. */
int sbm_mlp_shape(const void* mlp, int* F, int* Fpad, int* H, int* O, long long* nparam);
/* Host FP32 packed parameters in / out; setting them also resets the Adam state. */
int sbm_mlp_set_params(void* mlp, const float* params_host);
int sbm_mlp_get_params(const void* mlp, float* params_host);
/* GEMM implementation of the MLP: 0 (default) the tcgen05 tensor-core kernel (128 x 128 tiles,
 * FP32 accumulators in tensor memory), 1 the warp-level mma.sync kernel.  Both compute the same
 * BF16 x BF16 -> FP32 products (summation order differs).  A tensor-core commit that does not arrive
 * within a bounded wait makes the next synchronising MLP call return SBM_ERR_CUDA. */
int sbm_mlp_gemm_backend(void* mlp, int backend);
/* Y_dev[rows][O] = MLP(X_dev[rows][F]) (device FP32 buffers; X is rounded to BF16). */
int sbm_mlp_forward(void* mlp, const float* X_dev, int rows, float* Y_dev);
/* Gradient of the mean squared error mean((MLP(X) - T)^2) over the rows x O entries, in the
 * packed layout (host), and the loss.  X_dev [rows][F], T_dev [rows][O] device FP32. */
int sbm_mlp_gradients(void* mlp, const float* X_dev, const float* T_dev, int rows, float* grad_host,
                      double* loss);
/* Normalises the stored training targets to unit root mean square: computes rms = sqrt(mean T^2)
 * over every stored target entry (device, deterministic), divides the stored targets by it and
 * returns it in *rms (1 and no change if the targets are all zero).  A network trained afterwards
 * predicts targets / rms; attach it with scale = rms (sbm_attach_mlp) to restore the units.  The
 * training loss is then the mean squared error relative to the targets' mean square.
 * SBM_ERR_ARG if the set is empty. */
int sbm_mlp_target_scale(void* mlp, double* rms);
/* The MLP's training set (filled by sbm_collect): number of stored rows; empty it. */
int sbm_mlp_num_samples(const void* mlp, long long* n);
int sbm_mlp_clear_samples(void* mlp);
/* Adam (lr, beta = 0.9 / 0.999, eps 1e-8) on the mean squared error of the stored set for
 * `epochs` passes in minibatches of `batch` rows, shuffled each epoch by a splitmix64
 * Fisher-Yates permutation seeded by `seed`; *loss = mean batch loss of the last epoch.
 * SBM_ERR_ARG if the set is empty. */
int sbm_mlp_train(void* mlp, int epochs, int batch, float lr, unsigned long long seed, double* loss);
/* Checkpoint: "SBMMLP\0\0", int32 {version 1, dim, p, F, H, O}, packed FP32 parameters, CRC-32
 * (IEEE) of everything before it.  Load checks the shape and the checksum (SBM_ERR_ARG). */
int sbm_mlp_save(const void* mlp, const char* path);
int sbm_mlp_load(void* mlp, const char* path);

/* Finest-level features of every boundary cell from a residual res_dev (dtype SBM_F64 or
 * SBM_F32, compact layout): X_dev [n_bnd][F] FP32 (the BF16 values the MLP sees) and s_dev
 * [n_bnd].  Boundary cells are ordered as sbm_learned_cells lists them. */
int sbm_learned_features(void* ctx, int dtype, const void* res_dev, float* X_dev, float* s_dev);
/* Number of finest-level boundary cells and (if cells_host is non-NULL) their compact indices. */
int sbm_learned_cells(void* ctx, int* n_bnd, int* cells_host);
/* Training pairs: from each of the n_starts initial vectors u0_dev[k][N] (dtype, the V-cycle
 * precision used), run n_cycles steps of u <- u + V(-A u) on A u = 0 (plain V-cycles, exact
 * solution 0) and after each step append, for every boundary cell, (x_K from r = -A u,
 * target -u_K / (s_K h^(2-d))) to the MLP's training set.  *n_added = rows appended. */
int sbm_collect(void* ctx, void* mlp, int dtype, const void* u0_dev, int n_starts, int n_cycles,
                long long* n_added);
/* Attach (mlp non-NULL) or detach (NULL) the correction to the context's V-cycle with the given
 * scale.  fallback_rate > 0: a solve whose mean residual reduction per step over its first three
 * steps is worse (larger) than fallback_rate switches the correction off for the rest of that
 * solve (reported in sbm_solve_info.learned_fallback); 0 disables the rule. */
int sbm_attach_mlp(void* ctx, void* mlp, float scale, double fallback_rate);

#ifdef __cplusplus
}
#endif
#endif /* SBM_H */
