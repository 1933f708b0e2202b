// Thread-per-cell CUDA kernels for small cells ((p+1)^d <= 16: 2D p = 1..3 and 3D p = 1).
//
// One thread owns one cell: its (p+1)^d values, the interior-face couplings to its 2d
// neighbours, its surrogate-face terms and its block inverse live in registers.  Every loop
// over nodes, lines and directions is unrolled, so each 1D-matrix coefficient is a uniform,
// immediate-offset read of the kernel parameter block (constant cache broadcast) and no
// shared memory or barrier is needed.  The per-DoF kernels of level_ops.cu issue about 175
// instructions per DoF, mostly shared-memory traffic; here the arithmetic is the same
// (Eqs. 7, 10, 11, 14, 16, 18) but the instruction stream is a fraction of that.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "ops.h"

namespace sbm {
namespace {

constexpr int kCellThreads = 128;
constexpr int kTailThreads = 512;

template <int D, int N1>
struct CD {
  static constexpr int NP = D == 2 ? N1 * N1 : N1 * N1 * N1;
  static constexpr int NQ = D == 2 ? N1 : N1 * N1;
};

// Local dof of node k along `dir` on tangential line t (tangential dims ascending, first fastest).
template <int D, int N1>
__host__ __device__ constexpr int dof(int dir, int k, int t) {
  return D == 2 ? (dir == 0 ? k + N1 * t : t + N1 * k)
                : (dir == 0 ? k + N1 * (t % N1) + N1 * N1 * (t / N1)
                            : (dir == 1 ? (t % N1) + N1 * k + N1 * N1 * (t / N1)
                                        : (t % N1) + N1 * (t / N1) + N1 * N1 * k));
}

template <int D, int N1, typename R>
__device__ __forceinline__ R line_weight(const LevelConsts<R>& C, int t) {
  return D == 2 ? C.w[t] : C.w[t % N1] * C.w[t / N1];
}

// Component m of the tangential index t on faces normal to dir: tangential dims ascending.
template <int D>
__host__ __device__ constexpr int tang_dim(int dir, int q) {
  return D == 2 ? 1 - dir : (dir == 0 ? 1 + q : (dir == 1 ? 2 * q : q));
}

// Vector loads.  COH: through L2 only (ld.global.cg), for the cluster V-cycle, where values
// written by other CTAs in the previous phase are read after a cluster barrier and L1 is not
// coherent; otherwise ordinary L1-cached loads (a thread reads its cell's contiguous values,
// so consecutive load instructions of a warp hit the lines the first one brought in).
template <bool COH, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if (COH) return __ldcg(p);
  return *p;
}

template <int D, int N1, bool COH, typename TI, typename R>
__device__ __forceinline__ void load_cell(const TI* __restrict__ x, int a, R (&v)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
#pragma unroll
  for (int i = 0; i < NP; ++i) v[i] = (R)ldv<COH>(x + (size_t)a * NP + i);
}

// y += (sum over interior faces of A_KN u_N) for cell a (Eq. 10 couplings); neighbours of
// colour > col are skipped when zero_start (they hold zeros).
template <int D, int N1, bool COH, typename TI, typename R>
__device__ __forceinline__ void add_couplings(const LevelParams<R>& P, const TI* __restrict__ u, int a, int col,
                                              bool zero_start, int (&nb)[2 * D], R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP, NQ = CD<D, N1>::NQ;
  const LevelConsts<R>& C = P.k;
#pragma unroll
  for (int s = 0; s < 2 * D; ++s) {
    const int dir = s >> 1;
    const int n = nb[s];
    if (n < 0 || (zero_start && (col ^ (1 << dir)) > col)) continue;
    R un[NP];
    load_cell<D, N1, COH, TI, R>(u, n, un);
    const R* B = (s & 1) ? C.Bmp : C.Bpm;
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const R wt = line_weight<D, N1, R>(C, t);
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        R acc = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) acc += B[i * N1 + j] * un[dof<D, N1>(dir, j, t)];
        y[dof<D, N1>(dir, i, t)] += wt * acc;
      }
    }
  }
}

// y += A_KK v (volume + own halves of interior faces + surrogate faces), reference scaling.
template <int D, int N1, typename R>
__device__ __forceinline__ void add_self(const LevelParams<R>& P, const int (&nb)[2 * D], int bidx,
                                         const R (&v)[CD<D, N1>::NP], R (&y)[CD<D, N1>::NP]) {
  constexpr int NQ = CD<D, N1>::NQ;
  const LevelConsts<R>& C = P.k;
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    // self matrix by neighbour mask; the mask is uniform over a warp of interior cells
    const R* Lm = C.L[(nb[2 * dir] >= 0) + 2 * (nb[2 * dir + 1] >= 0)];
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const R wt = line_weight<D, N1, R>(C, t);
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        R acc = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) acc += Lm[i * N1 + k] * v[dof<D, N1>(dir, k, t)];
        y[dof<D, N1>(dir, i, t)] += wt * acc;
      }
    }
  }
  if (bidx < 0) return;
  // surrogate faces (Eq. 7): U_t, normal derivative G_t, extended value E_t per face point
#pragma unroll
  for (int s = 0; s < 2 * D; ++s) {
    if (nb[s] >= 0) continue;
    const int dir = s >> 1, side = s & 1;
    const R sg = side ? R(1) : R(-1);
    const R* es = side ? C.e1 : C.e0;
    const R* ds = side ? C.d1 : C.d0;
    const R* dh = P.dhat + ((size_t)bidx * 2 * D + s) * D * NQ;
    R U[NQ], G[NQ];
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      R su = 0, sd = 0;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        su += es[k] * v[dof<D, N1>(dir, k, t)];
        sd += ds[k] * v[dof<D, N1>(dir, k, t)];
      }
      U[t] = su;
      G[t] = sd;
    }
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      R E;
      if (P.extension == 0) {
        E = U[t] + dh[dir * NQ + t] * G[t];
#pragma unroll
        for (int q = 0; q < D - 1; ++q) {           // tangential derivatives of the trace
          const int m = tang_dim<D>(dir, q);
          const int stride = q == 0 ? 1 : N1;
          const int tm = (t / stride) % N1;
          R g = 0;
#pragma unroll
          for (int r = 0; r < N1; ++r) g += C.Dm[tm * N1 + r] * U[t + (r - tm) * stride];
          E += dh[m * NQ + t] * g;
        }
      } else {                                      // cell polynomial at x~ + d
        R lv[D][N1];
#pragma unroll
        for (int m = 0; m < D; ++m) {
          R xi;
          if (m == dir) {
            xi = R(side);
          } else {                                  // node of tangential dim m (position q) on line t
            const int q = m < dir ? m : m - 1;
            xi = C.x[(t / (q == 0 ? 1 : N1)) % N1];
          }
          const R yv = xi + dh[m * NQ + t];
#pragma unroll
          for (int k = 0; k < N1; ++k) {
            R val = C.inv_denom[k];
#pragma unroll
            for (int j = 0; j < N1; ++j)
              if (j != k) val *= (yv - C.x[j]);
            lv[m][k] = val;
          }
        }
        E = 0;
#pragma unroll
        for (int j = 0; j < CD<D, N1>::NP; ++j) {
          R ph = lv[0][j % N1] * lv[1][(j / N1) % N1];
          if (D == 3) ph *= lv[D - 1][j / (N1 * N1)];
          E += ph * v[j];
        }
      }
      const R wt = line_weight<D, N1, R>(C, t);
#pragma unroll
      for (int k = 0; k < N1; ++k)
        y[dof<D, N1>(dir, k, t)] += wt * (es[k] * (-sg * G[t] + P.sigG * E) - P.alpha * sg * ds[k] * E);
    }
  }
}

template <typename R>
__device__ __forceinline__ int boundary_index(const LevelParams<R>& P, int a, int ncol) {
  int c = 0;
#pragma unroll
  for (int k = 1; k < 8; ++k)
    if (k < ncol && a >= P.colour_start[k]) c = k;
  const int off = a - P.colour_start[c];
  return off < P.colour_nbnd[c] ? P.bstart[c] + off : -1;
}

template <int D, typename R>
__device__ __forceinline__ void load_nbr(const LevelParams<R>& P, int a, int (&nb)[2 * D]) {
#pragma unroll
  for (int s = 0; s < 2 * D; ++s) nb[s] = P.nbr[(size_t)s * P.n_act + a];
}

// y = (A x)_a with the reference scaling h^(d-2) applied.
template <int D, int N1, bool COH, typename TI, typename R>
__device__ __forceinline__ void cell_apply(const LevelParams<R>& P, const TI* __restrict__ x, int a,
                                           R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  int nb[2 * D];
  load_nbr<D, R>(P, a, nb);
  R v[NP];
  load_cell<D, N1, COH, TI, R>(x, a, v);
#pragma unroll
  for (int i = 0; i < NP; ++i) y[i] = 0;
  add_self<D, N1, R>(P, nb, boundary_index(P, a, 1 << D), v, y);
  add_couplings<D, N1, COH, TI, R>(P, x, a, 0, false, nb, y);
#pragma unroll
  for (int i = 0; i < NP; ++i) y[i] *= P.hscale;
}

template <int D, int N1, typename TI, typename R, int MODE>
__global__ void __launch_bounds__(kCellThreads) k_apply_cell(const __grid_constant__ LevelParams<R> P,
                                                             const TI* __restrict__ x, const R* __restrict__ f,
                                                             R* __restrict__ y) {
  constexpr int NP = CD<D, N1>::NP;
  const int a = blockIdx.x * kCellThreads + threadIdx.x;
  if (a >= P.n_act) return;
  R r[NP];
  cell_apply<D, N1, false, TI, R>(P, x, a, r);
#pragma unroll
  for (int i = 0; i < NP; ++i) y[(size_t)a * NP + i] = MODE == 1 ? f[(size_t)a * NP + i] - r[i] : r[i];
}

// One cell of one colour of the block Gauss-Seidel sweep (Eq. 16): cell a of the colour
// starting at cs whose first nbnd cells are boundary cells (dense inverse, boundary index
// b0 + a - cs); the others use the fast diagonalisation.  zero_start as in k_smooth.
template <int D, int N1, bool COH, typename R>
__device__ __forceinline__ void smooth_one(const LevelParams<R>& P, int col, int zero_start, int cs, int nbnd,
                                           int b0, int a, const R* __restrict__ f, R* __restrict__ u) {
  constexpr int NP = CD<D, N1>::NP, NQ = CD<D, N1>::NQ;
  const bool isB = a - cs < nbnd;
  int nb[2 * D];
  load_nbr<D, R>(P, a, nb);
  R c[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) c[i] = 0;
  add_couplings<D, N1, COH, R, R>(P, u, a, col, zero_start != 0, nb, c);
  R t[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) t[i] = ldv<COH>(f + (size_t)a * NP + i) - P.hscale * c[i];
  R y[NP];
  if (isB) {
    const R* Bi = P.binvT + (size_t)(b0 + (a - cs)) * NP * NP;
#pragma unroll
    for (int i = 0; i < NP; ++i) y[i] = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
      for (int i = 0; i < NP; ++i) y[i] += Bi[j * NP + i] * t[j];
  } else {
    const LevelConsts<R>& C = P.k;
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {            // (S^T)^(x d) t
      R w[NP];
#pragma unroll
      for (int tl = 0; tl < NQ; ++tl)
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          R acc = 0;
#pragma unroll
          for (int k = 0; k < N1; ++k) acc += C.S[k * N1 + m] * t[dof<D, N1>(dir, k, tl)];
          w[dof<D, N1>(dir, m, tl)] = acc;
        }
#pragma unroll
      for (int i = 0; i < NP; ++i) t[i] = w[i];
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      R lsum = C.lam[i % N1] + C.lam[(i / N1) % N1];
      if (D == 3) lsum += C.lam[i / (N1 * N1)];
      t[i] = t[i] / (P.hscale * lsum);
    }
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {            // S^(x d) v
      R w[NP];
#pragma unroll
      for (int tl = 0; tl < NQ; ++tl)
#pragma unroll
        for (int m = 0; m < N1; ++m) {
          R acc = 0;
#pragma unroll
          for (int k = 0; k < N1; ++k) acc += C.S[m * N1 + k] * t[dof<D, N1>(dir, k, tl)];
          w[dof<D, N1>(dir, m, tl)] = acc;
        }
#pragma unroll
      for (int i = 0; i < NP; ++i) t[i] = w[i];
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) y[i] = t[i];
  }
  if (P.omega == R(1)) {
#pragma unroll
    for (int i = 0; i < NP; ++i) u[(size_t)a * NP + i] = y[i];
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const R uo = zero_start ? R(0) : ldv<COH>(u + (size_t)a * NP + i);
      u[(size_t)a * NP + i] = (R(1) - P.omega) * uo + P.omega * y[i];
    }
  }
}

// One colour of the block Gauss-Seidel sweep, one thread per cell: boundary cells of the colour
// in blocks [0, nblk_b), interior cells in the remaining blocks.
template <int D, int N1, typename R>
__global__ void __launch_bounds__(kCellThreads) k_smooth_cell(const __grid_constant__ LevelParams<R> P, int col,
                                                              int zero_start, int cs, int nbnd, int ce, int nblk_b,
                                                              int b0, const R* __restrict__ f, R* __restrict__ u) {
  const bool isB = (int)blockIdx.x < nblk_b;
  const int first = isB ? cs + blockIdx.x * kCellThreads : cs + nbnd + (blockIdx.x - nblk_b) * kCellThreads;
  const int last = isB ? cs + nbnd : ce;
  const int a = first + threadIdx.x;
  if (a >= last) return;
  smooth_one<D, N1, false, R>(P, col, zero_start, cs, nbnd, b0, a, f, u);
}

// Residual and p-restriction fused, one thread per cell (Eqs. 11, 18).
template <int D, int N1, int NC, typename R>
__global__ void __launch_bounds__(kCellThreads) k_resid_restrict_p_cell(const __grid_constant__ LevelParams<R> P,
                                                                        const __grid_constant__ TransferParams<R> T,
                                                                        const R* __restrict__ u,
                                                                        const R* __restrict__ f, R* __restrict__ rc) {
  constexpr int NP = CD<D, N1>::NP;
  constexpr int NPC = D == 2 ? NC * NC : NC * NC * NC;
  const int a = blockIdx.x * kCellThreads + threadIdx.x;
  if (a >= P.n_act) return;
  R r[NP];
  cell_apply<D, N1, false, R, R>(P, u, a, r);
#pragma unroll
  for (int i = 0; i < NP; ++i) r[i] = f[(size_t)a * NP + i] - r[i];
#pragma unroll
  for (int j = 0; j < NPC; ++j) {
    const int j0 = j % NC, j1 = (j / NC) % NC, j2 = D == 3 ? j / (NC * NC) : 0;
    R acc = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const int i0 = i % N1, i1 = (i / N1) % N1, i2 = D == 3 ? i / (N1 * N1) : 0;
      R wgt = T.Pp[i0 * NC + j0] * T.Pp[i1 * NC + j1];
      if (D == 3) wgt *= T.Pp[i2 * NC + j2];
      acc += wgt * r[i];
    }
    rc[(size_t)a * NPC + j] = acc;
  }
}

// Residual and h-restriction fused for coarse cell cc (p = 1 on both meshes): the residuals of
// its active children are formed in registers and restricted (Eq. 18).
template <int D, bool COH, typename R>
__device__ __forceinline__ void resid_restrict_h_one(const LevelParams<R>& P, const TransferParams<R>& T,
                                                     const R* __restrict__ u, const R* __restrict__ f,
                                                     R* __restrict__ rc, int cc) {
  constexpr int NP = CD<D, 2>::NP;
  R out[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) out[j] = 0;
#pragma unroll
  for (int o = 0; o < (1 << D); ++o) {
    const int a = T.children[(size_t)o * T.n_act_c + cc];
    if (a < 0) continue;
    R r[NP];
    cell_apply<D, 2, COH, R, R>(P, u, a, r);
#pragma unroll
    for (int i = 0; i < NP; ++i) r[i] = ldv<COH>(f + (size_t)a * NP + i) - r[i];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      R acc = 0;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        R wgt = T.Ph[o & 1][(i & 1) * 2 + (j & 1)] * T.Ph[(o >> 1) & 1][((i >> 1) & 1) * 2 + ((j >> 1) & 1)];
        if (D == 3) wgt *= T.Ph[(o >> 2) & 1][((i >> 2) & 1) * 2 + ((j >> 2) & 1)];
        acc += wgt * r[i];
      }
      out[j] += acc;
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) rc[(size_t)cc * NP + j] = out[j];
}

template <int D, typename R>
__global__ void __launch_bounds__(kCellThreads) k_resid_restrict_h_cell(const __grid_constant__ LevelParams<R> P,
                                                                        const __grid_constant__ TransferParams<R> T,
                                                                        const R* __restrict__ u,
                                                                        const R* __restrict__ f, R* __restrict__ rc) {
  const int cc = blockIdx.x * kCellThreads + threadIdx.x;
  if (cc >= T.n_act_c) return;
  resid_restrict_h_one<D, false, R>(P, T, u, f, rc, cc);
}

// Prolongation into fine cell a (p = 1 on both meshes, Eq. 17): uf_a += (Ph x Ph ..) ec_parent.
template <int D, typename R>
__device__ __forceinline__ void prolong_h_one(const TransferParams<R>& T, const R* __restrict__ ec,
                                              R* __restrict__ uf, int a) {
  constexpr int NP = CD<D, 2>::NP;
  const int code = T.parent_code[a];
  if (code < 0) return;
  const int par = code >> 3, o = code & 7;
  R e[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) e[j] = ldv<true>(ec + (size_t)par * NP + j);
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    R acc = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      R wgt = T.Ph[o & 1][(i & 1) * 2 + (j & 1)] * T.Ph[(o >> 1) & 1][((i >> 1) & 1) * 2 + ((j >> 1) & 1)];
      if (D == 3) wgt *= T.Ph[(o >> 2) & 1][((i >> 2) & 1) * 2 + ((j >> 2) & 1)];
      acc += wgt * e[j];
    }
    uf[(size_t)a * NP + i] = ldv<true>(uf + (size_t)a * NP + i) + acc;
  }
}

// The V-cycle below and including level `top` (all of them p = 1 h-levels) in one launch of a
// thread-block cluster: every phase (one colour of a sweep, a fused residual/restriction, the
// coarse solve, a prolongation) is spread over the cluster's threads and closed by a fence and
// a hardware cluster barrier, which replaces the per-phase kernel launches.
template <int D, typename R>
__global__ void __launch_bounds__(kTailThreads, 1) k_vcycle_tail(const TailLevel<R>* __restrict__ TL, int top,
                                                                 const R* __restrict__ r_top, R* __restrict__ z_top,
                                                                 const double* __restrict__ coarse_inv, int pre,
                                                                 int post) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int nthr = (int)(cl.num_blocks() * blockDim.x);
  const int tid = (int)(cl.block_rank() * blockDim.x + threadIdx.x);
  constexpr int NCOL = 1 << D, NP = CD<D, 2>::NP;
  auto phase_end = [&]() {
    __threadfence();
    cl.sync();
  };
  for (int l = top; l >= 1; --l) {                 // down: pre-smooth, residual, restrict
    const TailLevel<R>& L = TL[l];
    const R* r = l == top ? r_top : L.rhs;
    R* z = l == top ? z_top : L.z;
    if (pre == 0) {
      for (size_t q = tid; q < (size_t)L.P.n_act * NP; q += nthr) z[q] = R(0);
      phase_end();
    }
    for (int k = 0; k < pre; ++k)
      for (int col = 0; col < NCOL; ++col) {
        const int cs = L.P.colour_start[col], ce = L.P.colour_start[col + 1];
        for (int a = cs + tid; a < ce; a += nthr)
          smooth_one<D, 2, true, R>(L.P, col, k == 0, cs, L.P.colour_nbnd[col], L.P.bstart[col], a, r, z);
        phase_end();
      }
    const TailLevel<R>& Lc = TL[l - 1];
    for (int cc = tid; cc < Lc.P.n_act; cc += nthr) resid_restrict_h_one<D, true, R>(L.P, L.T, z, r, Lc.rhs, cc);
    phase_end();
  }
  {                                                // coarse solve in FP64, one warp per row
    const TailLevel<R>& L0 = TL[0];
    const int n0 = L0.P.n_act * NP;
    R* z0 = top == 0 ? z_top : L0.z;
    const R* r0 = top == 0 ? r_top : L0.rhs;
    const int lane = threadIdx.x & 31;
    for (int row = tid >> 5; row < n0; row += nthr >> 5) {
      double acc = 0;
      for (int c = lane; c < n0; c += 32) acc += coarse_inv[(size_t)row * n0 + c] * (double)ldv<true>(r0 + c);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) z0[row] = (R)acc;
    }
    phase_end();
  }
  for (int l = 1; l <= top; ++l) {                 // up: prolongate, post-smooth
    const TailLevel<R>& L = TL[l];
    const R* r = l == top ? r_top : L.rhs;
    R* z = l == top ? z_top : L.z;
    const R* zc = l - 1 == 0 && top == 0 ? z_top : TL[l - 1].z;
    for (int a = tid; a < L.P.n_act; a += nthr) prolong_h_one<D, R>(L.T, zc, z, a);
    phase_end();
    for (int k = 0; k < post; ++k)
      for (int q = 0; q < NCOL; ++q) {
        const int col = NCOL - 1 - q;
        const int cs = L.P.colour_start[col], ce = L.P.colour_start[col + 1];
        for (int a = cs + tid; a < ce; a += nthr)
          smooth_one<D, 2, true, R>(L.P, col, 0, cs, L.P.colour_nbnd[col], L.P.bstart[col], a, r, z);
        phase_end();
      }
  }
}

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

bool cell_kernels(int dim, int p) { return dim == 2 || (dim == 3 && p == 1); }

#define SBM_CELL_DISPATCH(dim, p, MACRO)            \
  do {                                              \
    if (dim == 2 && p == 1) { MACRO(2, 2); }        \
    else if (dim == 2 && p == 2) { MACRO(2, 3); }   \
    else if (dim == 2 && p == 3) { MACRO(2, 4); }   \
    else if (dim == 3 && p == 1) { MACRO(3, 2); }   \
    else return cudaErrorInvalidValue;              \
  } while (0)

template <typename TI, typename R>
cudaError_t launch_apply_cell(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                              cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
#define SBM_AC(D, N1)                                                                           \
  {                                                                                             \
    if (mode == 0) k_apply_cell<D, N1, TI, R, 0><<<cdiv(P.n_act, kCellThreads), kCellThreads, 0, s>>>(P, x, f, y); \
    else k_apply_cell<D, N1, TI, R, 1><<<cdiv(P.n_act, kCellThreads), kCellThreads, 0, s>>>(P, x, f, y);          \
  }
  SBM_CELL_DISPATCH(dim, p, SBM_AC);
#undef SBM_AC
  count_launches();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_smooth_cell(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f,
                               R* u, cudaStream_t s) {
  if (reverse) zero_start = 0;
  const int ncol = 1 << dim;
  for (int q = 0; q < ncol; ++q) {   // (the launcher in level_ops.cu chose this path for the level)
    const int col = reverse ? ncol - 1 - q : q;
    const int cs = P.colour_start[col], ce = P.colour_start[col + 1], nbnd = P.colour_nbnd[col];
    const int nblk_b = (int)cdiv(nbnd, kCellThreads), nblk_i = (int)cdiv(ce - cs - nbnd, kCellThreads);
    if (nblk_b + nblk_i == 0) continue;
#define SBM_SC(D, N1)                                                                                    \
  k_smooth_cell<D, N1, R><<<nblk_b + nblk_i, kCellThreads, 0, s>>>(P, col, zero_start, cs, nbnd, ce, nblk_b, \
                                                                   P.bstart[col], f, u);
    SBM_CELL_DISPATCH(dim, p, SBM_SC);
#undef SBM_SC
    count_launches();
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_resid_restrict_p_cell(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T,
                                        const R* u, const R* f, R* rc, cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
  const unsigned g = cdiv(P.n_act, kCellThreads);
  if (dim == 2 && pf == 2) k_resid_restrict_p_cell<2, 3, 2, R><<<g, kCellThreads, 0, s>>>(P, T, u, f, rc);
  else if (dim == 2 && pf == 3) k_resid_restrict_p_cell<2, 4, 3, R><<<g, kCellThreads, 0, s>>>(P, T, u, f, rc);
  else return cudaErrorInvalidValue;
  count_launches();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_resid_restrict_h_cell(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                        const R* f, R* rc, cudaStream_t s) {
  if (T.n_act_c == 0) return cudaSuccess;
  const unsigned g = cdiv(T.n_act_c, kCellThreads);
  if (dim == 2) k_resid_restrict_h_cell<2, R><<<g, kCellThreads, 0, s>>>(P, T, u, f, rc);
  else if (dim == 3) k_resid_restrict_h_cell<3, R><<<g, kCellThreads, 0, s>>>(P, T, u, f, rc);
  else return cudaErrorInvalidValue;
  count_launches();
  return cudaGetLastError();
}

int tail_cluster_size(int dim, int prec) {
  static int cached[2][2] = {{-1, -1}, {-1, -1}};
  int& c = cached[dim == 3][prec];
  if (c >= 0) return c;
  c = 0;
  for (int size : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(size);
    cfg.blockDim = dim3(kTailThreads);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e;
    if (dim == 2 && prec == 0) {
      cudaFuncSetAttribute(k_vcycle_tail<2, double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_tail<2, double>, &cfg);
    } else if (dim == 2) {
      cudaFuncSetAttribute(k_vcycle_tail<2, float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_tail<2, float>, &cfg);
    } else if (prec == 0) {
      cudaFuncSetAttribute(k_vcycle_tail<3, double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_tail<3, double>, &cfg);
    } else {
      cudaFuncSetAttribute(k_vcycle_tail<3, float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      e = cudaOccupancyMaxActiveClusters(&nclusters, k_vcycle_tail<3, float>, &cfg);
    }
    if (e == cudaSuccess && nclusters >= 1) {
      c = size;
      break;
    }
    cudaGetLastError();                            // clear a refused query
  }
  return c;
}

template <typename R>
cudaError_t launch_vcycle_tail(int dim, const TailLevel<R>* TL, int top, const R* r, R* z, const double* coarse_inv,
                               int pre, int post, cudaStream_t s) {
  const int size = tail_cluster_size(dim, sizeof(R) == 8 ? 0 : 1);
  if (size == 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(size);
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (dim == 2) e = cudaLaunchKernelEx(&cfg, k_vcycle_tail<2, R>, TL, top, r, z, coarse_inv, pre, post);
  else e = cudaLaunchKernelEx(&cfg, k_vcycle_tail<3, R>, TL, top, r, z, coarse_inv, pre, post);
  count_launches();
  return e;
}

template cudaError_t launch_vcycle_tail<double>(int, const TailLevel<double>*, int, const double*, double*,
                                                const double*, int, int, cudaStream_t);
template cudaError_t launch_vcycle_tail<float>(int, const TailLevel<float>*, int, const float*, float*, const double*,
                                               int, int, cudaStream_t);
template cudaError_t launch_apply_cell<double, double>(int, int, const LevelParams<double>&, const double*,
                                                       const double*, double*, int, cudaStream_t);
template cudaError_t launch_apply_cell<float, float>(int, int, const LevelParams<float>&, const float*, const float*,
                                                     float*, int, cudaStream_t);
template cudaError_t launch_apply_cell<float, double>(int, int, const LevelParams<double>&, const float*,
                                                      const double*, double*, int, cudaStream_t);
template cudaError_t launch_smooth_cell<double>(int, int, const LevelParams<double>&, int, int, const double*,
                                                double*, cudaStream_t);
template cudaError_t launch_smooth_cell<float>(int, int, const LevelParams<float>&, int, int, const float*, float*,
                                               cudaStream_t);
template cudaError_t launch_resid_restrict_p_cell<double>(int, int, const LevelParams<double>&,
                                                          const TransferParams<double>&, const double*, const double*,
                                                          double*, cudaStream_t);
template cudaError_t launch_resid_restrict_p_cell<float>(int, int, const LevelParams<float>&,
                                                         const TransferParams<float>&, const float*, const float*,
                                                         float*, cudaStream_t);
template cudaError_t launch_resid_restrict_h_cell<double>(int, const LevelParams<double>&,
                                                          const TransferParams<double>&, const double*, const double*,
                                                          double*, cudaStream_t);
template cudaError_t launch_resid_restrict_h_cell<float>(int, const LevelParams<float>&, const TransferParams<float>&,
                                                         const float*, const float*, float*, cudaStream_t);

}  // namespace sbm
