// CUDA kernels of one multigrid level (sm_103a): matrix-free DG-SBM operator, coloured block
// Gauss-Seidel smoother, h- and p-transfers, coarse dense solve.
//
// Paper: arXiv 2506.12899.  Operator: Eqs. 7, 10, 11 (Sec. 2.2).  Smoother: Eqs. 14, 16 (Sec. 3.1).
// Transfers: Eqs. 17, 18 (Sec. 3.2).
//
// Thread mapping: one thread per degree of freedom, CPB = floor(256 / (p+1)^d) cells per block.
// A block stages its cells and their 2d face neighbours in shared memory with coalesced loads
// (each cell's (p+1)^d values are contiguous), then every thread contracts the 1D element
// matrices along each direction (sum factorisation on the Cartesian cell).
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ops.h"

namespace sbm {

namespace {

template <int D, int N1>
struct Dims {
  static constexpr int NP = D == 2 ? N1 * N1 : N1 * N1 * N1;
  static constexpr int NQ = D == 2 ? N1 : N1 * N1;
  static constexpr int NS = 2 * D;
  static constexpr int CPB = 256 / NP > 0 ? 256 / NP : 1;
  static constexpr int NT = CPB * NP;
};

template <int N1>
__device__ __forceinline__ int stride_of(int dir) {
  return dir == 0 ? 1 : (dir == 1 ? N1 : N1 * N1);
}

template <int D, int N1>
__device__ __forceinline__ void decompose(int i, int (&ii)[3]) {
  ii[0] = i % N1;
  ii[1] = (i / N1) % N1;
  ii[2] = D == 3 ? i / (N1 * N1) : 0;
}

// Tangential index t (tangential dims ascending, first fastest) and weight of dof ii on the
// faces normal to dir.
template <int D, int N1, typename R>
__device__ __forceinline__ int tang(const int (&ii)[3], int dir, const R* w, R& wt) {
  if (D == 2) {
    const int k = ii[1 - dir];
    wt = w[k];
    return k;
  }
  const int a = dir == 0 ? 1 : 0, b = dir == 2 ? 1 : 2;
  wt = w[ii[a]] * w[ii[b]];
  return ii[a] + N1 * ii[b];
}

template <typename R>
__device__ __forceinline__ void load_consts(const LevelConsts<R>& src, LevelConsts<R>& dst) {
  constexpr int n = sizeof(LevelConsts<R>) / sizeof(R);
  const R* s = reinterpret_cast<const R*>(&src);
  R* d = reinterpret_cast<R*>(&dst);
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

// Index of cell a among boundary cells (cells owning a surrogate face), or -1.
template <typename R>
__device__ __forceinline__ int bnd_index(const LevelParams<R>& P, int a, int ncol) {
  int c = 0;
#pragma unroll
  for (int k = 1; k < 8; ++k)
    if (k < ncol && a >= P.colour_start[k]) c = k;
  const int off = a - P.colour_start[c];
  return off < P.colour_nbnd[c] ? P.bstart[c] + off : -1;
}

// Nitsche-SBM surrogate-face terms of Eq. 7 for the dofs of one block (reference form; the
// caller multiplies by h^(d-2)).  Per face point t: trace U_t, normal derivative G_t,
// extended value E_t = U_t + d^.grad^u (extension 0) or the cell polynomial at x~ + d
// (extension 1); dof (k, t) receives w_t [ e_s[k] (-s G_t + sigma^ E_t) - alpha s d_s[k] E_t ].
// Every thread of the block must call this (it contains barriers).  smask bit s marks slot s
// (= 2 * direction + side) as a surrogate face of this thread's cell.
template <int D, int N1, typename R>
__device__ __forceinline__ R sbm_face_terms(const LevelParams<R>& P, const LevelConsts<R>& C, int bidx,
                                            unsigned smask, int c, int i, const int (&ii)[3], const R* sU, R* sA,
                                            R* sB, R* sE) {
  using Dm = Dims<D, N1>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NS = Dm::NS;
  R acc = 0;
#pragma unroll 1
  for (int slot = 0; slot < NS; ++slot) {
    const int dir = slot >> 1, side = slot & 1;
    const bool sf = bidx >= 0 && ((smask >> slot) & 1u);
    const int st = stride_of<N1>(dir), id = ii[dir], base = i - id * st;
    R wt;
    const int t = tang<D, N1>(ii, dir, C.w, wt);
    const R* es = side ? C.e1 : C.e0;
    const R* ds = side ? C.d1 : C.d0;
    if (sf && id == 0) {
      R su = 0, sd = 0;
#pragma unroll
      for (int k = 0; k < N1; ++k) {
        const R v = sU[c * NP + base + k * st];
        su += es[k] * v;
        sd += ds[k] * v;
      }
      sA[c * NQ + t] = su;
      sB[c * NQ + t] = sd;
    }
    __syncthreads();
    if (sf && id == 0) {
      const R* dh = P.dhat + ((size_t)bidx * NS + slot) * D * NQ;
      R E;
      if (P.extension == 0) {
        E = sA[c * NQ + t] + dh[dir * NQ + t] * sB[c * NQ + t];
        if (D == 2) {
          const int m = 1 - dir;
          R g = 0;
#pragma unroll
          for (int q = 0; q < N1; ++q) g += C.Dm[t * N1 + q] * sA[c * NQ + q];
          E += dh[m * NQ + t] * g;
        } else {
          const int ma = dir == 0 ? 1 : 0, mb = dir == 2 ? 1 : 2;
          const int ta = t % N1, tb = t / N1;
          R ga = 0, gb = 0;
#pragma unroll
          for (int q = 0; q < N1; ++q) {
            ga += C.Dm[ta * N1 + q] * sA[c * NQ + q + N1 * tb];
            gb += C.Dm[tb * N1 + q] * sA[c * NQ + ta + N1 * q];
          }
          E += dh[ma * NQ + t] * ga + dh[mb * NQ + t] * gb;
        }
      } else {
        R lv[3][N1];
#pragma unroll
        for (int m = 0; m < D; ++m) {
          const R y = (m == dir ? R(side) : C.x[ii[m]]) + dh[m * NQ + t];
#pragma unroll
          for (int k = 0; k < N1; ++k) {
            R v = C.inv_denom[k];
#pragma unroll
            for (int j = 0; j < N1; ++j)
              if (j != k) v *= (y - C.x[j]);
            lv[m][k] = v;
          }
        }
        E = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          R ph = lv[0][j % N1] * lv[1][(j / N1) % N1];
          if (D == 3) ph *= lv[2][j / (N1 * N1)];
          E += ph * sU[c * NP + j];
        }
      }
      sE[c * NQ + t] = E;
    }
    __syncthreads();
    if (sf) {
      const R sg = side ? R(1) : R(-1);
      const R E = sE[c * NQ + t], G = sB[c * NQ + t];
      acc += wt * (es[id] * (-sg * G + P.sigG * E) - P.alpha * sg * ds[id] * E);
    }
    __syncthreads();
  }
  return acc;
}

// Face neighbours of cell a (-1 on every slot when !valid): set-up data, read before pdl_wait().
template <int D, typename R>
__device__ __forceinline__ void dof_nbr(const LevelParams<R>& P, int a, bool valid, int (&nb)[2 * D]) {
#pragma unroll
  for (int s = 0; s < 2 * D; ++s) nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;
}

// (A x) at dof i of the block's cell slot c (cell a, neighbours nb from dof_nbr) on one level;
// every thread of the block calls this (it contains barriers).  Stages the block's cells and their
// face neighbours in shared memory.
template <int D, int N1, typename TI, typename R>
__device__ __forceinline__ R apply_dof(const LevelParams<R>& P, const LevelConsts<R>& C, const TI* __restrict__ x,
                                       int c, int i, int a, bool valid, const int (&nb)[2 * D], R* sU, R* sN,
                                       R* sA, R* sB, R* sE) {
  using Dm = Dims<D, N1>;
  constexpr int NP = Dm::NP, NS = Dm::NS;
  if (valid) {
    sU[c * NP + i] = (R)x[(size_t)a * NP + i];
#pragma unroll
    for (int s = 0; s < NS; ++s) sN[(c * NS + s) * NP + i] = nb[s] >= 0 ? (R)x[(size_t)nb[s] * NP + i] : R(0);
  }
  __syncthreads();
  int ii[3];
  decompose<D, N1>(i, ii);
  R acc = 0;
  if (valid) {
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      const int st = stride_of<N1>(dir), id = ii[dir], base = i - id * st;
      R wt;
      tang<D, N1>(ii, dir, C.w, wt);
      const int mask = (nb[2 * dir] >= 0) + 2 * (nb[2 * dir + 1] >= 0);
      const R* Lm = C.L[mask];
      R s = 0;
#pragma unroll
      for (int k = 0; k < N1; ++k) s += Lm[id * N1 + k] * sU[c * NP + base + k * st];
      if (nb[2 * dir] >= 0) {
#pragma unroll
        for (int k = 0; k < N1; ++k) s += C.Bpm[id * N1 + k] * sN[(c * NS + 2 * dir) * NP + base + k * st];
      }
      if (nb[2 * dir + 1] >= 0) {
#pragma unroll
        for (int k = 0; k < N1; ++k) s += C.Bmp[id * N1 + k] * sN[(c * NS + 2 * dir + 1) * NP + base + k * st];
      }
      acc += wt * s;
    }
  }
  const int bidx = valid ? bnd_index(P, a, 1 << D) : -1;
  unsigned smask = 0;                               // bit s: face slot s is a surrogate face
#pragma unroll
  for (int s = 0; s < NS; ++s) smask |= (nb[s] < 0 ? 1u : 0u) << s;
  if (__syncthreads_or(bidx >= 0)) acc += sbm_face_terms<D, N1, R>(P, C, bidx, smask, c, i, ii, sU, sA, sB, sE);
  return P.hscale * acc;
}

// y = A x  (MODE 0)  or  y = f - A x  (MODE 1).
template <int D, int N1, typename TI, typename R, int MODE>
__global__ void __launch_bounds__(256) k_apply(const __grid_constant__ LevelParams<R> P, const TI* __restrict__ x,
                                               const R* __restrict__ f, R* __restrict__ y) {
  using Dm = Dims<D, N1>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NS = Dm::NS, CPB = Dm::CPB;
  __shared__ LevelConsts<R> C;
  __shared__ R sU[CPB * NP];
  __shared__ R sN[CPB * NS * NP];
  __shared__ R sA[CPB * NQ], sB[CPB * NQ], sE[CPB * NQ];
  load_consts(P.k, C);
  const int c = threadIdx.x / NP, i = threadIdx.x - c * NP;
  const int a = blockIdx.x * CPB + c;
  const bool valid = threadIdx.x < CPB * NP && a < P.n_act;
  int nb[NS];
  dof_nbr<D, R>(P, a, valid, nb);
  pdl_wait();
  pdl_trigger();
  R v = apply_dof<D, N1, TI, R>(P, C, x, c, i, a, valid, nb, sU, sN, sA, sB, sE);
  if (valid) {
    if (MODE == 1) v = f[(size_t)a * NP + i] - v;
    y[(size_t)a * NP + i] = v;
  }
}

// Residual and p-restriction fused (Eqs. 11, 18; same mesh, degree N1-1 -> NC-1):
//   rc_K = (Pp^T (x) Pp^T) (f - A u)_K, the residual kept in shared memory.
template <int D, int N1, int NC, typename R>
__global__ void __launch_bounds__(256) k_resid_restrict_p(const __grid_constant__ LevelParams<R> P,
                                                          const __grid_constant__ TransferParams<R> T,
                                                          const R* __restrict__ u, const R* __restrict__ f,
                                                          R* __restrict__ rc, int early) {
  using Dm = Dims<D, N1>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NS = Dm::NS, CPB = Dm::CPB;
  constexpr int NPC = D == 2 ? NC * NC : NC * NC * NC;
  __shared__ LevelConsts<R> C;
  __shared__ R sU[CPB * NP];
  __shared__ R sN[CPB * NS * NP];
  __shared__ R sA[CPB * NQ], sB[CPB * NQ], sE[CPB * NQ];
  __shared__ R sPp[N1 * NC];
  load_consts(P.k, C);
  for (int q = threadIdx.x; q < N1 * NC; q += blockDim.x) sPp[q] = T.Pp[q];
  const int c = threadIdx.x / NP, i = threadIdx.x - c * NP;
  const int a = blockIdx.x * CPB + c;
  const bool valid = threadIdx.x < CPB * NP && a < P.n_act;
  int nb[NS];
  dof_nbr<D, R>(P, a, valid, nb);
  R fv = 0;
  if (valid && early) fv = __ldcg(f + (size_t)a * NP + i);   // f written two or more launches back (L2)
  pdl_wait();
  pdl_trigger();
  if (valid && !early) fv = f[(size_t)a * NP + i];
  R v = apply_dof<D, N1, R, R>(P, C, u, c, i, a, valid, nb, sU, sN, sA, sB, sE);
  __syncthreads();                                   // sU is reused for the residual
  sU[c * NP + i] = valid ? fv - v : R(0);
  __syncthreads();
  if (valid && i < NPC) {
    const int j0 = i % NC, j1 = (i / NC) % NC, j2 = D == 3 ? i / (NC * NC) : 0;
    const R* r = sU + c * NP;
    R s2 = 0;
#pragma unroll
    for (int i2 = 0; i2 < (D == 3 ? N1 : 1); ++i2) {
      R s1 = 0;
#pragma unroll
      for (int i1 = 0; i1 < N1; ++i1) {
        R s0 = 0;
#pragma unroll
        for (int i0 = 0; i0 < N1; ++i0) s0 += sPp[i0 * NC + j0] * r[i0 + N1 * i1 + N1 * N1 * i2];
        s1 += sPp[i1 * NC + j1] * s0;
      }
      s2 += (D == 3 ? sPp[i2 * NC + j2] : R(1)) * s1;
    }
    rc[(size_t)a * NPC + i] = s2;
  }
}

// Residual and h-restriction fused (Eqs. 11, 18; p = 1 on both meshes): a block takes CPB / 2^d
// coarse cells; block slot c = 2^d * (coarse cell) + o holds child o (o = child bits = colour of
// the fine cell).  The children's residuals f - A u stay in shared memory (0 for inactive
// children) and rc_C = sum_o (Ph[o_0] (x) Ph[o_1] ...)^T r_child(o).
template <int D, typename R>
__global__ void __launch_bounds__(256) k_resid_restrict_h(const __grid_constant__ LevelParams<R> P,
                                                          const __grid_constant__ TransferParams<R> T,
                                                          const R* __restrict__ u, const R* __restrict__ f,
                                                          R* __restrict__ rc, int early) {
  using Dm = Dims<D, 2>;
  constexpr int NP = Dm::NP, NQ = Dm::NQ, NS = Dm::NS, CPB = Dm::CPB;
  constexpr int NCH = 1 << D, CPC = CPB / NCH;       // children per coarse cell, coarse cells per block
  __shared__ LevelConsts<R> C;
  __shared__ R sU[CPB * NP];
  __shared__ R sN[CPB * NS * NP];
  __shared__ R sA[CPB * NQ], sB[CPB * NQ], sE[CPB * NQ];
  __shared__ R sPh[2][4];
  load_consts(P.k, C);
  if (threadIdx.x < 8) sPh[threadIdx.x >> 2][threadIdx.x & 3] = T.Ph[threadIdx.x >> 2][threadIdx.x & 3];
  const int c = threadIdx.x / NP, i = threadIdx.x - c * NP;
  const int cc = blockIdx.x * CPC + c / NCH, o = c % NCH;
  const int a = (threadIdx.x < CPB * NP && cc < T.n_act_c) ? T.children[(size_t)o * T.n_act_c + cc] : -1;
  const bool valid = a >= 0;
  int nb[NS];
  dof_nbr<D, R>(P, a, valid, nb);
  R fv = 0;
  if (valid && early) fv = __ldcg(f + (size_t)a * NP + i);   // f written two or more launches back (L2)
  pdl_wait();
  pdl_trigger();
  if (valid && !early) fv = f[(size_t)a * NP + i];
  R v = apply_dof<D, 2, R, R>(P, C, u, c, i, a, valid, nb, sU, sN, sA, sB, sE);
  __syncthreads();                                   // sU is reused for the residuals
  sU[c * NP + i] = valid ? fv - v : R(0);
  __syncthreads();
  const int t = threadIdx.x;
  if (t < CPC * NP) {                               // coarse dof j of coarse cell t / NP (NPC = NP for p = 1)
    const int ccl = t / NP, j = t % NP;
    const int cc2 = blockIdx.x * CPC + ccl;
    if (cc2 < T.n_act_c) {
      const int j0 = j & 1, j1 = (j >> 1) & 1, j2 = (j >> 2) & 1;
      R sum = 0;
#pragma unroll
      for (int oo = 0; oo < NCH; ++oo) {
        const R* r = sU + (ccl * NCH + oo) * NP;
        const R* P0 = sPh[oo & 1];
        const R* P1 = sPh[(oo >> 1) & 1];
        const R* P2 = sPh[(oo >> 2) & 1];
        R s2 = 0;
#pragma unroll
        for (int i2 = 0; i2 < (D == 3 ? 2 : 1); ++i2) {
          R s1 = 0;
#pragma unroll
          for (int i1 = 0; i1 < 2; ++i1) {
            const R s0 = P0[0 * 2 + j0] * r[0 + 2 * i1 + 4 * i2] + P0[1 * 2 + j0] * r[1 + 2 * i1 + 4 * i2];
            s1 += P1[i1 * 2 + j1] * s0;
          }
          s2 += (D == 3 ? P2[i2 * 2 + j2] : R(1)) * s1;
        }
        sum += s2;
      }
      rc[(size_t)cc2 * NP + j] = sum;
    }
  }
}

// One colour of the block Gauss-Seidel sweep (Eq. 16): for each cell K of the colour,
//   t_K = f_K - sum_{N != K} A_KN u_N  (interior-face couplings only; the SBM terms lie in A_KK),
//   u_K <- (1 - omega) u_K + omega A_KK^{-1} t_K,
// which equals u_K + omega A_KK^{-1}(f - A u)_K.  Blocks [0, nblk_b) take the colour's boundary
// cells (dense inverse), the remaining blocks its interior cells (fast diagonalisation
// A_KK^{-1} = h^(2-d) S^(x d) diag(1 / sum lambda) (S^T)^(x d)).
//
// zero_start: u is the zero vector before this forward sweep; cells of colours not yet visited
// (neighbour colour > col) are read as zero and u itself is not read, so no memset is needed.
template <int D, int N1, typename R>
__global__ void __launch_bounds__(256) k_smooth(const __grid_constant__ LevelParams<R> P,
                                                const __grid_constant__ SmoothSegs G, int zero_start,
                                                const R* __restrict__ f, R* __restrict__ u, int early) {
  using Dm = Dims<D, N1>;
  constexpr int NP = Dm::NP, NS = Dm::NS, CPB = Dm::CPB;
  __shared__ LevelConsts<R> C;
  __shared__ R sN[CPB * NS * NP];
  __shared__ R sT[CPB * NP], sW[CPB * NP];
  load_consts(P.k, C);
  int sg = 0;                                        // the segment of this block (one colour, one kind)
#pragma unroll
  for (int k = 1; k < SmoothSegs::kMax; ++k)
    if (k < G.n && (int)blockIdx.x >= G.blk[k]) sg = k;
  const int col = G.col[sg], cs = G.cs[sg], b0 = G.b0[sg];
  const bool isB = G.first[sg] < cs + G.nbnd[sg];
  const int first = G.first[sg] + ((int)blockIdx.x - G.blk[sg]) * CPB;
  const int last = G.last[sg];
  const int c = threadIdx.x / NP, i = threadIdx.x - c * NP;
  const int a = first + c;
  const bool valid = threadIdx.x < CPB * NP && a < last;
  int nb[NS];
  dof_nbr<D, R>(P, a, valid, nb);                    // set-up data: read before the wait
#pragma unroll
  for (int s = 0; s < NS; ++s)                       // neighbours that read as zero (kZero* modes)
    if ((zero_start == kZeroLater && (col ^ (1 << (s >> 1))) > col) || zero_start == kZeroAll) nb[s] = -1;
  R fv = 0;
  if (valid && early) fv = __ldcg(f + (size_t)a * NP + i);   // f written two or more launches back (L2)
  pdl_wait();
  pdl_trigger();
  if (valid && !early) fv = f[(size_t)a * NP + i];
  R uold = 0;
  if (valid) {
#pragma unroll
    for (int s = 0; s < NS; ++s) sN[(c * NS + s) * NP + i] = nb[s] >= 0 ? u[(size_t)nb[s] * NP + i] : R(0);
    if (P.omega != R(1) && !zero_start) uold = u[(size_t)a * NP + i];
  }
  __syncthreads();
  int ii[3];
  decompose<D, N1>(i, ii);
  R t = 0;
  if (valid) {
    R acc = 0;
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      const int st = stride_of<N1>(dir), id = ii[dir], base = i - id * st;
      R wt;
      tang<D, N1>(ii, dir, C.w, wt);
      R s = 0;
      if (nb[2 * dir] >= 0) {
#pragma unroll
        for (int k = 0; k < N1; ++k) s += C.Bpm[id * N1 + k] * sN[(c * NS + 2 * dir) * NP + base + k * st];
      }
      if (nb[2 * dir + 1] >= 0) {
#pragma unroll
        for (int k = 0; k < N1; ++k) s += C.Bmp[id * N1 + k] * sN[(c * NS + 2 * dir + 1) * NP + base + k * st];
      }
      acc += wt * s;
    }
    t = fv - P.hscale * acc;
  }
  sT[c * NP + i] = t;
  __syncthreads();
  R yv = 0;
  if (isB) {
    if (valid) {
      const R* Bi = P.binvT + (size_t)(b0 + (a - cs)) * NP * NP;
#pragma unroll 8
      for (int j = 0; j < NP; ++j) yv += Bi[(size_t)j * NP + i] * sT[c * NP + j];
    }
  } else {
    R* src = sT;
    R* dst = sW;
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {              // (S^T)^(x d) t
      const int st = stride_of<N1>(dir), id = ii[dir], base = i - id * st;
      R v = 0;
#pragma unroll
      for (int m = 0; m < N1; ++m) v += C.S[m * N1 + id] * src[c * NP + base + m * st];
      yv = v;
      dst[c * NP + i] = v;
      __syncthreads();
      R* tmp = src;
      src = dst;
      dst = tmp;
    }
    yv = yv * C.inv_diag[i];
    dst[c * NP + i] = yv;
    __syncthreads();
    {
      R* tmp = src;
      src = dst;
      dst = tmp;
    }
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {              // S^(x d) v
      const int st = stride_of<N1>(dir), id = ii[dir], base = i - id * st;
      R v = 0;
#pragma unroll
      for (int m = 0; m < N1; ++m) v += C.S[id * N1 + m] * src[c * NP + base + m * st];
      yv = v;
      if (dir + 1 < D) {
        dst[c * NP + i] = v;
        __syncthreads();
        R* tmp = src;
        src = dst;
        dst = tmp;
      }
    }
  }
  if (valid) u[(size_t)a * NP + i] = P.omega == R(1) ? yv : (R(1) - P.omega) * uold + P.omega * yv;
}

// Restriction rc = P^T rf (Eq. 18), gathered per coarse dof.
template <int D, int NF, int NC, typename R>
__global__ void __launch_bounds__(256) k_restrict(const __grid_constant__ TransferParams<R> T,
                                                  const R* __restrict__ rf, R* __restrict__ rc) {
  pdl_entry();
  constexpr int NPF = D == 2 ? NF * NF : NF * NF * NF;
  constexpr int NPC = D == 2 ? NC * NC : NC * NC * NC;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int cc = (int)(gid / NPC), j = (int)(gid % NPC);
  if (cc >= T.n_act_c) return;
  const int j0 = j % NC, j1 = (j / NC) % NC, j2 = D == 3 ? j / (NC * NC) : 0;
  R sum = 0;
  const int nchild = T.hmode ? (1 << D) : 1;
  for (int o = 0; o < nchild; ++o) {
    int src;
    const R *P0, *P1, *P2;
    if (T.hmode) {
      src = T.children[(size_t)o * T.n_act_c + cc];
      if (src < 0) continue;
      P0 = T.Ph[o & 1];
      P1 = T.Ph[(o >> 1) & 1];
      P2 = T.Ph[(o >> 2) & 1];
    } else {
      src = cc;
      P0 = P1 = P2 = T.Pp;
    }
    const R* r = rf + (size_t)src * NPF;
    R s2 = 0;
#pragma unroll
    for (int i2 = 0; i2 < (D == 3 ? NF : 1); ++i2) {
      R s1 = 0;
#pragma unroll
      for (int i1 = 0; i1 < NF; ++i1) {
        R s0 = 0;
#pragma unroll
        for (int i0 = 0; i0 < NF; ++i0) s0 += P0[i0 * NC + j0] * r[i0 + NF * i1 + NF * NF * i2];
        s1 += P1[i1 * NC + j1] * s0;
      }
      s2 += (D == 3 ? P2[i2 * NC + j2] : R(1)) * s1;
    }
    sum += s2;
  }
  rc[(size_t)cc * NPC + j] = sum;
}

// Prolongation uf += P ec (Eq. 17) per fine dof; fine cells without an active parent get 0.
template <int D, int NF, int NC, typename R>
__global__ void __launch_bounds__(256) k_prolong(const __grid_constant__ TransferParams<R> T,
                                                 const R* __restrict__ ec, R* __restrict__ uf, int early) {
  constexpr int NPF = D == 2 ? NF * NF : NF * NF * NF;
  constexpr int NPC = D == 2 ? NC * NC : NC * NC * NC;
  const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int a = (int)(gid / NPF), i = (int)(gid % NPF);
  const int code = T.hmode && a < T.n_act_f ? T.parent_code[a] : 0;   // set-up data: before the wait
  R uv = 0;
  if (early && a < T.n_act_f && code >= 0) uv = __ldcg(uf + (size_t)a * NPF + i);   // uf two launches back (L2)
  pdl_wait();
  pdl_trigger();
  if (a >= T.n_act_f) return;
  if (!early && code >= 0) uv = uf[(size_t)a * NPF + i];
  int par;
  const R *P0, *P1, *P2;
  if (T.hmode) {
    if (code < 0) return;
    par = code >> 3;
    P0 = T.Ph[code & 1];
    P1 = T.Ph[(code >> 1) & 1];
    P2 = T.Ph[(code >> 2) & 1];
  } else {
    par = a;
    P0 = P1 = P2 = T.Pp;
  }
  const int i0 = i % NF, i1 = (i / NF) % NF, i2 = D == 3 ? i / (NF * NF) : 0;
  const R* e = ec + (size_t)par * NPC;
  R s2 = 0;
#pragma unroll
  for (int j2 = 0; j2 < (D == 3 ? NC : 1); ++j2) {
    R s1 = 0;
#pragma unroll
    for (int j1 = 0; j1 < NC; ++j1) {
      R s0 = 0;
#pragma unroll
      for (int j0 = 0; j0 < NC; ++j0) s0 += P0[i0 * NC + j0] * e[j0 + NC * j1 + NC * NC * j2];
      s1 += P1[i1 * NC + j1] * s0;
    }
    s2 += (D == 3 ? P2[i2 * NC + j2] : R(1)) * s1;
  }
  uf[(size_t)a * NPF + i] = uv + s2;
}

// e = Ainv r in FP64; one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(const double* __restrict__ Ainv, int N, const T* __restrict__ r,
                                                T* __restrict__ e) {
  pdl_entry();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + warp;
  if (row >= N) return;
  double s = 0;
  for (int col = lane; col < N; col += 32) s += Ainv[(size_t)row * N + col] * (double)r[col];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) e[row] = (T)s;
}

inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

// ------------------------------------------------------------------------------------ launchers
#define SBM_DISPATCH_DP(dim, p, MACRO)                 \
  do {                                                 \
    if (dim == 2 && p == 1) { MACRO(2, 2); }           \
    else if (dim == 2 && p == 2) { MACRO(2, 3); }      \
    else if (dim == 2 && p == 3) { MACRO(2, 4); }      \
    else if (dim == 3 && p == 1) { MACRO(3, 2); }      \
    else if (dim == 3 && p == 2) { MACRO(3, 3); }      \
    else if (dim == 3 && p == 3) { MACRO(3, 4); }      \
    else return cudaErrorInvalidValue;                 \
  } while (0)

template <typename TI, typename R>
cudaError_t launch_apply(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                         cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
  // 3D p = 2 has a thread-per-cell operator for FP32 only (cell_kernels / cell_smoother)
  constexpr bool f32 = std::is_same<TI, float>::value && std::is_same<R, float>::value;
  if constexpr (f32) {
    if (staged_kernels(dim, p) && P.staged_min > 0 && P.n_act >= P.staged_min)
      return launch_apply_staged(dim, p, P, x, f, y, mode, s);
  }
  if constexpr (std::is_same<TI, float>::value && (std::is_same<R, float>::value || std::is_same<R, dfl>::value)) {
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    const bool use = std::is_same<R, dfl>::value ? line_kernels_df(dim, p) : line_kernels(dim, p);
    if (use && P.cell_min > 0 && P.n_act >= P.cell_min && al16(x) && al16(y) && (mode == 0 || al16(f)))
      return launch_apply_line<R>(p, P, x, f, y, mode, s);
  }
  if ((f32 ? cell_kernels(dim, p) : cell_smoother(dim, p)) && P.cell_min > 0 && P.n_act >= P.cell_min)
    return launch_apply_cell<TI, R>(dim, p, P, x, f, y, mode, s);
#define SBM_APPLY(D, N1)                                                                 \
  {                                                                                      \
    using Dm = Dims<D, N1>;                                                              \
    const unsigned grid = ceil_div(P.n_act, Dm::CPB);                                    \
    if (mode == 0) SBM_PDL((k_apply<D, N1, TI, R, 0>), grid, Dm::NT, 0, s, P, x, f, y);         \
    else SBM_PDL((k_apply<D, N1, TI, R, 1>), grid, Dm::NT, 0, s, P, x, f, y);                   \
    count_launches();                                                                    \
  }
  SBM_DISPATCH_DP(dim, p, SBM_APPLY);
#undef SBM_APPLY
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_smooth(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f, R* u,
                          cudaStream_t s, int early, int first_group) {
  if constexpr (std::is_same<R, float>::value) {
    if (staged_kernels(dim, p) && P.staged_min > 0 && P.n_act >= (1 << dim) * P.staged_min) {
      if (first_group != 0) return cudaErrorInvalidValue;
      return launch_smooth_staged(dim, p, P, reverse, zero_start, f, u, s, early);
    }
  }
  if (cell_smoother(dim, p) && P.cell_min > 0 && P.n_act >= (1 << dim) * P.cell_min)
    return launch_smooth_cell<R>(dim, p, P, reverse, zero_start, f, u, s, early, first_group);
  if constexpr (std::is_same<R, float>::value) {
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    if (line_smoother(dim, p) && P.cell_min > 0 && P.n_act >= (1 << dim) * P.cell_min && al16(f) && al16(u))
      return launch_smooth_line(p, P, reverse, zero_start, f, u, s, early, first_group);
  }
  if (first_group != 0) return cudaErrorInvalidValue;
  if (reverse) zero_start = 0;
  int launched = 0;
  const int ng = n_colour_groups(P, dim);
  for (int q = 0; q < ng; ++q) {
    const int g = reverse ? ng - 1 - q : q;
    const int zm = group_zero_mode(P, zero_start, q);
    const int fe = launched > 0 || early;            // after the sweep's first launch f is two back
#define SBM_SMOOTH(D, N1)                                                                          \
  {                                                                                                \
    using Dm = Dims<D, N1>;                                                                        \
    const SmoothSegs G = smooth_segs(P, dim, g, Dm::CPB);                                          \
    if (G.n > 0 && G.blk[G.n] > 0) {                                                               \
      SBM_PDL((k_smooth<D, N1, R>), G.blk[G.n], Dm::NT, 0, s, P, G, zm, f, u, fe);                 \
      count_launches();                                                                            \
      ++launched;                                                                                  \
    }                                                                                              \
  }
    SBM_DISPATCH_DP(dim, p, SBM_SMOOTH);
#undef SBM_SMOOTH
  }
  return cudaGetLastError();
}

namespace {
// The update of the additive smoothers (block Jacobi, Chebyshev) after y = D^-1 (f - A z):
//   mode 0: z = b y (first Jacobi step from z = 0)      mode 1: z += b y
//   mode 2: d = b y, z = d (first Chebyshev step from 0) mode 3: d = b y, z += d
//   mode 4: d = a d + b y, z += d
template <typename R>
__global__ void k_smoother_update(size_t n, R a, R b, const R* __restrict__ y, R* __restrict__ d, R* __restrict__ z,
                                  int mode) {
  pdl_entry();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const R by = b * y[i];
    if (mode == 0) {
      z[i] = by;
    } else if (mode == 1) {
      z[i] += by;
    } else {
      const R di = mode == 4 ? a * d[i] + by : by;
      d[i] = di;
      z[i] = mode == 2 ? di : z[i] + di;
    }
  }
}
}  // namespace

template <typename R>
cudaError_t launch_smoother_update(size_t n, R a, R b, const R* y, R* d, R* z, int mode, cudaStream_t s) {
  size_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 152 * 8) g = 152 * 8;
  SBM_PDL((k_smoother_update<R>), (unsigned)g, 256, 0, s, n, a, b, y, d, z, mode);
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_smoother_update<double>(size_t, double, double, const double*, double*, double*, int,
                                                    cudaStream_t);
template cudaError_t launch_smoother_update<float>(size_t, float, float, const float*, float*, float*, int,
                                                   cudaStream_t);

template <typename R>
bool restrict_fuses_first_group(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T, int pc,
                                const LevelParams<R>& Pc) {
  const bool fine_cell = T.hmode ? (P.cell_min > 0 && T.n_act_f >= P.cell_min)
                                 : (cell_kernels(dim, pf) && P.cell_min > 0 && P.n_act >= P.cell_min);
  bool coarse_cell = cell_smoother(dim, pc) && Pc.cell_min > 0 && Pc.n_act >= (1 << dim) * Pc.cell_min &&
                     Pc.ordering == 0;
  if constexpr (std::is_same<R, float>::value)
    coarse_cell = coarse_cell && !(staged_kernels(dim, pc) && Pc.staged_min > 0 && Pc.n_act >= (1 << dim) * Pc.staged_min);
  return fine_cell && coarse_cell;
}
template bool restrict_fuses_first_group<double>(int, int, const LevelParams<double>&, const TransferParams<double>&,
                                                 int, const LevelParams<double>&);
template bool restrict_fuses_first_group<float>(int, int, const LevelParams<float>&, const TransferParams<float>&, int,
                                                const LevelParams<float>&);

#define SBM_DISPATCH_T(dim, pf, pc, MACRO)                          \
  do {                                                              \
    if (dim == 2 && pf == 1 && pc == 1) { MACRO(2, 2, 2); }         \
    else if (dim == 2 && pf == 2 && pc == 1) { MACRO(2, 3, 2); }    \
    else if (dim == 2 && pf == 3 && pc == 2) { MACRO(2, 4, 3); }    \
    else if (dim == 3 && pf == 1 && pc == 1) { MACRO(3, 2, 2); }    \
    else if (dim == 3 && pf == 2 && pc == 1) { MACRO(3, 3, 2); }    \
    else if (dim == 3 && pf == 3 && pc == 2) { MACRO(3, 4, 3); }    \
    else return cudaErrorInvalidValue;                              \
  } while (0)

template <typename R>
cudaError_t launch_resid_restrict_p(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                   const R* f, R* rc, cudaStream_t s, int early, const LevelParams<R>* Pc, R* zc) {
  if (P.n_act == 0) return cudaSuccess;
  if (cell_kernels(dim, pf) && P.cell_min > 0 && P.n_act >= P.cell_min)
    return launch_resid_restrict_p_cell<R>(dim, pf, P, T, u, f, rc, s, early, Pc, zc);
  if (Pc || zc) return cudaErrorInvalidValue;       // the fused first group exists on the cell path only
  if constexpr (std::is_same<R, float>::value) {
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    if (dim == 3 && pf == 3 && P.cell_min > 0 && P.n_act >= P.cell_min && al16(u) && al16(f))
      return launch_resid_restrict_line(P, T, u, f, rc, s, early);
  }
#define SBM_RRP(D, N1, NC)                                                                         \
  {                                                                                                \
    using Dm = Dims<D, N1>;                                                                        \
    SBM_PDL((k_resid_restrict_p<D, N1, NC, R>), ceil_div(P.n_act, Dm::CPB), Dm::NT, 0, s, P, T, u, f, rc, early); \
    count_launches();                                                                              \
  }
  if (dim == 2 && pf == 2) { SBM_RRP(2, 3, 2); }
  else if (dim == 2 && pf == 3) { SBM_RRP(2, 4, 3); }
  else if (dim == 3 && pf == 2) { SBM_RRP(3, 3, 2); }
  else if (dim == 3 && pf == 3) { SBM_RRP(3, 4, 3); }
  else return cudaErrorInvalidValue;
#undef SBM_RRP
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_resid_restrict_h(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                   const R* f, R* rc, cudaStream_t s, int early, const LevelParams<R>* Pc, R* zc) {
  if (T.n_act_c == 0) return cudaSuccess;
  if (P.cell_min > 0 && T.n_act_f >= P.cell_min)
    return launch_resid_restrict_h_cell<R>(dim, P, T, u, f, rc, s, early, Pc, zc);
  if (Pc || zc) return cudaErrorInvalidValue;       // the fused first group exists on the cell path only
  if (dim == 2) {
    using Dm = Dims<2, 2>;
    SBM_PDL((k_resid_restrict_h<2, R>), ceil_div(T.n_act_c, Dm::CPB / 4), Dm::NT, 0, s, P, T, u, f, rc, early);
  } else if (dim == 3) {
    using Dm = Dims<3, 2>;
    SBM_PDL((k_resid_restrict_h<3, R>), ceil_div(T.n_act_c, Dm::CPB / 8), Dm::NT, 0, s, P, T, u, f, rc, early);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launches();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_restrict(int dim, int pf, int pc, const TransferParams<R>& T, const R* rf, R* rc, cudaStream_t s) {
  if (T.n_act_c == 0) return cudaSuccess;
#define SBM_RESTRICT(D, NF, NC)                                                   \
  {                                                                               \
    const size_t n = (size_t)T.n_act_c * (D == 2 ? NC * NC : NC * NC * NC);       \
    SBM_PDL((k_restrict<D, NF, NC, R>), ceil_div(n, 256), 256, 0, s, T, rf, rc);         \
    count_launches();                                                             \
  }
  SBM_DISPATCH_T(dim, pf, pc, SBM_RESTRICT);
#undef SBM_RESTRICT
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_prolong(int dim, int pf, int pc, const TransferParams<R>& T, const R* ec, R* uf, cudaStream_t s,
                           int early) {
  if (T.n_act_f == 0) return cudaSuccess;
#define SBM_PROLONG(D, NF, NC)                                                    \
  {                                                                               \
    const size_t n = (size_t)T.n_act_f * (D == 2 ? NF * NF : NF * NF * NF);       \
    SBM_PDL((k_prolong<D, NF, NC, R>), ceil_div(n, 256), 256, 0, s, T, ec, uf, early);   \
    count_launches();                                                             \
  }
  SBM_DISPATCH_T(dim, pf, pc, SBM_PROLONG);
#undef SBM_PROLONG
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse(const double* Ainv, int N, const T* r, T* e, cudaStream_t s) {
  if (N == 0) return cudaSuccess;
  SBM_PDL((k_coarse<T>), ceil_div(N, 8), 256, 0, s, Ainv, N, r, e);
  count_launches();
  return cudaGetLastError();
}

template cudaError_t launch_apply<double, double>(int, int, const LevelParams<double>&, const double*, const double*,
                                                  double*, int, cudaStream_t);
template cudaError_t launch_apply<float, float>(int, int, const LevelParams<float>&, const float*, const float*,
                                                float*, int, cudaStream_t);
template cudaError_t launch_apply<float, double>(int, int, const LevelParams<double>&, const float*, const double*,
                                                 double*, int, cudaStream_t);
template cudaError_t launch_apply<float, dfl>(int, int, const LevelParams<dfl>&, const float*, const dfl*, dfl*, int,
                                              cudaStream_t);
template cudaError_t launch_smooth<double>(int, int, const LevelParams<double>&, int, int, const double*, double*,
                                               cudaStream_t, int, int);
template cudaError_t launch_smooth<float>(int, int, const LevelParams<float>&, int, int, const float*, float*,
                                               cudaStream_t, int, int);
template cudaError_t launch_resid_restrict_p<double>(int, int, const LevelParams<double>&,
                                                     const TransferParams<double>&, const double*, const double*,
                                                     double*, cudaStream_t, int, const LevelParams<double>*, double*);
template cudaError_t launch_resid_restrict_p<float>(int, int, const LevelParams<float>&, const TransferParams<float>&,
                                                    const float*, const float*, float*, cudaStream_t, int,
                                                    const LevelParams<float>*, float*);
template cudaError_t launch_resid_restrict_h<double>(int, const LevelParams<double>&, const TransferParams<double>&,
                                                     const double*, const double*, double*, cudaStream_t, int,
                                                     const LevelParams<double>*, double*);
template cudaError_t launch_resid_restrict_h<float>(int, const LevelParams<float>&, const TransferParams<float>&,
                                                    const float*, const float*, float*, cudaStream_t, int,
                                                    const LevelParams<float>*, float*);
template cudaError_t launch_restrict<double>(int, int, int, const TransferParams<double>&, const double*, double*,
                                             cudaStream_t);
template cudaError_t launch_restrict<float>(int, int, int, const TransferParams<float>&, const float*, float*,
                                            cudaStream_t);
template cudaError_t launch_prolong<double>(int, int, int, const TransferParams<double>&, const double*, double*,
                                            cudaStream_t, int);
template cudaError_t launch_prolong<float>(int, int, int, const TransferParams<float>&, const float*, float*,
                                           cudaStream_t, int);
template cudaError_t launch_coarse<double>(const double*, int, const double*, double*, cudaStream_t);
template cudaError_t launch_coarse<float>(const double*, int, const float*, float*, cudaStream_t);

}  // namespace sbm
