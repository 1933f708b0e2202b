// Thread-per-cell CUDA kernels for small cells ((p+1)^d <= 16: 2D p = 1..3 and 3D p = 1; the FP32
// operator and residual + restriction also for 3D p = 2).
//
// One thread owns one cell: its (p+1)^d values, the interior-face couplings to its 2d
// neighbours, its surrogate-face terms and its block inverse live in registers.  Every loop
// over nodes, lines and directions is unrolled, so each 1D-matrix coefficient is a uniform,
// immediate-offset read of the kernel parameter block (constant cache broadcast).  The per-DoF
// kernels of level_ops.cu issue about 175 instructions per DoF, mostly shared-memory traffic;
// here the arithmetic is the same (Eqs. 7, 10, 11, 14, 16, 18) but the instruction stream is a
// fraction of that.  Cells of an odd number of values are read through their 16-byte-aligned
// window and stored through shared memory (cell_core.cuh); launches over a whole level take the
// colours interleaved (interleaved_warp).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "ops.h"

namespace sbm {
namespace {

#include "cell_core.cuh"

// Launches over all cells of a level interleave the colours: block b takes chunk b / 2^D (of
// blockDim.x consecutive cells) of colour b mod 2^D.  The face neighbours of a cell all have
// other colours, so with the colours taken one after another every colour's values would be read
// from DRAM once for its own pass and again in the passes of the colours next to it; interleaved,
// the blocks in flight cover the same stretch of the mesh in every colour and the neighbours'
// values are found in L2.  Sets the first cell of the calling thread's warp and the end of its
// colour (the warp holds min(32, end - a0w) cells, none if that is <= 0).
template <int D, typename R>
__device__ __forceinline__ void interleaved_warp(const LevelParams<R>& P, int& a0w, int& end) {
  constexpr int NCOL = 1 << D;
  const int c = (int)blockIdx.x % NCOL;
  a0w = P.colour_start[c] + ((int)blockIdx.x / NCOL) * (int)blockDim.x + ((int)threadIdx.x & ~31);
  end = P.colour_start[c + 1];
}

// y = A x (MODE 0) or y = f - A x (MODE 1), one thread per cell, colours interleaved.
template <int D, int N1, typename TI, typename R, int MODE>
__device__ __forceinline__ void apply_cell_body(const LevelParams<R>& P, const TI* __restrict__ x,
                                                const R* __restrict__ f, R* __restrict__ y) {
  constexpr int NP = CD<D, N1>::NP;
  int a0w, end;
  interleaved_warp<D, R>(P, a0w, end);
  const int a = a0w + ((int)threadIdx.x & 31);
  const bool valid = a < end;
  int nb[2 * D];
  if (valid) load_nbr<D, R>(P, a, nb);             // set-up data: read before the wait
  pdl_wait();
  pdl_trigger();
  R r[NP];
  if (valid) {
    cell_apply<D, N1, TI, R>(P, x, a, nb, r);
    if (MODE == 1) {
      R fv[NP];
      load_cell<D, N1, R, R>(f, a, P.n_act, fv);
#pragma unroll
      for (int i = 0; i < NP; ++i) r[i] = fv[i] - r[i];
    }
  }
  if constexpr (cell_vec16<NP, R>()) {
    if (valid) store_cell<D, N1, R>(y, a, r);
  } else {
    __shared__ WarpStage<NP, R> stage;
    if (a0w < end) warp_store_cells<NP, R>(y, a0w, min(32, end - a0w), r, stage.v[threadIdx.x >> 5]);
  }
}

template <int D, int N1, typename TI, typename R, int MODE>
__global__ void __launch_bounds__(kCellThreads) k_apply_cell(const __grid_constant__ LevelParams<R> P,
                                                             const TI* __restrict__ x, const R* __restrict__ f,
                                                             R* __restrict__ y) {
  apply_cell_body<D, N1, TI, R, MODE>(P, x, f, y);
}

// The same, compiled for 24 resident warps per SM (80 registers).  Used for the double-float
// operator of 2D p = 2: at its natural 96 registers an SM holds 20 warps, and the 512^2 p = 2 grid
// of 3164 warps then runs as 1.04 waves whose last warps run alone; at 80 every warp is resident
// at once.  (2D p = 3 spills heavily at 80; p = 1 needs fewer than 80.)
template <int D, int N1, typename TI, typename R, int MODE>
__global__ void __launch_bounds__(kCellThreads, 6) k_apply_cell_occ(const __grid_constant__ LevelParams<R> P,
                                                                    const TI* __restrict__ x,
                                                                    const R* __restrict__ f, R* __restrict__ y) {
  apply_cell_body<D, N1, TI, R, MODE>(P, x, f, y);
}


// One colour group of the block Gauss-Seidel sweep, one thread per cell: block b updates cells of
// the segment whose block range holds b.
template <int D, int N1, typename R>
__global__ void __launch_bounds__(kCellThreads) k_smooth_cell(const __grid_constant__ LevelParams<R> P,
                                                              const __grid_constant__ SmoothSegs G, int zero_start,
                                                              const R* __restrict__ f, R* __restrict__ u, int early) {
  constexpr int NP = CD<D, N1>::NP;
  int sg = 0;
#pragma unroll
  for (int k = 1; k < SmoothSegs::kMax; ++k)
    if (k < G.n && (int)blockIdx.x >= G.blk[k]) sg = k;
  const int a0w = G.first[sg] + ((int)blockIdx.x - G.blk[sg]) * (int)blockDim.x + ((int)threadIdx.x & ~31);
  const int end = G.last[sg];
  const int a = a0w + ((int)threadIdx.x & 31);
  const bool valid = a < end;
  int nb[2 * D];
  R t[NP];
  if (valid) {
    load_nbr<D, R>(P, a, nb);                        // set-up data: read before the wait
    if (early) load_cell_l2<D, N1, R, R>(f, a, P.n_act, t);   // f written two or more launches back
  }
  pdl_wait();
  pdl_trigger();
  R y[NP];
  if (valid) {
    if (!early) load_cell<D, N1, R, R>(f, a, P.n_act, t);
    smooth_rhs<D, N1, R>(P, G.col[sg], zero_start, nb, t, u);
    const int off = a - G.cs[sg];
    block_solve<D, N1, R>(P, off < G.nbnd[sg] ? G.b0[sg] + off : -1, t, y);
    smooth_relax<D, N1, R>(P, zero_start, a, u, y);
  }
  if constexpr (cell_vec16<NP, R>()) {
    if (valid) store_cell<D, N1, R>(u, a, y);
  } else {
    __shared__ WarpStage<NP, R> stage;
    if (a0w < end) warp_store_cells<NP, R>(u, a0w, min(32, end - a0w), y, stage.v[threadIdx.x >> 5]);
  }
}

// Residual and p-restriction fused, one thread per cell (Eqs. 11, 18).
// SM0: also the first colour group (colour 0) of the coarse level's first pre-smoothing sweep from
// zero, zc_K = omega A_KK^-1 rc_K for coarse cells K of colour 0 (their neighbours, of later
// colours, are still zero), with the coarse level's parameters Pc; that sweep then starts at group 1.
template <int D, int N1, int NC, typename R, bool SM0>
__global__ void __launch_bounds__(kCellThreads) k_resid_restrict_p_cell(const __grid_constant__ LevelParams<R> P,
                                                                        const __grid_constant__ TransferParams<R> T,
                                                                        const R* __restrict__ u,
                                                                        const R* __restrict__ f, R* __restrict__ rc,
                                                                        int early,
                                                                        const __grid_constant__ LevelParams<R> Pc,
                                                                        R* __restrict__ zc) {
  constexpr int NP = CD<D, N1>::NP;
  constexpr int NPC = D == 2 ? NC * NC : NC * NC * NC;
  int a0w, end;
  interleaved_warp<D, R>(P, a0w, end);               // colours interleaved
  const int a = a0w + ((int)threadIdx.x & 31);
  int nb[2 * D];
  R fa[NP];
  if (a < end) {
    load_nbr<D, R>(P, a, nb);                        // set-up data: read before the wait
    if (early) load_cell_l2<D, N1, R, R>(f, a, P.n_act, fa);  // f written two or more launches back
  }
  pdl_wait();
  pdl_trigger();
  if (a >= end) return;
  if (!early) load_cell<D, N1, R, R>(f, a, P.n_act, fa);
  R r[NP];
  cell_apply<D, N1, R, R>(P, u, a, nb, r);
#pragma unroll
  for (int i = 0; i < NP; ++i) r[i] = fa[i] - r[i];
  R out[NPC];
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
    out[j] = acc;
    rc[(size_t)a * NPC + j] = acc;
  }
  if constexpr (SM0) {
    if (a < Pc.colour_start[1]) {                    // same mesh: the coarse cell has index a
      R y[NPC];
      block_solve<D, NC, R>(Pc, a < Pc.colour_nbnd[0] ? Pc.bstart[0] + a : -1, out, y);
#pragma unroll
      for (int j = 0; j < NPC; ++j) y[j] = Pc.omega == R(1) ? y[j] : Pc.omega * y[j];
      store_cell<D, NC, R>(zc, a, y);
    }
  }
}

// h-transfer weight of fine node i (child o of its parent) and coarse node j, p = 1 on both
// meshes (Eqs. 17, 18): the tensor product of the 1D child matrices.
template <int D, typename R>
__device__ __forceinline__ R h_weight(const TransferParams<R>& T, int o, int i, int j) {
  R wgt = T.Ph[o & 1][(i & 1) * 2 + (j & 1)] * T.Ph[(o >> 1) & 1][((i >> 1) & 1) * 2 + ((j >> 1) & 1)];
  if (D == 3) wgt *= T.Ph[(o >> 2) & 1][((i >> 2) & 1) * 2 + ((j >> 2) & 1)];
  return wgt;
}

// One group of 2^D adjacent lanes per coarse cell, lane o of the group handling child o: the
// child's residual in registers, its restriction, then a fixed butterfly sum over the group.
// SM0: also the first colour group of the coarse level's first pre-smoothing sweep from zero (see
// k_resid_restrict_p_cell), computed by lane 0 of each coarse cell's group.
template <int D, typename R, bool SM0>
__global__ void __launch_bounds__(kCellThreads) k_resid_restrict_h_cell(const __grid_constant__ LevelParams<R> P,
                                                                        const __grid_constant__ TransferParams<R> T,
                                                                        const R* __restrict__ u,
                                                                        const R* __restrict__ f, R* __restrict__ rc,
                                                                        int early,
                                                                        const __grid_constant__ LevelParams<R> Pc,
                                                                        R* __restrict__ zc) {
  constexpr int NCOL = 1 << D, NP = CD<D, 2>::NP;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int cc = t / NCOL, o = t % NCOL;
  R out[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) out[j] = 0;
  // the child and its neighbours are set-up data: read before the wait
  const int a = cc < T.n_act_c ? T.children[(size_t)o * T.n_act_c + cc] : -1;
  int nb[2 * D];
  R fa[NP];
  if (a >= 0) {
    load_nbr<D, R>(P, a, nb);
    if (early) load_cell_l2<D, 2, R, R>(f, a, P.n_act, fa);   // f written two or more launches back
  }
  pdl_wait();
  pdl_trigger();
  if (a >= 0) {
    R r[NP];
    if (!early) load_cell<D, 2, R, R>(f, a, P.n_act, fa);
    cell_apply<D, 2, R, R>(P, u, a, nb, r);
#pragma unroll
    for (int i = 0; i < NP; ++i) r[i] = fa[i] - r[i];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      R acc = 0;
#pragma unroll
      for (int i = 0; i < NP; ++i) acc += h_weight<D, R>(T, o, i, j) * r[i];
      out[j] = acc;
    }
  }
#pragma unroll
  for (int off = 1; off < NCOL; off <<= 1)
#pragma unroll
    for (int j = 0; j < NP; ++j) out[j] += __shfl_xor_sync(0xffffffffu, out[j], off);
  if (o == 0 && cc < T.n_act_c) {
#pragma unroll
    for (int j = 0; j < NP; ++j) rc[(size_t)cc * NP + j] = out[j];
    if constexpr (SM0) {
      if (cc < Pc.colour_start[1]) {
        R y[NP];
        block_solve<D, 2, R>(Pc, cc < Pc.colour_nbnd[0] ? Pc.bstart[0] + cc : -1, out, y);
#pragma unroll
        for (int j = 0; j < NP; ++j) y[j] = Pc.omega == R(1) ? y[j] : Pc.omega * y[j];
        store_cell<D, 2, R>(zc, cc, y);
      }
    }
  }
}


// ----------------------------------------------------------------------------------------------
// The V-cycle below and including level `top` (all of them p = 1 h-levels) in one launch of a
// thread-block cluster, with every level vector held in the cluster's shared memory.
//
// Layout: colour c of a level (cells [cs_c, ce_c) of the colour-major order) is cut into
// chunks of m[c] consecutive cells, chunk k living on CTA k of the cluster; a CTA stores its
// chunks of all colours back to back (colour c from cell slot off[c]) once for z (element
// offset zoff) and once for the right-hand side (roff).  A CTA updates only the cells it
// stores; neighbour, child and parent values of other CTAs are read through distributed shared
// memory.  Every phase (one colour of a sweep, the fused residual/restriction, the coarse solve,
// a prolongation) ends with a cluster barrier, whose release/acquire semantics order the shared
// memory writes of the phase before the reads of the next.
// ----------------------------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ int colour_of(const TailLevel<R>& L, int a, int ncol) {
  int c = 0;
#pragma unroll
  for (int k = 1; k < 8; ++k)
    if (k < ncol && a >= L.P.colour_start[k]) c = k;
  return c;
}

// Generic address of the NP values of cell a (colour col) of vector `vo` (zoff or roff) of L.
template <int NP, typename R>
__device__ __forceinline__ R* tail_cell(const cooperative_groups::cluster_group& cl, R* sm, const TailLevel<R>& L,
                                        int vo, int a, int col) {
  const int rel = a - L.P.colour_start[col];
  const int rk = rel / L.m[col];
  R* p = sm + vo + (size_t)(L.off[col] + rel - rk * L.m[col]) * NP;
  return cl.map_shared_rank(p, (unsigned)rk);
}

template <int D, typename R>
__global__ void __launch_bounds__(kTailThreads, 1) k_vcycle_tail(const TailLevel<R>* __restrict__ TL, int top,
                                                                 const R* __restrict__ r_top, R* __restrict__ z_top,
                                                                 const double* __restrict__ coarse_inv, int pre,
                                                                 int post, int ssor, int gather_off) {
  namespace cg = cooperative_groups;
  const cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char tail_smem[];
  R* sm = reinterpret_cast<R*>(tail_smem);
  const int rank = (int)cl.block_rank();
  constexpr int NCOL = 1 << D, NP = CD<D, 2>::NP;

  // this CTA's cells of colour col of L: fn(cell, slot)
  auto for_own = [&](const TailLevel<R>& L, int col, auto&& fn) {
    const int cs = L.P.colour_start[col], ce = L.P.colour_start[col + 1], m = L.m[col];
    const int first = cs + rank * m;
    const int cnt = min(m, ce - first);
    for (int j = threadIdx.x; j < cnt; j += kTailThreads) fn(first + j, L.off[col] + j);
  };
  auto loader = [&cl, sm](const TailLevel<R>& L, int vo) {
    const TailLevel<R>* Lp = &L;
    return [&cl, sm, Lp, vo](int n, int ncol, R(&un)[NP]) {
      load_np_vec<NP, R>(tail_cell<NP>(cl, sm, *Lp, vo, n, ncol), un);
    };
  };
  auto smooth = [&](const TailLevel<R>& L, int col, bool zs) {
    for_own(L, col, [&](int a, int slot) {
      const LevelParams<R>& P = L.P;
      int nb[2 * D];
      load_nbr<D, R>(P, a, nb);
      R c[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) c[i] = 0;
      add_couplings_f<D, 2, R>(P.k, col, zs, nb, loader(L, L.zoff), c);
      R t[NP];
      load_np_vec<NP, R>(sm + L.roff + (size_t)slot * NP, t);
#pragma unroll
      for (int i = 0; i < NP; ++i) t[i] -= P.hscale * c[i];
      const int off = a - P.colour_start[col];
      R y[NP];
      block_solve<D, 2, R>(P, off < P.colour_nbnd[col] ? P.bstart[col] + off : -1, t, y);
      R* zu = sm + L.zoff + (size_t)slot * NP;
      if (P.omega != R(1)) {
        R uo[NP];
        if (zs) {
#pragma unroll
          for (int i = 0; i < NP; ++i) uo[i] = 0;
        } else {
          load_np_vec<NP, R>(zu, uo);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) y[i] = (R(1) - P.omega) * uo[i] + P.omega * y[i];
      }
      store_np_vec<NP, R>(zu, y);
    });
  };

  {                                                // right-hand side of the top level
    const TailLevel<R>& L = TL[top];
    for (int col = 0; col < NCOL; ++col)
      for_own(L, col, [&](int a, int slot) {
#pragma unroll
        for (int i = 0; i < NP; ++i) sm[L.roff + (size_t)slot * NP + i] = r_top[(size_t)a * NP + i];
      });
    cl.sync();
  }
  for (int l = top; l >= 1; --l) {                 // down: pre-smooth, residual, restrict
    const TailLevel<R>& L = TL[l];
    if (pre == 0) {
      for (int q = threadIdx.x; q < L.ncell * NP; q += kTailThreads) sm[L.zoff + q] = R(0);
      cl.sync();
    }
    for (int k = 0; k < pre; ++k) {
      for (int col = 0; col < NCOL; ++col) {
        smooth(L, col, k == 0);
        cl.sync();
      }
      if (ssor)
        for (int q = 0; q < NCOL; ++q) {
          smooth(L, NCOL - 1 - q, false);
          cl.sync();
        }
    }
    const TailLevel<R>& Lc = TL[l - 1];
    for (int ccol = 0; ccol < NCOL; ++ccol)
      for_own(Lc, ccol, [&](int cc, int slot) {
        R out[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) out[j] = 0;
#pragma unroll 1
        for (int o = 0; o < NCOL; ++o) {
          const int a = L.T.children[(size_t)o * L.T.n_act_c + cc];
          if (a < 0) continue;
          const int ca = colour_of(L, a, NCOL);
          int nb[2 * D];
          load_nbr<D, R>(L.P, a, nb);
          R v[NP], y[NP], f[NP];
          load_np_vec<NP, R>(tail_cell<NP>(cl, sm, L, L.zoff, a, ca), v);
          load_np_vec<NP, R>(tail_cell<NP>(cl, sm, L, L.roff, a, ca), f);
#pragma unroll
          for (int i = 0; i < NP; ++i) y[i] = 0;
          const int off = a - L.P.colour_start[ca];
          add_self<D, 2, R>(L.P, nb, off < L.P.colour_nbnd[ca] ? L.P.bstart[ca] + off : -1, v, y);
          add_couplings_f<D, 2, R>(L.P.k, ca, false, nb, loader(L, L.zoff), y);
#pragma unroll
          for (int i = 0; i < NP; ++i) y[i] = f[i] - L.P.hscale * y[i];
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            R acc = 0;
#pragma unroll
            for (int i = 0; i < NP; ++i) acc += h_weight<D, R>(L.T, o, i, j) * y[i];
            out[j] += acc;
          }
        }
        store_np_vec<NP, R>(sm + Lc.roff + (size_t)slot * NP, out);
      });
    cl.sync();
  }
  {                                                // coarse solve in FP64, one warp per row
    const TailLevel<R>& L0 = TL[0];
    const int n0 = L0.P.n_act * NP;
    R* g = sm + gather_off;                        // this CTA's copy of the whole coarse rhs
    for (int a = threadIdx.x; a < L0.P.n_act; a += kTailThreads) {
      R v[NP];
      load_np_vec<NP, R>(tail_cell<NP>(cl, sm, L0, L0.roff, a, colour_of(L0, a, NCOL)), v);
      store_np_vec<NP, R>(g + (size_t)a * NP, v);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nwarp = (int)cl.num_blocks() * (kTailThreads / 32);
    for (int row = rank * (kTailThreads / 32) + (threadIdx.x >> 5); row < n0; row += nwarp) {
      double acc = 0;
      for (int c = lane; c < n0; c += 32) acc += coarse_inv[(size_t)row * n0 + c] * (double)g[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (lane == 0) {
        const int cell = row / NP;
        tail_cell<NP>(cl, sm, L0, L0.zoff, cell, colour_of(L0, cell, NCOL))[row - cell * NP] = (R)acc;
      }
    }
    cl.sync();
  }
  for (int l = 1; l <= top; ++l) {                 // up: prolongate, post-smooth
    const TailLevel<R>& L = TL[l];
    const TailLevel<R>& Lc = TL[l - 1];
    for (int col = 0; col < NCOL; ++col)
      for_own(L, col, [&](int a, int slot) {
        const int code = L.T.parent_code[a];
        if (code < 0) return;
        const int par = code >> 3, o = code & 7;
        R e[NP], u[NP];
        load_np_vec<NP, R>(tail_cell<NP>(cl, sm, Lc, Lc.zoff, par, colour_of(Lc, par, NCOL)), e);
        R* zu = sm + L.zoff + (size_t)slot * NP;
        load_np_vec<NP, R>(zu, u);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          R acc = 0;
#pragma unroll
          for (int j = 0; j < NP; ++j) acc += h_weight<D, R>(L.T, o, i, j) * e[j];
          u[i] += acc;
        }
        store_np_vec<NP, R>(zu, u);
      });
    cl.sync();
    for (int k = 0; k < post; ++k) {
      if (ssor)
        for (int col = 0; col < NCOL; ++col) {
          smooth(L, col, false);
          cl.sync();
        }
      for (int q = 0; q < NCOL; ++q) {
        smooth(L, NCOL - 1 - q, false);
        cl.sync();
      }
    }
  }
  {                                                // correction of the top level out
    const TailLevel<R>& L = TL[top];
    for (int col = 0; col < NCOL; ++col)
      for_own(L, col, [&](int a, int slot) {
#pragma unroll
        for (int i = 0; i < NP; ++i) z_top[(size_t)a * NP + i] = sm[L.zoff + (size_t)slot * NP + i];
      });
  }
}

// ----------------------------------------------------------------------------------------------
// The V-cycle of levels 0..top (p = 1 h-levels) in one CTA: all data of those levels in shared
// memory, phases separated by __syncthreads(); see TailCta.
// ----------------------------------------------------------------------------------------------
// Threads of the one-CTA tail: 1024 for 2D FP32 (a colour group of the 64^2 level in one pass), 512
// otherwise (register budget).
template <int D, typename R>
constexpr int tail_cta_threads() {
  return D == 2 && sizeof(R) == 4 ? 1024 : 512;
}

// Set when the tail's staging copies did not complete within kAsyncSpin polls (the tail then
// copied the data itself); tail_fault_take() reads and clears it.
__device__ int g_tail_fault;

template <int D, typename R>
__global__ void __launch_bounds__(tail_cta_threads<D, R>(), 1) k_vcycle_tail_cta(const __grid_constant__ TailCta<R> TP,
                                                                        const R* __restrict__ r_top,
                                                                        R* __restrict__ z_top,
                                                                        const double* __restrict__ coarse_inv,
                                                                        const void* __restrict__ coarse_invT) {
  extern __shared__ __align__(16) unsigned char tcta_smem[];
  R* sm = reinterpret_cast<R*>(tcta_smem);
  int* si = reinterpret_cast<int*>(tcta_smem + TP.int_base);
  constexpr int NCOL = 1 << D, NP = CD<D, 2>::NP, NT = tail_cta_threads<D, R>();
  const int top = TP.top, tid = threadIdx.x;
  // Stage the tables and inverses of every level (set-up data, staged while the kernel before
  // finishes), then, after the wait, the top level's right-hand side.  With TP.bulk, thread 0
  // moves the 16-byte multiple part of every array with bulk asynchronous copies (all sources and
  // slots are 16-byte aligned) and the threads copy the few entries past it; otherwise (or if a
  // copy does not complete in bounded time) the threads copy everything.
  __shared__ __align__(8) unsigned long long tbar[2];
  const int nr = TP.P[top].n_act * NP;
  const bool rbulk = TP.bulk && reinterpret_cast<uintptr_t>(r_top) % 16 == 0;
  // visits every staged table: f(dst, src, count, element size)
  auto tables = [&](auto&& f) {
    for (int l = 0; l <= top; ++l) {
      const LevelParams<R>& P = TP.P[l];
      f(static_cast<void*>(si + TP.noff[l]), static_cast<const void*>(P.nbr), 2 * D * P.n_act, (int)sizeof(int));
      f(static_cast<void*>(sm + TP.boff[l]), static_cast<const void*>(P.binvT), TP.n_bnd[l] * NP * NP,
        (int)sizeof(R));
      if (l >= 1) {
        const TransferParams<R>& T = TP.T[l];
        f(static_cast<void*>(si + TP.coff[l]), static_cast<const void*>(T.children), NCOL * T.n_act_c, (int)sizeof(int));
        f(static_cast<void*>(si + TP.poff[l]), static_cast<const void*>(T.parent_code), T.n_act_f, (int)sizeof(int));
      }
    }
    if (TP.cinv_off) {
      const int n0 = TP.P[0].n_act * NP;
      f(static_cast<void*>(tcta_smem + TP.cinv_off), coarse_invT, n0 * n0, 8);
    }
  };
  auto plain = [&](void* dst, const void* src, int n, int es, int from) {   // entries [from, n)
    if (es == 4)
      for (int q = from + tid; q < n; q += NT) static_cast<int*>(dst)[q] = static_cast<const int*>(src)[q];
    else
      for (int q = from + tid; q < n; q += NT) static_cast<double*>(dst)[q] = static_cast<const double*>(src)[q];
  };
  if (TP.bulk) {
    if (tid == 0) {
      mbar_init(&tbar[0], 1);
      mbar_init(&tbar[1], 1);
      mbar_fence_init();
      unsigned total = 0;
      tables([&](void*, const void*, int n, int es) { total += (unsigned)(n * es) & ~15u; });
      mbar_arrive_tx(&tbar[0], total);
      tables([&](void* dst, const void* src, int n, int es) {
        const unsigned b = (unsigned)(n * es) & ~15u;
        if (b) bulk_load(dst, src, b, &tbar[0]);
      });
    }
    tables([&](void* dst, const void* src, int n, int es) { plain(dst, src, n, es, (int)(((unsigned)(n * es) & ~15u) / es)); });
    __syncthreads();                                 // barriers initialised before anyone polls them
  } else {
    tables([&](void* dst, const void* src, int n, int es) { plain(dst, src, n, es, 0); });
  }
  pdl_wait();
  pdl_trigger();
  if (rbulk) {
    if (tid == 0) {
      mbar_arrive_tx(&tbar[1], (unsigned)(nr * sizeof(R)));
      bulk_load(sm + TP.roff[top], r_top, (unsigned)(nr * sizeof(R)), &tbar[1]);
    }
  } else {
    for (int q = tid; q < nr; q += NT) sm[TP.roff[top] + q] = r_top[q];
  }
  if (TP.bulk) {
    const bool ok = mbar_wait(&tbar[0], 0) && (!rbulk || mbar_wait(&tbar[1], 0));
    if (!__syncthreads_and(ok)) {                    // record, let the copies land, copy by hand
      if (tid == 0) {
        atomicExch(&g_tail_fault, 1);
        mbar_wait(&tbar[0], 0);
        if (rbulk) mbar_wait(&tbar[1], 0);
      }
      __syncthreads();
      tables([&](void* dst, const void* src, int n, int es) { plain(dst, src, n, es, 0); });
      for (int q = tid; q < nr; q += NT) sm[TP.roff[top] + q] = r_top[q];
    }
  }
  __syncthreads();

  auto nbr_of = [&](int l, int a, int (&nb)[2 * D]) {
#pragma unroll
    for (int s = 0; s < 2 * D; ++s) nb[s] = si[TP.noff[l] + s * TP.P[l].n_act + a];
  };
  // one colour group g (colours with g odd index bits, which share no face): all its cells at once
  auto smooth = [&](int l, int g, bool zs) {
    const LevelParams<R>& P = TP.P[l];
    // the group's colours c0 < c1 < c2 (at most three) and the running cell counts before c1, c2
    int c0 = -1, c1 = -1, c2 = -1, n0 = 0, n1 = 0, n2 = 0;
#pragma unroll
    for (int c = 0; c < NCOL; ++c)
      if (__popc(c) == g) {
        const int n = P.colour_start[c + 1] - P.colour_start[c];
        if (c0 < 0) { c0 = c; n0 = n; }
        else if (c1 < 0) { c1 = c; n1 = n; }
        else { c2 = c; n2 = n; }
      }
    R* z = sm + TP.zoff[l];
    const R* f = sm + TP.roff[l];
    for (int idx = tid; idx < n0 + n1 + n2; idx += NT) {
      int col = c0, base = 0;
      if (idx >= n0 + n1) { col = c2; base = n0 + n1; }
      else if (idx >= n0) { col = c1; base = n0; }
      const int cs = P.colour_start[col], nbnd = P.colour_nbnd[col];
      const int a = cs + idx - base;
      int nb[2 * D];
      nbr_of(l, a, nb);
      R c[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) c[i] = 0;
      add_couplings_f<D, 2, R>(P.k, col, zs, nb, [&](int n, int, R(&un)[NP]) { load_np_vec<NP, R>(z + n * NP, un); },
                               c);
      R t[NP];
      load_np_vec<NP, R>(f + a * NP, t);
#pragma unroll
      for (int i = 0; i < NP; ++i) t[i] -= P.hscale * c[i];
      const int off = a - cs;
      R y[NP];
      block_solve_at<D, 2, R>(P, off < nbnd ? sm + TP.boff[l] + (size_t)(P.bstart[col] + off) * NP * NP : nullptr,
                              t, y);
      if (P.omega != R(1)) {
        R uo[NP];
        if (zs) {
#pragma unroll
          for (int i = 0; i < NP; ++i) uo[i] = 0;
        } else {
          load_np_vec<NP, R>(z + a * NP, uo);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) y[i] = (R(1) - P.omega) * uo[i] + P.omega * y[i];
      }
      store_np_vec<NP, R>(z + a * NP, y);
    }
  };

  for (int l = top; l >= 1; --l) {                 // down: pre-smooth, residual, restrict
    const LevelParams<R>& P = TP.P[l];
    if (TP.pre == 0) {
      for (int q = tid; q < P.n_act * NP; q += NT) sm[TP.zoff[l] + q] = R(0);
      __syncthreads();
    }
    for (int k = 0; k < TP.pre; ++k) {
      for (int g = 0; g <= D; ++g) {
        smooth(l, g, k == 0);
        __syncthreads();
      }
      if (TP.ssor)
        for (int g = D; g >= 0; --g) {
          smooth(l, g, false);
          __syncthreads();
        }
    }
    const TransferParams<R>& T = TP.T[l];
    const R* z = sm + TP.zoff[l];
    const R* f = sm + TP.roff[l];
    R* rc = sm + TP.roff[l - 1];
    // one thread per child: group of NCOL adjacent lanes per coarse cell (lane o: child o), the
    // child's residual restricted in registers, then a fixed butterfly sum over the group (every
    // lane of a warp takes part: the pass count is the same for the whole block)
    for (int base = 0; base < T.n_act_c * NCOL; base += NT) {
      const int t = base + tid, cc = t / NCOL, o = t % NCOL;
      const int a = cc < T.n_act_c ? si[TP.coff[l] + o * T.n_act_c + cc] : -1;
      R out[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) out[j] = 0;
      if (a >= 0) {
        int ca = 0;
#pragma unroll
        for (int q = 1; q < NCOL; ++q)
          if (a >= P.colour_start[q]) ca = q;
        int nb[2 * D];
        nbr_of(l, a, nb);
        R v[NP], y[NP], fa[NP];
        load_np_vec<NP, R>(z + a * NP, v);
        load_np_vec<NP, R>(f + a * NP, fa);
#pragma unroll
        for (int i = 0; i < NP; ++i) y[i] = 0;
        const int off = a - P.colour_start[ca];
        add_self<D, 2, R>(P, nb, off < P.colour_nbnd[ca] ? P.bstart[ca] + off : -1, v, y);
        add_couplings_f<D, 2, R>(P.k, ca, false, nb,
                                 [&](int n, int, R(&un)[NP]) { load_np_vec<NP, R>(z + n * NP, un); }, y);
#pragma unroll
        for (int i = 0; i < NP; ++i) y[i] = fa[i] - P.hscale * y[i];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          R acc = 0;
#pragma unroll
          for (int i = 0; i < NP; ++i) acc += h_weight<D, R>(T, o, i, j) * y[i];
          out[j] = acc;
        }
      }
#pragma unroll
      for (int sh = 1; sh < NCOL; sh <<= 1)
#pragma unroll
        for (int j = 0; j < NP; ++j) out[j] += __shfl_xor_sync(0xffffffffu, out[j], sh);
      if (o == 0 && cc < T.n_act_c) store_np_vec<NP, R>(rc + cc * NP, out);
    }
    __syncthreads();
  }
  {                                                // coarse solve in FP64, one warp per row
    const int n0 = TP.P[0].n_act * NP;
    const R* r0 = sm + TP.roff[0];
    R* z0 = sm + TP.zoff[0];
    if (TP.cinv_off) {
      // the transpose staged in shared memory, one thread per row, four accumulation chains;
      // consecutive threads read consecutive entries and r0[c] is a broadcast.  FP32 tail: the
      // inverse is stored as double-float and every product is exact (two_prod) and summed in
      // double-float on the FP32 pipes (about 48 bits; the input and the result are FP32), since
      // one SM's FP64 pipe made this the tail's longest phase.  FP64 tail: FP64 throughout.
      for (int row = tid; row < n0; row += NT) {
        if constexpr (sizeof(R) == 4) {
          const dfl* aT = reinterpret_cast<const dfl*>(tcta_smem + TP.cinv_off);
          dfl acc[4] = {dfl(0.f), dfl(0.f), dfl(0.f), dfl(0.f)};
          int c = 0;
          for (; c + 4 <= n0; c += 4)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += aT[(size_t)(c + k) * n0 + row] * dfl((float)r0[c + k]);
          for (; c < n0; ++c) acc[0] += aT[(size_t)c * n0 + row] * dfl((float)r0[c]);
          const dfl sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
          z0[row] = (R)__fadd_rn(sum.hi, sum.lo);
        } else {
          const double* aT = reinterpret_cast<const double*>(tcta_smem + TP.cinv_off);
          double acc[4] = {0.0, 0.0, 0.0, 0.0};
          int c = 0;
          for (; c + 4 <= n0; c += 4)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += aT[(size_t)(c + k) * n0 + row] * (double)r0[c + k];
          for (; c < n0; ++c) acc[0] += aT[(size_t)c * n0 + row] * (double)r0[c];
          z0[row] = (R)((acc[0] + acc[1]) + (acc[2] + acc[3]));
        }
      }
    } else {                                       // from global memory, one warp per row
      const int lane = tid & 31;
      for (int row = tid >> 5; row < n0; row += NT / 32) {
        double acc = 0;
        for (int c = lane; c < n0; c += 32) acc += coarse_inv[(size_t)row * n0 + c] * (double)r0[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) z0[row] = (R)acc;
      }
    }
    __syncthreads();
  }
  for (int l = 1; l <= top; ++l) {                 // up: prolongate, post-smooth
    const LevelParams<R>& P = TP.P[l];
    const TransferParams<R>& T = TP.T[l];
    R* z = sm + TP.zoff[l];
    const R* zc = sm + TP.zoff[l - 1];
    for (int a = tid; a < P.n_act; a += NT) {
      const int code = si[TP.poff[l] + a];
      if (code < 0) continue;
      const int par = code >> 3, o = code & 7;
      R e[NP], u[NP];
      load_np_vec<NP, R>(zc + par * NP, e);
      load_np_vec<NP, R>(z + a * NP, u);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        R acc = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) acc += h_weight<D, R>(T, o, i, j) * e[j];
        u[i] += acc;
      }
      store_np_vec<NP, R>(z + a * NP, u);
    }
    __syncthreads();
    for (int k = 0; k < TP.post; ++k) {
      if (TP.ssor)
        for (int g = 0; g <= D; ++g) {
          smooth(l, g, false);
          __syncthreads();
        }
      for (int g = D; g >= 0; --g) {
        smooth(l, g, false);
        __syncthreads();
      }
    }
  }
  for (int q = tid; q < TP.P[top].n_act * NP; q += NT) z_top[q] = sm[TP.zoff[top] + q];
}

inline unsigned cdiv(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Grid of an interleaved launch (interleaved_warp) over all cells of a level: 2^dim blocks per
// chunk, as many chunks as the largest colour needs.
template <typename R>
unsigned interleaved_grid(const LevelParams<R>& P, int dim, unsigned bs) {
  const int ncol = 1 << dim;
  int longest = 0;
  for (int c = 0; c < ncol; ++c) longest = std::max(longest, P.colour_start[c + 1] - P.colour_start[c]);
  return (unsigned)ncol * cdiv((size_t)longest, bs);
}

}  // namespace

bool cell_kernels(int dim, int p) { return dim == 2 || (dim == 3 && p <= 2); }
bool cell_smoother(int dim, int p) { return dim == 2 || (dim == 3 && p == 1); }

// (p+1)^d <= 16: every thread-per-cell kernel; SBM_CELL_DISPATCH3 adds 3D p = 2 (FP32 operator).
#define SBM_CELL_DISPATCH(dim, p, MACRO)            \
  do {                                              \
    if (dim == 2 && p == 1) { MACRO(2, 2); }        \
    else if (dim == 2 && p == 2) { MACRO(2, 3); }   \
    else if (dim == 2 && p == 3) { MACRO(2, 4); }   \
    else if (dim == 3 && p == 1) { MACRO(3, 2); }   \
    else return cudaErrorInvalidValue;              \
  } while (0)
#define SBM_CELL_DISPATCH3(dim, p, MACRO)           \
  do {                                              \
    if (dim == 3 && p == 2) { MACRO(3, 3); }        \
    else SBM_CELL_DISPATCH(dim, p, MACRO);          \
  } while (0)

template <typename TI, typename R>
cudaError_t launch_apply_cell(int dim, int p, const LevelParams<R>& P, const TI* x, const R* f, R* y, int mode,
                              cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
#define SBM_AC(D, N1)                                                                           \
  {                                                                                             \
    const unsigned bs = cell_block(P.n_act), g = interleaved_grid(P, dim, bs);                 \
    if constexpr (std::is_same<R, dfl>::value && D == 2 && N1 == 3) {                           \
      if (mode == 0) SBM_PDL((k_apply_cell_occ<D, N1, TI, R, 0>), g, bs, 0, s, P, x, f, y);    \
      else SBM_PDL((k_apply_cell_occ<D, N1, TI, R, 1>), g, bs, 0, s, P, x, f, y);              \
    } else {                                                                                    \
      if (mode == 0) SBM_PDL((k_apply_cell<D, N1, TI, R, 0>), g, bs, 0, s, P, x, f, y);        \
      else SBM_PDL((k_apply_cell<D, N1, TI, R, 1>), g, bs, 0, s, P, x, f, y);                  \
    }                                                                                           \
  }
  if constexpr (std::is_same<TI, float>::value && std::is_same<R, float>::value) SBM_CELL_DISPATCH3(dim, p, SBM_AC);
  else SBM_CELL_DISPATCH(dim, p, SBM_AC);
#undef SBM_AC
  count_launches();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_smooth_cell(int dim, int p, const LevelParams<R>& P, int reverse, int zero_start, const R* f,
                               R* u, cudaStream_t s, int early, int first_group) {
  if (reverse) zero_start = 0;
  int launched = 0;
  const int ng = n_colour_groups(P, dim);
  for (int q = first_group; q < ng; ++q) {   // (the launcher in level_ops.cu chose this path for the level)
    const int g = reverse ? ng - 1 - q : q;
    const int zm = group_zero_mode(P, zero_start, q);
    const unsigned bs = cell_block(group_cells(P, dim, g));
    const SmoothSegs G = smooth_segs(P, dim, g, (int)bs);
    if (G.n == 0 || G.blk[G.n] == 0) continue;
    const int fe = launched > 0 || early;            // after the sweep's first launch f is two back
#define SBM_SC(D, N1) SBM_PDL((k_smooth_cell<D, N1, R>), G.blk[G.n], bs, 0, s, P, G, zm, f, u, fe);
    SBM_CELL_DISPATCH(dim, p, SBM_SC);
#undef SBM_SC
    count_launches();
    ++launched;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_resid_restrict_p_cell(int dim, int pf, const LevelParams<R>& P, const TransferParams<R>& T,
                                        const R* u, const R* f, R* rc, cudaStream_t s, int early,
                                        const LevelParams<R>* Pc, R* zc) {
  if (P.n_act == 0) return cudaSuccess;
  const unsigned bs = cell_block(P.n_act), g = interleaved_grid(P, dim, bs);
  const bool sm0 = Pc != nullptr && zc != nullptr;
  const LevelParams<R>& Q = sm0 ? *Pc : P;           // unused without the fused first group
#define SBM_RRPC(D, N1, NC)                                                                                \
  {                                                                                                        \
    if (sm0) SBM_PDL((k_resid_restrict_p_cell<D, N1, NC, R, true>), g, bs, 0, s, P, T, u, f, rc, early, Q, zc); \
    else SBM_PDL((k_resid_restrict_p_cell<D, N1, NC, R, false>), g, bs, 0, s, P, T, u, f, rc, early, Q, zc);    \
  }
  if (dim == 2 && pf == 2) SBM_RRPC(2, 3, 2)
  else if (dim == 2 && pf == 3) SBM_RRPC(2, 4, 3)
  else if (dim == 3 && pf == 2) SBM_RRPC(3, 3, 2)
  else return cudaErrorInvalidValue;
#undef SBM_RRPC
  count_launches();
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_resid_restrict_h_cell(int dim, const LevelParams<R>& P, const TransferParams<R>& T, const R* u,
                                        const R* f, R* rc, cudaStream_t s, int early, const LevelParams<R>* Pc,
                                        R* zc) {
  if (T.n_act_c == 0) return cudaSuccess;
  const unsigned bs = cell_block((size_t)T.n_act_c << dim), g = cdiv((size_t)T.n_act_c << dim, bs);
  const bool sm0 = Pc != nullptr && zc != nullptr;
  const LevelParams<R>& Q = sm0 ? *Pc : P;
  if (dim == 2) {
    if (sm0) SBM_PDL((k_resid_restrict_h_cell<2, R, true>), g, bs, 0, s, P, T, u, f, rc, early, Q, zc);
    else SBM_PDL((k_resid_restrict_h_cell<2, R, false>), g, bs, 0, s, P, T, u, f, rc, early, Q, zc);
  } else if (dim == 3) {
    if (sm0) SBM_PDL((k_resid_restrict_h_cell<3, R, true>), g, bs, 0, s, P, T, u, f, rc, early, Q, zc);
    else SBM_PDL((k_resid_restrict_h_cell<3, R, false>), g, bs, 0, s, P, T, u, f, rc, early, Q, zc);
  } else {
    return cudaErrorInvalidValue;
  }
  count_launches();
  return cudaGetLastError();
}

size_t tail_smem_limit() {
  static size_t limit = 0;
  if (limit == 0) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    limit = optin > 1024 ? (size_t)optin - 1024 : 0;   // room for the kernels' static shared memory
  }
  return limit;
}

template <int D, typename R>
bool tail_fits_kernel(int size, size_t smem) {
  auto kern = k_vcycle_tail<D, R>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tail_smem_limit()) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(size);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) cudaGetLastError();          // clear a refused query
  return e == cudaSuccess && nclusters >= 1;
}

bool tail_cluster_fits(int dim, int prec, int size, size_t smem) {
  if (smem > tail_smem_limit()) return false;
  if (dim == 2) return prec == 0 ? tail_fits_kernel<2, double>(size, smem) : tail_fits_kernel<2, float>(size, smem);
  return prec == 0 ? tail_fits_kernel<3, double>(size, smem) : tail_fits_kernel<3, float>(size, smem);
}

template <typename R>
cudaError_t launch_vcycle_tail(int dim, const TailLevel<R>* TL, int top, const R* r, R* z, const double* coarse_inv,
                               int pre, int post, int ssor, const TailPlan& plan, cudaStream_t s) {
  if (plan.cluster < 1) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(plan.cluster);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = plan.smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (dim == 2) e = cudaLaunchKernelEx(&cfg, k_vcycle_tail<2, R>, TL, top, r, z, coarse_inv, pre, post, ssor, plan.gather_off);
  else e = cudaLaunchKernelEx(&cfg, k_vcycle_tail<3, R>, TL, top, r, z, coarse_inv, pre, post, ssor, plan.gather_off);
  count_launches();
  return e;
}

template <typename K>
bool tail_cta_fits_kernel(K kern, size_t smem) {
  cudaFuncAttributes fa{};
  int dev = 0, optin = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  if (smem > room) return false;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

bool tail_cta_fits(int dim, int prec, size_t smem, size_t param_bytes) {
  (void)param_bytes;
  if (dim == 2) return prec == 0 ? tail_cta_fits_kernel(k_vcycle_tail_cta<2, double>, smem)
                                 : tail_cta_fits_kernel(k_vcycle_tail_cta<2, float>, smem);
  return prec == 0 ? tail_cta_fits_kernel(k_vcycle_tail_cta<3, double>, smem)
                   : tail_cta_fits_kernel(k_vcycle_tail_cta<3, float>, smem);
}

int tail_fault_take() {
  int f = 0;
  if (cudaMemcpyFromSymbol(&f, g_tail_fault, sizeof(int)) != cudaSuccess) return -1;
  if (f) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_tail_fault, &zero, sizeof(int)) != cudaSuccess) return -1;
  }
  return f;
}

template <typename R>
cudaError_t launch_vcycle_tail_cta(int dim, const TailCta<R>& TP, const R* r, R* z, const double* coarse_inv,
                                   const void* coarse_invT, size_t smem, cudaStream_t s) {
  if (dim == 2)
    SBM_PDL((k_vcycle_tail_cta<2, R>), 1, (tail_cta_threads<2, R>()), smem, s, TP, r, z, coarse_inv, coarse_invT);
  else
    SBM_PDL((k_vcycle_tail_cta<3, R>), 1, (tail_cta_threads<3, R>()), smem, s, TP, r, z, coarse_inv, coarse_invT);
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_vcycle_tail_cta<double>(int, const TailCta<double>&, const double*, double*,
                                                    const double*, const void*, size_t, cudaStream_t);
template cudaError_t launch_vcycle_tail_cta<float>(int, const TailCta<float>&, const float*, float*, const double*,
                                                   const void*, size_t, cudaStream_t);

template cudaError_t launch_vcycle_tail<double>(int, const TailLevel<double>*, int, const double*, double*,
                                                const double*, int, int, int, const TailPlan&, cudaStream_t);
template cudaError_t launch_vcycle_tail<float>(int, const TailLevel<float>*, int, const float*, float*, const double*,
                                               int, int, int, const TailPlan&, cudaStream_t);
template cudaError_t launch_apply_cell<double, double>(int, int, const LevelParams<double>&, const double*,
                                                       const double*, double*, int, cudaStream_t);
template cudaError_t launch_apply_cell<float, float>(int, int, const LevelParams<float>&, const float*, const float*,
                                                     float*, int, cudaStream_t);
template cudaError_t launch_apply_cell<float, double>(int, int, const LevelParams<double>&, const float*,
                                                      const double*, double*, int, cudaStream_t);
template cudaError_t launch_apply_cell<float, dfl>(int, int, const LevelParams<dfl>&, const float*, const dfl*,
                                                   dfl*, int, cudaStream_t);
template cudaError_t launch_smooth_cell<double>(int, int, const LevelParams<double>&, int, int, const double*,
                                                double*, cudaStream_t, int, int);
template cudaError_t launch_smooth_cell<float>(int, int, const LevelParams<float>&, int, int, const float*, float*,
                                               cudaStream_t, int, int);
template cudaError_t launch_resid_restrict_p_cell<double>(int, int, const LevelParams<double>&,
                                                          const TransferParams<double>&, const double*, const double*,
                                                          double*, cudaStream_t, int, const LevelParams<double>*,
                                                          double*);
template cudaError_t launch_resid_restrict_p_cell<float>(int, int, const LevelParams<float>&,
                                                         const TransferParams<float>&, const float*, const float*,
                                                         float*, cudaStream_t, int, const LevelParams<float>*, float*);
template cudaError_t launch_resid_restrict_h_cell<double>(int, const LevelParams<double>&,
                                                          const TransferParams<double>&, const double*, const double*,
                                                          double*, cudaStream_t, int, const LevelParams<double>*,
                                                          double*);
template cudaError_t launch_resid_restrict_h_cell<float>(int, const LevelParams<float>&, const TransferParams<float>&,
                                                         const float*, const float*, float*, cudaStream_t, int,
                                                         const LevelParams<float>*, float*);

}  // namespace sbm
