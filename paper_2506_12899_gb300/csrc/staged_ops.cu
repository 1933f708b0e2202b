// Staged thread-per-cell kernels: the operator (Eqs. 7, 10, 11) and one colour group of the block
// Gauss-Seidel smoother (Eqs. 14, 16) for cells of (p+1)^d <= 27 values (2D p = 1..3, 3D p = 1, 2).
//
// The thread-per-cell kernels of cell_ops.cu let every thread fetch its own cell and its 2d face
// neighbours: one warp-wide load instruction then touches 32 different cells, (p+1)^d * 4 bytes
// apart, and the L1 request stream, not DRAM, limits them (22-25 sectors per request at 3D p = 1).
// Here a CTA of CB threads takes CB consecutive cells of the compact order and first copies, with
// all its threads, the values of those cells and of their neighbours into shared memory: consecutive
// threads copy consecutive values of a cell, and the neighbours of consecutive cells are mostly
// consecutive cells of another colour, so the copies are coalesced.  The copies are asynchronous
// (cp.async, LDGSTS), all issued before the first wait.  Rows are stored with an odd stride, so the
// thread-per-cell reads that follow are free of bank conflicts.  Each thread then runs the same
// per-cell arithmetic as the cell_ops.cu kernels on its registers; its results replace its own row,
// and the CTA writes the rows back with coalesced stores.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ops.h"

namespace sbm {
namespace {

#include "cell_core.cuh"

// Row stride (in elements) of a staged cell: n_p, made odd so that threads reading their rows at
// the same offset hit 32 distinct banks.
template <int NP>
constexpr int srow() {
  return (NP & 1) ? NP : NP + 1;
}

// Asynchronous 4- or 8-byte copy global -> shared; src_bytes 0 writes zeros (no global access).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Copies the values of the m cells ids[0..m) (id < 0: zeros) into rows dst + j * ST.
template <int NP, int ST, int CB, typename T>
__device__ __forceinline__ void stage_cells(const T* __restrict__ x, const int* ids, int m, T* dst) {
  for (int e = threadIdx.x; e < m * NP; e += CB) {
    const int j = e / NP, k = e - j * NP;
    const int c = ids[j];
    cp_async_elem(dst + j * ST + k, x + (size_t)(c < 0 ? 0 : c) * NP + k, c >= 0);
  }
}

// Copies the values of the m consecutive cells a0 .. a0+m-1 into rows dst + j * ST.
template <int NP, int ST, int CB, typename T>
__device__ __forceinline__ void stage_range(const T* __restrict__ x, int a0, int m, T* dst) {
  const T* src = x + (size_t)a0 * NP;
  for (int e = threadIdx.x; e < m * NP; e += CB) {
    const int j = e / NP, k = e - j * NP;
    cp_async_elem(dst + j * ST + k, src + e, true);
  }
}

// Writes rows src + j * ST of the m consecutive cells a0 .. back to y (MODE 1: y = f - row).
template <int NP, int ST, int CB, int MODE, typename T>
__device__ __forceinline__ void store_range(T* __restrict__ y, const T* __restrict__ f, int a0, int m, const T* src) {
  T* dst = y + (size_t)a0 * NP;
  for (int e = threadIdx.x; e < m * NP; e += CB) {
    const int j = e / NP, k = e - j * NP;
    const T v = src[j * ST + k];
    dst[e] = MODE == 1 ? f[(size_t)a0 * NP + e] - v : v;
  }
}

// y += sum over the interior faces of A_KN u_N (Eq. 10 couplings) with the neighbour on slot s
// read from its staged row rows[s] (valid where nb[s] >= 0).
template <int D, int N1, typename R, typename T>
__device__ __forceinline__ void add_couplings_rows(const LevelConsts<R>& C, const int (&nb)[2 * D],
                                                   const T* const (&rows)[2 * D], R (&y)[CD<D, N1>::NP]) {
  constexpr int NQ = CD<D, N1>::NQ;
#pragma unroll
  for (int s = 0; s < 2 * D; ++s) {
    if (nb[s] < 0) continue;
    const int dir = s >> 1;
    const T* un = rows[s];
    const R* B = (s & 1) ? C.Bmp : C.Bpm;
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
      const R wt = line_weight<D, N1, R>(C, t);
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        R acc = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) acc += B[i * N1 + j] * (R)un[dof<D, N1>(dir, j, t)];
        y[dof<D, N1>(dir, i, t)] += wt * acc;
      }
    }
  }
}

// Dynamic shared memory of a staged launch: `sets` row sets of CB cells (own values or f, the 2d
// neighbours, u_K for the smoother) and the neighbour table.
template <int D, int N1, int CB, int sets>
constexpr size_t staged_smem() {
  return (size_t)sets * CB * srow<CD<D, N1>::NP>() * sizeof(float) + (size_t)2 * D * CB * sizeof(int);
}

// y = A x (MODE 0) or y = f - A x (MODE 1), FP32, CB consecutive cells per CTA.
template <int D, int N1, int MODE, int CB>
__global__ void __launch_bounds__(CB) k_apply_staged(const __grid_constant__ LevelParams<float> P,
                                                     const float* __restrict__ x, const float* __restrict__ f,
                                                     float* __restrict__ y) {
  constexpr int NP = CD<D, N1>::NP, NS = 2 * D, ST = srow<NP>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sX = reinterpret_cast<float*>(smem_raw);                      // [1 + NS][CB][ST]
  int* sNb = reinterpret_cast<int*>(sX + (size_t)(1 + NS) * CB * ST);  // [NS][CB]
  const int a0 = blockIdx.x * CB;
  const int m = min(CB, P.n_act - a0);
  const int a = a0 + (int)threadIdx.x;
  const bool own = (int)threadIdx.x < m;
  int nb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) nb[s] = -1;
  if (own) load_nbr<D, float>(P, a, nb);                               // set-up data: before the wait
#pragma unroll
  for (int s = 0; s < NS; ++s) sNb[s * CB + threadIdx.x] = nb[s];
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  stage_range<NP, ST, CB>(x, a0, m, sX);
#pragma unroll
  for (int s = 0; s < NS; ++s) stage_cells<NP, ST, CB>(x, sNb + s * CB, m, sX + (size_t)(1 + s) * CB * ST);
  cp_async_wait_all();
  __syncthreads();
  float* row = sX + threadIdx.x * ST;
  if (own) {
    float v[NP], r[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      v[i] = row[i];
      r[i] = 0.f;
    }
    add_self<D, N1, float>(P, nb, boundary_index(P, a, 1 << D), v, r);
    const float* rows[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) rows[s] = sX + ((size_t)(1 + s) * CB + threadIdx.x) * ST;
    add_couplings_rows<D, N1, float>(P.k, nb, rows, r);
#pragma unroll
    for (int i = 0; i < NP; ++i) row[i] = P.hscale * r[i];             // own row: read by this thread only
  }
  __syncthreads();
  store_range<NP, ST, CB, MODE>(y, f, a0, m, sX);
}

// One colour group of the block Gauss-Seidel sweep (Eq. 16), FP32, CB consecutive cells of one
// segment per CTA:  t_K = f_K - sum_N A_KN u_N over interior faces (the SBM terms lie in A_KK),
// u_K <- (1 - omega) u_K + omega A_KK^-1 t_K.  zero_start: u is zero on entry (forward sweep from
// zero), so neighbours of colours not yet visited and u_K itself are not read.
template <int D, int N1, int CB>
__global__ void __launch_bounds__(CB) k_smooth_staged(const __grid_constant__ LevelParams<float> P,
                                                      const __grid_constant__ SmoothSegs G, int zero_start,
                                                      const float* __restrict__ f, float* __restrict__ u,
                                                      int early) {
  constexpr int NP = CD<D, N1>::NP, NS = 2 * D, ST = srow<NP>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sX = reinterpret_cast<float*>(smem_raw);                      // [2 + NS][CB][ST]: f, neighbours, u_K
  int* sNb = reinterpret_cast<int*>(sX + (size_t)(2 + NS) * CB * ST);  // [NS][CB]
  float* sU = sX + (size_t)(1 + NS) * CB * ST;
  int sg = 0;
#pragma unroll
  for (int k = 1; k < SmoothSegs::kMax; ++k)
    if (k < G.n && (int)blockIdx.x >= G.blk[k]) sg = k;
  const int col = G.col[sg];
  const int a0 = G.first[sg] + ((int)blockIdx.x - G.blk[sg]) * CB;
  const int m = min(CB, G.last[sg] - a0);
  const int a = a0 + (int)threadIdx.x;
  const bool own = (int)threadIdx.x < m;
  const bool isB = a0 < G.cs[sg] + G.nbnd[sg];                         // segments are all-boundary or all-interior
  int nb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) nb[s] = -1;
  if (own) load_nbr<D, float>(P, a, nb);                               // set-up data: before the wait
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const bool later = (zero_start == kZeroLater && (col ^ (1 << (s >> 1))) > col) || zero_start == kZeroAll;
    sNb[s * CB + threadIdx.x] = later ? -1 : nb[s];
  }
  if (early) {                                 // f written two or more launches back: L2-only loads
    for (int e = threadIdx.x; e < m * NP; e += CB) {
      const int j = e / NP, k = e - j * NP;
      sX[j * ST + k] = __ldcg(f + (size_t)a0 * NP + e);
    }
  }
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  if (!early) stage_range<NP, ST, CB>(f, a0, m, sX);
#pragma unroll
  for (int s = 0; s < NS; ++s) stage_cells<NP, ST, CB>(u, sNb + s * CB, m, sX + (size_t)(1 + s) * CB * ST);
  const bool relax = P.omega != 1.f && !zero_start;
  if (relax) stage_range<NP, ST, CB>(u, a0, m, sU);
  cp_async_wait_all();
  __syncthreads();
  float* row = sX + threadIdx.x * ST;
  if (own) {
    float t[NP], c[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      t[i] = row[i];
      c[i] = 0.f;
    }
    int nbs[NS];
    const float* rows[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      nbs[s] = sNb[s * CB + threadIdx.x];
      rows[s] = sX + ((size_t)(1 + s) * CB + threadIdx.x) * ST;
    }
    add_couplings_rows<D, N1, float>(P.k, nbs, rows, c);
#pragma unroll
    for (int i = 0; i < NP; ++i) t[i] -= P.hscale * c[i];
    float yv[NP];
    block_solve<D, N1, float>(P, isB ? G.b0[sg] + (a - G.cs[sg]) : -1, t, yv);
    if (P.omega != 1.f) {
      const float* urow = sU + threadIdx.x * ST;
#pragma unroll
      for (int i = 0; i < NP; ++i) yv[i] = (1.f - P.omega) * (relax ? urow[i] : 0.f) + P.omega * yv[i];
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) row[i] = yv[i];
  }
  __syncthreads();
  store_range<NP, ST, CB, 0>(u, (const float*)nullptr, a0, m, sX);
}

inline unsigned cdiv_s(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

template <typename K>
cudaError_t allow_smem(K kern, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool staged_kernels(int dim, int p) { return dim == 2 || (dim == 3 && p <= 2); }

#define SBM_STAGED_DISPATCH(dim, p, MACRO)          \
  do {                                              \
    if (dim == 2 && p == 1) { MACRO(2, 2); }        \
    else if (dim == 2 && p == 2) { MACRO(2, 3); }   \
    else if (dim == 2 && p == 3) { MACRO(2, 4); }   \
    else if (dim == 3 && p == 1) { MACRO(3, 2); }   \
    else if (dim == 3 && p == 2) { MACRO(3, 3); }   \
    else return cudaErrorInvalidValue;              \
  } while (0)

// Cells per CTA: 32 for launches of up to 32 warps per SM (short launches spread over every SM),
// else 128 (64 for 3D p = 2, whose CTA stages 48 KB).
template <int D, int N1, int MODE, int CB>
cudaError_t launch_apply_staged_cb(const LevelParams<float>& P, const float* x, const float* f, float* y,
                                   cudaStream_t s) {
  constexpr size_t sm = staged_smem<D, N1, CB, 1 + 2 * D>();
  auto kern = k_apply_staged<D, N1, MODE, CB>;
  cudaError_t e = allow_smem(kern, sm);
  if (e != cudaSuccess) return e;
  SBM_PDL(kern, cdiv_s(P.n_act, CB), CB, sm, s, P, x, f, y);
  return cudaSuccess;
}

cudaError_t launch_apply_staged(int dim, int p, const LevelParams<float>& P, const float* x, const float* f,
                                float* y, int mode, cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
  const bool small = (size_t)P.n_act <= (size_t)152 * 32 * 32;
  cudaError_t e = cudaSuccess;
#define SBM_AS(D, N1)                                                                              \
  {                                                                                                \
    constexpr int CBL = CD<D, N1>::NP > 16 ? 64 : 128;                                             \
    if (mode == 0) e = small ? launch_apply_staged_cb<D, N1, 0, 32>(P, x, f, y, s)                 \
                             : launch_apply_staged_cb<D, N1, 0, CBL>(P, x, f, y, s);               \
    else e = small ? launch_apply_staged_cb<D, N1, 1, 32>(P, x, f, y, s)                           \
                   : launch_apply_staged_cb<D, N1, 1, CBL>(P, x, f, y, s);                         \
  }
  SBM_STAGED_DISPATCH(dim, p, SBM_AS);
#undef SBM_AS
  if (e != cudaSuccess) return e;
  count_launches();
  return cudaGetLastError();
}

template <int D, int N1, int CB>
cudaError_t launch_smooth_staged_cb(const LevelParams<float>& P, const SmoothSegs& G, int zero_start,
                                    const float* f, float* u, int early, cudaStream_t s) {
  constexpr size_t sm = staged_smem<D, N1, CB, 2 + 2 * D>();
  auto kern = k_smooth_staged<D, N1, CB>;
  cudaError_t e = allow_smem(kern, sm);
  if (e != cudaSuccess) return e;
  SBM_PDL(kern, G.blk[G.n], CB, sm, s, P, G, zero_start, f, u, early);
  return cudaSuccess;
}

cudaError_t launch_smooth_staged(int dim, int p, const LevelParams<float>& P, int reverse, int zero_start,
                                 const float* f, float* u, cudaStream_t s, int early) {
  if (reverse) zero_start = 0;
  int launched = 0;
  const int ng = n_colour_groups(P, dim);
  for (int q = 0; q < ng; ++q) {
    const int g = reverse ? ng - 1 - q : q;
    const int zm = group_zero_mode(P, zero_start, q);
    const int cells = group_cells(P, dim, g);
    const bool small = (size_t)cells <= (size_t)152 * 32 * 32;
    const int fe = launched > 0 || early;            // after the sweep's first launch f is two back
    cudaError_t e = cudaSuccess;
    bool any = false;
#define SBM_SS(D, N1)                                                                              \
  {                                                                                                \
    constexpr int CBL = CD<D, N1>::NP > 16 ? 64 : 128;                                             \
    const int cb = small ? 32 : CBL;                                                               \
    const SmoothSegs G = smooth_segs(P, dim, g, cb);                                               \
    if (G.n > 0 && G.blk[G.n] > 0) {                                                               \
      any = true;                                                                                  \
      e = small ? launch_smooth_staged_cb<D, N1, 32>(P, G, zm, f, u, fe, s)                        \
                : launch_smooth_staged_cb<D, N1, CBL>(P, G, zm, f, u, fe, s);                      \
    }                                                                                              \
  }
    SBM_STAGED_DISPATCH(dim, p, SBM_SS);
#undef SBM_SS
    if (e != cudaSuccess) return e;
    if (any) {
      count_launches();
      ++launched;
    }
  }
  return cudaGetLastError();
}

}  // namespace sbm
