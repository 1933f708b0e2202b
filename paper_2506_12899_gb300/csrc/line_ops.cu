// Thread-per-line kernels for 3D cells of degree p = 2 and 3 (Eqs. 7, 10, 11, 14, 16, 18).
//
// A 3D cell holds N1^3 values (N1 = p + 1, dof i + N1 j + N1^2 k).  The thread-per-DoF kernels of
// level_ops.cu give every value its own thread and spend hundreds of instructions per value on
// index arithmetic and scalar shared-memory reads; one thread per cell needs 100-200 registers.
// Here a cell's N1^2 lines along x take N1^2 consecutive lanes of one warp (16 at p = 3, two cells
// per warp; 9 at p = 2, three cells per warp and lanes 27-31 idle); lane l owns the line
// (j, k) = (l mod N1, l / N1) and computes at its N1 values i = 0..N1-1:
//   - the block copies its cells and their 6 face neighbours into shared memory (a cell's values
//     are contiguous, so the copies are coalesced: 16-byte words at p = 3, 4-byte at p = 2), every
//     line in its own 16-byte word;
//   - x terms (volume, both x faces): the thread's own line, N1 x N1 matrices;
//   - y terms: plane k of the cell and of its y neighbours (the lines through (i, ., k));
//   - z terms: the (i, j, .) rows of the cell and of its z neighbours;
// the 1D matrices come from the kernel's parameter block.  Surrogate faces (Eq. 7) follow in three
// barrier-separated phases per face slot: the cell's lanes take the N1^2 points of the face (trace
// and normal derivative, then the extended value), then every lane adds the face terms at its own
// values.  The smoother's fast diagonalisation contracts x on the thread's line and y, z after
// exchanges through shared memory; a cell's lanes lie in one warp, so those exchanges need only
// warp barriers.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ops.h"

namespace sbm {
namespace {

#include "cell_core.cuh"

constexpr int kLineThreads = 128;                // 4 warps per block

// A cell's lanes: LPC consecutive lanes of one warp (16 at p = 3, 9 at p = 2, so that a warp holds
// CPW = 2 or 3 cells and a cell's exchanges need only warp barriers; at p = 2 lanes 27-31 idle).
template <int N1>
struct LD {
  static constexpr int NP = N1 * N1 * N1;        // values of a cell
  static constexpr int NL = N1 * N1;             // lines (and face points) of a cell
  static constexpr int ST = N1 == 4 ? 68 : 40;   // staged row of a cell (floats, 16-byte multiple; banks)
  static constexpr int LPC = N1 == 4 ? 16 : 9;   // lanes per cell
  static constexpr int CPW = 32 / LPC;           // cells per warp
  static constexpr int CPB = 4 * CPW;            // cells per block
};

// Staged rows keep every line of a cell in its own 16-byte word: value (i, j, k) at
// i + 4 (j + N1 k), so that a line, and a row of a plane, is one 16-byte shared-memory access (at
// p = 2 the fourth word of a line is padding); sp(q) maps the dense index q = i + N1 j + N1^2 k.
template <int N1>
__host__ __device__ constexpr int sp(int q) {
  return (q % N1) + 4 * (q / N1);
}

// The calling thread's cell slot c in the block and lane l within the cell; false for the idle
// lanes past the warp's last cell (they take slot and lane of the warp's first line and must
// not write).
template <int N1>
__device__ __forceinline__ bool line_lane(int& c, int& l) {
  constexpr int LPC = LD<N1>::LPC, CPW = LD<N1>::CPW;
  const int w = (int)threadIdx.x >> 5, L = (int)threadIdx.x & 31;
  const bool ok = L < CPW * LPC;
  c = w * CPW + (ok ? L / LPC : 0);
  l = ok ? L % LPC : 0;
  return ok;
}

// acc += a b and a b in the arithmetic R: FP32, or double-float (the Arnoldi operator's).
__device__ __forceinline__ void madd(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void madd(dfl& acc, dfl a, dfl b) { acc += a * b; }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ dfl mul(dfl a, dfl b) { return dfl(a * b); }

// One staged line (a 16-byte word, see sp).
template <int N1>
__device__ __forceinline__ void lds_line(const float* p, float (&v)[N1]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  if constexpr (N1 == 4) v[3] = q.w;
}
template <int N1>
__device__ __forceinline__ void sts_line(float* p, const float (&v)[N1]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], N1 == 4 ? v[3] : 0.f);
}

// The thread's line of a global FP32 vector (at offset o); CG: L2-only loads (data written two or
// more launches back, read before the dependency wait).
template <int N1, bool CG>
__device__ __forceinline__ void ldg_line(const float* __restrict__ x, size_t o, float (&v)[N1]) {
  if constexpr (N1 == 4) {
    const float4 q = CG ? __ldcg(reinterpret_cast<const float4*>(x + o)) : *reinterpret_cast<const float4*>(x + o);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = CG ? __ldcg(x + o + i) : x[o + i];
  }
}
template <int N1>
__device__ __forceinline__ void stg_line(float* __restrict__ y, size_t o, const float (&v)[N1]) {
  if constexpr (N1 == 4) {
    *reinterpret_cast<float4*>(y + o) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < N1; ++i) y[o + i] = v[i];
  }
}
template <int N1>
__device__ __forceinline__ void stg_line(dfl* __restrict__ y, size_t o, const dfl (&v)[N1]) {
  if constexpr (N1 == 4) {
    reinterpret_cast<float4*>(y + o)[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
    reinterpret_cast<float4*>(y + o)[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
  } else {
#pragma unroll
    for (int i = 0; i < N1; ++i) reinterpret_cast<float2*>(y + o)[i] = make_float2(v[i].hi, v[i].lo);
  }
}

// Copies the values of cell a (row X0, unless null) and of its face neighbours nb (rows N[s])
// into shared memory; lane l of the cell's LPC copies its share of every row.
template <int N1>
__device__ __forceinline__ void line_stage(const float* __restrict__ x, int a, const int (&nb)[6], int l, float* X0,
                                           float (*N)[LD<N1>::ST]) {
  constexpr int NP = LD<N1>::NP;
  if constexpr (N1 == 4) {
    if (X0) reinterpret_cast<float4*>(X0)[l] = reinterpret_cast<const float4*>(x + (size_t)a * NP)[l];
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (nb[s] >= 0) reinterpret_cast<float4*>(N[s])[l] = reinterpret_cast<const float4*>(x + (size_t)nb[s] * NP)[l];
  } else {
#pragma unroll
    for (int w = l; w < NP; w += LD<N1>::LPC) {
      if (X0) X0[sp<N1>(w)] = x[(size_t)a * NP + w];
#pragma unroll
      for (int s = 0; s < 6; ++s)
        if (nb[s] >= 0) N[s][sp<N1>(w)] = x[(size_t)nb[s] * NP + w];
    }
  }
}

// The volume and interior-face terms (Eq. 10, reference scaling) at the N1 values (i, j, k) of the
// thread's line, from the cell's staged row own and the staged rows N[s] of its neighbours (slot
// s = 2 dir + side, valid where nb[s] >= 0).  SELF: with the volume and the cell's own face terms
// (the operator); without them only the couplings to the neighbours (the smoother's right-hand
// side; own is not read).
template <bool SELF, int N1, typename R>
__device__ __forceinline__ void line_interior(const LevelConsts<R>& C, const float* own,
                                              const float (*N)[LD<N1>::ST], const int (&nb)[6], int j, int k,
                                              R (&acc)[N1]) {
  {                                                // x: the thread's own line (j, k)
    R s[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) s[i] = R(0.f);
#pragma unroll
    for (int q = SELF ? -1 : 0; q < 2; ++q) {      // q = -1: the cell itself
      if (q >= 0 && nb[q] < 0) continue;
      const R* M = q < 0 ? C.L[(nb[0] >= 0) + 2 * (nb[1] >= 0)] : (q == 0 ? C.Bpm : C.Bmp);
      float v[N1];
      lds_line<N1>((q < 0 ? own : N[q]) + 4 * (j + N1 * k), v);
#pragma unroll
      for (int i = 0; i < N1; ++i)
#pragma unroll
        for (int m = 0; m < N1; ++m) madd(s[i], M[N1 * i + m], R(v[m]));
    }
    const R wt = mul(C.w[j], C.w[k]);
#pragma unroll
    for (int i = 0; i < N1; ++i) madd(acc[i], wt, s[i]);
  }
#pragma unroll
  for (int dir = 1; dir < 3; ++dir) {              // y: lines (i, ., k), row j; z: lines (i, j, .), row k
    const int row = dir == 1 ? j : k;
    R s[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) s[i] = R(0.f);
#pragma unroll
    for (int q = SELF ? -1 : 0; q < 2; ++q) {
      if (q >= 0 && nb[2 * dir + q] < 0) continue;
      const R* M = q < 0 ? C.L[(nb[2 * dir] >= 0) + 2 * (nb[2 * dir + 1] >= 0)] : (q == 0 ? C.Bpm : C.Bmp);
      const float* xs = q < 0 ? own : N[2 * dir + q];
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        float v[N1];
        lds_line<N1>(xs + 4 * (dir == 1 ? m + N1 * k : j + N1 * m), v);
        const R cm = M[N1 * row + m];
#pragma unroll
        for (int i = 0; i < N1; ++i) madd(s[i], cm, R(v[i]));
      }
    }
    const R wo = C.w[dir == 1 ? k : j];
#pragma unroll
    for (int i = 0; i < N1; ++i) madd(acc[i], mul(C.w[i], wo), s[i]);
  }
}

// Surrogate-face terms (Eq. 7) of the block's boundary cells at the calling thread's values,
// reference scaling; every thread of the block calls it (barriers).  own: the cell's staged row;
// line: whether the thread owns a line.
template <int N1, typename R>
__device__ __forceinline__ void line_sbm_terms(const LevelParams<R>& P, const float* own, R (*sU)[16], R (*sG)[16],
                                               R (*sE)[16], int c, int l, bool line, int j, int k, int bidx,
                                               const int (&nb)[6], R (&acc)[N1]) {
  constexpr int NQ = N1 * N1;
  const LevelConsts<R>& C = P.k;
#pragma unroll 1
  for (int slot = 0; slot < 6; ++slot) {
    const bool sf = bidx >= 0 && nb[slot] < 0;
    if (!__syncthreads_or(sf)) continue;
    const int dir = slot >> 1, side = slot & 1;
    const R* es = side ? C.e1 : C.e0;
    const R* ds = side ? C.d1 : C.d0;
    const R* dh = sf ? P.dhat + ((size_t)bidx * 6 + slot) * 3 * NQ : nullptr;
    const int t = l;                             // this thread's face point (t < NQ)
    if (sf && t < NQ) {                          // trace and normal derivative at face point t
      R su = R(0.f), sd = R(0.f);
#pragma unroll
      for (int kn = 0; kn < N1; ++kn) {
        const R v = R(own[sp<N1>(dof<3, N1>(dir, kn, t))]);
        madd(su, es[kn], v);
        madd(sd, ds[kn], v);
      }
      sU[c][t] = su;
      sG[c][t] = sd;
    }
    __syncthreads();
    if (sf && t < NQ) {                          // extended value at face point t
      R E;
      if (P.extension == 0) {
        E = sU[c][t];
        madd(E, dh[dir * NQ + t], sG[c][t]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {            // tangential derivatives of the trace
          const int m = tang_dim<3>(dir, q);
          const int stride = q == 0 ? 1 : N1;
          const int tm = (t / stride) % N1;
          R g = R(0.f);
#pragma unroll
          for (int r = 0; r < N1; ++r) madd(g, C.Dm[tm * N1 + r], sU[c][t + (r - tm) * stride]);
          madd(E, dh[m * NQ + t], g);
        }
      } else {                                   // cell polynomial at x~ + d
        R lv[3][N1];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          R xi;
          if (m == dir) {
            xi = R((float)side);
          } else {
            const int q = m < dir ? m : m - 1;
            xi = C.x[(t / (q == 0 ? 1 : N1)) % N1];
          }
          const R yv = xi + dh[m * NQ + t];
#pragma unroll
          for (int kk = 0; kk < N1; ++kk) {
            R val = C.inv_denom[kk];
#pragma unroll
            for (int jj = 0; jj < N1; ++jj)
              if (jj != kk) val = mul(val, yv - C.x[jj]);
            lv[m][kk] = val;
          }
        }
        E = R(0.f);
#pragma unroll
        for (int q = 0; q < N1 * NQ; ++q)
          madd(E, mul(mul(lv[0][q % N1], lv[1][(q / N1) % N1]), lv[2][q / NQ]), R(own[sp<N1>(q)]));
      }
      sE[c][t] = E;
    }
    __syncthreads();
    if (sf && line) {                            // terms at the thread's values (i, j, k)
      const R sg = R(side ? 1.f : -1.f);
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        int tp, kn;                              // face point and normal position of value (i, j, k)
        if (dir == 0) {
          tp = j + N1 * k;
          kn = i;
        } else if (dir == 1) {
          tp = i + N1 * k;
          kn = j;
        } else {
          tp = i + N1 * j;
          kn = k;
        }
        const R wt = mul(C.w[tp % N1], C.w[tp / N1]);
        const R E = sE[c][tp], G = sG[c][tp];
        R term = mul(es[kn], mul(P.sigG, E) - mul(sg, G));
        term = term - mul(mul(P.alpha, sg), mul(ds[kn], E));
        madd(acc[i], wt, term);
      }
    }
    __syncthreads();
  }
}

// y = A x (MODE 0) or y = f - A x (MODE 1) for a 3D level of degree N1 - 1; x FP32, arithmetic
// and y in R (FP32, or double-float for the Arnoldi operator).
template <int N1, typename R, int MODE>
__global__ void __launch_bounds__(kLineThreads) k_apply_line(const __grid_constant__ LevelParams<R> P,
                                                             const float* __restrict__ x, const R* __restrict__ f,
                                                             R* __restrict__ y) {
  constexpr int NP = LD<N1>::NP, NL = LD<N1>::NL, ST = LD<N1>::ST, CPB = LD<N1>::CPB;
  __shared__ __align__(16) float sX[CPB][7][ST];
  __shared__ R sU[CPB][16], sG[CPB][16], sE[CPB][16];
  int c, l;
  const bool lane_ok = line_lane<N1>(c, l);
  const int j = l % N1, k = l / N1;
  const int a = blockIdx.x * CPB + c;
  const bool valid = lane_ok && a < P.n_act;
  const bool line = valid && l < NL;
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;   // set-up data
  pdl_wait();
  pdl_trigger();
  if (valid) line_stage<N1>(x, a, nb, l, sX[c][0], sX[c] + 1);
  __syncthreads();
  R acc[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) acc[i] = R(0.f);
  if (line) line_interior<true, N1, R>(P.k, sX[c][0], sX[c] + 1, nb, j, k, acc);
  const int bidx = valid ? boundary_index(P, a, 8) : -1;
  if (__syncthreads_or(bidx >= 0))
    line_sbm_terms<N1, R>(P, sX[c][0], sU, sG, sE, c, l, line, j, k, bidx, nb, acc);
  if (line) {
    const size_t o = (size_t)a * NP + N1 * j + N1 * N1 * k;
    R out[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) out[i] = mul(P.hscale, acc[i]);
    if (MODE == 1) {
#pragma unroll
      for (int i = 0; i < N1; ++i) out[i] = f[o + i] - out[i];
    }
    stg_line<N1>(y, o, out);
  }
}

// Residual and p-restriction fused (Eqs. 11, 18) from a 3D p = 3 level to p = 2 on the same mesh,
// FP32: r = f - A u at the thread's four values as in k_apply_line, then
// rc_K = (Pp^T (x) Pp^T (x) Pp^T) r_K by three one-direction contractions (4 -> 3 values), the x
// one on the thread's line, the y and z ones after warp-level exchanges through shared memory.
__global__ void __launch_bounds__(kLineThreads) k_resid_restrict_line(const __grid_constant__ LevelParams<float> P,
                                                                      const __grid_constant__ TransferParams<float> T,
                                                                      const float* __restrict__ u,
                                                                      const float* __restrict__ f,
                                                                      float* __restrict__ rc, int early) {
  constexpr int CPB = LD<4>::CPB;
  __shared__ __align__(16) float sX[CPB][7][LD<4>::ST];
  __shared__ float sU[CPB][16], sG[CPB][16], sE[CPB][16];
  __shared__ float sR1[CPB][48], sR2[CPB][36];
  const int c = threadIdx.x >> 4, l = threadIdx.x & 15, j = l & 3, k = l >> 2;
  const int a = blockIdx.x * CPB + c;
  const bool valid = a < P.n_act;
  const size_t o = (size_t)a * 64 + 4 * j + 16 * k;
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;   // set-up data
  float fv[4] = {0.f, 0.f, 0.f, 0.f};
  if (valid && early) ldg_line<4, true>(f, o, fv);   // f written two or more launches back
  pdl_wait();
  pdl_trigger();
  if (valid) {
    if (!early) ldg_line<4, false>(f, o, fv);
    line_stage<4>(u, a, nb, l, sX[c][0], sX[c] + 1);
  }
  __syncthreads();
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (valid) line_interior<true, 4, float>(P.k, sX[c][0], sX[c] + 1, nb, j, k, acc);
  const int bidx = valid ? boundary_index(P, a, 8) : -1;
  if (__syncthreads_or(bidx >= 0)) line_sbm_terms<4, float>(P, sX[c][0], sU, sG, sE, c, l, valid, j, k, bidx, nb, acc);
  float r[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) r[i] = fv[i] - P.hscale * acc[i];
#pragma unroll
  for (int j0 = 0; j0 < 3; ++j0) {                 // x: (j0, j, k) = sum_i Pp[i][j0] r(i, j, k)
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) v = fmaf(T.Pp[i * 3 + j0], r[i], v);
    sR1[c][j0 + 3 * j + 12 * k] = v;
  }
  __syncwarp();
  if (j < 3) {                                     // y: (j0, j1 = j, k) = sum_q Pp[q][j1] (j0, q, k)
#pragma unroll
    for (int j0 = 0; j0 < 3; ++j0) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) v = fmaf(T.Pp[q * 3 + j], sR1[c][j0 + 3 * q + 12 * k], v);
      sR2[c][j0 + 3 * j + 9 * k] = v;
    }
  }
  __syncwarp();
  if (valid && j < 3 && k < 3) {                   // z: (j0, j1 = j, j2 = k) = sum_q Pp[q][j2] (j0, j1, q)
#pragma unroll
    for (int j0 = 0; j0 < 3; ++j0) {
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) v = fmaf(T.Pp[q * 3 + k], sR2[c][j0 + 3 * j + 9 * q], v);
      rc[(size_t)a * 27 + j0 + 3 * j + 9 * k] = v;
    }
  }
}

// One colour group of the block Gauss-Seidel sweep (Eq. 16) on a 3D level of degree N1 - 1, FP32,
// 8 cells of one segment per block:
//   t_K = f_K - sum over interior faces of A_KN u_N (the SBM terms lie in A_KK),
//   u_K <- (1 - omega) u_K + omega A_KK^-1 t_K.
// The couplings take the same line, plane and row reads as the operator.  Boundary cells apply
// their dense inverse (each thread its N1 rows, t from shared memory); interior cells the fast
// diagonalisation (S^T)^(x3), 1 / (h^(d-2) sum lambda), S^(x3).  zero_start: a kZero* mode (ops.h).
template <int N1>
__global__ void __launch_bounds__(kLineThreads) k_smooth_line(const __grid_constant__ LevelParams<float> P,
                                                              const __grid_constant__ SmoothSegs G, int zero_start,
                                                              const float* __restrict__ f, float* __restrict__ u,
                                                              int early) {
  constexpr int NP = LD<N1>::NP, NL = LD<N1>::NL, ST = LD<N1>::ST, Q = N1 * N1, CPB = LD<N1>::CPB;
  __shared__ __align__(16) float sN[CPB][6][ST];
  __shared__ __align__(16) float sT[CPB][ST], sW[CPB][ST];
  int c, l;
  const bool lane_ok = line_lane<N1>(c, l);          // idle lanes mirror line 0 of the warp (no stores)
  const int j = l % N1, k = l / N1;
  int sg = 0;
#pragma unroll
  for (int q = 1; q < SmoothSegs::kMax; ++q)
    if (q < G.n && (int)blockIdx.x >= G.blk[q]) sg = q;
  const int col = G.col[sg], cs = G.cs[sg];
  const bool isB = G.first[sg] < cs + G.nbnd[sg];    // segments are all-boundary or all-interior
  const int a = G.first[sg] + ((int)blockIdx.x - G.blk[sg]) * CPB + c;
  const bool valid = lane_ok && a < G.last[sg];
  const bool line = valid && l < NL;
  const size_t o = (size_t)a * NP + N1 * j + Q * k;  // the thread's line
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {                      // set-up data: read before the wait
    nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;
    if ((zero_start == kZeroLater && (col ^ (1 << (s >> 1))) > col) || zero_start == kZeroAll) nb[s] = -1;
  }
  float fv[N1], uold[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) fv[i] = uold[i] = 0.f;
  if (line && early) ldg_line<N1, true>(f, o, fv);   // f written two or more launches back
  pdl_wait();
  pdl_trigger();
  if (valid) {
    if (line && !early) ldg_line<N1, false>(f, o, fv);
    line_stage<N1>(u, a, nb, l, nullptr, sN[c]);
    if (line && P.omega != 1.f && zero_start == kZeroNone) ldg_line<N1, false>(u, o, uold);
  }
  __syncthreads();
  const LevelConsts<float>& C = P.k;
  float t[N1];
  {                                                  // couplings (Eq. 10, interior faces)
    float acc[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) acc[i] = 0.f;
    if (line) line_interior<false, N1, float>(C, nullptr, sN[c], nb, j, k, acc);
#pragma unroll
    for (int i = 0; i < N1; ++i) t[i] = fv[i] - P.hscale * acc[i];
  }
  float y[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) y[i] = 0.f;
  float* lt = sT[c] + 4 * (j + N1 * k);
  float* lw = sW[c] + 4 * (j + N1 * k);
  const bool owner = lane_ok && l < NL;              // writes its line in the exchanges
  if (isB) {                                         // dense inverse: y = Binv t
    if (owner) sts_line<N1>(lt, t);
    __syncwarp();
    if (line) {
      const float* Bi = P.binvT + (size_t)(G.b0[sg] + (a - cs)) * NP * NP + N1 * j + Q * k;
#pragma unroll(N1 == 4 ? 8 : 9)
      for (int q = 0; q < NP; ++q) {
        float b[N1];
        ldg_line<N1, false>(Bi, (size_t)q * NP, b);
        const float tq = sT[c][sp<N1>(q)];
#pragma unroll
        for (int i = 0; i < N1; ++i) y[i] = fmaf(b[i], tq, y[i]);
      }
    }
  } else {                                           // fast diagonalisation
    float w[N1], v[N1], z[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) {                   // x: S^T on the thread's line
      w[m] = 0.f;
#pragma unroll
      for (int q = 0; q < N1; ++q) w[m] = fmaf(C.S[q * N1 + m], t[q], w[m]);
    }
    if (owner) sts_line<N1>(lt, w);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = 0.f;         // y: S^T along the lines (i, ., k)
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      float r[N1];
      lds_line<N1>(sT[c] + 4 * (q + N1 * k), r);
      const float cq = C.S[N1 * q + j];
#pragma unroll
      for (int i = 0; i < N1; ++i) v[i] = fmaf(cq, r[i], v[i]);
    }
    __syncwarp();
    if (owner) sts_line<N1>(lw, v);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < N1; ++i) z[i] = 0.f;         // z: S^T along the lines (i, j, .)
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      float r[N1];
      lds_line<N1>(sW[c] + 4 * (j + N1 * q), r);
      const float cq = C.S[N1 * q + k];
#pragma unroll
      for (int i = 0; i < N1; ++i) z[i] = fmaf(cq, r[i], z[i]);
    }
#pragma unroll
    for (int i = 0; i < N1; ++i) z[i] *= C.inv_diag[i + N1 * j + Q * k];
#pragma unroll
    for (int m = 0; m < N1; ++m) {                   // x: S on the thread's line
      w[m] = 0.f;
#pragma unroll
      for (int q = 0; q < N1; ++q) w[m] = fmaf(C.S[m * N1 + q], z[q], w[m]);
    }
    __syncwarp();
    if (owner) sts_line<N1>(lt, w);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < N1; ++i) v[i] = 0.f;         // y: S along (i, ., k)
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      float r[N1];
      lds_line<N1>(sT[c] + 4 * (q + N1 * k), r);
      const float cq = C.S[N1 * j + q];
#pragma unroll
      for (int i = 0; i < N1; ++i) v[i] = fmaf(cq, r[i], v[i]);
    }
    __syncwarp();
    if (owner) sts_line<N1>(lw, v);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < N1; ++q) {                   // z: S along (i, j, .)
      float r[N1];
      lds_line<N1>(sW[c] + 4 * (j + N1 * q), r);
      const float cq = C.S[N1 * k + q];
#pragma unroll
      for (int i = 0; i < N1; ++i) y[i] = fmaf(cq, r[i], y[i]);
    }
  }
  if (line) {
    if (P.omega != 1.f) {
#pragma unroll
      for (int i = 0; i < N1; ++i) y[i] = (1.f - P.omega) * uold[i] + P.omega * y[i];
    }
    stg_line<N1>(u, o, y);
  }
}

}  // namespace

// Where the thread-per-line kernels run (measured at 128^3 p = 2 and 96^3 p = 3 against the
// thread-per-cell FP32 operator and the thread-per-DoF smoother): the FP32 operator and residual +
// restriction at p = 3 (at p = 2 the line operator took 135 us against 53 us for the thread-per-
// cell one); the FP32 smoother and the double-float Arnoldi operator at p = 2 and 3.
bool line_kernels(int dim, int p) { return dim == 3 && p == 3; }
bool line_smoother(int dim, int p) { return dim == 3 && (p == 2 || p == 3); }
bool line_kernels_df(int dim, int p) { return dim == 3 && (p == 2 || p == 3); }

#define SBM_LINE_DISPATCH(p, MACRO)     \
  do {                                  \
    if (p == 2) { MACRO(3); }           \
    else if (p == 3) { MACRO(4); }      \
    else return cudaErrorInvalidValue;  \
  } while (0)

template <typename R>
cudaError_t launch_apply_line(int p, const LevelParams<R>& P, const float* x, const R* f, R* y, int mode,
                              cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
#define SBM_AL(N1)                                                                          \
  {                                                                                         \
    const unsigned grid = (unsigned)((P.n_act + LD<N1>::CPB - 1) / LD<N1>::CPB);            \
    if (mode == 0) SBM_PDL((k_apply_line<N1, R, 0>), grid, kLineThreads, 0, s, P, x, f, y); \
    else SBM_PDL((k_apply_line<N1, R, 1>), grid, kLineThreads, 0, s, P, x, f, y);           \
  }
  SBM_LINE_DISPATCH(p, SBM_AL);
#undef SBM_AL
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_apply_line<float>(int, const LevelParams<float>&, const float*, const float*, float*, int,
                                              cudaStream_t);
template cudaError_t launch_apply_line<dfl>(int, const LevelParams<dfl>&, const float*, const dfl*, dfl*, int,
                                            cudaStream_t);

cudaError_t launch_resid_restrict_line(const LevelParams<float>& P, const TransferParams<float>& T, const float* u,
                                       const float* f, float* rc, cudaStream_t s, int early) {
  if (P.n_act == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((P.n_act + LD<4>::CPB - 1) / LD<4>::CPB);
  SBM_PDL(k_resid_restrict_line, grid, kLineThreads, 0, s, P, T, u, f, rc, early);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_smooth_line(int p, const LevelParams<float>& P, int reverse, int zero_start, const float* f,
                               float* u, cudaStream_t s, int early, int first_group) {
  if (p != 2 && p != 3) return cudaErrorInvalidValue;
  if (reverse) zero_start = 0;
  int launched = 0;
  const int ng = n_colour_groups(P, 3);
  for (int q = first_group; q < ng; ++q) {
    const int g = reverse ? ng - 1 - q : q;
    const SmoothSegs G = smooth_segs(P, 3, g, p == 3 ? LD<4>::CPB : LD<3>::CPB);
    if (G.n == 0 || G.blk[G.n] == 0) continue;
    const int fe = launched > 0 || early;            // after the sweep's first launch f is two back
    const int zm = group_zero_mode(P, zero_start, q);
#define SBM_SL(N1) SBM_PDL((k_smooth_line<N1>), G.blk[G.n], kLineThreads, 0, s, P, G, zm, f, u, fe);
    SBM_LINE_DISPATCH(p, SBM_SL);
#undef SBM_SL
    count_launches();
    ++launched;
  }
  return cudaGetLastError();
}

}  // namespace sbm
