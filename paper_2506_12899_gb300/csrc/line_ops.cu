// Thread-per-line operator for 3D p = 3 cells (Eqs. 7, 10, 11), FP32.
//
// A p = 3 cell holds 64 values (4 x 4 x 4, dof i + 4 j + 16 k).  The thread-per-DoF kernels of
// level_ops.cu give every value its own thread and spend about 470 instructions per value on
// index arithmetic and scalar shared-memory reads; a thread per cell would need some 200
// registers.  Here a cell's 16 threads each own one line along x, (j, k) = (l mod 4, l / 4) for
// thread l, and compute the operator at its four values i = 0..3:
//   - the block copies its 8 cells and their 6 face neighbours into shared memory, one 16-byte
//     word per thread and cell (a cell's 256 bytes are contiguous, so the copies are coalesced);
//   - x terms (volume, both x faces): the thread's own line, 4 x 4 matrices;
//   - y terms: plane k of the cell and of its y neighbours (the lines through (i, ., k));
//   - z terms: the (i, j, .) lines, rows j of the cell and its z neighbours;
// every read is a 16-byte shared-memory word, and the 1D matrices come from the kernel's
// parameter block.  Surrogate faces (Eq. 7) follow in three barrier-separated phases per face
// slot: the 16 threads of a cell take the 16 points of the face (trace and normal derivative,
// then the extended value), then every thread adds the face terms at its own four values.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ops.h"

namespace sbm {
namespace {

#include "cell_core.cuh"

constexpr int kLineCells = 8;                    // cells per block
constexpr int kLineThreads = 16 * kLineCells;    // 16 lines per cell
constexpr int kLineStride = 68;                  // staged row of a cell: 64 values, padded (banks)

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// acc += a b and a b in the arithmetic R: FP32, or double-float (the Arnoldi operator's).
__device__ __forceinline__ void madd(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void madd(dfl& acc, dfl a, dfl b) { acc += a * b; }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ dfl mul(dfl a, dfl b) { return dfl(a * b); }

// s[i] += sum_m M[4 i + m] v[m]: a full 4 x 4 matrix on one line.
template <typename R>
__device__ __forceinline__ void mat4(const R* M, const float4 v, R (&s)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    madd(s[i], M[4 * i], R(v.x));
    madd(s[i], M[4 * i + 1], R(v.y));
    madd(s[i], M[4 * i + 2], R(v.z));
    madd(s[i], M[4 * i + 3], R(v.w));
  }
}

// The volume and interior-face terms (Eq. 10, reference scaling) at the four values (i, j, k),
// i = 0..3, of the thread's line, from the cell's staged row own and the staged rows N[s] of its
// neighbours (slot s = 2 dir + side, valid where nb[s] >= 0).  SELF: with the volume and the
// cell's own face terms (the operator); without them only the couplings to the neighbours (the
// smoother's right-hand side; own is not read).
template <bool SELF, typename R>
__device__ __forceinline__ void line_interior(const LevelConsts<R>& C, const float* own, const float (*N)[kLineStride],
                                              const int (&nb)[6], int j, int k, R (&acc)[4]) {
  {                                                // x: the thread's own line (j, k)
    R s[4] = {R(0.f), R(0.f), R(0.f), R(0.f)};
    if (SELF) mat4(C.L[(nb[0] >= 0) + 2 * (nb[1] >= 0)], lds4(own + 4 * j + 16 * k), s);
    if (nb[0] >= 0) mat4(C.Bpm, lds4(N[0] + 4 * j + 16 * k), s);
    if (nb[1] >= 0) mat4(C.Bmp, lds4(N[1] + 4 * j + 16 * k), s);
    const R wt = mul(C.w[j], C.w[k]);
#pragma unroll
    for (int i = 0; i < 4; ++i) madd(acc[i], wt, s[i]);
  }
#pragma unroll
  for (int dir = 1; dir < 3; ++dir) {              // y: lines (i, ., k), row j; z: lines (i, j, .), row k
    const int row = dir == 1 ? j : k;
    R s[4] = {R(0.f), R(0.f), R(0.f), R(0.f)};
#pragma unroll
    for (int q = SELF ? -1 : 0; q < 2; ++q) {      // q = -1: the cell itself
      if (q >= 0 && nb[2 * dir + q] < 0) continue;
      const R* M = q < 0 ? C.L[(nb[2 * dir] >= 0) + 2 * (nb[2 * dir + 1] >= 0)] : (q == 0 ? C.Bpm : C.Bmp);
      const float* xs = q < 0 ? own : N[2 * dir + q];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float4 v = lds4(xs + (dir == 1 ? 4 * m + 16 * k : 4 * j + 16 * m));
        const R cm = M[4 * row + m];
        madd(s[0], cm, R(v.x));
        madd(s[1], cm, R(v.y));
        madd(s[2], cm, R(v.z));
        madd(s[3], cm, R(v.w));
      }
    }
    const R wo = C.w[dir == 1 ? k : j];
#pragma unroll
    for (int i = 0; i < 4; ++i) madd(acc[i], mul(C.w[i], wo), s[i]);
  }
}

// Surrogate-face terms (Eq. 7) of the block's boundary cells at the calling thread's four
// values, reference scaling; every thread of the block calls it (barriers).
template <typename R>
__device__ __forceinline__ void line_sbm_terms(const LevelParams<R>& P, float (*sX)[7][kLineStride], R (*sU)[16],
                                               R (*sG)[16], R (*sE)[16], int c, int l, int j, int k, int bidx,
                                               const int (&nb)[6], R (&acc)[4]) {
  const LevelConsts<R>& C = P.k;
  const float* own = sX[c][0];
#pragma unroll 1
  for (int slot = 0; slot < 6; ++slot) {
    const bool sf = bidx >= 0 && nb[slot] < 0;
    if (!__syncthreads_or(sf)) continue;
    const int dir = slot >> 1, side = slot & 1;
    const R* es = side ? C.e1 : C.e0;
    const R* ds = side ? C.d1 : C.d0;
    const R* dh = sf ? P.dhat + ((size_t)bidx * 6 + slot) * 3 * 16 : nullptr;
    const int t = l;                             // this thread's face point
    if (sf) {                                    // trace and normal derivative at face point t
      R su = R(0.f), sd = R(0.f);
#pragma unroll
      for (int kn = 0; kn < 4; ++kn) {
        const R v = R(own[dof<3, 4>(dir, kn, t)]);
        madd(su, es[kn], v);
        madd(sd, ds[kn], v);
      }
      sU[c][t] = su;
      sG[c][t] = sd;
    }
    __syncthreads();
    if (sf) {                                    // extended value at face point t
      R E;
      if (P.extension == 0) {
        E = sU[c][t];
        madd(E, dh[dir * 16 + t], sG[c][t]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {            // tangential derivatives of the trace
          const int m = tang_dim<3>(dir, q);
          const int stride = q == 0 ? 1 : 4;
          const int tm = (t / stride) % 4;
          R g = R(0.f);
#pragma unroll
          for (int r = 0; r < 4; ++r) madd(g, C.Dm[tm * 4 + r], sU[c][t + (r - tm) * stride]);
          madd(E, dh[m * 16 + t], g);
        }
      } else {                                   // cell polynomial at x~ + d
        R lv[3][4];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          R xi;
          if (m == dir) {
            xi = R((float)side);
          } else {
            const int q = m < dir ? m : m - 1;
            xi = C.x[(t / (q == 0 ? 1 : 4)) % 4];
          }
          const R yv = xi + dh[m * 16 + t];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            R val = C.inv_denom[kk];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
              if (jj != kk) val = mul(val, yv - C.x[jj]);
            lv[m][kk] = val;
          }
        }
        E = R(0.f);
#pragma unroll
        for (int q = 0; q < 64; ++q) madd(E, mul(mul(lv[0][q % 4], lv[1][(q / 4) % 4]), lv[2][q / 16]), R(own[q]));
      }
      sE[c][t] = E;
    }
    __syncthreads();
    if (sf) {                                    // terms at the thread's values (i, j, k), i = 0..3
      const R sg = R(side ? 1.f : -1.f);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int tp, kn;                              // face point and normal position of value (i, j, k)
        if (dir == 0) {
          tp = j + 4 * k;
          kn = i;
        } else if (dir == 1) {
          tp = i + 4 * k;
          kn = j;
        } else {
          tp = i + 4 * j;
          kn = k;
        }
        const R wt = mul(C.w[tp % 4], C.w[tp / 4]);
        const R E = sE[c][tp], G = sG[c][tp];
        R term = mul(es[kn], mul(P.sigG, E) - mul(sg, G));
        term = term - mul(mul(P.alpha, sg), mul(ds[kn], E));
        madd(acc[i], wt, term);
      }
    }
    __syncthreads();
  }
}

// Stages word l of cell a and of its face neighbours nb into X (rows of kLineStride floats).
__device__ __forceinline__ void line_stage(const float* __restrict__ x, int a, const int (&nb)[6], int l,
                                           float (*X)[kLineStride]) {
  reinterpret_cast<float4*>(X[0])[l] = reinterpret_cast<const float4*>(x + (size_t)a * 64)[l];
#pragma unroll
  for (int s = 0; s < 6; ++s)
    if (nb[s] >= 0) reinterpret_cast<float4*>(X[1 + s])[l] = reinterpret_cast<const float4*>(x + (size_t)nb[s] * 64)[l];
}

// y = A x (MODE 0) or y = f - A x (MODE 1) for a 3D p = 3 level; x FP32, arithmetic and y in R
// (FP32, or double-float for the Arnoldi operator).
template <typename R, int MODE>
__global__ void __launch_bounds__(kLineThreads) k_apply_line(const __grid_constant__ LevelParams<R> P,
                                                             const float* __restrict__ x, const R* __restrict__ f,
                                                             R* __restrict__ y) {
  __shared__ __align__(16) float sX[kLineCells][7][kLineStride];
  __shared__ R sU[kLineCells][16], sG[kLineCells][16], sE[kLineCells][16];
  const int c = threadIdx.x >> 4, l = threadIdx.x & 15, j = l & 3, k = l >> 2;
  const int a = blockIdx.x * kLineCells + c;
  const bool valid = a < P.n_act;
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;   // set-up data
  pdl_wait();
  pdl_trigger();
  if (valid) line_stage(x, a, nb, l, sX[c]);
  __syncthreads();
  R acc[4] = {R(0.f), R(0.f), R(0.f), R(0.f)};
  if (valid) line_interior<true, R>(P.k, sX[c][0], sX[c] + 1, nb, j, k, acc);
  const int bidx = valid ? boundary_index(P, a, 8) : -1;
  if (__syncthreads_or(bidx >= 0)) line_sbm_terms<R>(P, sX, sU, sG, sE, c, l, j, k, bidx, nb, acc);
  if (valid) {
    const size_t o = (size_t)a * 64 + 4 * j + 16 * k;
    R out[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = mul(P.hscale, acc[i]);
    if (MODE == 1) {
#pragma unroll
      for (int i = 0; i < 4; ++i) out[i] = f[o + i] - out[i];
    }
    if constexpr (sizeof(R) == 4) {
      *reinterpret_cast<float4*>(y + o) = make_float4(out[0], out[1], out[2], out[3]);
    } else {
      reinterpret_cast<float4*>(y + o)[0] = make_float4(out[0].hi, out[0].lo, out[1].hi, out[1].lo);
      reinterpret_cast<float4*>(y + o)[1] = make_float4(out[2].hi, out[2].lo, out[3].hi, out[3].lo);
    }
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
  __shared__ __align__(16) float sX[kLineCells][7][kLineStride];
  __shared__ float sU[kLineCells][16], sG[kLineCells][16], sE[kLineCells][16];
  __shared__ float sR1[kLineCells][48], sR2[kLineCells][36];
  const int c = threadIdx.x >> 4, l = threadIdx.x & 15, j = l & 3, k = l >> 2;
  const int a = blockIdx.x * kLineCells + c;
  const bool valid = a < P.n_act;
  const size_t o = (size_t)a * 64 + 4 * j + 16 * k;
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;   // set-up data
  float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid && early) fv = __ldcg(reinterpret_cast<const float4*>(f + o));   // f written two or more launches back
  pdl_wait();
  pdl_trigger();
  if (valid) {
    if (!early) fv = *reinterpret_cast<const float4*>(f + o);
    line_stage(u, a, nb, l, sX[c]);
  }
  __syncthreads();
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (valid) line_interior<true, float>(P.k, sX[c][0], sX[c] + 1, nb, j, k, acc);
  const int bidx = valid ? boundary_index(P, a, 8) : -1;
  if (__syncthreads_or(bidx >= 0)) line_sbm_terms<float>(P, sX, sU, sG, sE, c, l, j, k, bidx, nb, acc);
  const float r[4] = {fv.x - P.hscale * acc[0], fv.y - P.hscale * acc[1], fv.z - P.hscale * acc[2],
                      fv.w - P.hscale * acc[3]};
  // x: (j0, j, k) = sum_i Pp[i][j0] r(i, j, k)
#pragma unroll
  for (int j0 = 0; j0 < 3; ++j0) {
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

// One colour group of the block Gauss-Seidel sweep (Eq. 16) on a 3D p = 3 level, FP32, one thread
// per x-line, 8 cells of one segment per block:
//   t_K = f_K - sum over interior faces of A_KN u_N (the SBM terms lie in A_KK),
//   u_K <- (1 - omega) u_K + omega A_KK^-1 t_K.
// The couplings take the same line, plane and row reads as the operator.  Boundary cells apply
// their dense inverse (each thread four rows, 16-byte reads of the transposed inverse, t from
// shared memory); interior cells the fast diagonalisation (S^T)^(x3), 1 / (h^(d-2) sum lambda),
// S^(x3): the x contractions on the thread's own line in registers, the y and z contractions
// after an exchange of the cell's values through shared memory.  A cell's 16 threads lie in one
// warp, so the exchanges need only warp barriers.  zero_start: a kZero* mode (ops.h).
__global__ void __launch_bounds__(kLineThreads) k_smooth_line(const __grid_constant__ LevelParams<float> P,
                                                              const __grid_constant__ SmoothSegs G, int zero_start,
                                                              const float* __restrict__ f, float* __restrict__ u,
                                                              int early) {
  __shared__ __align__(16) float sN[kLineCells][6][kLineStride];
  __shared__ __align__(16) float sT[kLineCells][kLineStride], sW[kLineCells][kLineStride];
  const int c = threadIdx.x >> 4, l = threadIdx.x & 15, j = l & 3, k = l >> 2;
  int sg = 0;
#pragma unroll
  for (int q = 1; q < SmoothSegs::kMax; ++q)
    if (q < G.n && (int)blockIdx.x >= G.blk[q]) sg = q;
  const int col = G.col[sg], cs = G.cs[sg];
  const bool isB = G.first[sg] < cs + G.nbnd[sg];    // segments are all-boundary or all-interior
  const int a = G.first[sg] + ((int)blockIdx.x - G.blk[sg]) * kLineCells + c;
  const bool valid = a < G.last[sg];
  const size_t o = (size_t)a * 64 + 4 * j + 16 * k;  // the thread's line
  int nb[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) {                      // set-up data: read before the wait
    nb[s] = valid ? P.nbr[(size_t)s * P.n_act + a] : -1;
    if ((zero_start == kZeroLater && (col ^ (1 << (s >> 1))) > col) || zero_start == kZeroAll) nb[s] = -1;
  }
  float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid && early) fv = __ldcg(reinterpret_cast<const float4*>(f + o));   // f written two or more launches back
  pdl_wait();
  pdl_trigger();
  float4 uold = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    if (!early) fv = *reinterpret_cast<const float4*>(f + o);
#pragma unroll
    for (int s = 0; s < 6; ++s)
      if (nb[s] >= 0)
        reinterpret_cast<float4*>(sN[c][s])[l] = reinterpret_cast<const float4*>(u + (size_t)nb[s] * 64)[l];
    if (P.omega != 1.f && zero_start == kZeroNone) uold = *reinterpret_cast<const float4*>(u + o);
  }
  __syncthreads();
  const LevelConsts<float>& C = P.k;
  float t[4];
  {                                                  // couplings (Eq. 10, interior faces)
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (valid) line_interior<false, float>(P.k, nullptr, sN[c], nb, j, k, acc);
    t[0] = fv.x - P.hscale * acc[0];
    t[1] = fv.y - P.hscale * acc[1];
    t[2] = fv.z - P.hscale * acc[2];
    t[3] = fv.w - P.hscale * acc[3];
  }
  float y[4] = {0.f, 0.f, 0.f, 0.f};
  float* lt = sT[c] + 4 * j + 16 * k;
  float* lw = sW[c] + 4 * j + 16 * k;
  if (isB) {                                         // dense inverse: y = Binv t
    *reinterpret_cast<float4*>(lt) = make_float4(t[0], t[1], t[2], t[3]);
    __syncwarp();
    if (valid) {
      const float* Bi = P.binvT + (size_t)(G.b0[sg] + (a - cs)) * 64 * 64 + 4 * j + 16 * k;
#pragma unroll 8
      for (int q = 0; q < 64; ++q) {
        const float4 b = *reinterpret_cast<const float4*>(Bi + (size_t)q * 64);
        const float tq = sT[c][q];
        y[0] += b.x * tq; y[1] += b.y * tq; y[2] += b.z * tq; y[3] += b.w * tq;
      }
    }
  } else {                                           // fast diagonalisation
    float w[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) w[m] = C.S[m] * t[0] + C.S[4 + m] * t[1] + C.S[8 + m] * t[2] + C.S[12 + m] * t[3];
    *reinterpret_cast<float4*>(lt) = make_float4(w[0], w[1], w[2], w[3]);
    __syncwarp();
    float v[4] = {0.f, 0.f, 0.f, 0.f};               // y: (S^T) along the lines (i, ., k)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 r = lds4(sT[c] + 4 * q + 16 * k);
      const float cq = C.S[4 * q + j];
      v[0] += cq * r.x; v[1] += cq * r.y; v[2] += cq * r.z; v[3] += cq * r.w;
    }
    *reinterpret_cast<float4*>(lw) = make_float4(v[0], v[1], v[2], v[3]);
    __syncwarp();
    float z[4] = {0.f, 0.f, 0.f, 0.f};               // z: (S^T) along the lines (i, j, .)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 r = lds4(sW[c] + 4 * j + 16 * q);
      const float cq = C.S[4 * q + k];
      z[0] += cq * r.x; z[1] += cq * r.y; z[2] += cq * r.z; z[3] += cq * r.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i] *= C.inv_diag[i + 4 * j + 16 * k];
#pragma unroll
    for (int m = 0; m < 4; ++m) w[m] = C.S[4 * m] * z[0] + C.S[4 * m + 1] * z[1] + C.S[4 * m + 2] * z[2] + C.S[4 * m + 3] * z[3];
    *reinterpret_cast<float4*>(lt) = make_float4(w[0], w[1], w[2], w[3]);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = 0.f;          // y: S along (i, ., k)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 r = lds4(sT[c] + 4 * q + 16 * k);
      const float cq = C.S[4 * j + q];
      v[0] += cq * r.x; v[1] += cq * r.y; v[2] += cq * r.z; v[3] += cq * r.w;
    }
    *reinterpret_cast<float4*>(lw) = make_float4(v[0], v[1], v[2], v[3]);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q) {                    // z: S along (i, j, .)
      const float4 r = lds4(sW[c] + 4 * j + 16 * q);
      const float cq = C.S[4 * k + q];
      y[0] += cq * r.x; y[1] += cq * r.y; y[2] += cq * r.z; y[3] += cq * r.w;
    }
  }
  if (valid) {
    float4 out = make_float4(y[0], y[1], y[2], y[3]);
    if (P.omega != 1.f) {
      const float om = P.omega, rm = 1.f - P.omega;
      out = make_float4(rm * uold.x + om * y[0], rm * uold.y + om * y[1], rm * uold.z + om * y[2],
                        rm * uold.w + om * y[3]);
    }
    *reinterpret_cast<float4*>(u + o) = out;
  }
}

}  // namespace

bool line_kernels(int dim, int p) { return dim == 3 && p == 3; }

template <typename R>
cudaError_t launch_apply_line(const LevelParams<R>& P, const float* x, const R* f, R* y, int mode, cudaStream_t s) {
  if (P.n_act == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((P.n_act + kLineCells - 1) / kLineCells);
  if (mode == 0) SBM_PDL((k_apply_line<R, 0>), grid, kLineThreads, 0, s, P, x, f, y);
  else SBM_PDL((k_apply_line<R, 1>), grid, kLineThreads, 0, s, P, x, f, y);
  count_launches();
  return cudaGetLastError();
}
template cudaError_t launch_apply_line<float>(const LevelParams<float>&, const float*, const float*, float*, int,
                                              cudaStream_t);
template cudaError_t launch_apply_line<dfl>(const LevelParams<dfl>&, const float*, const dfl*, dfl*, int,
                                            cudaStream_t);

cudaError_t launch_resid_restrict_line(const LevelParams<float>& P, const TransferParams<float>& T, const float* u,
                                       const float* f, float* rc, cudaStream_t s, int early) {
  if (P.n_act == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((P.n_act + kLineCells - 1) / kLineCells);
  SBM_PDL(k_resid_restrict_line, grid, kLineThreads, 0, s, P, T, u, f, rc, early);
  count_launches();
  return cudaGetLastError();
}

cudaError_t launch_smooth_line(const LevelParams<float>& P, int reverse, int zero_start, const float* f, float* u,
                               cudaStream_t s, int early, int first_group) {
  if (reverse) zero_start = 0;
  int launched = 0;
  const int ng = n_colour_groups(P, 3);
  for (int q = first_group; q < ng; ++q) {
    const int g = reverse ? ng - 1 - q : q;
    const SmoothSegs G = smooth_segs(P, 3, g, kLineCells);
    if (G.n == 0 || G.blk[G.n] == 0) continue;
    const int fe = launched > 0 || early;            // after the sweep's first launch f is two back
    SBM_PDL(k_smooth_line, G.blk[G.n], kLineThreads, 0, s, P, G, group_zero_mode(P, zero_start, q), f, u, fe);
    count_launches();
    ++launched;
  }
  return cudaGetLastError();
}

}  // namespace sbm
