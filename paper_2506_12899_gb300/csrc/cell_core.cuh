// Device helpers shared by the thread-per-cell kernels (cell_ops.cu) and the staged
// thread-per-cell kernels (staged_ops.cu): cell layout, cell loads and stores, the operator
// pieces of one cell (Eqs. 7, 10, 11) and the block solve of the smoother (Eqs. 14, 16).
// Included inside namespace sbm { namespace { ... } }.
#pragma once

constexpr int kCellThreads = 128;   // largest block of the thread-per-cell kernels

// Block size of a thread-per-cell launch over `cells` threads: 32 for launches of up to 32 warps
// per SM (more, smaller blocks spread a short launch over all SMs: with 32 everywhere the 2D p=2
// 512^2 solve was 3% faster and the 3D p=1 64^3 one 16%), 128 above.
inline unsigned cell_block(size_t cells) { return cells <= (size_t)152 * 32 * 32 ? 32u : (unsigned)kCellThreads; }
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

// Global loads are ordinary L1-cached loads (a thread reads its cell's contiguous values, so
// consecutive load instructions of a warp hit the lines the first one brought in).
template <typename T>
__device__ __forceinline__ T ldv(const T* p) {
  return *p;
}

// 32-byte global load / store (sm_100 and later), p 32-byte aligned.
__device__ __forceinline__ void ld32B(const void* p, unsigned (&r)[8]) {
  asm volatile("ld.global.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "l"(p));
}
__device__ __forceinline__ void st32B(void* p, const unsigned (&r)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(r[0]), "r"(r[1]), "r"(r[2]),
               "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// The NP values of cell a when they do not fill whole 16-byte words (an odd (p+1)^d, i.e. 2D and 3D
// p = 2): the thread reads the 16-byte-aligned window of the vector that holds them, with
// 16-byte loads, and moves its values to the front by two word-shift selects.  A warp's scalar
// loads of such cells each touch as many 128-byte lines as the cells span (27 for 3D p = 2 in
// FP32), and the L1 request stream, not DRAM, then bounds the kernel; the window loads touch the
// same lines with a fraction of the requests.  The window may cover words of the adjacent cells,
// which are read and discarded (in a smoother launch those words can belong to cells another
// thread is updating; no value taken from them is used).  Returns false, loading nothing, when the window would pass the
// end of the vector (n_act cells) or the vector is not 16-byte aligned; the caller then loads the
// values one by one.  CG: loads that go to L2 only (see load_cell_l2).
template <int NP, typename T, bool CG>
__device__ __forceinline__ bool load_window(const T* __restrict__ x, int a, int n_act, T (&v)[NP]) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  constexpr int NW = NP * (int)sizeof(T) / 4;                 // 32-bit words of one cell
  constexpr int MAXSH = sizeof(T) == 8 ? 2 : 3;               // largest word shift of a cell start
  constexpr int NV = (NW + MAXSH + 3) / 4;                    // 16-byte loads of the window
  if ((reinterpret_cast<uintptr_t>(x) & 15) != 0) return false;
  const size_t g = (size_t)a * NW;
  const size_t st = g & ~(size_t)3;
  if (st + 4 * NV > (size_t)n_act * NW) return false;
  const int sh = (int)(g - st);
  const uint4* q = reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned*>(x) + st);
  unsigned w[4 * NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const uint4 u4 = CG ? __ldcg(q + c) : q[c];
    w[4 * c] = u4.x;
    w[4 * c + 1] = u4.y;
    w[4 * c + 2] = u4.z;
    w[4 * c + 3] = u4.w;
  }
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i + 1 < 4 * NV; ++i) w[i] = (sh & 1) ? w[i + 1] : w[i];
  }
  unsigned o[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) o[i] = (sh & 2) ? w[i + 2] : w[i];
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    if constexpr (sizeof(T) == 4) {
      v[i] = __uint_as_float(o[i]);
    } else {
      const unsigned pair[2] = {o[2 * i], o[2 * i + 1]};
      memcpy(&v[i], pair, sizeof(T));
    }
  }
  return true;
}

// The (p+1)^d values of cell a (of a vector of n_act cells).  When a cell's values fill whole
// 32-byte words (3D p = 1 and 2D p = 3 in FP32, 3D p = 1 in FP64) and the vector is 32-byte
// aligned, they are read with 32-byte loads (one L1 request per warp and word instead of two);
// when they fill 16-byte words (2D p = 1 as well), with 16-byte loads; otherwise through their
// 16-byte-aligned window (load_window).
template <int D, int N1, typename TI, typename R>
__device__ __forceinline__ void load_cell(const TI* __restrict__ x, int a, int n_act, R (&v)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  if constexpr ((NP * sizeof(TI)) % 32 == 0) {
    if ((reinterpret_cast<uintptr_t>(x) & 31) == 0) {
      TI t[NP];
      const unsigned char* q = reinterpret_cast<const unsigned char*>(x + (size_t)a * NP);
#pragma unroll
      for (int c = 0; c < (int)(NP * sizeof(TI) / 32); ++c) {
        unsigned r[8];
        ld32B(q + 32 * c, r);
#pragma unroll
        for (int k = 0; k < 8; ++k) reinterpret_cast<unsigned*>(t)[8 * c + k] = r[k];
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = (R)t[i];
      return;
    }
  }
  if constexpr ((NP * sizeof(TI)) % 16 == 0) {
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
      TI t[NP];
      const uint4* q = reinterpret_cast<const uint4*>(x + (size_t)a * NP);
#pragma unroll
      for (int c = 0; c < (int)(NP * sizeof(TI) / 16); ++c) reinterpret_cast<uint4*>(t)[c] = q[c];
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = (R)t[i];
      return;
    }
  } else if constexpr (sizeof(TI) == 4 || sizeof(TI) == 8) {
    TI t[NP];
    if (load_window<NP, TI, false>(x, a, n_act, t)) {
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = (R)t[i];
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) v[i] = (R)ldv(x + (size_t)a * NP + i);
}

// load_cell for data that earlier kernels wrote, read before griddepcontrol.wait (the `early`
// reads): every access goes to L2 only (ld.global.cg), the coherence point that the writer's
// completion has reached, so a line another kernel left in this SM's L1 is never used.
template <int D, int N1, typename TI, typename R>
__device__ __forceinline__ void load_cell_l2(const TI* __restrict__ x, int a, int n_act, R (&v)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  const TI* p = x + (size_t)a * NP;
  if constexpr ((NP * sizeof(TI)) % 32 == 0) {
    if ((reinterpret_cast<uintptr_t>(x) & 31) == 0) {
      TI t[NP];
#pragma unroll
      for (int c = 0; c < (int)(NP * sizeof(TI) / 32); ++c) {
        unsigned r[8];
        asm volatile("ld.global.cg.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                       "=r"(r[7])
                     : "l"(reinterpret_cast<const unsigned char*>(p) + 32 * c));
#pragma unroll
        for (int k = 0; k < 8; ++k) reinterpret_cast<unsigned*>(t)[8 * c + k] = r[k];
      }
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = (R)t[i];
      return;
    }
  }
  if constexpr ((NP * sizeof(TI)) % 16 == 0) {
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
      TI t[NP];
#pragma unroll
      for (int c = 0; c < (int)(NP * sizeof(TI) / 16); ++c)
        reinterpret_cast<uint4*>(t)[c] = __ldcg(reinterpret_cast<const uint4*>(p) + c);
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = (R)t[i];
      return;
    }
  } else if constexpr (sizeof(TI) == 4 || sizeof(TI) == 8) {
    TI t[NP];
    if (load_window<NP, TI, true>(x, a, n_act, t)) {
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = (R)t[i];
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) v[i] = (R)__ldcg(p + i);
}

// Whether the values of a cell fill whole 16-byte words (then stored with vector stores by each
// thread; otherwise warp_store_cells).
template <int NP, typename R>
constexpr bool cell_vec16() {
  return (NP * sizeof(R)) % 16 == 0;
}

// Shared-memory staging buffer of warp_store_cells: 32 cells per warp of a kCellThreads block.
template <int NP, typename R>
struct WarpStage {
  R v[kCellThreads / 32][cell_vec16<NP, R>() ? 1 : 32 * NP];
};

// Stores the values v of cells a0 + lane, for the lanes lane < m, of a warp whose lanes own
// consecutive cells: through the warp's slice sw of shared memory, so that the global stores are
// coalesced (lane k of every store instruction writes word k of a 128-byte run) instead of one
// scattered 4- or 8-byte store per value and thread.  Every lane of the warp must call it.
template <int NP, typename R>
__device__ __forceinline__ void warp_store_cells(R* __restrict__ y, int a0, int m, const R (&v)[NP], R* sw) {
  const int lane = threadIdx.x & 31;
  __syncwarp();                                   // earlier readers of sw are done
  if (lane < m) {
#pragma unroll
    for (int i = 0; i < NP; ++i) sw[lane * NP + i] = v[i];
  }
  __syncwarp();
  R* dst = y + (size_t)a0 * NP;
  const int cnt = m * NP;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int e = lane + 32 * k;
    if (e < cnt) dst[e] = sw[e];
  }
}

// Stores the values of cell a, with 32- or 16-byte stores under the same conditions as load_cell.
template <int D, int N1, typename R>
__device__ __forceinline__ void store_cell(R* __restrict__ x, int a, const R (&v)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  if constexpr ((NP * sizeof(R)) % 32 == 0) {
    if ((reinterpret_cast<uintptr_t>(x) & 31) == 0) {
      unsigned char* q = reinterpret_cast<unsigned char*>(x + (size_t)a * NP);
#pragma unroll
      for (int c = 0; c < (int)(NP * sizeof(R) / 32); ++c) {
        unsigned r[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = reinterpret_cast<const unsigned*>(v)[8 * c + k];
        st32B(q + 32 * c, r);
      }
      return;
    }
  }
  if constexpr ((NP * sizeof(R)) % 16 == 0) {
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0) {
      uint4* q = reinterpret_cast<uint4*>(x + (size_t)a * NP);
#pragma unroll
      for (int c = 0; c < (int)(NP * sizeof(R) / 16); ++c) q[c] = reinterpret_cast<const uint4*>(v)[c];
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) x[(size_t)a * NP + i] = v[i];
}

// Loads the 16-byte aligned values of one cell from shared memory (local or another CTA of the
// cluster) with vector loads.
template <int NP, typename R>
__device__ __forceinline__ void load_np_vec(const R* p, R (&v)[NP]) {
  static_assert((NP * sizeof(R)) % 16 == 0, "cell values must fill 16-byte words");
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int c = 0; c < NP / 4; ++c) {
      const float4 w = reinterpret_cast<const float4*>(p)[c];
      v[4 * c] = w.x;
      v[4 * c + 1] = w.y;
      v[4 * c + 2] = w.z;
      v[4 * c + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) {
      const double2 w = reinterpret_cast<const double2*>(p)[c];
      v[2 * c] = w.x;
      v[2 * c + 1] = w.y;
    }
  }
}

template <int NP, typename R>
__device__ __forceinline__ void store_np_vec(R* p, const R (&v)[NP]) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int c = 0; c < NP / 4; ++c)
      reinterpret_cast<float4*>(p)[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  } else {
#pragma unroll
    for (int c = 0; c < NP / 2; ++c) reinterpret_cast<double2*>(p)[c] = make_double2(v[2 * c], v[2 * c + 1]);
  }
}

// y += (sum over interior faces of A_KN u_N) for a cell of colour col (Eq. 10 couplings);
// loadn(n, colour of n, values) fetches neighbour n.  Neighbours of colour > col are skipped
// when zero_start (they hold zeros).
template <int D, int N1, typename R, typename LoadN>
__device__ __forceinline__ void add_couplings_f(const LevelConsts<R>& C, int col, bool zero_start,
                                                const int (&nb)[2 * D], LoadN loadn, R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP, NQ = CD<D, N1>::NQ;
#pragma unroll
  for (int s = 0; s < 2 * D; ++s) {
    const int dir = s >> 1;
    const int n = nb[s];
    if (n < 0 || (zero_start && (col ^ (1 << dir)) > col)) continue;
    R un[NP];
    loadn(n, col ^ (1 << dir), un);
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

// Couplings with the neighbour values read from the global vector u.
template <int D, int N1, typename TI, typename R>
__device__ __forceinline__ void add_couplings(const LevelParams<R>& P, const TI* __restrict__ u, int col,
                                              bool zero_start, const int (&nb)[2 * D], R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  add_couplings_f<D, N1, R>(P.k, col, zero_start, nb,
                            [&](int n, int, R(&un)[NP]) { load_cell<D, N1, TI, R>(u, n, P.n_act, un); }, y);
}

// y += the surrogate-face terms of boundary cell bidx (Eq. 7) with the line weights wq (the
// quadrature weights of the face points, times any scale folded into them); nothing when bidx < 0.
// V: the type of the cell values v (FP32 values under a double-float R are exact in it).
template <int D, int N1, typename R, typename V>
__device__ __forceinline__ void add_surrogate(const LevelParams<R>& P, const int (&nb)[2 * D], int bidx,
                                              const R (&wq)[CD<D, N1>::NQ], const V (&v)[CD<D, N1>::NP],
                                              R (&y)[CD<D, N1>::NP]) {
  constexpr int NQ = CD<D, N1>::NQ;
  const LevelConsts<R>& C = P.k;
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
      const R wt = wq[t];
#pragma unroll
      for (int k = 0; k < N1; ++k)
        y[dof<D, N1>(dir, k, t)] += wt * (es[k] * (-sg * G[t] + P.sigG * E) - P.alpha * sg * ds[k] * E);
    }
  }
}

// y += A_KK v (volume + own halves of interior faces + surrogate faces), reference scaling.
template <int D, int N1, typename R>
__device__ __forceinline__ void add_self(const LevelParams<R>& P, const int (&nb)[2 * D], int bidx,
                                         const R (&v)[CD<D, N1>::NP], R (&y)[CD<D, N1>::NP]) {
  constexpr int NQ = CD<D, N1>::NQ;
  const LevelConsts<R>& C = P.k;
  R wq[NQ];
#pragma unroll
  for (int t = 0; t < NQ; ++t) wq[t] = line_weight<D, N1, R>(C, t);
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    // self matrix by neighbour mask; the mask is uniform over a warp of interior cells
    const R* Lm = C.L[(nb[2 * dir] >= 0) + 2 * (nb[2 * dir + 1] >= 0)];
#pragma unroll
    for (int t = 0; t < NQ; ++t) {
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        R acc = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) acc += Lm[i * N1 + k] * v[dof<D, N1>(dir, k, t)];
        y[dof<D, N1>(dir, i, t)] += wq[t] * acc;
      }
    }
  }
  add_surrogate<D, N1, R, R>(P, nb, bidx, wq, v, y);
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

// y = (A x)_a with the reference scaling h^(d-2) applied; nb: the neighbours of a (load_nbr).
//
// Double-float accumulation (the Arnoldi operator on the FP32 V-cycle output): the FP32 values
// stay FP32 (exact, and the double-float x FP32 products are the shorter form), and per direction
// the self line matrix and the couplings to the two neighbours across the faces normal to it act
// on the lines along that direction, their sum weighted once per line point by the face-point
// weight times h^(d-2); a missing neighbour contributes zeros.  This executes about a quarter
// fewer FP32 instructions than the face-by-face form.  FP32 and FP64 keep the face-by-face form,
// which holds one neighbour at a time in registers.
template <int D, int N1, typename TI, typename R>
__device__ __forceinline__ void cell_apply(const LevelParams<R>& P, const TI* __restrict__ x, int a,
                                           const int (&nb)[2 * D], R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP, NQ = CD<D, N1>::NQ;
  const LevelConsts<R>& C = P.k;
  if constexpr (std::is_same<R, dfl>::value && std::is_same<TI, float>::value) {
    R wq[NQ];
#pragma unroll
    for (int t = 0; t < NQ; ++t) wq[t] = R(line_weight<D, N1, R>(C, t) * P.hscale);
    // 3D p = 1: a boundary cell applies its stored self block (bself) instead of the self line
    // matrices and the surrogate-face terms
    constexpr bool kDenseSelf = D == 3 && N1 == 2;
    int bidx = -1;
    bool dense = false;
    if constexpr (kDenseSelf) {
      bidx = boundary_index(P, a, 1 << D);
      dense = bidx >= 0 && P.bself != nullptr;
    }
    float v[NP];
    load_cell<D, N1, TI, float>(x, a, P.n_act, v);
    if (dense) {                                   // the self terms come from the dense block below
#pragma unroll
      for (int i = 0; i < NP; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      const int nm = nb[2 * dir], npl = nb[2 * dir + 1];
      float um[NP], up[NP];
      if (nm >= 0) {
        load_cell<D, N1, TI, float>(x, nm, P.n_act, um);
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) um[i] = 0.f;
      }
      if (npl >= 0) {
        load_cell<D, N1, TI, float>(x, npl, P.n_act, up);
      } else {
#pragma unroll
        for (int i = 0; i < NP; ++i) up[i] = 0.f;
      }
      const R* Lm = C.L[(nm >= 0) + 2 * (npl >= 0)];   // self matrix by neighbour mask
#pragma unroll
      for (int t = 0; t < NQ; ++t) {
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          R acc = R(Lm[i * N1] * v[dof<D, N1>(dir, 0, t)]);
#pragma unroll
          for (int k = 1; k < N1; ++k) acc += Lm[i * N1 + k] * v[dof<D, N1>(dir, k, t)];
#pragma unroll
          for (int k = 0; k < N1; ++k) acc += C.Bpm[i * N1 + k] * um[dof<D, N1>(dir, k, t)];
#pragma unroll
          for (int k = 0; k < N1; ++k) acc += C.Bmp[i * N1 + k] * up[dof<D, N1>(dir, k, t)];
          if (dir == 0) y[dof<D, N1>(dir, i, t)] = R(wq[t] * acc);   // dir 0 visits every dof once
          else y[dof<D, N1>(dir, i, t)] += wq[t] * acc;
        }
      }
    }
    if constexpr (kDenseSelf) {
      if (dense) {                                 // y += h^(d-2) A_KK v, two block entries per 16-byte load
        load_cell<D, N1, TI, float>(x, a, P.n_act, v);
        const float4* Ab = reinterpret_cast<const float4*>(P.bself + (size_t)bidx * P.bself_ld);
#pragma unroll
        for (int e = 0; e < (NP * NP + 1) / 2; ++e) {
          const float4 q = Ab[e];
          y[(2 * e) % NP] += dfl(q.x, q.y) * v[(2 * e) / NP];
          if (2 * e + 1 < NP * NP) y[(2 * e + 1) % NP] += dfl(q.z, q.w) * v[(2 * e + 1) / NP];
        }
      } else {
        add_surrogate<D, N1, R, float>(P, nb, bidx, wq, v, y);
      }
    } else {
      add_surrogate<D, N1, R, float>(P, nb, boundary_index(P, a, 1 << D), wq, v, y);
    }
  } else {
    R v[NP];
    load_cell<D, N1, TI, R>(x, a, P.n_act, v);
#pragma unroll
    for (int i = 0; i < NP; ++i) y[i] = 0;
    add_self<D, N1, R>(P, nb, boundary_index(P, a, 1 << D), v, y);
    add_couplings<D, N1, TI, R>(P, x, 0, false, nb, y);
#pragma unroll
    for (int i = 0; i < NP; ++i) y[i] *= P.hscale;
  }
}


// y = A_KK^{-1} t / hscale-scaled block solve of one cell: the dense inverse of boundary cell
// bidx, or the fast diagonalisation (S^T)^(x d), 1 / (hscale sum lambda), S^(x d) when bidx < 0.
template <int D, int N1, typename R>
__device__ __forceinline__ void block_solve_at(const LevelParams<R>& P, const R* Bi, R (&t)[CD<D, N1>::NP],
                                               R (&y)[CD<D, N1>::NP]);

template <int D, int N1, typename R>
__device__ __forceinline__ void block_solve(const LevelParams<R>& P, int bidx, R (&t)[CD<D, N1>::NP],
                                            R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  block_solve_at<D, N1, R>(P, bidx >= 0 ? P.binvT + (size_t)bidx * NP * NP : nullptr, t, y);
}

// Bi: the cell's transposed dense inverse, or null for the fast diagonalisation.
template <int D, int N1, typename R>
__device__ __forceinline__ void block_solve_at(const LevelParams<R>& P, const R* Bi, R (&t)[CD<D, N1>::NP],
                                               R (&y)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP, NQ = CD<D, N1>::NQ;
  if (Bi) {
#pragma unroll
    for (int i = 0; i < NP; ++i) y[i] = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
      for (int i = 0; i < NP; ++i) y[i] += Bi[j * NP + i] * t[j];
    return;
  }
  const LevelConsts<R>& C = P.k;
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {              // (S^T)^(x d) t
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
    t[i] = t[i] * C.inv_diag[i];
  }
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {              // S^(x d) v
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

// One cell of one colour of the block Gauss-Seidel sweep (Eq. 16), in three steps: smooth_rhs
// forms t_K = f_K - sum over interior faces of A_KN u_N (t: f_K on entry; the SBM terms lie in
// A_KK), the caller solves A_KK y = t (dense inverse for boundary cells, fast diagonalisation
// otherwise), and smooth_relax applies the relaxation factor.  zero_start: a kZero* mode (ops.h).
template <int D, int N1, typename R>
__device__ __forceinline__ void smooth_rhs(const LevelParams<R>& P, int col, int zero_start, const int (&nb)[2 * D],
                                           R (&t)[CD<D, N1>::NP], const R* __restrict__ u) {
  constexpr int NP = CD<D, N1>::NP;
  R c[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) c[i] = 0;
  int nbz[2 * D];                                   // kZeroAll: every neighbour reads as zero
#pragma unroll
  for (int q = 0; q < 2 * D; ++q) nbz[q] = zero_start == kZeroAll ? -1 : nb[q];
  add_couplings<D, N1, R, R>(P, u, col, zero_start == kZeroLater, nbz, c);
#pragma unroll
  for (int i = 0; i < NP; ++i) t[i] -= P.hscale * c[i];
}

// un = (1 - omega) u_K + omega un for cell a (u_K = 0 when zero_start).
template <int D, int N1, typename R>
__device__ __forceinline__ void smooth_relax(const LevelParams<R>& P, int zero_start, int a, const R* __restrict__ u,
                                             R (&un)[CD<D, N1>::NP]) {
  constexpr int NP = CD<D, N1>::NP;
  if (P.omega == R(1)) return;
  R uo[NP];
  if (zero_start) {
#pragma unroll
    for (int i = 0; i < NP; ++i) uo[i] = R(0);
  } else {
    load_cell<D, N1, R, R>(u, a, P.n_act, uo);
  }
#pragma unroll
  for (int i = 0; i < NP; ++i) un[i] = (R(1) - P.omega) * uo[i] + P.omega * un[i];
}
