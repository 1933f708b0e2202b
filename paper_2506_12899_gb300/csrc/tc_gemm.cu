// BF16 GEMM of the learned correction's MLP on the fifth-generation tensor cores (tcgen05, sm_100
// family): C = opA(A) opB(B) (+ bias) (ReLU), BF16 operands, FP32 accumulation in tensor memory.
//
// One CTA of 128 threads computes a 128 x 128 tile of C.  For each K chunk of 64 the threads stage
// the A tile (128 rows x 64) and the B tile (128 columns x 64) in shared memory in the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes
// apart, 8-row groups 1024 bytes apart; out-of-range rows, columns and K entries are zero.  One
// thread then issues four tcgen05.mma (M = 128, N = 128, K = 16 each) that accumulate into a
// 128 x 128 FP32 tile in tensor memory, and commits them to the stage's mbarrier.  Two stages
// alternate, so the threads stage chunk i + 1 while the tensor core works on chunk i; a stage is
// overwritten only after its commit arrived (at most kAsyncSpin polls per wait; a wait that runs out
// records the failure in a device flag, lets the MMAs in flight land and skips the epilogue).
// Finally each warp reads its 32 rows of the accumulator with tcgen05.ld and applies bias and ReLU.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ops.h"

namespace sbm {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;
constexpr int kTcThreads = 128;

__device__ int g_tc_fault = 0;

// Shared-memory matrix descriptor (tcgen05): start address, leading (K direction) and stride
// (8-row groups) byte offsets, all >> 4; bits 46-48 hold the fixed value 1; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = (uint64_t)(smem_addr(p) >> 4) & 0x3FFFu;
  return a | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row r, k) of a 128 x 64 K-major no-swizzle tile.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 8 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Stages the K chunk k0 .. k0+63 of rows r0 .. r0+127 of the operand X (op(X)(r, k) = X[r*ld + k] when
// KMAJ, else X[k*ld + r]) into the 128 x 64 K-major tile T.  16-byte pieces (8 consecutive k of one
// row, one row of a core matrix) are loaded with 16-byte loads where the piece lies inside the
// matrix and is 16-byte aligned (KMAJ); otherwise (MN-major storage: 8 consecutive r of one k, or the
// ragged edges) element by element.  Entries outside R x K are zero.
template <bool KMAJ>
__device__ __forceinline__ void stage_tile(unsigned char* T, const __nv_bfloat16* __restrict__ X, int ld, int R,
                                           int K, int r0, int k0, bool vec_ok) {
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  if (KMAJ) {
    for (int q = threadIdx.x; q < 128 * 8; q += kTcThreads) {   // piece q: row q / 8, k chunk q % 8
      const int r = q >> 3, c = q & 7;
      const int gr = r0 + r, gk = k0 + 8 * c;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gr < R) {
        const __nv_bfloat16* src = X + (size_t)gr * ld + gk;
        if (vec_ok && gk + 8 <= K) {
          v = *reinterpret_cast<const uint4*>(src);
        } else {
          __nv_bfloat16 t[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) t[j] = gk + j < K ? src[j] : zero;
          v = *reinterpret_cast<const uint4*>(t);
        }
      }
      *reinterpret_cast<uint4*>(T + tile_off(r, 8 * c)) = v;
    }
  } else {
    for (int q = threadIdx.x; q < 64 * 16; q += kTcThreads) {   // piece q: k = q / 16, rows 8 (q % 16) ..
      const int kk = q >> 4, rc = (q & 15) * 8;
      const int gk = k0 + kk, gr = r0 + rc;
      __nv_bfloat16 t[8];
      if (gk < K) {
        const __nv_bfloat16* src = X + (size_t)gk * ld + gr;
        if (vec_ok && gr + 8 <= R) {
          *reinterpret_cast<uint4*>(t) = *reinterpret_cast<const uint4*>(src);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) t[j] = gr + j < R ? src[j] : zero;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = zero;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) *reinterpret_cast<__nv_bfloat16*>(T + tile_off(rc + j, kk)) = t[j];
    }
  }
}

template <int TA, int TB>
__global__ void __launch_bounds__(kTcThreads) k_gemm_tc(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                        int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                        const float* __restrict__ bias, int relu,
                                                        float* __restrict__ Cf, __nv_bfloat16* __restrict__ Cb,
                                                        int ldc) {
  // two stages of (A tile, B tile), 32 KB each, in dynamic shared memory (1024-byte aligned)
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int stop;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {                                   // 128 FP32 columns of tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_addr(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    stop = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(TBM, TBN);
  // 16-byte loads need 16-byte aligned rows
  const bool va = (reinterpret_cast<uintptr_t>(A) & 15) == 0 && ((size_t)lda * 2) % 16 == 0;
  const bool vb = (reinterpret_cast<uintptr_t>(B) & 15) == 0 && ((size_t)ldb * 2) % 16 == 0;
  unsigned phase[2] = {0u, 0u};
  int it = 0;
  bool failed = false;
  for (int k0 = 0; k0 < K; k0 += TBK, ++it) {
    const int b = it & 1;
    unsigned char* As = tc_smem + b * 2 * (TBM * TBK * 2);
    unsigned char* Bs = As + TBM * TBK * 2;
    if (it >= 2) {                                   // the MMAs of chunk it - 2 read this stage
      const bool ok = stop ? true : mbar_wait(&bar[b], phase[b]);
      phase[b] ^= 1u;
      if (!__syncthreads_and(ok)) {
        failed = true;
        break;
      }
    }
    stage_tile<TA == 0>(As, A, lda, M, K, m0, k0, va);
    stage_tile<TB == 1>(Bs, B, ldb, N, K, n0, k0, vb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < TBK / 16; ++ks) {        // K = 16 per instruction: two core matrices
        const uint64_t ad = smem_desc(As + ks * 256, 128, 1024);
        const uint64_t bd = smem_desc(Bs + ks * 256, 128, 1024);
        const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bar[b]))
                   : "memory");
    }
  }
  // wait for the commits still outstanding (the last one or two chunks), bounded
  if (!failed) {
    bool ok = true;
    for (int j = (it >= 2 ? it - 2 : 0); j < it; ++j) {
      const int b = j & 1;
      ok = ok && mbar_wait(&bar[b], phase[b]);
      phase[b] ^= 1u;
    }
    failed = !__syncthreads_and(ok);
  }
  if (failed && threadIdx.x == 0) {                  // record it and let the MMAs in flight land
    atomicExch(&g_tc_fault, 1);
    mbar_wait(&bar[0], phase[0]);
    mbar_wait(&bar[1], phase[1]);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp w owns accumulator rows (TMEM lanes) 32 w .. 32 w + 31
  const int m = m0 + warp * 32 + lane;
  if (!failed && K > 0) {
#pragma unroll 1
    for (int c0 = 0; c0 < TBN; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
          "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c0 + j;
          if (n < N) {
            float v = __uint_as_float(r[j]);
            if (bias) v += bias[n];
            if (relu) v = fmaxf(v, 0.f);
            if (Cf) Cf[(size_t)m * ldc + n] = v;
            if (Cb) Cb[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
          }
        }
      }
    }
  } else if (K == 0 && m < M) {                      // empty contraction: C = bias (ReLU)
    for (int n = n0; n < n0 + TBN && n < N; ++n) {
      float v = bias ? bias[n] : 0.f;
      if (relu) v = fmaxf(v, 0.f);
      if (Cf) Cf[(size_t)m * ldc + n] = v;
      if (Cb) Cb[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

}  // namespace

// Two stages of 32 KB: at most 3 CTAs per SM, so the CTAs of an SM never ask for more than 3 x 128
// of its 512 tensor-memory columns (tcgen05.alloc would wait).
constexpr size_t kTcSmem = 2 * 2 * (size_t)TBM * TBK * 2;

template <int TA, int TB>
cudaError_t launch_tc(dim3 grid, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B,
                      int ldb, const float* bias, int relu, float* Cf, __nv_bfloat16* Cb, int ldc, cudaStream_t s) {
  const cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTcSmem);
  if (e != cudaSuccess) return e;
  k_gemm_tc<TA, TB><<<grid, kTcThreads, kTcSmem, s>>>(M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc);
  return cudaSuccess;
}

cudaError_t launch_gemm_tc(int M, int N, int K, int ta, int tb, const __nv_bfloat16* A, int lda,
                           const __nv_bfloat16* B, int ldb, const float* bias, int relu, float* Cf,
                           __nv_bfloat16* Cb, int ldc, cudaStream_t s) {
  if (M == 0 || N == 0) return cudaSuccess;
  const dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
  cudaError_t e;
  if (!ta && !tb) e = launch_tc<0, 0>(grid, M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc, s);
  else if (!ta && tb) e = launch_tc<0, 1>(grid, M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc, s);
  else if (ta && !tb) e = launch_tc<1, 0>(grid, M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc, s);
  else e = launch_tc<1, 1>(grid, M, N, K, A, lda, B, ldb, bias, relu, Cf, Cb, ldc, s);
  if (e != cudaSuccess) return e;
  count_launches();
  return cudaGetLastError();
}

int tc_fault_take() {
  int f = 0;
  if (cudaMemcpyFromSymbol(&f, g_tc_fault, sizeof(int)) != cudaSuccess) return -1;
  if (f) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_tc_fault, &zero, sizeof(int)) != cudaSuccess) return -1;
  }
  return f;
}

}  // namespace sbm
