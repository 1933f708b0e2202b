// C ABI of libsbm: context set-up, level operations, the V-cycle (Sec. 3) and FGMRES.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "ops.h"

namespace sbm {
namespace {

thread_local std::string g_last_error;

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                             \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) throw SetupError{SBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

template <typename R>
constexpr int prec_index() {
  return sizeof(R) == 8 ? 0 : 1;
}

struct DevLevel {
  HostLevel H;
  int* nbr = nullptr;
  double* dhat64 = nullptr;
  float* dhat32 = nullptr;
  double* binv64 = nullptr;
  float* binv32 = nullptr;
  int* parent_code = nullptr;
  int* children = nullptr;
  double* coarse_inv = nullptr;
  double* coarse_invT = nullptr;     // its transpose (the one-CTA tail reads it a row per thread)
  dfl* coarse_invT_df = nullptr;     // the transpose rounded to double-float (FP32 tail)
  LevelParams<double> P64{};
  LevelParams<float> P32{};
  LevelParams<dfl> Pdf{};         // double-float operator constants (finest level, thread-per-cell shapes)
  dfl* dhat_df = nullptr;
  dfl* bself_df = nullptr;        // dense boundary self blocks of the double-float operator
  bool has_df = false;
  TransferParams<double> T64{};   // transfer between level l-1 (coarse) and this level
  TransferParams<float> T32{};
  void* z[2] = {nullptr, nullptr};
  void* rhs[2] = {nullptr, nullptr};
  void* res[2] = {nullptr, nullptr};
  void* tmp[2] = {nullptr, nullptr};   // additive smoothers: y = D^-1 r
  void* dir[2] = {nullptr, nullptr};   // Chebyshev: the update direction d
  double lam_max = 0.0;                // Chebyshev: estimate of lambda_max(D^-1 A) (set-up)
};


// The learned boundary-cell correction: a two-hidden-layer ReLU MLP (FP32 master parameters,
// BF16 copies for the tensor-core GEMMs), its Adam state, a device training set and the
// per-batch activation buffers.  Parameters are packed W1[Fpad][H] b1[H] W2[H][H] b2[H]
// W3[H][O] b3[O] (input-major); rows F..Fpad-1 of W1 are zero and stay zero (their gradient
// is zero because the padded feature columns are zero).
// The MLP's GEMMs: tcgen05 (backend 0) or mma.sync (1).
inline cudaError_t gemm_bf16(int backend, int M, int N, int K, int ta, int tb, const __nv_bfloat16* A, int lda,
                             const __nv_bfloat16* B, int ldb, const float* bias, int relu, float* Cf,
                             __nv_bfloat16* Cb, int ldc, cudaStream_t s) {
  return backend == 0 ? launch_gemm_tc(M, N, K, ta, tb, A, lda, B, ldb, bias, relu, Cf, Cb, ldc, s)
                      : launch_gemm_bf16(M, N, K, ta, tb, A, lda, B, ldb, bias, relu, Cf, Cb, ldc, s);
}

struct Mlp {
  int dim = 2, p = 1, np = 4, npatch = 9, nstat = 0, F = 0, Fpad = 0, H = 128, O = 4;
  size_t nparam = 0, oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  float* P = nullptr;                // master parameters
  float* G = nullptr;                // gradients
  float* Am = nullptr;               // Adam first moments
  float* Av = nullptr;               // Adam second moments
  __nv_bfloat16* Pb = nullptr;       // BF16 copy of the parameters
  int adam_t = 0;
  int gemm = 0;                      // 0: tcgen05 tensor cores (tc_gemm.cu), 1: warp-level mma.sync
  size_t cap = 0, count = 0;         // training set rows
  __nv_bfloat16* Xd = nullptr;       // [cap][Fpad]
  float* Td = nullptr;               // [cap][O]
  int* idx_all = nullptr;            // [cap] epoch permutation
  int bcap = 0;                      // batch buffers
  __nv_bfloat16 *Xb = nullptr, *H1 = nullptr, *H2 = nullptr, *dYb = nullptr, *dZ2b = nullptr, *dZ1b = nullptr;
  float *Tb = nullptr, *Y = nullptr, *dYf = nullptr, *dH2 = nullptr, *dH1 = nullptr, *loss_part = nullptr,
        *loss_tmp = nullptr, *loss_acc = nullptr;
  ~Mlp() {
    for (void* q : allocs) cudaFree(q);
  }
  template <typename T>
  T* alloc(size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(T));
    if (e != cudaSuccess) throw SetupError{SBM_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    allocs.push_back(q);
    return static_cast<T*>(q);
  }
  void release(void* q) {
    if (!q) return;
    for (auto it = allocs.begin(); it != allocs.end(); ++it)
      if (*it == q) {
        cudaFree(q);
        allocs.erase(it);
        return;
      }
  }
  const __nv_bfloat16* W1b() const { return Pb + oW1; }
  const __nv_bfloat16* W2b() const { return Pb + oW2; }
  const __nv_bfloat16* W3b() const { return Pb + oW3; }
  void ensure_batch(int B) {
    if (B <= bcap) return;
    for (void* q : {(void*)Xb, (void*)H1, (void*)H2, (void*)dYb, (void*)dZ2b, (void*)dZ1b, (void*)Tb, (void*)Y,
                    (void*)dYf, (void*)dH2, (void*)dH1})
      release(q);
    Xb = alloc<__nv_bfloat16>((size_t)B * Fpad);
    H1 = alloc<__nv_bfloat16>((size_t)B * H);
    H2 = alloc<__nv_bfloat16>((size_t)B * H);
    dYb = alloc<__nv_bfloat16>((size_t)B * O);
    dZ2b = alloc<__nv_bfloat16>((size_t)B * H);
    dZ1b = alloc<__nv_bfloat16>((size_t)B * H);
    Tb = alloc<float>((size_t)B * O);
    Y = alloc<float>((size_t)B * O);
    dYf = alloc<float>((size_t)B * O);
    dH2 = alloc<float>((size_t)B * H);
    dH1 = alloc<float>((size_t)B * H);
    bcap = B;
  }
  // Training-set capacity for `rows` rows, keeping the stored ones.
  void reserve(size_t rows) {
    if (rows <= cap) return;
    const size_t ncap = std::max(rows, cap * 2);
    __nv_bfloat16* nX = alloc<__nv_bfloat16>(ncap * Fpad);
    float* nT = alloc<float>(ncap * O);
    if (count) {
      CUDA_TRY(cudaMemcpyAsync(nX, Xd, count * Fpad * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(nT, Td, count * O * sizeof(float), cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    }
    release(Xd);
    release(Td);
    release(idx_all);
    Xd = nX;
    Td = nT;
    idx_all = alloc<int>(ncap);
    cap = ncap;
  }
  // Yout[rows][O] = MLP(X) with the BF16 weights, hidden activations into h1, h2 ([rows][H]).
  void forward(const __nv_bfloat16* X, int rows, float* Yout, __nv_bfloat16* h1, __nv_bfloat16* h2,
               cudaStream_t st) const {
    CUDA_TRY(gemm_bf16(gemm, rows, H, Fpad, 0, 0, X, Fpad, W1b(), H, P + ob1, 1, nullptr, h1, H, st));
    CUDA_TRY(gemm_bf16(gemm, rows, H, H, 0, 0, h1, H, W2b(), H, P + ob2, 1, nullptr, h2, H, st));
    CUDA_TRY(gemm_bf16(gemm, rows, O, H, 0, 0, h2, H, W3b(), O, P + ob3, 0, Yout, nullptr, O, st));
  }
  // G = gradient of the mean squared error over the rows of (X, T), after forward(X, rows, Y,
  // H1, H2); loss_part receives per-block partial sums of the squared errors.
  void backward(const __nv_bfloat16* X, const float* T, int rows) {
    CUDA_TRY(launch_mse_grad(rows, O, Y, T, dYf, dYb, 1.0f / ((float)rows * O), loss_part, 152, s));
    CUDA_TRY(gemm_bf16(gemm, H, O, rows, 1, 0, H2, H, dYb, O, nullptr, 0, G + oW3, nullptr, O, s));
    CUDA_TRY(launch_colsum(rows, O, dYf, G + ob3, s));
    CUDA_TRY(gemm_bf16(gemm, rows, H, O, 0, 1, dYb, O, W3b(), O, nullptr, 0, dH2, nullptr, H, s));
    CUDA_TRY(launch_relu_mask(rows * H, dH2, H2, dZ2b, s));
    CUDA_TRY(gemm_bf16(gemm, H, H, rows, 1, 0, H1, H, dZ2b, H, nullptr, 0, G + oW2, nullptr, H, s));
    CUDA_TRY(launch_colsum(rows, H, dH2, G + ob2, s));
    CUDA_TRY(gemm_bf16(gemm, rows, H, H, 0, 1, dZ2b, H, W2b(), H, nullptr, 0, dH1, nullptr, H, s));
    CUDA_TRY(launch_relu_mask(rows * H, dH1, H1, dZ1b, s));
    CUDA_TRY(gemm_bf16(gemm, Fpad, H, rows, 1, 0, X, Fpad, dZ1b, H, nullptr, 0, G + oW1, nullptr, H, s));
    CUDA_TRY(launch_colsum(rows, H, dH1, G + ob1, s));
  }
};

struct Context {
  sbm_setup_desc desc{};
  cudaStream_t stream = nullptr;
  std::vector<DevLevel> lv;
  std::vector<double> rhs_host;
  std::vector<void*> allocs;
  bool work_ready[2] = {false, false};
  int tail_cand = -1;                // highest level the cluster tail may start at (-1: none)
  TailPlan tail_plan[2];             // per precision: levels 0..top in one cluster launch
  void* tail[2] = {nullptr, nullptr};  // TailLevel<double> / TailLevel<float> arrays
  std::unique_ptr<TailCta<double>> tail_cta64;   // one-CTA tail parameter blocks
  std::unique_ptr<TailCta<float>> tail_cta32;
  // FGMRES workspace
  int ws_m = 0, ws_prec = -1;
  double* V = nullptr;               // FP64 basis [m+1][N] (krylov_basis = 1)
  float2* V2 = nullptr;              // double-float basis [m+1][ldv] (krylov_basis = 0)
  size_t ldv = 0;                    // leading dimension of V2: N rounded up to 32 entries
  float2* wdf = nullptr;             // w as double-float between the Gram-Schmidt sweeps
  void* Z = nullptr;
  double* w = nullptr;
  float* r32 = nullptr;
  double* v64 = nullptr;             // FP64 copy of v_j for the FP64 V-cycle on a double-float basis
  int ws_basis = -1;
  double* partial = nullptr;
  double* dots = nullptr;          // [0,32) h1, [32,64) h2, [64] norm, [96, 128) Hessenberg column
  double* ydev = nullptr;
  double* bbuf = nullptr;
  double* xbuf = nullptr;
  double* host_pinned = nullptr;   // 192 doubles: [0,64) scalars and y; [64,128), [128,192) the
                                   // Hessenberg columns of even and odd Arnoldi steps
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t step_done[2] = {};   // end of the last even / odd Arnoldi step launched
  bool host_only = false;
  double* dots_scratch = nullptr;  // partial sums of sbm_dots
  size_t dots_scratch_len = 0;
  // sbm_gram_schmidt: its own copy of the basis and of w (padded rows), partial sums and results
  float2* gsV2 = nullptr;          // [32][ldv] double-float basis rows
  double* gsw = nullptr;           // [ldv] w, FP64
  float2* gswdf = nullptr;         // [ldv] w, double-float
  double* gspartial = nullptr;
  double* gsdots = nullptr;        // [0,32) h1, [32,64) h2, [64] |w|, [65] 1.0, [128,161) column
  // sbm_l2_error: background indices of the finest cells, partial sums, result
  int* l2cell = nullptr;
  double* l2partial = nullptr;
  double* l2out = nullptr;
  // FGMRES runs on an internal non-blocking stream (the legacy default stream cannot be captured
  // into a graph), joined to the caller's stream with events.  Each Arnoldi step j of each
  // V-cycle precision is captured once into a CUDA graph and replayed.
  cudaStream_t ws = nullptr;
  cudaEvent_t join_in = nullptr, join_out = nullptr;
  cudaGraphExec_t arnoldi[2][2][32] = {};   // [precision][learned correction on][j]
  long long arnoldi_kernels[2][2][32] = {};
  // learned boundary-cell correction attached to this context (not owned)
  Mlp* mlp = nullptr;
  bool mlp_on = false;                 // correction active in the next V-cycles
  float mlp_scale = 1.f;
  double mlp_rate_ref = 0.0;           // fallback when the per-step rate is worse than this (0: never)
  // finest-level feature data (uploaded on first use) and inference buffers
  int lf_F = 0, lf_Fpad = 0, lf_npatch = 0, lf_nstat = 0, lf_nb = 0;
  int* mlp_cells = nullptr;            // [n_bnd] compact cell of each boundary cell (finest level)
  int* mlp_patch = nullptr;            // [n_bnd][3^d]
  float* mlp_stat = nullptr;           // [n_bnd][nstat]
  __nv_bfloat16* mlp_X = nullptr;      // [n_bnd][Fpad] inference features
  float* mlp_s = nullptr;              // [n_bnd]
  int mlp_bufH = 0, mlp_bufO = 0;      // sizes of the buffers below
  float* mlp_Y = nullptr;              // [n_bnd][O]
  __nv_bfloat16* mlp_H1 = nullptr;     // [n_bnd][H]
  __nv_bfloat16* mlp_H2 = nullptr;
  void* col_vec[2][4] = {};            // training-data collection: u, rhs, z, zero (per precision)

  void drop_graphs() {
    for (auto& a : arnoldi)
      for (auto& row : a)
        for (auto& g : row)
          if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
          }
  }

  ~Context() {
    drop_graphs();
    if (ws) cudaStreamDestroy(ws);
    if (join_in) cudaEventDestroy(join_in);
    if (join_out) cudaEventDestroy(join_out);
    for (void* p : allocs) cudaFree(p);
    if (host_pinned) cudaFreeHost(host_pinned);
    for (cudaEvent_t e : step_done)
      if (e) cudaEventDestroy(e);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }

  template <typename T>
  T* dalloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) throw SetupError{SBM_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    allocs.push_back(p);
    return static_cast<T*>(p);
  }
  template <typename T>
  T* upload(const std::vector<T>& v) {
    T* p = dalloc<T>(v.size());
    if (!v.empty()) CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  int finest() const { return (int)lv.size() - 1; }
};

template <typename R>
const LevelParams<R>& params(const DevLevel& L);
template <>
const LevelParams<double>& params<double>(const DevLevel& L) { return L.P64; }
template <>
const LevelParams<float>& params<float>(const DevLevel& L) { return L.P32; }
template <typename R>
const TransferParams<R>& tparams(const DevLevel& L);
template <>
const TransferParams<double>& tparams<double>(const DevLevel& L) { return L.T64; }
template <>
const TransferParams<float>& tparams<float>(const DevLevel& L) { return L.T32; }

template <typename R>
LevelParams<R> make_params(const DevLevel& D, const R* dhat, const R* binv) {
  const HostLevel& H = D.H;
  LevelParams<R> P;
  std::memset(&P, 0, sizeof(P));
  P.n_act = H.n_act;
  for (int c = 0; c < 9; ++c) P.colour_start[c] = H.colour_start[c];
  for (int c = 0; c < 8; ++c) {
    P.colour_nbnd[c] = H.colour_nbnd[c];
    P.bstart[c] = H.bstart[c];
  }
  P.nbr = D.nbr;
  P.dhat = dhat;
  P.binvT = binv;
  P.hscale = (R)std::pow(H.h, H.dim - 2);
  P.sigG = (R)H.sigG_hat;
  P.alpha = (R)H.alpha;
  P.omega = (R)H.omega;
  P.extension = H.extension;
  const int n1 = H.n1;
  for (int m = 0; m < 4; ++m)
    for (int ij = 0; ij < n1 * n1; ++ij) P.k.L[m][ij] = (R)H.L[m][ij];
  for (int ij = 0; ij < n1 * n1; ++ij) {
    P.k.Bmp[ij] = (R)H.Bmp[ij];
    P.k.Bpm[ij] = (R)H.Bpm[ij];
    P.k.Kh[ij] = (R)H.B.Khat[ij];
    P.k.Bmm[ij] = (R)H.Bmm[ij];
    P.k.Bpp[ij] = (R)H.Bpp[ij];
    P.k.Dm[ij] = (R)H.B.Dm[ij];
    P.k.S[ij] = (R)H.S[ij];
  }
  for (int k = 0; k < n1; ++k) {
    P.k.w[k] = (R)H.B.w[k];
    P.k.e0[k] = (R)H.B.e0[k];
    P.k.e1[k] = (R)H.B.e1[k];
    P.k.d0[k] = (R)H.B.d0[k];
    P.k.d1[k] = (R)H.B.d1[k];
    P.k.x[k] = (R)H.B.x[k];
    double den = 1.0;
    for (int j = 0; j < n1; ++j)
      if (j != k) den *= H.B.x[k] - H.B.x[j];
    P.k.inv_denom[k] = (R)(1.0 / den);
    P.k.lam[k] = (R)H.lam[k];
  }
  const double hs = std::pow(H.h, H.dim - 2);
  for (int i = 0; i < H.np; ++i) {
    double ls = H.lam[i % n1] + H.lam[(i / n1) % n1];
    if (H.dim == 3) ls += H.lam[i / (n1 * n1)];
    P.k.inv_diag[i] = (R)(1.0 / (hs * ls));
  }
  return P;
}

template <typename R>
TransferParams<R> make_transfer(const DevLevel& C, const DevLevel& F) {
  TransferParams<R> T;
  std::memset(&T, 0, sizeof(T));
  T.n_act_f = F.H.n_act;
  T.n_act_c = C.H.n_act;
  T.hmode = C.H.n != F.H.n;
  T.parent_code = F.parent_code;
  T.children = C.children;
  const int nf = F.H.n1, nc = C.H.n1;
  double v[kMaxN1];
  for (int o = 0; o < 2; ++o)
    for (int i = 0; i < nf; ++i) {
      lagrange_eval(nc, C.H.B.x, 0.5 * (o + F.H.B.x[i]), v, nullptr);
      for (int j = 0; j < nc; ++j) T.Ph[o][i * nc + j] = (R)v[j];
    }
  for (int i = 0; i < nf; ++i) {
    lagrange_eval(nc, C.H.B.x, F.H.B.x[i], v, nullptr);
    for (int j = 0; j < nc; ++j) T.Pp[i * nc + j] = (R)v[j];
  }
  return T;
}

template <typename T>
std::vector<float> to_f32(const std::vector<T>& v) {
  return std::vector<float>(v.begin(), v.end());
}

void validate(const sbm_setup_desc& d) {
  auto bad = [](const std::string& m) { throw SetupError{SBM_ERR_ARG, m}; };
  if (d.dim != 2 && d.dim != 3) bad("dim must be 2 or 3");
  if (d.p < 1 || d.p > 3) bad("p must be 1, 2 or 3");
  if (d.n < 1 || d.n > 4096) bad("n out of range");
  if (d.coarsest_n < 1) bad("coarsest_n must be >= 1");
  if (!(d.lambda >= 0.0 && d.lambda <= 1.0)) bad("lambda must lie in [0,1]");
  if (d.pre_smooth < 0 || d.post_smooth < 0 || d.pre_smooth > 16 || d.post_smooth > 16) bad("smoothing steps");
  if (d.ssor_each != 0 && d.ssor_each != 1) bad("ssor_each must be 0 or 1");
  if (d.precision != SBM_F64 && d.precision != SBM_F32) bad("precision must be SBM_F64 or SBM_F32");
  if (d.extension != 0 && d.extension != 1) bad("extension must be 0 or 1");
  if (d.krylov_basis < 0 || d.krylov_basis > 2) bad("krylov_basis must be 0, 1 or 2");
  if (d.smoother < 0 || d.smoother > 2) bad("smoother must be 0, 1 or 2");
  if (d.ordering != 0 && d.ordering != 1) bad("ordering must be 0 or 1");
  if (d.smoother == 2 && (d.cheb_degree < 1 || d.cheb_degree > 16 || !(d.cheb_ratio > 1.0)))
    bad("Chebyshev smoother: 1 <= cheb_degree <= 16 and cheb_ratio > 1");
  if (d.tail_cluster_ctas < 0 || d.tail_cluster_ctas > 16 || (d.tail_cluster_ctas & (d.tail_cluster_ctas - 1)))
    bad("tail_cluster_ctas must be 0, 1, 2, 4, 8 or 16");
  const double w0 = d.hi[0] - d.lo[0];
  if (!(w0 > 0) || !std::isfinite(w0)) bad("empty or non-finite box");
  for (int k = 1; k < d.dim; ++k)
    if (!(std::fabs((d.hi[k] - d.lo[k]) - w0) <= 1e-12 * w0)) bad("cells must be square: equal box extents");
  if (!(d.sigma_face_c > 0 && d.sigma_bnd_c >= 0)) bad("penalty constants");
  if (d.shape.kind < 0 || d.shape.kind > 4) bad("unknown shape");
  if (d.shape.kind == SBM_SHAPE_STAR && d.dim != 2) bad("star shape is 2D");
  if (d.shape.kind == SBM_SHAPE_COMPLEX2D && d.dim != 2) bad("complex2d shape is 2D");
  if (d.shape.kind == SBM_SHAPE_ELLIPSOID && d.dim != 3) bad("ellipsoid shape is 3D");
}

// Start vector of the power iteration: entry (cell, node l) = 1 + 0.5 sin(0.7 (i + 2.1 j + 3.3 k) +
// 1.3 l) from the cell's background index, the same vector in any cell order.
std::vector<double> power_start(const HostLevel& H) {
  std::vector<double> v((size_t)H.n_dof());
  for (int a = 0; a < H.n_act; ++a) {
    const double base = H.cell[3 * a] + 2.1 * H.cell[3 * a + 1] + (H.dim == 3 ? 3.3 * H.cell[3 * a + 2] : 0.0);
    for (int l = 0; l < H.np; ++l) v[(size_t)a * H.np + l] = 1.0 + 0.5 * std::sin(0.7 * base + 1.3 * l);
  }
  return v;
}

constexpr int kPowerSteps = 15;       // power-iteration steps for lambda_max(D^-1 A)
constexpr double kChebSafety = 1.1;   // upper end of the Chebyshev interval: 1.1 times the estimate

// lambda_max(D^-1 A) of every level above the coarsest by kPowerSteps power-iteration steps in FP64
// on the device: w = D^-1 (A v) (the operator, then the block solves of the smoother kernels with
// every neighbour read as zero and omega = 1), lambda = |w| / |v|, v <- w (the normalisation of v
// before each step is folded into the quotient).
void estimate_lambda_max(Context& C) {
  const cudaStream_t s = C.stream;
  for (size_t l = 1; l < C.lv.size(); ++l) {
    DevLevel& L = C.lv[l];
    const size_t N = L.H.n_dof();
    double* v = C.dalloc<double>(N);
    double* av = C.dalloc<double>(N);
    double* w = C.dalloc<double>(N);
    double* part = C.dalloc<double>((size_t)dot_blocks(N) * 32);
    double* nrm = C.dalloc<double>(2);
    const std::vector<double> v0 = power_start(L.H);
    CUDA_TRY(cudaMemcpy(v, v0.data(), N * sizeof(double), cudaMemcpyHostToDevice));
    LevelParams<double> P1 = L.P64;
    P1.omega = 1.0;
    double lam = 0.0;
    for (int it = 0; it < kPowerSteps; ++it) {
      CUDA_TRY((launch_apply<double, double>(L.H.dim, L.H.p, L.P64, v, nullptr, av, 0, s)));
      CUDA_TRY(launch_smooth<double>(L.H.dim, L.H.p, P1, 0, kZeroAll, av, w, s));
      CUDA_TRY(launch_multi_dot(v, N, 1, v, N, part, nrm, 1, s));
      CUDA_TRY(launch_multi_dot(w, N, 1, w, N, part, nrm + 1, 1, s));
      CUDA_TRY(cudaMemcpyAsync(C.host_pinned, nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      lam = C.host_pinned[1] / C.host_pinned[0];
      std::swap(v, w);
    }
    L.lam_max = lam;
  }
}

Context* build_context(const sbm_setup_desc& d, bool device) {
  validate(d);
  auto C = std::make_unique<Context>();
  C->desc = d;
  C->stream = static_cast<cudaStream_t>(d.stream);
  std::vector<int> ns{d.n};
  while (ns.back() % 2 == 0 && ns.back() / 2 >= d.coarsest_n) ns.push_back(ns.back() / 2);
  std::vector<std::pair<int, int>> seq;
  for (auto it = ns.rbegin(); it != ns.rend(); ++it) seq.emplace_back(*it, 1);
  for (int q = 2; q <= d.p; ++q) seq.emplace_back(d.n, q);
  std::vector<int> counts;                 // volume-fraction counts of the last mesh size built
  int counts_n = -1;
  for (auto& np : seq) {
    DevLevel L;
    if (np.first != counts_n) counts.clear();
    counts_n = np.first;
    L.H = build_level(d, np.first, np.second, device, &counts);
    if (L.H.n_act == 0) {
      C->lv.clear();                       // an empty level: everything coarser is dropped
      continue;
    }
    C->lv.push_back(std::move(L));
  }
  if (C->lv.empty()) throw SetupError{SBM_ERR_GEOMETRY, "finest level has no active cells"};
  for (size_t l = 1; l < C->lv.size(); ++l) link_levels(C->lv[l - 1].H, C->lv[l].H);
  build_coarse_inverse(C->lv[0].H);
  C->rhs_host = build_rhs(d, C->lv.back().H);
  if (!device) return C.release();
  for (auto& L : C->lv) {
    L.nbr = C->upload(L.H.nbr);
    L.dhat64 = C->upload(L.H.dhat);
    L.dhat32 = C->upload(to_f32(L.H.dhat));
    L.binv64 = C->upload(L.H.binvT);
    L.binv32 = C->upload(to_f32(L.H.binvT));
    if (!L.H.parent_code.empty()) L.parent_code = C->upload(L.H.parent_code);
    if (!L.H.children.empty()) L.children = C->upload(L.H.children);
    if (!L.H.coarse_inv.empty()) {
      L.coarse_inv = C->upload(L.H.coarse_inv);
      const size_t n = L.H.n_dof();
      std::vector<double> t(n * n);
      for (size_t i = 0; i < n; ++i)
        for (size_t j = 0; j < n; ++j) t[j * n + i] = L.H.coarse_inv[i * n + j];
      L.coarse_invT = C->upload(t);
      std::vector<dfl> tdf(t.size());
      for (size_t i = 0; i < t.size(); ++i) tdf[i] = dfl(t[i]);
      L.coarse_invT_df = C->upload(tdf);
    }
    L.P64 = make_params<double>(L, L.dhat64, L.binv64);
    L.P32 = make_params<float>(L, L.dhat32, L.binv32);
    L.P64.ordering = L.P32.ordering = d.ordering;
    if (&L == &C->lv.back()) {                     // Arnoldi operator in double-float
      std::vector<dfl> dh(L.H.dhat.size());
      for (size_t i = 0; i < dh.size(); ++i) dh[i] = dfl(L.H.dhat[i]);
      L.dhat_df = C->upload(dh);
      L.Pdf = make_params<dfl>(L, L.dhat_df, nullptr);
      L.has_df = true;
      // 3D p = 1: the boundary cells' self blocks h^(d-2) A_KK, assembled in FP64 column by column
      // with the host operator and rounded to double-float; the thread-per-cell operator applies
      // them densely instead of evaluating the surrogate-face terms (blocks padded to an even
      // length so that every block starts on a 16-byte boundary).  2D keeps the surrogate-face
      // terms: there the dense blocks made the solve slower.
      const HostLevel& H = L.H;
      if (H.dim == 3 && H.p == 1 && H.n_bnd > 0) {
        const int np = H.np, ld = (np * np + 1) & ~1;
        std::vector<dfl> bs((size_t)H.n_bnd * ld, dfl(0.0));
        std::vector<double> e(np), col(np);
        for (int c = 0; c < H.ncol; ++c)
          for (int off = 0; off < H.colour_nbnd[c]; ++off) {
            const int a = H.colour_start[c] + off, b = H.bstart[c] + off;
            for (int j = 0; j < np; ++j) {
              std::fill(e.begin(), e.end(), 0.0);
              e[j] = 1.0;
              cell_self_apply(H, a, b, e.data(), col.data());
              for (int i = 0; i < np; ++i) bs[(size_t)b * ld + (size_t)j * np + i] = dfl(col[i]);
            }
          }
        L.bself_df = C->upload(bs);
        L.Pdf.bself = L.bself_df;
        L.Pdf.bself_ld = ld;
      }
    }
    // default: thread-per-cell kernels for FP32 (measured faster at every size from 512^2 to
    // 2048^2 cells), per-dof block kernels for FP64 (FP64 ALU bound; measured faster)
    if (d.cell_kernel_min_cells == 0) {
      L.P32.cell_min = 1;
      L.P64.cell_min = 0;
    } else {
      L.P64.cell_min = L.P32.cell_min = d.cell_kernel_min_cells < 0 ? 0 : d.cell_kernel_min_cells;
    }
    L.Pdf.cell_min = L.P32.cell_min;               // the double-float operator follows the FP32 choice
    // staged thread-per-cell kernels (FP32): launches over at least staged_min cells
    L.P32.staged_min = d.staged_min_cells == 0 ? 0 : (d.staged_min_cells < 0 ? 0 : d.staged_min_cells);
  }
  for (size_t l = 1; l < C->lv.size(); ++l) {
    C->lv[l].T64 = make_transfer<double>(C->lv[l - 1], C->lv[l]);
    C->lv[l].T32 = make_transfer<float>(C->lv[l - 1], C->lv[l]);
  }
  {
    const long long cap = d.tail_max_cells == 0 ? (1LL << 40) : d.tail_max_cells;
    int top = -1;
    for (int l = 0; l < (int)C->lv.size(); ++l) {
      const HostLevel& H = C->lv[l].H;
      const bool h_level = l == 0 || (H.n == 2 * C->lv[l - 1].H.n && H.p == 1);
      if (H.p != 1 || !h_level || H.n_act > cap) break;
      top = l;
    }
    // the one-launch tail runs the coloured Gauss-Seidel of the 2^d-colour ordering only
    C->tail_cand = cap > 0 && top >= 1 && d.smoother == 0 && d.ordering == 0 ? top : -1;
  }
  CUDA_TRY(cudaMallocHost(&C->host_pinned, 192 * sizeof(double)));
  if (d.smoother == 2) estimate_lambda_max(*C);
  CUDA_TRY(cudaEventCreate(&C->ev0));
  CUDA_TRY(cudaEventCreate(&C->ev1));
  CUDA_TRY(cudaStreamCreateWithFlags(&C->ws, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&C->join_in, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&C->join_out, cudaEventDisableTiming));
  for (cudaEvent_t& e : C->step_done) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CUDA_TRY(cudaDeviceSynchronize());
  return C.release();
}

template <typename R>
void ensure_work(Context& C) {
  const int pi = prec_index<R>();
  if (C.work_ready[pi]) return;
  for (auto& L : C.lv) {
    size_t N = L.H.n_dof();
    L.z[pi] = C.dalloc<R>(N);
    L.rhs[pi] = C.dalloc<R>(N);
    L.res[pi] = C.dalloc<R>(N);
    if (C.desc.smoother != 0) {
      L.tmp[pi] = C.dalloc<R>(N);
      if (C.desc.smoother == 2) L.dir[pi] = C.dalloc<R>(N);
    }
  }
  // cluster tail: the highest candidate level whose vectors (levels 0..top) fit in the shared
  // memory of a resident cluster of 16, else 8, CTAs
  C.tail_plan[pi] = TailPlan{};
  const int NP = C.lv[0].H.dim == 2 ? 4 : 8;
  // default (tail_max_cells = 0): the one-CTA tail for FP32 V-cycles, none for FP64 ones (one
  // SM's FP64 pipe makes it slower than per-level launches: measured)
  const bool tail_default = C.desc.tail_max_cells == 0;
  const int ctas = C.desc.tail_cluster_ctas == 0 ? 1 : C.desc.tail_cluster_ctas;
  if (ctas == 1 && !(tail_default && sizeof(R) == 8)) {
    // one CTA: the highest candidate level whose data (levels 0..top) fit in its shared memory
    const int dim = C.lv[0].H.dim, ncol = 1 << dim;
    for (int top = std::min(C.tail_cand, kMaxTailCta - 1); top >= 1; --top) {
      auto tp = std::make_unique<TailCta<R>>();
      std::memset(tp.get(), 0, sizeof(TailCta<R>));
      size_t re = 0, ie = 0;                        // R elements, ints
      // every array starts on a 16-byte boundary, so that bulk copies can stage the tables
      const size_t ra = 16 / sizeof(R), ia = 4;
      auto up = [](size_t v, size_t a) { return (v + a - 1) / a * a; };
      bool aligned = true;
      auto al16 = [&](const void* p) { aligned = aligned && reinterpret_cast<uintptr_t>(p) % 16 == 0; };
      for (int l = 0; l <= top; ++l) {
        const HostLevel& H = C.lv[l].H;
        tp->P[l] = params<R>(C.lv[l]);
        if (l >= 1) tp->T[l] = tparams<R>(C.lv[l]);
        tp->n_bnd[l] = H.n_bnd;
        tp->zoff[l] = (int)re;
        re = up(re + (size_t)H.n_act * NP, ra);
        tp->roff[l] = (int)re;
        re = up(re + (size_t)H.n_act * NP, ra);
        tp->boff[l] = (int)re;
        re = up(re + (size_t)H.n_bnd * NP * NP, ra);
        tp->noff[l] = (int)ie;
        ie = up(ie + (size_t)2 * dim * H.n_act, ia);
        al16(tp->P[l].nbr);
        al16(tp->P[l].binvT);
        if (l >= 1) {
          tp->coff[l] = (int)ie;
          ie = up(ie + (size_t)ncol * C.lv[l - 1].H.n_act, ia);
          tp->poff[l] = (int)ie;
          ie = up(ie + (size_t)H.n_act, ia);
          al16(tp->T[l].children);
          al16(tp->T[l].parent_code);
        }
      }
      tp->bulk = aligned ? 1 : 0;
      const size_t int_base = (re * sizeof(R) + 15) / 16 * 16;
      size_t smem = int_base + ie * sizeof(int);
      // the coarse inverse (FP64, n0 x n0) joins the staged data when it fits
      const size_t n0 = (size_t)C.lv[0].H.n_act * NP;
      const size_t cinv_off = up(smem, 16), smem_c = cinv_off + n0 * n0 * sizeof(double);
      tp->cinv_off = 0;
      const void* cinvT = sizeof(R) == 4 ? static_cast<const void*>(C.lv[0].coarse_invT_df)
                                         : static_cast<const void*>(C.lv[0].coarse_invT);
      if (cinvT && reinterpret_cast<uintptr_t>(cinvT) % 16 == 0 &&
          tail_cta_fits(dim, pi, smem_c, sizeof(TailCta<R>))) {
        tp->cinv_off = (unsigned)cinv_off;
        smem = smem_c;
      }
      tp->top = top;
      tp->pre = C.desc.pre_smooth;
      tp->post = C.desc.post_smooth;
      tp->ssor = C.desc.ssor_each;
      tp->int_base = (unsigned)int_base;
      if (!tail_cta_fits(dim, pi, smem, sizeof(TailCta<R>))) continue;
      C.tail_plan[pi].top = top;
      C.tail_plan[pi].cluster = 1;
      C.tail_plan[pi].smem_bytes = smem;
      if constexpr (sizeof(R) == 8) C.tail_cta64 = std::move(tp);
      else C.tail_cta32 = std::move(tp);
      break;
    }
  }
  std::vector<int> sizes = {ctas};
  if (ctas == 1 || (tail_default && sizeof(R) == 8)) sizes.clear();
  for (int size : sizes) {
    if (C.tail_plan[pi].top >= 1) break;
    for (int top = C.tail_cand; top >= 1; --top) {
      std::vector<TailLevel<R>> tl(top + 1);
      size_t elems = 0;
      for (int l = 0; l <= top; ++l) {
        std::memset(&tl[l], 0, sizeof(TailLevel<R>));
        tl[l].P = params<R>(C.lv[l]);
        if (l >= 1) tl[l].T = tparams<R>(C.lv[l]);
        int ncell = 0;
        for (int c = 0; c < (1 << C.lv[l].H.dim); ++c) {
          const int cnt = tl[l].P.colour_start[c + 1] - tl[l].P.colour_start[c];
          tl[l].m[c] = (cnt + size - 1) / size;
          tl[l].off[c] = ncell;
          ncell += tl[l].m[c];
        }
        tl[l].ncell = ncell;
        tl[l].zoff = (int)elems;
        tl[l].roff = (int)(elems + (size_t)ncell * NP);
        elems += 2 * (size_t)ncell * NP;
      }
      const int gather_off = (int)elems;
      elems += (size_t)C.lv[0].H.n_act * NP;
      const size_t smem = elems * sizeof(R);
      if (!tail_cluster_fits(C.lv[0].H.dim, pi, size, smem)) continue;
      TailLevel<R>* d = C.dalloc<TailLevel<R>>(tl.size());
      CUDA_TRY(cudaMemcpy(d, tl.data(), tl.size() * sizeof(TailLevel<R>), cudaMemcpyHostToDevice));
      C.tail[pi] = d;
      C.tail_plan[pi].top = top;
      C.tail_plan[pi].cluster = size;
      C.tail_plan[pi].smem_bytes = smem;
      C.tail_plan[pi].gather_off = gather_off;
      break;
    }
  }
  C.work_ready[pi] = true;
}

// Feature layout of the finest level: F = 3^d (p+1)^d patch values + 2d (p+1)^(d-1) d face
// components + kappa + 2d face mask, padded to a multiple of 32; uploads the patch table, the
// static features and the boundary-cell list on first use.
void ensure_learned(Context& C) {
  if (C.lf_F > 0) return;
  const HostLevel& H = C.lv[C.finest()].H;
  const int dim = H.dim, np = H.np, nq = H.nq;
  C.lf_npatch = dim == 2 ? 9 : 27;
  C.lf_nstat = 2 * dim * nq * dim + 1 + 2 * dim;
  C.lf_F = C.lf_npatch * np + C.lf_nstat;
  C.lf_Fpad = (C.lf_F + 31) / 32 * 32;
  C.lf_nb = H.n_bnd;
  const int nb = H.n_bnd;
  C.mlp_cells = C.dalloc<int>(nb);
  C.mlp_patch = C.dalloc<int>((size_t)nb * C.lf_npatch);
  C.mlp_stat = C.dalloc<float>((size_t)nb * C.lf_nstat);
  C.mlp_X = C.dalloc<__nv_bfloat16>((size_t)nb * C.lf_Fpad);
  C.mlp_s = C.dalloc<float>(nb);
  std::vector<float> st(H.mlp_static.begin(), H.mlp_static.end());
  if (nb) {
    CUDA_TRY(cudaMemcpy(C.mlp_cells, H.bnd_cell.data(), nb * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(C.mlp_patch, H.patch.data(), H.patch.size() * sizeof(int), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(C.mlp_stat, st.data(), st.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
}

// Learned boundary-cell correction after the finest-level post-smoothing: features from the
// residual r - A z, then z_K += scale * s_K * MLP(x_K) on every boundary cell.
template <typename R>
void apply_learned(Context& C, DevLevel& L, const R* r, R* z, cudaStream_t s) {
  const Mlp& M = *C.mlp;
  const int pi = prec_index<R>();
  R* res = static_cast<R*>(L.res[pi]);
  CUDA_TRY((launch_apply<R, R>(L.H.dim, L.H.p, params<R>(L), z, r, res, 1, s)));
  const int nb = C.lf_nb;
  CUDA_TRY(launch_mlp_features<R>(nb, C.lf_npatch, L.H.np, C.lf_nstat, C.lf_Fpad, C.mlp_patch, C.mlp_stat, res,
                                  C.mlp_X, C.mlp_s, s));
  M.forward(C.mlp_X, nb, C.mlp_Y, C.mlp_H1, C.mlp_H2, s);
  // the network predicts the correction in units of s h^(2-d) (A scales like h^(d-2))
  const float hs = (float)std::pow(L.H.h, 2 - L.H.dim);
  CUDA_TRY(launch_mlp_scatter<R>(nb, M.np, M.O, C.mlp_cells, C.mlp_Y, C.mlp_s, C.mlp_scale * hs, z, s));
}

// y = D^-1 t on level L: the smoother kernels with every neighbour read as zero and omega = 1 apply
// the cell-block inverses of Eq. 14 (dense for boundary cells, fast diagonalisation otherwise).
template <typename R>
void block_inverse(const DevLevel& L, const R* t, R* y, cudaStream_t s) {
  LevelParams<R> P1 = params<R>(L);
  P1.omega = R(1);
  CUDA_TRY(launch_smooth<R>(L.H.dim, L.H.p, P1, 0, kZeroAll, t, y, s));
}

// One step of the additive smoothers on z for the right-hand side r (zero: z = 0 on entry):
// block Jacobi z += omega_l D^-1 (r - A z), or cheb_degree Chebyshev steps with D^-1 on the
// interval [b / cheb_ratio, b], b = 1.1 lambda_max (three-term recurrence: rho_0 = 1 / sigma,
// d_0 = D^-1 r_0 / theta, rho_k = 1 / (2 sigma - rho_(k-1)), d_k = rho_k rho_(k-1) d_(k-1)
// + (2 rho_k / delta) D^-1 r_k, z += d_k).
template <typename R>
void additive_smooth(Context& C, DevLevel& L, const R* r, R* z, bool zero, cudaStream_t s) {
  const int pi = prec_index<R>();
  const size_t N = L.H.n_dof();
  const int dim = L.H.dim, p = L.H.p;
  R* res = static_cast<R*>(L.res[pi]);
  R* y = static_cast<R*>(L.tmp[pi]);
  const LevelParams<R>& P = params<R>(L);
  auto residual_inverse = [&](bool from_zero) {      // y = D^-1 (r - A z)
    if (from_zero) {
      block_inverse<R>(L, r, y, s);
    } else {
      CUDA_TRY((launch_apply<R, R>(dim, p, P, z, r, res, 1, s)));
      block_inverse<R>(L, res, y, s);
    }
  };
  if (C.desc.smoother == 1) {
    const R omega = (R)(p == 3 ? C.desc.omega_p3 : C.desc.omega);
    residual_inverse(zero);
    CUDA_TRY(launch_smoother_update<R>(N, R(0), omega, y, nullptr, z, zero ? 0 : 1, s));
    return;
  }
  R* d = static_cast<R*>(L.dir[pi]);
  const double b = kChebSafety * L.lam_max, a = b / C.desc.cheb_ratio;
  const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
  double rho = 1.0 / sigma;
  residual_inverse(zero);
  CUDA_TRY(launch_smoother_update<R>(N, R(0), (R)(1.0 / theta), y, d, z, zero ? 2 : 3, s));
  for (int k = 1; k < C.desc.cheb_degree; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    residual_inverse(false);
    CUDA_TRY(launch_smoother_update<R>(N, (R)(rho_new * rho), (R)(2.0 * rho_new / delta), y, d, z, 4, s));
    rho = rho_new;
  }
}

// One V-cycle on level l (Sec. 3): zero initial guess, pre-smoothing with forward colour order,
// residual, restriction (Eq. 18), recursion, prolongation (Eq. 17), post-smoothing with reverse
// colour order; level 0 is solved with the dense coarse inverse.
template <typename R>
void vcycle_rec(Context& C, int l, const R* r, R* z, cudaStream_t s, bool first_group_done = false) {
  DevLevel& L = C.lv[l];
  const int pi = prec_index<R>();
  if (l == 0) {
    CUDA_TRY(launch_coarse<R>(L.coarse_inv, L.H.n_dof(), r, z, s));
    return;
  }
  if (l == C.tail_plan[pi].top && !(C.mlp_on && l == C.finest())) {   // levels 0..l in one launch
    if (C.tail_plan[pi].cluster == 1) {
      const TailCta<R>* tp;
      if constexpr (sizeof(R) == 8) tp = C.tail_cta64.get();
      else tp = C.tail_cta32.get();
      const void* cinvT = sizeof(R) == 4 ? static_cast<const void*>(C.lv[0].coarse_invT_df)
                                         : static_cast<const void*>(C.lv[0].coarse_invT);
      CUDA_TRY(launch_vcycle_tail_cta<R>(L.H.dim, *tp, r, z, C.lv[0].coarse_inv, cinvT, C.tail_plan[pi].smem_bytes, s));
    } else {
      CUDA_TRY(launch_vcycle_tail<R>(L.H.dim, static_cast<const TailLevel<R>*>(C.tail[pi]), l, r, z,
                                     C.lv[0].coarse_inv, C.desc.pre_smooth, C.desc.post_smooth, C.desc.ssor_each,
                                     C.tail_plan[pi], s));
    }
    return;
  }
  const int dim = L.H.dim;
  const LevelParams<R>& P = params<R>(L);
  // `early` (the last launcher argument): r, resp. the fine z, was written two or more launches
  // before, so the kernels read it before their dependency wait.  Only the first pre-smoothing
  // sweep may follow r's writer directly (the restriction from the level above); the residual
  // comes after the pre-smoothing sweeps or the memset of z, the prolongation after the residual.
  if (C.desc.pre_smooth == 0) CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)L.H.n_dof() * sizeof(R), s));
  for (int k = 0; k < C.desc.pre_smooth; ++k) {
    if (C.desc.smoother != 0) {
      additive_smooth<R>(C, L, r, z, k == 0, s);
      continue;
    }
    // the first sweep's first colour group may have been done by the restriction from the level above
    CUDA_TRY(launch_smooth<R>(dim, L.H.p, P, 0, k == 0, r, z, s, k > 0, k == 0 && first_group_done ? 1 : 0));
    if (C.desc.ssor_each) CUDA_TRY(launch_smooth<R>(dim, L.H.p, P, 1, 0, r, z, s, 1));
  }
  DevLevel& Lc = C.lv[l - 1];
  R* rc = static_cast<R*>(Lc.rhs[pi]);
  R* zc = static_cast<R*>(Lc.z[pi]);
  // The coarse level's first colour group (colour 0) of its first pre-smoothing sweep from zero
  // needs only its own restricted residual (every neighbour is still zero): the restriction kernel
  // does it too, unless the coarse level is solved directly or by the one-launch tail.
  const LevelParams<R>& Pc = params<R>(Lc);
  const bool fuse = C.desc.smoother == 0 && C.desc.ordering == 0 && C.desc.pre_smooth >= 1 && l - 1 >= 1 &&
                    l - 1 != C.tail_plan[pi].top &&
                    restrict_fuses_first_group<R>(dim, L.H.p, P, tparams<R>(L), Lc.H.p, Pc);
  if (Lc.H.n == L.H.n) {                          // p-transfer: residual restricted in the same kernel
    CUDA_TRY(launch_resid_restrict_p<R>(dim, L.H.p, P, tparams<R>(L), z, r, rc, s, 1, fuse ? &Pc : nullptr,
                                        fuse ? zc : nullptr));
  } else {                                        // h-transfer: coarse cells gather their children
    CUDA_TRY(launch_resid_restrict_h<R>(dim, P, tparams<R>(L), z, r, rc, s, 1, fuse ? &Pc : nullptr,
                                        fuse ? zc : nullptr));
  }
  vcycle_rec<R>(C, l - 1, rc, zc, s, fuse);
  CUDA_TRY(launch_prolong<R>(dim, L.H.p, Lc.H.p, tparams<R>(L), zc, z, s, 1));
  for (int k = 0; k < C.desc.post_smooth; ++k) {
    if (C.desc.smoother != 0) {
      additive_smooth<R>(C, L, r, z, false, s);
      continue;
    }
    if (C.desc.ssor_each) CUDA_TRY(launch_smooth<R>(dim, L.H.p, P, 0, 0, r, z, s, 1));
    CUDA_TRY(launch_smooth<R>(dim, L.H.p, P, 1, 0, r, z, s, 1));
  }
  if (C.mlp_on && l == C.finest()) apply_learned<R>(C, L, r, z, s);
}

void ensure_krylov(Context& C, int m) {
  const int prec = C.desc.precision;
  const int basis = C.desc.krylov_basis;
  if (C.ws_m >= m && C.ws_prec == prec && C.ws_basis == basis) return;
  C.drop_graphs();                                  // captured pointers change
  const size_t N = C.lv.back().H.n_dof();
  // the staged sweeps copy whole 16-byte units from 16-byte aligned rows: rows of ldv entries,
  // and w, wdf padded to the same length (the padding is never used in the arithmetic)
  C.ldv = (N + 31) / 32 * 32;
  if (basis == 1) {                                 // FP64 basis
    C.V = C.dalloc<double>((size_t)(m + 1) * N);
  } else {
    C.V2 = C.dalloc<float2>((size_t)(m + 1) * C.ldv);
    C.wdf = C.dalloc<float2>(C.ldv);
    if (prec == SBM_F64) C.v64 = C.dalloc<double>(N);
  }
  C.ws_basis = basis;
  C.Z = prec == SBM_F32 ? (void*)C.dalloc<float>((size_t)m * N) : (void*)C.dalloc<double>((size_t)m * N);
  C.w = C.dalloc<double>(C.ldv);
  if (prec == SBM_F32) C.r32 = C.dalloc<float>(N);
  C.partial = C.dalloc<double>((size_t)std::max(dot_blocks(N), gs_blocks(N)) * 32);   // rows of either grid
  C.dots = C.dalloc<double>(128);
  C.ydev = C.dalloc<double>(32);
  C.ws_m = m;
  C.ws_prec = prec;
}

double device_norm(Context& C, const double* v, size_t N, double* out_dev, cudaStream_t s) {
  CUDA_TRY(launch_multi_dot(v, N, 1, v, N, C.partial, out_dev, 1, s));
  CUDA_TRY(cudaMemcpyAsync(C.host_pinned, out_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return C.host_pinned[0];
}

// Pinned host slot of the Hessenberg column of Arnoldi step j (two slots, so that step j + 1 can
// be in flight while the host reads column j).
double* column_slot(Context& C, int j) { return C.host_pinned + 64 * (1 + (j & 1)); }

// All device work of Arnoldi step j (Sec. 3: one V-cycle, then the FP64 operator and two
// classical Gram-Schmidt passes), ending with the copy of Hessenberg column j to pinned memory.
void arnoldi_step_work(Context& C, int j, cudaStream_t s) {
  const int prec = C.desc.precision;
  const int Lf = C.finest();
  DevLevel& F = C.lv[Lf];
  const size_t N = F.H.n_dof();
  const int dim = F.H.dim, p = F.H.p;
  double* h1 = C.dots;
  double* h2 = C.dots + 32;
  double* hn = C.dots + 64;
  double* col = C.dots + 96;
  if (C.desc.krylov_basis == 1) {                 // FP64 basis
    double* Vj = C.V + (size_t)j * N;
    if (prec == SBM_F32) {
      float* Zj = static_cast<float*>(C.Z) + (size_t)j * N;
      CUDA_TRY((launch_cast<double, float>(Vj, C.r32, N, s)));
      vcycle_rec<float>(C, Lf, C.r32, Zj, s);
      CUDA_TRY((launch_apply<float, double>(dim, p, F.P64, Zj, nullptr, C.w, 0, s)));
    } else {
      double* Zj = static_cast<double*>(C.Z) + (size_t)j * N;
      vcycle_rec<double>(C, Lf, Vj, Zj, s);
      CUDA_TRY((launch_apply<double, double>(dim, p, F.P64, Zj, nullptr, C.w, 0, s)));
    }
    // CGS2 in three sweeps over V: h1 = V^T w; w -= V h1 and h2 = V^T w; w -= V h2 and |w|
    CUDA_TRY(launch_multi_dot(C.V, N, j + 1, C.w, N, C.partial, h1, 0, s));
    CUDA_TRY(launch_axpy_dot(C.V, N, j + 1, h1, C.w, N, C.partial, h2, s));
    CUDA_TRY(launch_axpy_norm(C.V, N, j + 1, h2, C.w, N, C.partial, hn, s));
    CUDA_TRY(launch_div_scalar(C.w, hn, C.V + (size_t)(j + 1) * N, N, s));
  } else {                                          // double-float basis, same three sweeps
    // v_j rounded to the V-cycle precision is in r32 / v64 (written with v_j itself)
    if (prec == SBM_F32) {
      float* Zj = static_cast<float*>(C.Z) + (size_t)j * N;
      vcycle_rec<float>(C, Lf, C.r32, Zj, s);
      if (C.desc.krylov_basis == 0 && F.has_df) {   // w = A z in double-float, straight into wdf
        dfl* wd = reinterpret_cast<dfl*>(C.wdf);
        if (cell_smoother(dim, p)) CUDA_TRY((launch_apply_cell<float, dfl>(dim, p, F.Pdf, Zj, nullptr, wd, 0, s)));
        else CUDA_TRY((launch_apply<float, dfl>(dim, p, F.Pdf, Zj, nullptr, wd, 0, s)));   // one thread per DoF
        CUDA_TRY(launch_gs_dot_df(C.V2, C.ldv, j + 1, C.wdf, N, C.partial, h1, s));
      } else {
        CUDA_TRY((launch_apply<float, double>(dim, p, F.P64, Zj, nullptr, C.w, 0, s)));
        CUDA_TRY(launch_gs_dot(C.V2, C.ldv, j + 1, C.w, C.wdf, N, C.partial, h1, s));
      }
    } else {
      double* Zj = static_cast<double*>(C.Z) + (size_t)j * N;
      vcycle_rec<double>(C, Lf, C.v64, Zj, s);
      CUDA_TRY((launch_apply<double, double>(dim, p, F.P64, Zj, nullptr, C.w, 0, s)));
      CUDA_TRY(launch_gs_dot(C.V2, C.ldv, j + 1, C.w, C.wdf, N, C.partial, h1, s));
    }
    CUDA_TRY(launch_gs_axpy_dot(C.V2, C.ldv, j + 1, h1, C.wdf, N, C.partial, h2, s));
    CUDA_TRY(launch_gs_axpy_norm(C.V2, C.ldv, j + 1, h2, C.wdf, N, C.partial, hn, s, h1, col));   // + column
    float2* vnext = C.V2 + (size_t)(j + 1) * C.ldv;
    if (prec == SBM_F32) CUDA_TRY((launch_gs_scale<float2, float>(C.wdf, hn, vnext, C.r32, N, s)));
    else CUDA_TRY((launch_gs_scale<float2, double>(C.wdf, hn, vnext, C.v64, N, s)));
  }
  if (C.desc.krylov_basis == 1) CUDA_TRY(launch_hess_column(h1, h2, hn, j + 1, col, s));
  CUDA_TRY(cudaMemcpyAsync(column_slot(C, j), col, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
}

// Runs step j from its captured graph (captured on first use).
void run_arnoldi_step(Context& C, int j, cudaStream_t s) {
  const int pi = C.desc.precision == SBM_F32 ? 1 : 0;
  const int li = C.mlp_on ? 1 : 0;
  auto& graph = C.arnoldi[pi][li][j];
  auto& nkern = C.arnoldi_kernels[pi][li][j];
  if (!graph) {
    const long long before = g_kernel_launches.load();
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      arnoldi_step_work(C, j, s);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamEndCapture(s, &g));
    cudaGraphExec_t ge = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
    graph = ge;
    nkern = g_kernel_launches.load() - before;
    g_kernel_launches.fetch_sub(nkern);             // captured, not executed
  }
  CUDA_TRY(cudaGraphLaunch(graph, s));
  CUDA_TRY(cudaEventRecord(C.step_done[j & 1], s));
  count_launches(nkern);
}

// Step j + 1 is queued before the host has read column j when the residual after step j, predicted
// from the smallest of the last two per-step reduction factors, stays this many times above the
// tolerance.  A step queued in vain (the cycle ended at step j) costs one step; iterates and
// results do not depend on it.
constexpr double kQueueMargin = 8.0;

// Right-preconditioned flexible GMRES(m) with two classical Gram-Schmidt passes, FP64.
int solve_impl(Context& C, const double* b, double* x, double tol, int m, int max_it, sbm_solve_info* info) {
  if (m < 1 || m > 31) throw SetupError{SBM_ERR_ARG, "restart must be in 1..31"};
  if (!(tol > 0)) throw SetupError{SBM_ERR_ARG, "tol must be > 0"};
  ensure_krylov(C, m);
  const int prec = C.desc.precision;
  if (prec == SBM_F32) ensure_work<float>(C); else ensure_work<double>(C);
  const int Lf = C.finest();
  DevLevel& F = C.lv[Lf];
  const size_t N = F.H.n_dof();
  const cudaStream_t s = C.ws;
  const int dim = F.H.dim, p = F.H.p;
  double* hn = C.dots + 64;
  sbm_solve_info loc{};
  const bool mlp_was_on = C.mlp_on;
  loc.learned = C.mlp_on ? 1 : 0;
  struct Restore {                                  // the fallback lasts for this solve only
    Context& C;
    bool on;
    ~Restore() { C.mlp_on = on; }
  } restore{C, mlp_was_on};
  CUDA_TRY(cudaEventRecord(C.join_in, C.stream));   // b and x are ready on the caller's stream
  CUDA_TRY(cudaStreamWaitEvent(s, C.join_in, 0));
  CUDA_TRY(cudaEventRecord(C.ev0, s));
  const double bnorm = device_norm(C, b, N, hn, s);
  if (!std::isfinite(bnorm)) throw SetupError{SBM_ERR_NAN, "non-finite ||b||"};
  int status = SBM_OK;
  if (bnorm == 0.0) {
    CUDA_TRY(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    loc.converged = 1;
    loc.true_rel_residual = 0.0;
  } else {
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    double q_last = 0.0, q_prev = 0.0;              // |sn| of the last two steps: their residual factors
    while (true) {
      double* r0 = C.desc.krylov_basis == 1 ? C.V : C.w;   // r = b - A x, FP64
      CUDA_TRY((launch_apply<double, double>(dim, p, F.P64, x, b, r0, 1, s)));
      const double beta = device_norm(C, r0, N, hn, s);
      loc.true_rel_residual = beta / bnorm;
      if (!std::isfinite(beta)) {
        status = SBM_ERR_NAN;
        break;
      }
      if (beta <= tol * bnorm) {
        loc.converged = 1;
        break;
      }
      if (loc.iterations >= max_it) {
        status = SBM_ERR_NOT_CONVERGED;
        break;
      }
      if (C.desc.krylov_basis == 1) CUDA_TRY(launch_div_scalar(r0, hn, r0, N, s));
      else if (prec == SBM_F32) CUDA_TRY((launch_gs_scale<double, float>(r0, hn, C.V2, C.r32, N, s)));
      else CUDA_TRY((launch_gs_scale<double, double>(r0, hn, C.V2, C.v64, N, s)));
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int k = 0;
      bool nan = false;
      int queued = -1;                              // last step launched in this cycle
      for (int j = 0; j < m; ++j) {
        if (queued < j) {
          run_arnoldi_step(C, j, s);
          queued = j;
        }
        // queue step j + 1 behind step j when step j will not end the cycle: the next steps exist,
        // the learned-correction decision (after the third step of the first cycle) is not
        // pending, and the predicted residual stays well above the tolerance
        const double q_lo = std::min(q_last, q_prev);
        if (j + 1 < m && loc.iterations + 1 < max_it && q_lo > 0.0 &&
            !(C.mlp_on && loc.restarts == 0 && loc.iterations + 1 == 3) &&
            std::fabs(g[j]) * q_lo > kQueueMargin * tol * bnorm) {
          run_arnoldi_step(C, j + 1, s);
          queued = j + 1;
        }
        CUDA_TRY(cudaEventSynchronize(C.step_done[j & 1]));
        const double* colh = column_slot(C, j);
        for (int i = 0; i <= j + 1; ++i) {
          H[(size_t)i * m + j] = colh[i];
          if (!std::isfinite(colh[i])) nan = true;
        }
        const double hnorm = colh[j + 1];
        for (int i = 0; i < j; ++i) {              // previous Givens rotations
          const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
          H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = t;
        }
        const double rr = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
        cs[j] = H[(size_t)j * m + j] / rr;
        sn[j] = H[(size_t)(j + 1) * m + j] / rr;
        H[(size_t)j * m + j] = rr;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        q_prev = q_last;
        q_last = std::isfinite(sn[j]) ? std::fabs(sn[j]) : 0.0;
        k = j + 1;
        if (loc.iterations < 512) loc.history[loc.iterations] = std::fabs(g[j + 1]) / bnorm;
        loc.iterations += 1;
        // learned-correction fallback: after 3 steps of the first cycle, a mean residual reduction
        // per step worse than the reference rate switches the correction off; FGMRES tolerates
        // the change of preconditioner (every z_j is stored)
        if (C.mlp_on && C.mlp_rate_ref > 0 && loc.restarts == 0 && loc.iterations == 3 &&
            std::pow(std::fabs(g[j + 1]) / beta, 1.0 / 3.0) > C.mlp_rate_ref) {
          C.mlp_on = false;
          loc.learned_fallback = 1;
        }
        if (nan || !std::isfinite(g[j + 1])) {
          nan = true;
          break;
        }
        if (std::fabs(g[j + 1]) <= tol * bnorm || loc.iterations >= max_it || hnorm == 0.0) break;
      }
      if (nan) {
        status = SBM_ERR_NAN;
        break;
      }
      for (int i = k - 1; i >= 0; --i) {           // back substitution H y = g
        double acc = g[i];
        for (int q = i + 1; q < k; ++q) acc -= H[(size_t)i * m + q] * y[q];
        y[i] = acc / H[(size_t)i * m + i];
      }
      for (int i = 0; i < k; ++i) C.host_pinned[i] = y[i];
      CUDA_TRY(cudaMemcpyAsync(C.ydev, C.host_pinned, k * sizeof(double), cudaMemcpyHostToDevice, s));
      if (prec == SBM_F32)
        CUDA_TRY(launch_multi_axpy<float>(static_cast<float*>(C.Z), N, k, C.ydev, 1.0, x, N, s));
      else
        CUDA_TRY(launch_multi_axpy<double>(static_cast<double*>(C.Z), N, k, C.ydev, 1.0, x, N, s));
      CUDA_TRY(cudaStreamSynchronize(s));          // host_pinned is reused by the next norm
      loc.restarts += 1;
    }
  }
  CUDA_TRY(cudaEventRecord(C.ev1, s));
  CUDA_TRY(cudaEventRecord(C.join_out, s));
  CUDA_TRY(cudaStreamWaitEvent(C.stream, C.join_out, 0));
  CUDA_TRY(cudaEventSynchronize(C.ev1));
  float ms = 0;
  CUDA_TRY(cudaEventElapsedTime(&ms, C.ev0, C.ev1));
  loc.ms_total = ms;
  if (info) *info = loc;
  if (sweep_fault_take() != 0)
    return set_error(SBM_ERR_CUDA, "Gram-Schmidt sweep: staged copies did not complete in bounded time");
  if (tail_fault_take() != 0)
    return set_error(SBM_ERR_CUDA, "V-cycle tail: staging copies did not complete in bounded time");
  if (status == SBM_ERR_NAN) return set_error(status, "non-finite value in FGMRES");
  if (status == SBM_ERR_NOT_CONVERGED) return set_error(status, "FGMRES did not reach the tolerance");
  return SBM_OK;
}

// Training pairs from the stationary iteration u <- u + V(-A u) on A u = 0 (exact solution 0):
// after each V-cycle (the finest post-smoothing is its last step) the error of the iterate is -u,
// so every boundary cell K gives features x_K from r = -A u and the target -u_K / s_K.
template <typename R>
long long collect_impl(Context& C, Mlp& M, const R* u0, int n_starts, int n_cycles) {
  ensure_work<R>(C);
  ensure_learned(C);
  const int pi = prec_index<R>();
  const int Lf = C.finest();
  DevLevel& F = C.lv[Lf];
  const size_t N = F.H.n_dof();
  const int nb = C.lf_nb;
  const cudaStream_t s = C.stream;
  for (int k = 0; k < 4; ++k)
    if (!C.col_vec[pi][k]) C.col_vec[pi][k] = C.dalloc<R>(N);
  R* u = static_cast<R*>(C.col_vec[pi][0]);
  R* rhs = static_cast<R*>(C.col_vec[pi][1]);
  R* z = static_cast<R*>(C.col_vec[pi][2]);
  R* zero = static_cast<R*>(C.col_vec[pi][3]);
  CUDA_TRY(cudaMemsetAsync(zero, 0, N * sizeof(R), s));
  M.reserve(M.count + (size_t)n_starts * n_cycles * nb);
  const bool was_on = C.mlp_on;
  C.mlp_on = false;                                 // plain V-cycles
  const LevelParams<R>& P = params<R>(F);
  for (int k = 0; k < n_starts; ++k) {
    CUDA_TRY(cudaMemcpyAsync(u, u0 + (size_t)k * N, N * sizeof(R), cudaMemcpyDeviceToDevice, s));
    for (int c = 0; c < n_cycles; ++c) {
      CUDA_TRY((launch_apply<R, R>(F.H.dim, F.H.p, P, u, zero, rhs, 1, s)));     // rhs = -A u
      vcycle_rec<R>(C, Lf, rhs, z, s);
      CUDA_TRY(launch_add<R>(N, z, u, s));
      CUDA_TRY((launch_apply<R, R>(F.H.dim, F.H.p, P, u, zero, rhs, 1, s)));     // r = -A u
      __nv_bfloat16* X = M.Xd + M.count * M.Fpad;
      CUDA_TRY(launch_mlp_features<R>(nb, C.lf_npatch, F.H.np, C.lf_nstat, C.lf_Fpad, C.mlp_patch, C.mlp_stat, rhs, X,
                                      C.mlp_s, s));
      const float hfac = (float)std::pow(F.H.h, F.H.dim - 2);     // targets -u_K / (s h^(2-d))
      CUDA_TRY(launch_mlp_targets<R>(nb, F.H.np, C.mlp_cells, u, C.mlp_s, hfac, M.Td + M.count * M.O, s));
      M.count += nb;
    }
  }
  C.mlp_on = was_on;
  CUDA_TRY(cudaStreamSynchronize(s));
  return (long long)nb * n_starts * n_cycles;
}

// splitmix64 (Steele, Lea, Flood 2014): the seeded generator of the host-side MLP set-up.
uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& x) { return ((splitmix64(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
double normal01(uint64_t& x) {                      // Box-Muller
  const double u1 = uniform01(x), u2 = uniform01(x);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320), bitwise.
uint32_t crc32(const unsigned char* p, size_t n) {
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) {
    c ^= p[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return c ^ 0xFFFFFFFFu;
}

// Packed unpadded parameter vector (W1 F x H, b1, W2, b2, W3, b3) <-> the padded device layout.
size_t packed_size(const Mlp& M) { return M.nparam - (size_t)(M.Fpad - M.F) * M.H; }

void set_params(Mlp& M, const float* host) {
  std::vector<float> full(M.nparam, 0.f);
  std::memcpy(full.data(), host, (size_t)M.F * M.H * sizeof(float));
  std::memcpy(full.data() + M.ob1, host + (size_t)M.F * M.H, (M.nparam - M.ob1) * sizeof(float));
  CUDA_TRY(cudaMemcpy(M.P, full.data(), M.nparam * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(launch_to_bf16((int)M.nparam, M.P, M.Pb, M.s));
  CUDA_TRY(cudaMemsetAsync(M.Am, 0, M.nparam * sizeof(float), M.s));
  CUDA_TRY(cudaMemsetAsync(M.Av, 0, M.nparam * sizeof(float), M.s));
  CUDA_TRY(cudaStreamSynchronize(M.s));
  M.adam_t = 0;
}

void get_packed(const Mlp& M, const float* dev, float* host) {
  std::vector<float> full(M.nparam);
  CUDA_TRY(cudaMemcpy(full.data(), dev, M.nparam * sizeof(float), cudaMemcpyDeviceToHost));
  std::memcpy(host, full.data(), (size_t)M.F * M.H * sizeof(float));
  std::memcpy(host + (size_t)M.F * M.H, full.data() + M.ob1, (M.nparam - M.ob1) * sizeof(float));
}

// Sum of the squared-error partials of the last backward pass, on the host.
double read_loss(Mlp& M, int rows) {
  float part[152];
  CUDA_TRY(cudaMemcpyAsync(part, M.loss_part, sizeof(part), cudaMemcpyDeviceToHost, M.s));
  CUDA_TRY(cudaStreamSynchronize(M.s));
  double t = 0;
  for (float v : part) t += v;
  return t / ((double)rows * M.O);
}

// The context handle of an ABI call; also selects, for the calling thread, whether the
// launches of this call use programmatic dependent launch (the context's launch_overlap).
Context* ctx_of(void* p) {
  Context* C = static_cast<Context*>(p);
  if (C) pdl_enabled() = C->desc.launch_overlap > 0 || (C->desc.launch_overlap == 0 && C->desc.precision == SBM_F32);
  return C;
}
Mlp* mlp_of(void* p) { return static_cast<Mlp*>(p); }

int check_level(const Context* C, int& level) {
  if (!C) return set_error(SBM_ERR_ARG, "null context");
  if (C->lv.empty()) return set_error(SBM_ERR_ARG, "context has no levels");
  if (level < 0) level = (int)C->lv.size() - 1;
  if (level >= (int)C->lv.size()) return set_error(SBM_ERR_ARG, "level out of range");
  return SBM_OK;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const SetupError& e) {
    return set_error(e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return set_error(SBM_ERR_ALLOC, "host allocation failed");
  } catch (const std::exception& e) {
    return set_error(SBM_ERR_ARG, e.what());
  }
}

}  // namespace

int record_error(int code, const std::string& msg) { return set_error(code, msg); }

}  // namespace sbm

using namespace sbm;

extern "C" {

int sbm_setup(const sbm_setup_desc* desc, void** out) {
  if (out) *out = nullptr;
  if (!desc || !out) return set_error(SBM_ERR_ARG, "null argument");
  return guarded([&]() -> int {
    *out = build_context(*desc, true);
    return SBM_OK;
  });
}

int sbm_setup_host(const sbm_setup_desc* desc, void** out) {
  if (out) *out = nullptr;
  if (!desc || !out) return set_error(SBM_ERR_ARG, "null argument");
  return guarded([&]() -> int {
    *out = build_context(*desc, false);
    static_cast<Context*>(*out)->host_only = true;
    return SBM_OK;
  });
}

int sbm_host_apply(const void* ctx, int level, const double* x_host, double* y_host) {
  const Context* C = static_cast<const Context*>(ctx);
  if (int e = check_level(C, level)) return e;
  if (!x_host || !y_host || x_host == y_host) return set_error(SBM_ERR_ARG, "bad vector pointers");
  return guarded([&]() -> int {
    host_apply_level(C->lv[level].H, x_host, y_host);
    return SBM_OK;
  });
}

int sbm_host_rhs(const void* ctx, double* b_host) {
  const Context* C = static_cast<const Context*>(ctx);
  if (!C || !b_host) return set_error(SBM_ERR_ARG, "null argument");
  std::memcpy(b_host, C->rhs_host.data(), C->rhs_host.size() * sizeof(double));
  return SBM_OK;
}

void sbm_destroy(void* ctx) { delete ctx_of(ctx); }

const char* sbm_last_error(void) { return g_last_error.c_str(); }

long long sbm_kernel_launches(void) { return g_kernel_launches.load(); }

int sbm_num_levels(const void* ctx, int* out) {
  if (!ctx || !out) return set_error(SBM_ERR_ARG, "null argument");
  *out = (int)static_cast<const Context*>(ctx)->lv.size();
  return SBM_OK;
}

int sbm_info(const void* ctx, int level, sbm_level_info* out) {
  const Context* C = static_cast<const Context*>(ctx);
  if (int e = check_level(C, level)) return e;
  if (!out) return set_error(SBM_ERR_ARG, "null output");
  const HostLevel& H = C->lv[level].H;
  std::memset(out, 0, sizeof(*out));
  out->n = H.n;
  out->p = H.p;
  out->h = H.h;
  out->n_active = H.n_act;
  out->n_dof = H.n_dof();
  out->n_boundary = H.n_bnd;
  out->n_sface = H.n_sface;
  for (int c = 0; c < 9; ++c) out->colour_start[c] = H.colour_start[c];
  for (int c = 0; c < 8; ++c) out->colour_nbnd[c] = H.colour_nbnd[c];
  return SBM_OK;
}

int sbm_layout(const void* ctx, int level, int* coords_host) {
  const Context* C = static_cast<const Context*>(ctx);
  if (int e = check_level(C, level)) return e;
  if (!coords_host) return set_error(SBM_ERR_ARG, "null output");
  const HostLevel& H = C->lv[level].H;
  std::memcpy(coords_host, H.cell.data(), H.cell.size() * sizeof(int));
  return SBM_OK;
}

int sbm_export_geometry(const void* ctx, int level, int* n_faces, int* cell_host, int* slot_host, double* d_host) {
  const Context* C = static_cast<const Context*>(ctx);
  if (int e = check_level(C, level)) return e;
  const HostLevel& H = C->lv[level].H;
  if (n_faces) *n_faces = H.n_sface;
  if (cell_host) std::memcpy(cell_host, H.sf_cell.data(), H.sf_cell.size() * sizeof(int));
  if (slot_host) std::memcpy(slot_host, H.sf_slot.data(), H.sf_slot.size() * sizeof(int));
  if (d_host) std::memcpy(d_host, H.sf_d.data(), H.sf_d.size() * sizeof(double));
  return SBM_OK;
}

int sbm_rhs(void* ctx, double* b_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !b_dev) return set_error(SBM_ERR_ARG, "null argument");
  return guarded([&]() -> int {
    CUDA_TRY(cudaMemcpyAsync(b_dev, C->rhs_host.data(), C->rhs_host.size() * sizeof(double),
                             cudaMemcpyHostToDevice, C->stream));
    CUDA_TRY(cudaStreamSynchronize(C->stream));
    return SBM_OK;
  });
}

int sbm_apply(void* ctx, int level, int dtype, const void* x_dev, void* y_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (int e = check_level(C, level)) return e;
  if (!x_dev || !y_dev || x_dev == y_dev) return set_error(SBM_ERR_ARG, "bad vector pointers");
  return guarded([&]() -> int {
    DevLevel& L = C->lv[level];
    if (dtype == SBM_F64)
      CUDA_TRY((launch_apply<double, double>(L.H.dim, L.H.p, L.P64, (const double*)x_dev, nullptr, (double*)y_dev, 0,
                                             C->stream)));
    else if (dtype == SBM_F32)
      CUDA_TRY((launch_apply<float, float>(L.H.dim, L.H.p, L.P32, (const float*)x_dev, nullptr, (float*)y_dev, 0,
                                           C->stream)));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    return SBM_OK;
  });
}

int sbm_residual(void* ctx, int level, int dtype, const void* f_dev, const void* u_dev, void* r_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (int e = check_level(C, level)) return e;
  if (!f_dev || !u_dev || !r_dev || u_dev == r_dev) return set_error(SBM_ERR_ARG, "bad vector pointers");
  return guarded([&]() -> int {
    DevLevel& L = C->lv[level];
    if (dtype == SBM_F64)
      CUDA_TRY((launch_apply<double, double>(L.H.dim, L.H.p, L.P64, (const double*)u_dev, (const double*)f_dev,
                                             (double*)r_dev, 1, C->stream)));
    else if (dtype == SBM_F32)
      CUDA_TRY((launch_apply<float, float>(L.H.dim, L.H.p, L.P32, (const float*)u_dev, (const float*)f_dev,
                                           (float*)r_dev, 1, C->stream)));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    return SBM_OK;
  });
}

int sbm_smooth(void* ctx, int level, int dtype, int reverse, const void* f_dev, void* u_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (int e = check_level(C, level)) return e;
  if (!f_dev || !u_dev || f_dev == u_dev) return set_error(SBM_ERR_ARG, "bad vector pointers");
  return guarded([&]() -> int {
    DevLevel& L = C->lv[level];
    if (dtype == SBM_F64)
      CUDA_TRY(launch_smooth<double>(L.H.dim, L.H.p, L.P64, reverse, 0, (const double*)f_dev, (double*)u_dev,
                                     C->stream));
    else if (dtype == SBM_F32)
      CUDA_TRY(launch_smooth<float>(L.H.dim, L.H.p, L.P32, reverse, 0, (const float*)f_dev, (float*)u_dev,
                                    C->stream));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    return SBM_OK;
  });
}

int sbm_restrict(void* ctx, int level, int dtype, const void* rf_dev, void* rc_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (int e = check_level(C, level)) return e;
  if (level < 1) return set_error(SBM_ERR_ARG, "restriction needs level >= 1");
  if (!rf_dev || !rc_dev) return set_error(SBM_ERR_ARG, "null vector");
  return guarded([&]() -> int {
    DevLevel& L = C->lv[level];
    const int pc = C->lv[level - 1].H.p;
    if (dtype == SBM_F64)
      CUDA_TRY(launch_restrict<double>(L.H.dim, L.H.p, pc, L.T64, (const double*)rf_dev, (double*)rc_dev, C->stream));
    else if (dtype == SBM_F32)
      CUDA_TRY(launch_restrict<float>(L.H.dim, L.H.p, pc, L.T32, (const float*)rf_dev, (float*)rc_dev, C->stream));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    return SBM_OK;
  });
}

int sbm_prolong_add(void* ctx, int level, int dtype, const void* ec_dev, void* uf_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (int e = check_level(C, level)) return e;
  if (level < 1) return set_error(SBM_ERR_ARG, "prolongation needs level >= 1");
  if (!ec_dev || !uf_dev) return set_error(SBM_ERR_ARG, "null vector");
  return guarded([&]() -> int {
    DevLevel& L = C->lv[level];
    const int pc = C->lv[level - 1].H.p;
    if (dtype == SBM_F64)
      CUDA_TRY(launch_prolong<double>(L.H.dim, L.H.p, pc, L.T64, (const double*)ec_dev, (double*)uf_dev, C->stream));
    else if (dtype == SBM_F32)
      CUDA_TRY(launch_prolong<float>(L.H.dim, L.H.p, pc, L.T32, (const float*)ec_dev, (float*)uf_dev, C->stream));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    return SBM_OK;
  });
}

int sbm_coarse_solve(void* ctx, int dtype, const void* r_dev, void* e_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !r_dev || !e_dev || r_dev == e_dev) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    DevLevel& L = C->lv[0];
    if (dtype == SBM_F64)
      CUDA_TRY(launch_coarse<double>(L.coarse_inv, L.H.n_dof(), (const double*)r_dev, (double*)e_dev, C->stream));
    else if (dtype == SBM_F32)
      CUDA_TRY(launch_coarse<float>(L.coarse_inv, L.H.n_dof(), (const float*)r_dev, (float*)e_dev, C->stream));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    return SBM_OK;
  });
}

int sbm_vcycle(void* ctx, int dtype, const void* r_dev, void* z_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !r_dev || !z_dev || r_dev == z_dev) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    if (dtype == SBM_F64) {
      ensure_work<double>(*C);
      vcycle_rec<double>(*C, C->finest(), (const double*)r_dev, (double*)z_dev, C->stream);
    } else if (dtype == SBM_F32) {
      ensure_work<float>(*C);
      vcycle_rec<float>(*C, C->finest(), (const float*)r_dev, (float*)z_dev, C->stream);
    } else {
      return set_error(SBM_ERR_ARG, "dtype");
    }
    return SBM_OK;
  });
}

int sbm_dots(void* ctx, const double* V_dev, long long ldv, int nv, const double* w_dev, long long n,
             double* out_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !V_dev || !w_dev || !out_dev || nv < 1 || nv > 32 || n < 0 || ldv < n)
    return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    const size_t need = (size_t)dot_blocks((size_t)n) * 32;
    if (C->dots_scratch_len < need) {
      C->dots_scratch = C->dalloc<double>(need);
      C->dots_scratch_len = need;
    }
    CUDA_TRY(launch_multi_dot(V_dev, (size_t)ldv, nv, w_dev, (size_t)n, C->dots_scratch, out_dev, 0, C->stream));
    return SBM_OK;
  });
}

int sbm_l2_error(void* ctx, const double* x_dev, double* err_host) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !x_dev || !err_host) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    const HostLevel& H = C->lv.back().H;
    const cudaStream_t s = C->stream;
    if (!C->l2cell) {
      C->l2cell = C->upload(H.cell);
      C->l2partial = C->dalloc<double>((size_t)l2_error_blocks(H.n_act));
      C->l2out = C->dalloc<double>(1);
    }
    L2ErrorParams E;
    std::memset(&E, 0, sizeof(E));
    E.n_act = H.n_act;
    E.kind = C->desc.exact;
    E.h = H.h;
    for (int k = 0; k < 3; ++k) E.lo[k] = C->desc.lo[k];
    const int m1 = H.p + 3;
    gauss_legendre01(m1, E.xq, E.wq);
    for (int q = 0; q < m1; ++q) lagrange_eval(H.n1, H.B.x, E.xq[q], E.V + q * kMaxN1, nullptr);
    CUDA_TRY(launch_l2_error(H.dim, H.p, E, C->l2cell, x_dev, C->l2partial, C->l2out, s));
    CUDA_TRY(cudaMemcpyAsync(C->host_pinned, C->l2out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    *err_host = C->host_pinned[0];
    return SBM_OK;
  });
}

int sbm_gram_schmidt(void* ctx, int variant, const double* V_dev, int nv, const double* w_dev, double* h_dev,
                     double* w_out_dev, double* norm_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !V_dev || !w_dev || !h_dev || !w_out_dev || !norm_dev || nv < 1 || nv > 32 || variant < 0 ||
      variant > 2)
    return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    const size_t N = C->lv.back().H.n_dof();
    const size_t ldv = (N + 31) / 32 * 32;           // the solve's padded row length
    const cudaStream_t s = C->stream;
    if (!C->gsw) {
      C->gsw = C->dalloc<double>(ldv);
      C->gswdf = C->dalloc<float2>(ldv);
      C->gspartial = C->dalloc<double>((size_t)std::max(dot_blocks(N), gs_blocks(N)) * 32);
      C->gsdots = C->dalloc<double>(256);
      const double one = 1.0;
      CUDA_TRY(cudaMemcpy(C->gsdots + 65, &one, sizeof(double), cudaMemcpyHostToDevice));
    }
    if (sweep_fault_take() < 0) return set_error(SBM_ERR_CUDA, "cannot read the fault flag");
    double* h1 = C->gsdots;
    double* h2 = C->gsdots + 32;
    double* hn = C->gsdots + 64;
    const double* one = C->gsdots + 65;
    double* col = C->gsdots + 128;
    // w into the padded buffer (the staged copies read whole 16-byte units past an odd N)
    CUDA_TRY(cudaMemsetAsync(C->gsw, 0, ldv * sizeof(double), s));
    CUDA_TRY(cudaMemcpyAsync(C->gsw, w_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (variant == 2) {                              // FP64 basis: the sweeps of krylov_basis = 1
      CUDA_TRY(launch_multi_dot(V_dev, N, nv, C->gsw, N, C->gspartial, h1, 0, s));
      CUDA_TRY(launch_axpy_dot(V_dev, N, nv, h1, C->gsw, N, C->gspartial, h2, s));
      CUDA_TRY(launch_axpy_norm(V_dev, N, nv, h2, C->gsw, N, C->gspartial, hn, s));
      CUDA_TRY(cudaMemcpyAsync(w_out_dev, C->gsw, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {                                         // double-float basis: the staged sweeps
      if (!C->gsV2) {
        C->gsV2 = C->dalloc<float2>(32 * ldv);
        CUDA_TRY(cudaMemsetAsync(C->gsV2, 0, 32 * ldv * sizeof(float2), s));
      }
      for (int k = 0; k < nv; ++k)                   // rows rounded to double-float (exact split)
        CUDA_TRY((launch_gs_scale<double, double>(V_dev + (size_t)k * N, one, C->gsV2 + (size_t)k * ldv,
                                                  (double*)nullptr, N, s)));
      if (variant == 1) {                            // w handed over as double-float (FP32-V-cycle solves)
        CUDA_TRY(cudaMemsetAsync(C->gswdf, 0, ldv * sizeof(float2), s));
        CUDA_TRY((launch_gs_scale<double, double>(C->gsw, one, C->gswdf, (double*)nullptr, N, s)));
        CUDA_TRY(launch_gs_dot_df(C->gsV2, ldv, nv, C->gswdf, N, C->gspartial, h1, s));
      } else {                                       // w in FP64, converted by the first sweep
        CUDA_TRY(launch_gs_dot(C->gsV2, ldv, nv, C->gsw, C->gswdf, N, C->gspartial, h1, s));
      }
      CUDA_TRY(launch_gs_axpy_dot(C->gsV2, ldv, nv, h1, C->gswdf, N, C->gspartial, h2, s));
      CUDA_TRY(launch_gs_axpy_norm(C->gsV2, ldv, nv, h2, C->gswdf, N, C->gspartial, hn, s, h1, col));
      CUDA_TRY(launch_df_to<double>(C->gswdf, w_out_dev, N, s));
    }
    CUDA_TRY(cudaMemcpyAsync(h_dev, h1, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h_dev + nv, h2, nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(norm_dev, hn, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const int f = sweep_fault_take();
    if (f < 0) return set_error(SBM_ERR_CUDA, "cannot read the fault flag");
    if (f) return set_error(SBM_ERR_CUDA, "a bounded mbarrier wait of a Gram-Schmidt sweep gave up");
    return SBM_OK;
  });
}

int sbm_solve(void* ctx, const double* b_dev, double* x_dev, double tol, int restart, int max_it,
              sbm_solve_info* info) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !b_dev || !x_dev || (const void*)b_dev == (void*)x_dev) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int { return solve_impl(*C, b_dev, x_dev, tol, restart, max_it, info); });
}

int sbm_solve_host(void* ctx, const double* b_host, double* x_host, double tol, int restart, int max_it,
                   sbm_solve_info* info) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !b_host || !x_host) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    const size_t N = C->lv.back().H.n_dof();
    if (!C->bbuf) {
      C->bbuf = C->dalloc<double>(N);
      C->xbuf = C->dalloc<double>(N);
    }
    CUDA_TRY(cudaMemcpyAsync(C->bbuf, b_host, N * sizeof(double), cudaMemcpyHostToDevice, C->stream));
    CUDA_TRY(cudaMemsetAsync(C->xbuf, 0, N * sizeof(double), C->stream));
    int rc = solve_impl(*C, C->bbuf, C->xbuf, tol, restart, max_it, info);
    CUDA_TRY(cudaMemcpyAsync(x_host, C->xbuf, N * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
    CUDA_TRY(cudaStreamSynchronize(C->stream));
    return rc;
  });
}


// ------------------------------------------------------------------ learned boundary correction
int sbm_mlp_create(int dim, int p, int hidden, unsigned long long seed, void* stream, void** out) {
  if (!out) return set_error(SBM_ERR_ARG, "null output");
  *out = nullptr;
  if ((dim != 2 && dim != 3) || p < 1 || p > 3 || hidden < 8 || hidden > 1024)
    return set_error(SBM_ERR_ARG, "bad MLP shape");
  return guarded([&]() -> int {
    auto M = std::make_unique<Mlp>();
    M->dim = dim;
    M->p = p;
    M->np = dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
    const int nq = dim == 2 ? p + 1 : (p + 1) * (p + 1);
    M->npatch = dim == 2 ? 9 : 27;
    M->nstat = 2 * dim * nq * dim + 1 + 2 * dim;
    M->F = M->npatch * M->np + M->nstat;
    M->Fpad = (M->F + 31) / 32 * 32;
    M->H = hidden;
    M->O = M->np;
    M->s = static_cast<cudaStream_t>(stream);
    const size_t F = M->Fpad, H = M->H, O = M->O;
    M->oW1 = 0;
    M->ob1 = F * H;
    M->oW2 = M->ob1 + H;
    M->ob2 = M->oW2 + H * H;
    M->oW3 = M->ob2 + H;
    M->ob3 = M->oW3 + H * O;
    M->nparam = M->ob3 + O;
    M->P = M->alloc<float>(M->nparam);
    M->G = M->alloc<float>(M->nparam);
    M->Am = M->alloc<float>(M->nparam);
    M->Av = M->alloc<float>(M->nparam);
    M->Pb = M->alloc<__nv_bfloat16>(M->nparam);
    M->loss_part = M->alloc<float>(152);
    M->loss_tmp = M->alloc<float>(1);
    M->loss_acc = M->alloc<float>(1);
    // He-normal hidden layers, 1/H output layer, zero biases
    std::vector<float> packed(packed_size(*M), 0.f);
    uint64_t st = seed;
    size_t o = 0;
    for (size_t i = 0; i < (size_t)M->F * H; ++i) packed[o++] = (float)(normal01(st) * std::sqrt(2.0 / M->F));
    o += H;
    for (size_t i = 0; i < H * H; ++i) packed[o++] = (float)(normal01(st) * std::sqrt(2.0 / H));
    o += H;
    for (size_t i = 0; i < H * O; ++i) packed[o++] = (float)(normal01(st) * std::sqrt(1.0 / H));
    set_params(*M, packed.data());
    *out = M.release();
    return SBM_OK;
  });
}

void sbm_mlp_destroy(void* mlp) { delete mlp_of(mlp); }

int sbm_mlp_shape(const void* mlp, int* F, int* Fpad, int* H, int* O, long long* nparam) {
  const Mlp* M = static_cast<const Mlp*>(mlp);
  if (!M) return set_error(SBM_ERR_ARG, "null MLP");
  if (F) *F = M->F;
  if (Fpad) *Fpad = M->Fpad;
  if (H) *H = M->H;
  if (O) *O = M->O;
  if (nparam) *nparam = (long long)packed_size(*M);
  return SBM_OK;
}

int sbm_mlp_set_params(void* mlp, const float* params_host) {
  Mlp* M = mlp_of(mlp);
  if (!M || !params_host) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    set_params(*M, params_host);
    return SBM_OK;
  });
}

int sbm_mlp_get_params(const void* mlp, float* params_host) {
  const Mlp* M = static_cast<const Mlp*>(mlp);
  if (!M || !params_host) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    get_packed(*M, M->P, params_host);
    return SBM_OK;
  });
}

int sbm_mlp_gemm_backend(void* mlp, int backend) {
  Mlp* M = mlp_of(mlp);
  if (!M || backend < 0 || backend > 1) return set_error(SBM_ERR_ARG, "bad argument");
  M->gemm = backend;
  return SBM_OK;
}

int sbm_mlp_forward(void* mlp, const float* X_dev, int rows, float* Y_dev) {
  Mlp* M = mlp_of(mlp);
  if (!M || !X_dev || !Y_dev || rows < 0) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    M->ensure_batch(std::max(rows, 1));
    CUDA_TRY(launch_pack_bf16(rows, M->F, M->Fpad, X_dev, M->Xb, M->s));
    M->forward(M->Xb, rows, Y_dev, M->H1, M->H2, M->s);
    return SBM_OK;
  });
}

int sbm_mlp_gradients(void* mlp, const float* X_dev, const float* T_dev, int rows, float* grad_host,
                      double* loss) {
  Mlp* M = mlp_of(mlp);
  if (!M || !X_dev || !T_dev || rows < 1) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    M->ensure_batch(rows);
    CUDA_TRY(launch_pack_bf16(rows, M->F, M->Fpad, X_dev, M->Xb, M->s));
    CUDA_TRY(cudaMemcpyAsync(M->Tb, T_dev, (size_t)rows * M->O * sizeof(float), cudaMemcpyDeviceToDevice, M->s));
    M->forward(M->Xb, rows, M->Y, M->H1, M->H2, M->s);
    M->backward(M->Xb, M->Tb, rows);
    const double l = read_loss(*M, rows);
    if (tc_fault_take() != 0) return set_error(SBM_ERR_CUDA, "a tensor-core GEMM commit did not arrive in time");
    if (loss) *loss = l;
    if (grad_host) get_packed(*M, M->G, grad_host);
    return SBM_OK;
  });
}

int sbm_mlp_num_samples(const void* mlp, long long* n) {
  const Mlp* M = static_cast<const Mlp*>(mlp);
  if (!M || !n) return set_error(SBM_ERR_ARG, "bad argument");
  *n = (long long)M->count;
  return SBM_OK;
}

int sbm_mlp_clear_samples(void* mlp) {
  Mlp* M = mlp_of(mlp);
  if (!M) return set_error(SBM_ERR_ARG, "null MLP");
  M->count = 0;
  return SBM_OK;
}

int sbm_mlp_train(void* mlp, int epochs, int batch, float lr, unsigned long long seed, double* loss) {
  Mlp* M = mlp_of(mlp);
  if (!M || epochs < 0 || batch < 1 || !(lr > 0)) return set_error(SBM_ERR_ARG, "bad argument");
  if (M->count == 0) return set_error(SBM_ERR_ARG, "no training samples");
  return guarded([&]() -> int {
    M->ensure_batch(batch);
    const size_t n = M->count;
    std::vector<int> perm(n);
    uint64_t st = seed;
    double last = 0;
    for (int e = 0; e < epochs; ++e) {
      for (size_t i = 0; i < n; ++i) perm[i] = (int)i;
      for (size_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix64(st) % (i + 1)]);   // Fisher-Yates
      CUDA_TRY(cudaMemcpyAsync(M->idx_all, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, M->s));
      CUDA_TRY(cudaMemsetAsync(M->loss_acc, 0, sizeof(float), M->s));
      int nbatch = 0;
      for (size_t b0 = 0; b0 < n; b0 += batch) {
        const int rows = (int)std::min<size_t>(batch, n - b0);
        CUDA_TRY(launch_rows_gather(rows, M->Fpad, M->idx_all + b0, M->Xd, M->Xb, M->O, M->Td, M->Tb, M->s));
        M->forward(M->Xb, rows, M->Y, M->H1, M->H2, M->s);
        M->backward(M->Xb, M->Tb, rows);
        M->adam_t += 1;
        CUDA_TRY(launch_adam((int)M->nparam, M->P, M->G, M->Am, M->Av, M->Pb, lr, 0.9f, 0.999f, 1e-8f, M->adam_t, M->s));
        CUDA_TRY(launch_colsum(152, 1, M->loss_part, M->loss_tmp, M->s));
        CUDA_TRY(launch_axpy_f(1, 1.0f / ((float)rows * M->O), M->loss_tmp, M->loss_acc, M->s));
        ++nbatch;
      }
      float acc = 0;
      CUDA_TRY(cudaMemcpyAsync(&acc, M->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, M->s));
      CUDA_TRY(cudaStreamSynchronize(M->s));
      if (tc_fault_take() != 0) return set_error(SBM_ERR_CUDA, "a tensor-core GEMM commit did not arrive in time");
      last = acc / nbatch;
    }
    if (loss) *loss = last;
    return SBM_OK;
  });
}

int sbm_mlp_target_scale(void* mlp, double* rms) {
  Mlp* M = mlp_of(mlp);
  if (!M || !rms) return set_error(SBM_ERR_ARG, "bad argument");
  if (M->count == 0) return set_error(SBM_ERR_ARG, "no training samples");
  return guarded([&]() -> int {
    const size_t n = M->count * (size_t)M->O;
    const int nblk = 152 * 4;
    double* part = M->alloc<double>(nblk + 1);
    double sum = 0.0;
    cudaError_t e = launch_sumsq(n, M->Td, part, nblk, part + nblk, M->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sum, part + nblk, sizeof(double), cudaMemcpyDeviceToHost, M->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->s);
    M->release(part);
    CUDA_TRY(e);
    double r = std::sqrt(sum / (double)n);
    if (!(r > 0.0) || !std::isfinite(r)) r = 1.0;
    else CUDA_TRY(launch_scale_f(n, (float)(1.0 / r), M->Td, M->s));
    CUDA_TRY(cudaStreamSynchronize(M->s));
    *rms = r;
    return SBM_OK;
  });
}

int sbm_mlp_save(const void* mlp, const char* path) {
  const Mlp* M = static_cast<const Mlp*>(mlp);
  if (!M || !path) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    std::vector<float> w(packed_size(*M));
    get_packed(*M, M->P, w.data());
    int32_t hdr[6] = {1, M->dim, M->p, M->F, M->H, M->O};
    static const unsigned char magic[8] = {'S', 'B', 'M', 'M', 'L', 'P', 0, 0};
    std::vector<unsigned char> buf;
    buf.reserve(8 + sizeof(hdr) + w.size() * sizeof(float));
    buf.insert(buf.end(), magic, magic + 8);
    const unsigned char* hb = reinterpret_cast<const unsigned char*>(hdr);
    buf.insert(buf.end(), hb, hb + sizeof(hdr));
    const unsigned char* wb = reinterpret_cast<const unsigned char*>(w.data());
    buf.insert(buf.end(), wb, wb + w.size() * sizeof(float));
    const uint32_t crc = crc32(buf.data(), buf.size());
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_error(SBM_ERR_ARG, std::string("cannot write ") + path);
    const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size() && std::fwrite(&crc, 4, 1, f) == 1;
    std::fclose(f);
    return ok ? SBM_OK : set_error(SBM_ERR_ARG, std::string("short write to ") + path);
  });
}

int sbm_mlp_load(void* mlp, const char* path) {
  Mlp* M = mlp_of(mlp);
  if (!M || !path) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_error(SBM_ERR_ARG, std::string("cannot read ") + path);
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t k;
    while ((k = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + k);
    std::fclose(f);
    const size_t want = 8 + 24 + packed_size(*M) * sizeof(float) + 4;
    if (buf.size() != want || std::memcmp(buf.data(), "SBMMLP\0\0", 8) != 0)
      return set_error(SBM_ERR_ARG, "not an MLP file of this shape");
    int32_t hdr[6];
    std::memcpy(hdr, buf.data() + 8, sizeof(hdr));
    if (hdr[0] != 1 || hdr[1] != M->dim || hdr[2] != M->p || hdr[3] != M->F || hdr[4] != M->H || hdr[5] != M->O)
      return set_error(SBM_ERR_ARG, "MLP file shape differs");
    uint32_t crc;
    std::memcpy(&crc, buf.data() + want - 4, 4);
    if (crc != crc32(buf.data(), want - 4)) return set_error(SBM_ERR_ARG, "MLP file checksum mismatch");
    std::vector<float> w(packed_size(*M));
    std::memcpy(w.data(), buf.data() + 32, w.size() * sizeof(float));
    set_params(*M, w.data());
    return SBM_OK;
  });
}

int sbm_learned_features(void* ctx, int dtype, const void* res_dev, float* X_dev, float* s_dev) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !res_dev || !X_dev || !s_dev) return set_error(SBM_ERR_ARG, "bad argument");
  return guarded([&]() -> int {
    ensure_learned(*C);
    const HostLevel& H = C->lv[C->finest()].H;
    if (dtype == SBM_F64)
      CUDA_TRY(launch_mlp_features<double>(C->lf_nb, C->lf_npatch, H.np, C->lf_nstat, C->lf_Fpad, C->mlp_patch,
                                           C->mlp_stat, (const double*)res_dev, C->mlp_X, s_dev, C->stream));
    else if (dtype == SBM_F32)
      CUDA_TRY(launch_mlp_features<float>(C->lf_nb, C->lf_npatch, H.np, C->lf_nstat, C->lf_Fpad, C->mlp_patch,
                                          C->mlp_stat, (const float*)res_dev, C->mlp_X, s_dev, C->stream));
    else
      return set_error(SBM_ERR_ARG, "dtype");
    CUDA_TRY(launch_unpack_bf16(C->lf_nb, C->lf_F, C->lf_Fpad, C->mlp_X, X_dev, C->stream));
    return SBM_OK;
  });
}

int sbm_learned_cells(void* ctx, int* n_bnd, int* cells_host) {
  Context* C = ctx_of(ctx);
  if (!C || !n_bnd) return set_error(SBM_ERR_ARG, "bad argument");
  const HostLevel& H = C->lv[C->finest()].H;
  *n_bnd = H.n_bnd;
  if (cells_host && H.n_bnd) std::memcpy(cells_host, H.bnd_cell.data(), H.n_bnd * sizeof(int));
  return SBM_OK;
}

int sbm_collect(void* ctx, void* mlp, int dtype, const void* u0_dev, int n_starts, int n_cycles,
                long long* n_added) {
  Context* C = ctx_of(ctx);
  Mlp* M = mlp_of(mlp);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C || !M || !u0_dev || n_starts < 0 || n_cycles < 0) return set_error(SBM_ERR_ARG, "bad argument");
  const HostLevel& H = C->lv[C->finest()].H;
  if (M->dim != H.dim || M->p != H.p) return set_error(SBM_ERR_ARG, "MLP shape does not match the finest level");
  return guarded([&]() -> int {
    long long n = 0;
    if (dtype == SBM_F64) n = collect_impl<double>(*C, *M, (const double*)u0_dev, n_starts, n_cycles);
    else if (dtype == SBM_F32) n = collect_impl<float>(*C, *M, (const float*)u0_dev, n_starts, n_cycles);
    else return set_error(SBM_ERR_ARG, "dtype");
    if (n_added) *n_added = n;
    return SBM_OK;
  });
}

int sbm_attach_mlp(void* ctx, void* mlp, float scale, double fallback_rate) {
  Context* C = ctx_of(ctx);
  if (C && C->host_only) return set_error(SBM_ERR_ARG, "host-only context");
  if (!C) return set_error(SBM_ERR_ARG, "null context");
  Mlp* M = mlp_of(mlp);
  if (M) {
    const HostLevel& H = C->lv[C->finest()].H;
    if (M->dim != H.dim || M->p != H.p) return set_error(SBM_ERR_ARG, "MLP shape does not match the finest level");
  }
  return guarded([&]() -> int {
    CUDA_TRY(cudaStreamSynchronize(C->stream));
    C->drop_graphs();                               // the captured V-cycles change
    C->mlp = M;
    C->mlp_on = M != nullptr;
    C->mlp_scale = scale;
    C->mlp_rate_ref = fallback_rate;
    if (M) {
      ensure_learned(*C);
      const int nb = std::max(C->lf_nb, 1);
      if (C->mlp_bufH < M->H || C->mlp_bufO < M->O) {   // inference buffers before any capture
        C->mlp_H1 = C->dalloc<__nv_bfloat16>((size_t)nb * M->H);
        C->mlp_H2 = C->dalloc<__nv_bfloat16>((size_t)nb * M->H);
        C->mlp_Y = C->dalloc<float>((size_t)nb * M->O);
        C->mlp_bufH = M->H;
        C->mlp_bufO = M->O;
      }
    }
    return SBM_OK;
  });
}

}  // extern "C"
