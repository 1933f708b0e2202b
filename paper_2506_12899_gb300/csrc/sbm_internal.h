// Internal data structures of libsbm: host-side level set-up and the device parameter blocks.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "sbm.h"

namespace sbm {

constexpr int kMaxN1 = 4;          // p + 1 <= 4
constexpr int kMaxLevels = 16;

// ---------------------------------------------------------------------------------------------
// One-dimensional reference data of the nodal Gauss-Legendre Lagrange basis of degree p on [0,1].
struct Basis1D {
  int p = 1, n1 = 2;
  double x[kMaxN1] = {}, w[kMaxN1] = {};          // nodes and weights
  double Dm[kMaxN1 * kMaxN1] = {};                // Dm[i*n1+k] = l_k'(x_i)
  double e0[kMaxN1] = {}, e1[kMaxN1] = {};        // l_k(0), l_k(1)
  double d0[kMaxN1] = {}, d1[kMaxN1] = {};        // l_k'(0), l_k'(1)
  double Khat[kMaxN1 * kMaxN1] = {};              // sum_q w_q l_i'(x_q) l_j'(x_q)
};

void gauss_legendre01(int n, double* x, double* w);
void lagrange_eval(int n1, const double* nodes, double y, double* val, double* der);
Basis1D make_basis(int p);

// ---------------------------------------------------------------------------------------------
// Host copy of everything one multigrid level needs.
struct HostLevel {
  int dim = 2, n = 0, p = 1, n1 = 2, np = 4, nq = 2, nslot = 4, ncol = 4;
  double h = 0, lo[3] = {0, 0, 0};
  double sigF_hat = 0, sigG_hat = 0, alpha = 1, omega = 1;
  int extension = 0;
  int n_act = 0, n_bnd = 0, n_sface = 0;
  std::vector<int> cell;            // [n_act][3] background multi-index, compact order
  std::vector<int> bg2act;          // [n^dim] compact index or -1
  std::vector<int> nbr;             // [nslot][n_act] neighbour compact index or -1 (slot = 2*dir+side)
  int colour_start[9] = {}, colour_nbnd[8] = {}, bstart[8] = {};
  std::vector<double> dhat;         // [n_bnd][nslot][dim][nq]  d / h (zero on non-surrogate slots)
  std::vector<double> binvT;        // [n_bnd][np][np]  (A_KK^{-1})^T: element (j, i) at j*np + i
  std::vector<int> parent_code;     // [n_act] (parent compact index << 3) | child bits, or -1
  std::vector<int> children;        // [2^dim][n_act] compact index of child in the next finer level
  std::vector<int> sf_cell, sf_slot;
  std::vector<double> sf_d;         // [n_sface][nq][3]
  Basis1D B;
  double L[4][kMaxN1 * kMaxN1] = {}; // self 1D matrices by neighbour mask (left active) + 2*(right active)
  double Bmp[kMaxN1 * kMaxN1] = {};  // coupling to the right neighbour (this cell is K-)
  double Bpm[kMaxN1 * kMaxN1] = {};  // coupling to the left neighbour (this cell is K+)
  double Bmm[kMaxN1 * kMaxN1] = {};  // own half of the right interior face (this cell is K-)
  double Bpp[kMaxN1 * kMaxN1] = {};  // own half of the left interior face (this cell is K+)
  double S[kMaxN1 * kMaxN1] = {}, lam[kMaxN1] = {};   // W-orthonormal eigenvectors / values of L[3]
  std::vector<double> coarse_inv;   // [N*N] on the coarsest level only
  // learned boundary-cell correction: per boundary cell the compact indices of the 3^dim patch
  // cells K + o (o in {-1,0,1}^dim, x fastest; -1 inactive or outside) and the static features
  // [d/h per (slot, face point, component)], kappa, [surrogate mask per slot]
  std::vector<int> patch;           // [n_bnd][3^dim]
  std::vector<int> bnd_cell;        // [n_bnd] compact index of each boundary cell
  std::vector<double> mlp_static;   // [n_bnd][2 dim nq dim + 1 + 2 dim]
  int n_dof() const { return n_act * np; }
  bool is_boundary(int a, int* bidx) const;
};

struct SetupError {
  int code;
  std::string msg;
};

// Builds one level; throws SetupError.  (Geometry of Sec. 2.1 / Sec. 4.2, element data of Eq. 11.)
// device: the volume fractions and the closest points run as device kernels (geometry_ops.cu)
// unless d.device_geometry < 0.
// counts_cache: the sub-cell sample counts of the volume fractions on an n-cell mesh, shared by the
// levels of one mesh size (the p-levels): used when it holds n^dim entries, else filled.
HostLevel build_level(const sbm_setup_desc& d, int n, int p, bool device = false,
                      std::vector<int>* counts_cache = nullptr);
// Device set-up kernels (geometry_ops.cu); throw SetupError on CUDA failures.
void device_volume_counts(const sbm_setup_desc& d, int n, double h, int s, std::vector<int>& counts);
void device_closest_points(const sbm_setup_desc& d, const std::vector<double>& samples, const std::vector<double>& X,
                           std::vector<double>& C, std::vector<int>& ok);
// Links a coarse and the next finer level (parent / children tables for h-transfers).
void link_levels(HostLevel& coarse, HostLevel& fine);
// Dense coarse inverse (host LU with partial pivoting).
void build_coarse_inverse(HostLevel& L0);
// Finest-level right-hand side of Eq. 11 in compact layout.
std::vector<double> build_rhs(const sbm_setup_desc& d, const HostLevel& L);
// Host evaluation of y = A x on a whole level (set-up checks without a GPU).
void host_apply_level(const HostLevel& L, const double* x, double* y);
// Host evaluation of A_KK applied to one local vector (used for the dense cell blocks).
void cell_self_apply(const HostLevel& L, int a, int bidx, const double* u, double* y);

// ---------------------------------------------------------------------------------------------
// Small 1D element matrices of one level (copied to shared memory by every kernel block).
template <typename R>
struct LevelConsts {
  R L[4][kMaxN1 * kMaxN1];          // self matrices by neighbour mask
  R Bmp[kMaxN1 * kMaxN1], Bpm[kMaxN1 * kMaxN1];
  R Kh[kMaxN1 * kMaxN1];            // volume stiffness alone
  R Bmm[kMaxN1 * kMaxN1], Bpp[kMaxN1 * kMaxN1];   // own halves of the right / left interior face
  R Dm[kMaxN1 * kMaxN1];
  R S[kMaxN1 * kMaxN1];             // fast-diagonalisation eigenvectors (columns)
  R w[kMaxN1], e0[kMaxN1], e1[kMaxN1], d0[kMaxN1], d1[kMaxN1];
  R x[kMaxN1], inv_denom[kMaxN1];   // nodes and 1 / prod_{j != k}(x_k - x_j)
  R lam[kMaxN1];
  R inv_diag[kMaxN1 * kMaxN1 * kMaxN1];   // 1 / (h^(d-2) (lam_i + lam_j (+ lam_k))), x fastest
};

// Parameters of the L2-error kernel (error_ops.cu): finest level, (p+3)-point Gauss-Legendre rule on
// [0, 1], the 1D Lagrange values V[q * kMaxN1 + k] = l_k(xq[q]) of the cell basis at its points.
struct L2ErrorParams {
  int n_act, kind;
  double h, lo[3];
  double xq[8], wq[8];
  double V[8 * kMaxN1];
};

// Device parameter block of one level for one precision (passed by value to the kernels).
template <typename R>
struct LevelParams {
  int n_act;
  int colour_start[9], colour_nbnd[8], bstart[8];
  const int* nbr;
  const R* dhat;
  const R* binvT;
  // dense self blocks h^(d-2) A_KK of the boundary cells (Eqs. 10, 7), column j at bself_ld * b + np * j
  // (double-float operator of a 3D p = 1 finest level only; null elsewhere)
  const R* bself;
  int bself_ld;
  R hscale;                        // h^(dim-2)
  R sigG, alpha, omega;
  int extension;
  int cell_min;                    // launches over >= cell_min cells use thread-per-cell kernels (0: never)
  int staged_min;                  // FP32 launches over >= staged_min cells use the staged kernels (0: never)
  int ordering;                    // smoother colour groups: 0 by odd-bit count of the colour, 1 red-black
  LevelConsts<R> k;
};

// The cells one smoother launch updates: the colours of one colour group (equal number of odd
// index bits), each as a boundary segment then an interior segment.  Segment k covers cells
// [first[k], last[k]) of colour col[k] (colour starting at cs[k], nbnd[k] boundary cells, boundary
// index b0[k] of its first cell) and blocks [blk[k], blk[k + 1]) of the grid.
struct SmoothSegs {
  static constexpr int kMax = 8;
  int n;
  int first[kMax], last[kMax], col[kMax], cs[kMax], nbnd[kMax], b0[kMax];
  int blk[kMax + 1];
};

// Transfer parameter block between level l-1 (coarse) and l (fine).
template <typename R>
struct TransferParams {
  int n_act_f, n_act_c;
  int hmode;                       // 1: h-transfer (both p = 1), 0: p-transfer on the same mesh
  const int* parent_code;          // fine [n_act_f]
  const int* children;             // coarse [2^d][n_act_c]
  R Ph[2][kMaxN1 * kMaxN1];        // h: Ph[o][i*nc + j] = l^c_j((o + x^f_i)/2)
  R Pp[kMaxN1 * kMaxN1];           // p: Pp[i*nc + j] = l^c_j(x^f_i)
};

// One level of the cluster V-cycle tail (device memory): parameters, the transfer from the next
// coarser level, and where the level's vectors live in every CTA's shared memory: colour c is
// cut into chunks of m[c] cells (chunk k on CTA k), stored from cell slot off[c]; z and the
// right-hand side start at element offsets zoff and roff, ncell cell slots each.
template <typename R>
struct TailLevel {
  LevelParams<R> P;
  TransferParams<R> T;
  int m[8], off[8];
  int ncell, zoff, roff;
};

// One-CTA V-cycle tail: the coarse p = 1 levels 0..top in a single CTA, with every level vector,
// neighbour table, transfer table and boundary-cell inverse staged in its shared memory.  The
// whole block is a kernel parameter (__grid_constant__), so every level constant is a constant-
// bank read.  Offsets are in elements of R (vectors, inverses) or of int (tables).
constexpr int kMaxTailCta = 6;
template <typename R>
struct TailCta {
  int top, pre, post, ssor;
  int zoff[kMaxTailCta], roff[kMaxTailCta], boff[kMaxTailCta];
  int noff[kMaxTailCta], coff[kMaxTailCta], poff[kMaxTailCta];   // nbr, children, parent codes
  int n_bnd[kMaxTailCta];
  unsigned int_base;               // byte offset of the int area
  int bulk;                        // 1: tables staged by bulk asynchronous copies (every table and
                                   // its shared-memory slot 16-byte aligned), 0: by plain loads
  unsigned cinv_off;               // byte offset of the staged FP64 coarse inverse, 0: read from global
  LevelParams<R> P[kMaxTailCta];
  TransferParams<R> T[kMaxTailCta];
};

// Launch shape of the cluster tail of one precision: cluster size (CTAs), dynamic shared
// memory per CTA, and the element offset of the coarse right-hand-side gather buffer.
struct TailPlan {
  int top = -1;
  int cluster = 0;                 // 1: the one-CTA tail kernel
  size_t smem_bytes = 0;
  int gather_off = 0;
};

}  // namespace sbm
