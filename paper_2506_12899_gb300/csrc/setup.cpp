// Host-side, one-time set-up of libsbm (FP64): geometry, 1D element data, dense cell blocks,
// fast-diagonalisation factors, the coarse inverse and the right-hand side.
//
// Paper: arXiv 2506.12899.  Sec. 2.1 (volume fraction Eq. 4, active cells, shift d = x - x~),
// Sec. 4.2 (closest point by Newton on the Lagrangian, Eqs. 19-22), Sec. 2.2 (DG-SBM form,
// Eqs. 7, 10, 11), Sec. 3.1 (cell blocks A_i = R_i A R_i^T, Eq. 14).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>

#include "sbm_internal.h"
#include "geometry.cuh"

namespace sbm {

namespace {


int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int num_threads() {
  unsigned t = std::thread::hardware_concurrency();
  return t == 0 ? 4 : (int)std::min(t, 64u);
}

// Runs body(i) for i in [0, n) on all host cores (static chunks).
void parallel_for(int n, const std::function<void(int, int)>& body) {
  int nt = std::min(num_threads(), std::max(1, n / 64));
  if (nt <= 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  int chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    int b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back(body, b, e);
  }
  for (auto& x : th) x.join();
}

[[noreturn]] void fail(int code, const std::string& msg) { throw SetupError{code, msg}; }

// Fixed sampling of the true boundary (start points for the closest-point Newton solve):
// star / deformed 2D domain: 1024 rays theta_k = 2 pi k / 1024 (the deformed domain's radius by
// 64 bisection steps on [0, 2]); ellipsoid: 64 x 128 points u_i = pi (i + 1/2) / 64,
// v_j = 2 pi j / 128 of c + R diag(semi) (sin u cos v, sin u sin v, cos u).  Row-major [k][dim].
std::vector<double> boundary_samples(const Shape& sh) {
  std::vector<double> out;
  const double* c = sh.s.center;
  if (sh.s.kind == SBM_SHAPE_STAR || sh.s.kind == SBM_SHAPE_COMPLEX2D) {
    for (int k = 0; k < 1024; ++k) {
      const double th = 2.0 * kPi * k / 1024.0;
      double r;
      if (sh.s.kind == SBM_SHAPE_STAR) {
        r = sh.s.radius * (1.0 + sh.s.amp * std::sin(sh.s.freq * th + sh.s.phase));
      } else {
        double lo = 0.0, hi = 2.0;
        for (int it = 0; it < 64; ++it) {
          const double mid = 0.5 * (lo + hi);
          const double X[2] = {mid * std::cos(th), mid * std::sin(th)};
          if (sh.phi(X) < 0.0) lo = mid; else hi = mid;
        }
        r = 0.5 * (lo + hi);
      }
      const double ox = sh.s.kind == SBM_SHAPE_STAR ? c[0] : 0.0, oy = sh.s.kind == SBM_SHAPE_STAR ? c[1] : 0.0;
      out.push_back(ox + r * std::cos(th));
      out.push_back(oy + r * std::sin(th));
    }
  } else if (sh.s.kind == SBM_SHAPE_ELLIPSOID) {
    for (int i = 0; i < 64; ++i)
      for (int j = 0; j < 128; ++j) {
        const double u = kPi * (i + 0.5) / 64.0, v = 2.0 * kPi * j / 128.0;
        const double l[3] = {sh.s.semi[0] * std::sin(u) * std::cos(v), sh.s.semi[1] * std::sin(u) * std::sin(v),
                             sh.s.semi[2] * std::cos(u)};
        for (int r = 0; r < 3; ++r)
          out.push_back(c[r] + sh.s.rot[r * 3 + 0] * l[0] + sh.s.rot[r * 3 + 1] * l[1] + sh.s.rot[r * 3 + 2] * l[2]);
      }
  }
  return out;
}

// --------------------------------------------------------------------- manufactured solutions
double u_exact(int kind, int dim, const double* X) {
  double x = X[0], y = X[1], z = dim > 2 ? X[2] : 0.0;
  switch (kind) {
    case SBM_U_SINPROD: {
      double v = std::sin(kPi * x) * std::sin(kPi * y);
      return dim == 3 ? v * std::sin(kPi * z) : v;
    }
    case SBM_U_EXPCOS: return std::exp(x) * std::cos(2 * y);
    case SBM_U_LINEAR: return 0.5 + x - 0.7 * y + 0.3 * z;
    case SBM_U_COSSIN: return 2 * std::cos(x) * std::sin(y);
    case SBM_U_QUADRATIC:
      return 0.5 + x - 0.7 * y + 0.3 * z + x * x - 0.5 * y * y + 0.25 * x * y - 0.4 * z * z + 0.2 * y * z;
    case SBM_U_PHIP1: {
      double s = std::sin(kPi * x);
      return (1 - 0.75 * s * s) * (x * x + y * y) + 0.8;
    }
  }
  return 0.0;
}

double f_source(int kind, int dim, const double* X) {
  double x = X[0], y = X[1];
  switch (kind) {
    case SBM_U_SINPROD: return dim * kPi * kPi * u_exact(kind, dim, X);
    case SBM_U_EXPCOS: return 3.0 * u_exact(kind, dim, X);
    case SBM_U_LINEAR: return 0.0;
    case SBM_U_COSSIN: return 2.0 * u_exact(kind, dim, X);
    case SBM_U_QUADRATIC: return dim == 3 ? -0.2 : -1.0;
    case SBM_U_PHIP1: {
      double s2 = std::sin(kPi * x);
      s2 *= s2;
      double a = 1 - 0.75 * s2, ap = -0.75 * kPi * std::sin(2 * kPi * x);
      double app = -1.5 * kPi * kPi * std::cos(2 * kPi * x);
      return -(app * (x * x + y * y) + 4 * ap * x + 4 * a);
    }
  }
  return 0.0;
}

// --------------------------------------------------------------------- dense inverse
// Gauss-Jordan with partial pivoting; returns min|pivot| / max|pivot| (0 if singular).
double dense_inverse(int n, std::vector<double>& A, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  double pmin = 1e300, pmax = 0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > std::fabs(A[(size_t)piv * n + k])) piv = i;
    double pv = A[(size_t)piv * n + k];
    if (pv == 0.0 || !std::isfinite(pv)) return 0.0;
    pmin = std::min(pmin, std::fabs(pv));
    pmax = std::max(pmax, std::fabs(pv));
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)k * n + j], A[(size_t)piv * n + j]);
        std::swap(inv[(size_t)k * n + j], inv[(size_t)piv * n + j]);
      }
    }
    double ip = 1.0 / A[(size_t)k * n + k];
    for (int j = 0; j < n; ++j) {
      A[(size_t)k * n + j] *= ip;
      inv[(size_t)k * n + j] *= ip;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      double f = A[(size_t)i * n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
        inv[(size_t)i * n + j] -= f * inv[(size_t)k * n + j];
      }
    }
  }
  return pmin / pmax;
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (n <= 4): A = Q diag(lam) Q^T.
void jacobi_eigen(int n, const double* A_in, double* Q, double* lam) {
  double A[16];
  std::memcpy(A, A_in, sizeof(double) * n * n);
  for (int i = 0; i < n * n; ++i) Q[i] = 0;
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-30) break;
    for (int pq = 0; pq < n * n; ++pq) {
      int p = pq / n, q = pq % n;
      if (q <= p || std::fabs(A[p * n + q]) < 1e-300) continue;
      double theta = (A[q * n + q] - A[p * n + p]) / (2 * A[p * n + q]);
      double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
      double cs = 1 / std::sqrt(t * t + 1), sn = t * cs;
      for (int k = 0; k < n; ++k) {              // A <- J^T A J (columns p, q)
        double akp = A[k * n + p], akq = A[k * n + q];
        A[k * n + p] = cs * akp - sn * akq;
        A[k * n + q] = sn * akp + cs * akq;
      }
      for (int k = 0; k < n; ++k) {              // rows p, q
        double apk = A[p * n + k], aqk = A[q * n + k];
        A[p * n + k] = cs * apk - sn * aqk;
        A[q * n + k] = sn * apk + cs * aqk;
      }
      for (int k = 0; k < n; ++k) {
        double qkp = Q[k * n + p], qkq = Q[k * n + q];
        Q[k * n + p] = cs * qkp - sn * qkq;
        Q[k * n + q] = sn * qkp + cs * qkq;
      }
    }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[i * n + i];
}

int digit(int i, int k, int n1) {
  for (int j = 0; j < k; ++j) i /= n1;
  return i % n1;
}

// Tangential index t of local dof i on a face normal to `dir` (tangential dims ascending,
// first one fastest) and the tensor weight w_t.
int tangential_index(const HostLevel& L, int i, int dir, double* wt) {
  int t = 0, mul = 1;
  double w = 1;
  for (int k = 0; k < L.dim; ++k) {
    if (k == dir) continue;
    int dk = digit(i, k, L.n1);
    t += dk * mul;
    mul *= L.n1;
    w *= L.B.w[dk];
  }
  if (wt) *wt = w;
  return t;
}

// Local dof index from (k along dir, tangential index t).
int dof_index(const HostLevel& L, int dir, int k, int t) {
  int i = 0, stride = 1;
  for (int m = 0; m < L.dim; ++m) {
    int dm;
    if (m == dir) {
      dm = k;
    } else {
      dm = t % L.n1;
      t /= L.n1;
    }
    i += dm * stride;
    stride *= L.n1;
  }
  return i;
}

}  // namespace

// ------------------------------------------------------------------------------ basis
void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double p0 = 1, p1 = z, dp = 1;
    for (int it = 0; it < 100; ++it) {
      p0 = 1;
      p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    p0 = 1;
    p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1 - z * z) * dp * dp);
  }
}

void lagrange_eval(int n1, const double* nodes, double y, double* val, double* der) {
  for (int k = 0; k < n1; ++k) {
    double v = 1;
    for (int j = 0; j < n1; ++j)
      if (j != k) v *= (y - nodes[j]) / (nodes[k] - nodes[j]);
    val[k] = v;
    if (der) {
      double d = 0;
      for (int i = 0; i < n1; ++i) {
        if (i == k) continue;
        double term = 1.0 / (nodes[k] - nodes[i]);
        for (int j = 0; j < n1; ++j)
          if (j != k && j != i) term *= (y - nodes[j]) / (nodes[k] - nodes[j]);
        d += term;
      }
      der[k] = d;
    }
  }
}

Basis1D make_basis(int p) {
  Basis1D B;
  B.p = p;
  B.n1 = p + 1;
  const int n1 = B.n1;
  gauss_legendre01(n1, B.x, B.w);
  double v[kMaxN1], dv[kMaxN1];
  for (int i = 0; i < n1; ++i) {
    lagrange_eval(n1, B.x, B.x[i], v, dv);
    for (int k = 0; k < n1; ++k) B.Dm[i * n1 + k] = dv[k];
  }
  lagrange_eval(n1, B.x, 0.0, B.e0, B.d0);
  lagrange_eval(n1, B.x, 1.0, B.e1, B.d1);
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      double acc = 0;
      for (int q = 0; q < n1; ++q) acc += B.w[q] * B.Dm[q * n1 + i] * B.Dm[q * n1 + j];
      B.Khat[i * n1 + j] = acc;
    }
  return B;
}

bool HostLevel::is_boundary(int a, int* bidx) const {
  int c = 0;
  while (c + 1 < ncol && a >= colour_start[c + 1]) ++c;
  int off = a - colour_start[c];
  if (off < colour_nbnd[c]) {
    if (bidx) *bidx = bstart[c] + off;
    return true;
  }
  if (bidx) *bidx = -1;
  return false;
}

// ------------------------------------------------------------------------------ cell operator
// y = A_KK u for one cell (reference form times h^(dim-2)): volume stiffness, the cell's own
// halves of interior-face terms (Eq. 10) and the Nitsche-SBM terms of its surrogate faces (Eq. 7).
void cell_self_apply(const HostLevel& L, int a, int bidx, const double* u, double* y) {
  const int n1 = L.n1, np = L.np, dim = L.dim, nq = L.nq;
  for (int i = 0; i < np; ++i) y[i] = 0;
  for (int dir = 0; dir < dim; ++dir) {
    int stride = ipow(n1, dir);
    int aL = L.nbr[(size_t)(2 * dir) * L.n_act + a] >= 0;
    int aR = L.nbr[(size_t)(2 * dir + 1) * L.n_act + a] >= 0;
    const double* M = L.L[aL + 2 * aR];
    for (int i = 0; i < np; ++i) {
      int id = digit(i, dir, n1), base = i - id * stride;
      double wt;
      tangential_index(L, i, dir, &wt);
      double s = 0;
      for (int k = 0; k < n1; ++k) s += M[id * n1 + k] * u[base + k * stride];
      y[i] += wt * s;
    }
  }
  if (bidx >= 0) {
    for (int slot = 0; slot < 2 * dim; ++slot) {
      if (L.nbr[(size_t)slot * L.n_act + a] >= 0) continue;
      const int dir = slot >> 1, side = slot & 1;
      const double sg = side ? 1.0 : -1.0;
      const double* es = side ? L.B.e1 : L.B.e0;
      const double* ds = side ? L.B.d1 : L.B.d0;
      const double* dh = &L.dhat[((size_t)bidx * L.nslot + slot) * dim * nq];
      std::vector<double> U(nq), Gn(nq), E(nq);
      for (int t = 0; t < nq; ++t) {
        double su = 0, sd = 0;
        for (int k = 0; k < n1; ++k) {
          double uk = u[dof_index(L, dir, k, t)];
          su += es[k] * uk;
          sd += ds[k] * uk;
        }
        U[t] = su;
        Gn[t] = sd;
      }
      for (int t = 0; t < nq; ++t) {
        if (L.extension == 0) {
          double e = U[t] + dh[dir * nq + t] * Gn[t];
          int tt = t, mul = 1;
          for (int m = 0; m < dim; ++m) {        // tangential derivatives from the trace values
            if (m == dir) continue;
            int tm = tt % n1;
            tt /= n1;
            double g = 0;
            for (int q = 0; q < n1; ++q) g += L.B.Dm[tm * n1 + q] * U[t + (q - tm) * mul];
            e += dh[m * nq + t] * g;
            mul *= n1;
          }
          E[t] = e;
        } else {                                   // cell polynomial at x~ + d
          double lv[3][kMaxN1];
          int tt = t;
          for (int m = 0; m < dim; ++m) {
            double xi;
            if (m == dir) {
              xi = side;
            } else {
              xi = L.B.x[tt % n1];
              tt /= n1;
            }
            lagrange_eval(n1, L.B.x, xi + dh[m * nq + t], lv[m], nullptr);
          }
          double e = 0;
          for (int j = 0; j < np; ++j) {
            double ph = 1;
            for (int m = 0; m < dim; ++m) ph *= lv[m][digit(j, m, n1)];
            e += ph * u[j];
          }
          E[t] = e;
        }
      }
      for (int i = 0; i < np; ++i) {
        int id = digit(i, dir, n1);
        double wt;
        int t = tangential_index(L, i, dir, &wt);
        y[i] += wt * (es[id] * (-sg * Gn[t] + L.sigG_hat * E[t]) - L.alpha * sg * ds[id] * E[t]);
      }
    }
  }
  const double hs = std::pow(L.h, dim - 2);
  for (int i = 0; i < np; ++i) y[i] *= hs;
}

// ------------------------------------------------------------------------------ level set-up
HostLevel build_level(const sbm_setup_desc& d, int n, int p, bool device, std::vector<int>* counts_cache) {
  HostLevel L;
  L.dim = d.dim;
  L.n = n;
  L.p = p;
  L.n1 = p + 1;
  L.np = ipow(L.n1, d.dim);
  L.nq = ipow(L.n1, d.dim - 1);
  L.nslot = 2 * d.dim;
  L.ncol = 1 << d.dim;
  const int dim = d.dim, n1 = L.n1, np = L.np, nq = L.nq;
  L.h = (d.hi[0] - d.lo[0]) / n;
  for (int k = 0; k < dim; ++k) L.lo[k] = d.lo[k];
  L.sigF_hat = d.sigma_face_c * (p + 1) * (p + 1);
  L.sigG_hat = d.sigma_bnd_c * (p + 1) * (p + 1);
  L.alpha = d.alpha;
  L.omega = (p == 3) ? d.omega_p3 : d.omega;
  L.extension = d.extension;
  L.B = make_basis(p);
  Shape sh{d.shape, dim};

  // volume fractions from sub-cell midpoint signs (Eq. 4 with the cheap surrogate of Sec. 2.1)
  const int s = d.vf_samples > 0 ? d.vf_samples : (dim == 2 ? 16 : 8);
  const int S = ipow(s, dim);
  const size_t nbg = (size_t)ipow(n, dim);
  std::vector<unsigned char> active(nbg, 0);
  std::vector<int> counts(nbg, 0);
  const double thr = d.lambda * S;
  const bool dev_geo = device && d.device_geometry >= 0;
  if (counts_cache && counts_cache->size() == nbg) {   // a level of the same mesh counted them
    counts = *counts_cache;
    for (size_t lin = 0; lin < nbg; ++lin)
      active[lin] = d.lambda_inclusive ? (counts[lin] >= thr) : (counts[lin] > thr);
  } else if (dev_geo) {                            // counts on the device (geometry_ops.cu)
    device_volume_counts(d, n, L.h, s, counts);
    for (size_t lin = 0; lin < nbg; ++lin)
      active[lin] = d.lambda_inclusive ? (counts[lin] >= thr) : (counts[lin] > thr);
  } else parallel_for((int)nbg, [&](int b, int e) {
    for (int lin = b; lin < e; ++lin) {
      int idx[3] = {lin % n, (lin / n) % n, dim > 2 ? lin / (n * n) : 0};
      int count = 0;
      for (int q = 0; q < S; ++q) {
        double X[3];
        int qq = q;
        for (int k = 0; k < dim; ++k) {
          X[k] = d.lo[k] + L.h * (idx[k] + ((qq % s) + 0.5) / s);
          qq /= s;
        }
        count += sh.phi(X) < 0.0;
      }
      counts[lin] = count;
      active[lin] = d.lambda_inclusive ? (count >= thr) : (count > thr);
    }
  });
  if (counts_cache && counts_cache->size() != nbg) *counts_cache = counts;

  auto lin_of = [&](const int* idx) {
    int lin = 0;
    for (int k = dim - 1; k >= 0; --k) lin = lin * n + idx[k];
    return lin;
  };
  auto nb_lin = [&](const int* idx, int slot) {
    int j[3] = {idx[0], idx[1], idx[2]};
    int dir = slot >> 1;
    j[dir] += (slot & 1) ? 1 : -1;
    if (j[dir] < 0 || j[dir] >= n) return -1;
    return lin_of(j);
  };

  // compact order: colour-major; within a colour, boundary cells then interior cells.  The
  // boundary cells are ordered by the set of their faces without a neighbour (the surrogate
  // faces), then by background index: a warp of boundary cells then mostly evaluates one set of
  // surrogate-face terms, not the union of its lanes' sets.  Cells of one colour do not couple,
  // so the order within a colour changes no result of the smoother or the operator.
  std::vector<std::vector<std::pair<int, int>>> bnd_keyed(L.ncol);
  std::vector<std::vector<int>> bnd(L.ncol), inner(L.ncol);
  for (size_t lin = 0; lin < nbg; ++lin) {
    if (!active[lin]) continue;
    int idx[3] = {(int)(lin % n), (int)((lin / n) % n), dim > 2 ? (int)(lin / ((size_t)n * n)) : 0};
    int col = 0;
    for (int k = 0; k < dim; ++k) col |= (idx[k] & 1) << k;
    int mask = 0;
    for (int slot = 0; slot < 2 * dim; ++slot) {
      int nl = nb_lin(idx, slot);
      if (nl < 0 || !active[nl]) mask |= 1 << slot;
    }
    if (mask) bnd_keyed[col].push_back({mask, (int)lin});
    else inner[col].push_back((int)lin);
  }
  for (int c = 0; c < L.ncol; ++c) {
    std::sort(bnd_keyed[c].begin(), bnd_keyed[c].end());
    for (const auto& e : bnd_keyed[c]) bnd[c].push_back(e.second);
  }
  L.bg2act.assign(nbg, -1);
  std::vector<int> order;
  int nb_total = 0;
  for (int c = 0; c < L.ncol; ++c) {
    L.colour_start[c] = (int)order.size();
    L.colour_nbnd[c] = (int)bnd[c].size();
    L.bstart[c] = nb_total;
    nb_total += (int)bnd[c].size();
    order.insert(order.end(), bnd[c].begin(), bnd[c].end());
    order.insert(order.end(), inner[c].begin(), inner[c].end());
  }
  L.n_act = (int)order.size();
  L.n_bnd = nb_total;
  for (int c = L.ncol; c < 9; ++c) L.colour_start[c] = L.n_act;
  L.cell.assign((size_t)L.n_act * 3, 0);
  for (int a = 0; a < L.n_act; ++a) {
    int lin = order[a];
    L.bg2act[lin] = a;
    L.cell[3 * a + 0] = lin % n;
    L.cell[3 * a + 1] = (lin / n) % n;
    L.cell[3 * a + 2] = dim > 2 ? lin / (n * n) : 0;
  }
  L.nbr.assign((size_t)L.nslot * L.n_act, -1);
  for (int a = 0; a < L.n_act; ++a)
    for (int slot = 0; slot < L.nslot; ++slot) {
      int nl = nb_lin(&L.cell[3 * a], slot);
      L.nbr[(size_t)slot * L.n_act + a] = nl >= 0 ? L.bg2act[nl] : -1;
    }
  if (L.n_act == 0) return L;

  // 1D matrices with penalties (reference form of Eq. 10, factor h^(dim-2) applied separately)
  const Basis1D& B = L.B;
  const double sg = L.sigF_hat;
  double Bmm[16], Bpp[16];
  for (int i = 0; i < n1; ++i)
    for (int j = 0; j < n1; ++j) {
      int ij = i * n1 + j;
      Bmm[ij] = -0.5 * B.e1[i] * B.d1[j] - 0.5 * B.d1[i] * B.e1[j] + sg * B.e1[i] * B.e1[j];
      L.Bmp[ij] = -0.5 * B.e1[i] * B.d0[j] + 0.5 * B.d1[i] * B.e0[j] - sg * B.e1[i] * B.e0[j];
      L.Bpm[ij] = 0.5 * B.e0[i] * B.d1[j] - 0.5 * B.d0[i] * B.e1[j] - sg * B.e0[i] * B.e1[j];
      Bpp[ij] = 0.5 * B.e0[i] * B.d0[j] + 0.5 * B.d0[i] * B.e0[j] + sg * B.e0[i] * B.e0[j];
    }
  for (int mask = 0; mask < 4; ++mask)
    for (int ij = 0; ij < n1 * n1; ++ij)
      L.L[mask][ij] = B.Khat[ij] + ((mask & 2) ? Bmm[ij] : 0.0) + ((mask & 1) ? Bpp[ij] : 0.0);
  for (int ij = 0; ij < n1 * n1; ++ij) {
    L.Bmm[ij] = Bmm[ij];
    L.Bpp[ij] = Bpp[ij];
  }

  // fast diagonalisation of the interior block: L[3] s = lambda W s
  {
    double M[16], Q[16];
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) M[i * n1 + j] = L.L[3][i * n1 + j] / std::sqrt(B.w[i] * B.w[j]);
    jacobi_eigen(n1, M, Q, L.lam);
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) L.S[i * n1 + j] = Q[i * n1 + j] / std::sqrt(B.w[i]);
    double lmin = 1e300, lmax = 0;
    for (int i = 0; i < n1; ++i) {
      lmin = std::min(lmin, std::fabs(L.lam[i]));
      lmax = std::max(lmax, std::fabs(L.lam[i]));
    }
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j)
        if (std::fabs(L.lam[i] + L.lam[j]) < 1e-13 * lmax) fail(SBM_ERR_SINGULAR_BLOCK, "interior block is singular");
  }

  // surrogate faces: points x~ and shifts d (Sec. 2.1, Sec. 4.2)
  L.dhat.assign((size_t)L.n_bnd * L.nslot * dim * nq, 0.0);
  std::vector<int> bcell(L.n_bnd);
  for (int a = 0; a < L.n_act; ++a) {
    int bidx;
    if (L.is_boundary(a, &bidx)) bcell[bidx] = a;
  }
  std::vector<int> newton_fail(L.n_bnd, 0);
  const std::vector<double> samples = boundary_samples(sh);
  // surrogate-face point t of slot `slot` of cell a: X (3 entries, zero beyond dim)
  auto face_point = [&](int a, int slot, int t, double* X) {
    const int dir = slot >> 1, side = slot & 1;
    int tt = t;
    for (int k = 0; k < 3; ++k) X[k] = 0.0;
    for (int k = 0; k < dim; ++k) {
      double xi;
      if (k == dir) {
        xi = side;
      } else {
        xi = B.x[tt % n1];
        tt /= n1;
      }
      X[k] = d.lo[k] + L.h * (L.cell[3 * a + k] + xi);
    }
  };
  if (dev_geo) {                                   // closest points on the device (geometry_ops.cu)
    std::vector<double> Xs, Cs;
    std::vector<int> oks;
    for (int b = 0; b < L.n_bnd; ++b)
      for (int slot = 0; slot < L.nslot; ++slot) {
        if (L.nbr[(size_t)slot * L.n_act + bcell[b]] >= 0) continue;
        for (int t = 0; t < nq; ++t) {
          double X[3];
          face_point(bcell[b], slot, t, X);
          Xs.insert(Xs.end(), X, X + 3);
        }
      }
    device_closest_points(d, samples, Xs, Cs, oks);
    size_t i = 0;
    for (int b = 0; b < L.n_bnd; ++b)
      for (int slot = 0; slot < L.nslot; ++slot) {
        if (L.nbr[(size_t)slot * L.n_act + bcell[b]] >= 0) continue;
        for (int t = 0; t < nq; ++t, ++i) {
          if (!oks[i]) newton_fail[b] = 1;
          for (int k = 0; k < dim; ++k)
            L.dhat[(((size_t)b * L.nslot + slot) * dim + k) * nq + t] = (Cs[3 * i + k] - Xs[3 * i + k]) / L.h;
        }
      }
  } else parallel_for(L.n_bnd, [&](int b0, int b1) {
    for (int b = b0; b < b1; ++b) {
      int a = bcell[b];
      for (int slot = 0; slot < L.nslot; ++slot) {
        if (L.nbr[(size_t)slot * L.n_act + a] >= 0) continue;
        int dir = slot >> 1, side = slot & 1;
        for (int t = 0; t < nq; ++t) {
          double X[3] = {0, 0, 0}, C[3] = {0, 0, 0};
          int tt = t;
          for (int k = 0; k < dim; ++k) {
            double xi;
            if (k == dir) {
              xi = side;
            } else {
              xi = B.x[tt % n1];
              tt /= n1;
            }
            X[k] = d.lo[k] + L.h * (L.cell[3 * a + k] + xi);
          }
          if (!closest_point(sh, samples.data(), samples.size() / dim, X, C)) newton_fail[b] = 1;
          for (int k = 0; k < dim; ++k)
            L.dhat[(((size_t)b * L.nslot + slot) * dim + k) * nq + t] = (C[k] - X[k]) / L.h;
        }
      }
    }
  });
  for (int b = 0; b < L.n_bnd; ++b)
    if (newton_fail[b]) fail(SBM_ERR_GEOMETRY, "closest-point Newton did not converge");
  for (int b = 0; b < L.n_bnd; ++b) {
    int a = bcell[b];
    for (int slot = 0; slot < L.nslot; ++slot) {
      if (L.nbr[(size_t)slot * L.n_act + a] >= 0) continue;
      L.sf_cell.push_back(a);
      L.sf_slot.push_back(slot);
      for (int t = 0; t < nq; ++t)
        for (int k = 0; k < 3; ++k)
          L.sf_d.push_back(k < dim ? L.h * L.dhat[(((size_t)b * L.nslot + slot) * dim + k) * nq + t] : 0.0);
    }
  }
  L.n_sface = (int)L.sf_cell.size();

  // learned-correction data of boundary cells: 3^d patch table and static features
  {
    const int npatch = ipow(3, dim), nstat = 2 * dim * nq * dim + 1 + 2 * dim;
    L.patch.assign((size_t)L.n_bnd * npatch, -1);
    L.bnd_cell = bcell;
    L.mlp_static.assign((size_t)L.n_bnd * nstat, 0.0);
    for (int b = 0; b < L.n_bnd; ++b) {
      const int a = bcell[b];
      for (int o = 0; o < npatch; ++o) {
        int j[3] = {L.cell[3 * a], L.cell[3 * a + 1], L.cell[3 * a + 2]};
        bool inside = true;
        for (int k = 0, oo = o; k < dim; ++k, oo /= 3) {
          j[k] += oo % 3 - 1;
          inside = inside && j[k] >= 0 && j[k] < n;
        }
        if (inside) L.patch[(size_t)b * npatch + o] = L.bg2act[lin_of(j)];
      }
      double* st = &L.mlp_static[(size_t)b * nstat];
      for (int slot = 0; slot < L.nslot; ++slot)
        for (int t = 0; t < nq; ++t)
          for (int k = 0; k < dim; ++k)
            st[(slot * nq + t) * dim + k] = L.dhat[(((size_t)b * L.nslot + slot) * dim + k) * nq + t];
      st[2 * dim * nq * dim] = (double)counts[lin_of(&L.cell[3 * a])] / S;
      for (int slot = 0; slot < L.nslot; ++slot)
        st[2 * dim * nq * dim + 1 + slot] = L.nbr[(size_t)slot * L.n_act + a] < 0 ? 1.0 : 0.0;
    }
  }

  // dense blocks A_KK of boundary cells (Eq. 14) and their inverses, stored transposed
  L.binvT.assign((size_t)L.n_bnd * np * np, 0.0);
  std::vector<double> ratio(L.n_bnd, 1.0);
  parallel_for(L.n_bnd, [&](int b0, int b1) {
    std::vector<double> A((size_t)np * np), inv, e(np), col(np);
    for (int b = b0; b < b1; ++b) {
      int a = bcell[b];
      for (int j = 0; j < np; ++j) {
        std::fill(e.begin(), e.end(), 0.0);
        e[j] = 1.0;
        cell_self_apply(L, a, b, e.data(), col.data());
        for (int i = 0; i < np; ++i) A[(size_t)i * np + j] = col[i];
      }
      ratio[b] = dense_inverse(np, A, inv);
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) L.binvT[((size_t)b * np + j) * np + i] = inv[(size_t)i * np + j];
    }
  });
  for (int b = 0; b < L.n_bnd; ++b)
    if (!(ratio[b] >= 1e-13)) fail(SBM_ERR_SINGULAR_BLOCK, "boundary cell block is (nearly) singular");
  return L;
}

void host_apply_level(const HostLevel& L, const double* x, double* y) {
  const int np = L.np, n1 = L.n1, dim = L.dim;
  const double hs = std::pow(L.h, dim - 2);
  parallel_for(L.n_act, [&](int a0, int a1) {
    for (int a = a0; a < a1; ++a) {
      int bidx;
      L.is_boundary(a, &bidx);
      double* ya = y + (size_t)a * np;
      cell_self_apply(L, a, bidx, x + (size_t)a * np, ya);
      for (int slot = 0; slot < L.nslot; ++slot) {
        const int nb = L.nbr[(size_t)slot * L.n_act + a];
        if (nb < 0) continue;
        const int dir = slot >> 1, stride = ipow(n1, dir);
        const double* M = (slot & 1) ? L.Bmp : L.Bpm;
        const double* xn = x + (size_t)nb * np;
        for (int i = 0; i < np; ++i) {
          double wt;
          tangential_index(L, i, dir, &wt);
          const int id = digit(i, dir, n1), base = i - id * stride;
          double s = 0;
          for (int k = 0; k < n1; ++k) s += M[id * n1 + k] * xn[base + k * stride];
          ya[i] += hs * wt * s;
        }
      }
    }
  });
}

void link_levels(HostLevel& C, HostLevel& F) {
  const int dim = C.dim;
  if (C.n == F.n) {                  // p-transfer: identical active sets and compact order
    if (C.n_act != F.n_act || C.cell != F.cell) fail(SBM_ERR_ARG, "p-levels with different active sets");
    return;
  }
  if (F.n != 2 * C.n) fail(SBM_ERR_ARG, "h-levels must halve the mesh");
  F.parent_code.assign(F.n_act, -1);
  C.children.assign((size_t)(1 << dim) * C.n_act, -1);
  for (int a = 0; a < F.n_act; ++a) {
    int pidx[3] = {F.cell[3 * a] / 2, F.cell[3 * a + 1] / 2, F.cell[3 * a + 2] / 2};
    int o = 0;
    for (int k = 0; k < dim; ++k) o |= (F.cell[3 * a + k] & 1) << k;
    int lin = 0;
    for (int k = dim - 1; k >= 0; --k) lin = lin * C.n + pidx[k];
    int pc = C.bg2act[lin];
    if (pc < 0) continue;
    F.parent_code[a] = (pc << 3) | o;
    C.children[(size_t)o * C.n_act + pc] = a;
  }
}

void build_coarse_inverse(HostLevel& L) {
  const int np = L.np, n1 = L.n1, dim = L.dim;
  const int N = L.n_dof();
  std::vector<double> A((size_t)N * N, 0.0), e(np), col(np);
  const double hs = std::pow(L.h, dim - 2);
  for (int a = 0; a < L.n_act; ++a) {
    int bidx;
    L.is_boundary(a, &bidx);
    for (int j = 0; j < np; ++j) {
      std::fill(e.begin(), e.end(), 0.0);
      e[j] = 1.0;
      cell_self_apply(L, a, bidx, e.data(), col.data());
      for (int i = 0; i < np; ++i) A[(size_t)(a * np + i) * N + a * np + j] = col[i];
    }
    for (int slot = 0; slot < L.nslot; ++slot) {
      int nb = L.nbr[(size_t)slot * L.n_act + a];
      if (nb < 0) continue;
      int dir = slot >> 1;
      const double* M = (slot & 1) ? L.Bmp : L.Bpm;
      for (int i = 0; i < np; ++i) {
        double wt;
        int ti = tangential_index(L, i, dir, &wt);
        int id = digit(i, dir, n1);
        for (int j = 0; j < np; ++j) {
          if (tangential_index(L, j, dir, nullptr) != ti) continue;
          A[(size_t)(a * np + i) * N + nb * np + j] += hs * wt * M[id * n1 + digit(j, dir, n1)];
        }
      }
    }
  }
  double r = dense_inverse(N, A, L.coarse_inv);
  if (!(r >= 1e-13)) fail(SBM_ERR_SINGULAR_BLOCK, "coarse matrix is (nearly) singular");
}

std::vector<double> build_rhs(const sbm_setup_desc& d, const HostLevel& L) {
  const int dim = L.dim, n1 = L.n1, np = L.np, nq = L.nq;
  std::vector<double> b((size_t)L.n_dof(), 0.0);
  const int m1 = L.p + 3;
  double xq[8], wq[8];
  gauss_legendre01(m1, xq, wq);
  double V[8][kMaxN1];
  for (int q = 0; q < m1; ++q) lagrange_eval(n1, L.B.x, xq[q], V[q], nullptr);
  const int nvq = ipow(m1, dim);
  const double hd = std::pow(L.h, dim);
  parallel_for(L.n_act, [&](int a0, int a1) {
    std::vector<double> fq(nvq);
    for (int a = a0; a < a1; ++a) {
      for (int q = 0; q < nvq; ++q) {
        double X[3] = {0, 0, 0}, wt = 1;
        int qq = q;
        for (int k = 0; k < dim; ++k) {
          X[k] = d.lo[k] + L.h * (L.cell[3 * a + k] + xq[qq % m1]);
          wt *= wq[qq % m1];
          qq /= m1;
        }
        fq[q] = wt * f_source(d.exact, dim, X);
      }
      for (int i = 0; i < np; ++i) {
        int i0 = i % n1, i1 = (i / n1) % n1, i2 = i / (n1 * n1);
        double acc = 0;
        for (int q = 0; q < nvq; ++q) {
          int q0 = q % m1, q1 = (q / m1) % m1, q2 = q / (m1 * m1);
          double ph = V[q0][i0] * V[q1][i1];
          if (dim == 3) ph *= V[q2][i2];
          acc += ph * fq[q];
        }
        b[(size_t)a * np + i] = hd * acc;
      }
    }
  });
  const double hs = std::pow(L.h, dim - 2);
  Shape sh{d.shape, dim};
  (void)sh;
  for (int f = 0; f < L.n_sface; ++f) {
    int a = L.sf_cell[f], slot = L.sf_slot[f], dir = slot >> 1, side = slot & 1;
    const double sgn = side ? 1.0 : -1.0;
    const double* es = side ? L.B.e1 : L.B.e0;
    const double* ds = side ? L.B.d1 : L.B.d0;
    for (int t = 0; t < nq; ++t) {
      double X[3] = {0, 0, 0};
      int tt = t;
      double wt = 1;
      for (int k = 0; k < dim; ++k) {
        double xi;
        if (k == dir) {
          xi = side;
        } else {
          xi = L.B.x[tt % n1];
          wt *= L.B.w[tt % n1];
          tt /= n1;
        }
        X[k] = d.lo[k] + L.h * (L.cell[3 * a + k] + xi) + L.sf_d[((size_t)f * nq + t) * 3 + k];
      }
      double g = u_exact(d.exact, dim, X);
      for (int k = 0; k < n1; ++k)
        b[(size_t)a * np + dof_index(L, dir, k, t)] += hs * wt * g * (L.sigG_hat * es[k] - L.alpha * sgn * ds[k]);
    }
  }
  return b;
}

}  // namespace sbm
