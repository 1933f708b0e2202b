// Level-set shapes (Sec. 4.1: Omega = {phi < 0}) and the closest-point projection of Sec. 4.2
// (Eqs. 19-22), compiled for the host set-up (setup.cpp) and for the device set-up kernels
// (geometry_ops.cu) from the same source, so that both evaluate phi and run the Newton iteration
// with the same operations.
#pragma once

#include <cmath>
#include <cstddef>

#include "sbm.h"

#if defined(__CUDACC__)
#define SBM_HD __host__ __device__
#else
#define SBM_HD
#endif

namespace sbm {

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------------- level-set shapes
struct Shape {
  sbm_shape s;
  int dim;

  SBM_HD double phi(const double* x) const {
    const double* c = s.center;
    switch (s.kind) {
      case SBM_SHAPE_DISK: {
        double r2 = 0;
        for (int k = 0; k < dim; ++k) r2 += (x[k] - c[k]) * (x[k] - c[k]);
        return sqrt(r2) - s.radius;
      }
      case SBM_SHAPE_BOX: {
        double m = 0;
        for (int k = 0; k < dim; ++k) m = fmax(m, fabs(x[k] - c[k]));
        return m - s.radius;
      }
      case SBM_SHAPE_STAR: {
        double y0 = x[0] - c[0], y1 = x[1] - c[1];
        double rho = sqrt(y0 * y0 + y1 * y1), th = atan2(y1, y0);
        return rho - s.radius * (1.0 + s.amp * sin(s.freq * th + s.phase));
      }
      case SBM_SHAPE_ELLIPSOID: {
        double y[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
        double q2 = 0;
        for (int i = 0; i < 3; ++i) {          // q_i = (R^T y)_i / semi_i
          double t = s.rot[0 * 3 + i] * y[0] + s.rot[1 * 3 + i] * y[1] + s.rot[2 * 3 + i] * y[2];
          t /= s.semi[i];
          q2 += t * t;
        }
        return sqrt(q2) - 1.0;
      }
      case SBM_SHAPE_COMPLEX2D: {
        double sx = sin(kPi * x[0]);
        return (1.0 - 0.75 * sx * sx) * (x[0] * x[0] + x[1] * x[1]) - 0.2;
      }
    }
    return 1.0;
  }

  // Gradient g[dim] and Hessian H[dim*dim] of phi (smooth shapes).
  SBM_HD void grad_hess(const double* x, double* g, double* H) const {
    const double* c = s.center;
    if (s.kind == SBM_SHAPE_STAR) {
      double y0 = x[0] - c[0], y1 = x[1] - c[1];
      double r2 = y0 * y0 + y1 * y1, rho = sqrt(r2), th = atan2(y1, y0);
      double arg = s.freq * th + s.phase;
      double R1 = s.radius * s.amp * s.freq * cos(arg);
      double R2 = -s.radius * s.amp * s.freq * s.freq * sin(arg);
      double n0 = y0 / rho, n1 = y1 / rho;
      double t0 = -y1 / r2, t1 = y0 / r2;                 // grad theta
      g[0] = n0 - R1 * t0;
      g[1] = n1 - R1 * t1;
      double r4 = r2 * r2;
      double Hth00 = 2 * y0 * y1 / r4, Hth01 = (y1 * y1 - y0 * y0) / r4, Hth11 = -2 * y0 * y1 / r4;
      H[0] = (1 - n0 * n0) / rho - R2 * t0 * t0 - R1 * Hth00;
      H[1] = (-n0 * n1) / rho - R2 * t0 * t1 - R1 * Hth01;
      H[2] = H[1];
      H[3] = (1 - n1 * n1) / rho - R2 * t1 * t1 - R1 * Hth11;
      return;
    }
    if (s.kind == SBM_SHAPE_ELLIPSOID) {
      double y[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
      double q[3], M[9];                                   // M = R S^-1
      for (int i = 0; i < 3; ++i)
        q[i] = (s.rot[0 * 3 + i] * y[0] + s.rot[1 * 3 + i] * y[1] + s.rot[2 * 3 + i] * y[2]) / s.semi[i];
      for (int r = 0; r < 3; ++r)
        for (int i = 0; i < 3; ++i) M[r * 3 + i] = s.rot[r * 3 + i] / s.semi[i];
      double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
      for (int r = 0; r < 3; ++r) g[r] = (M[r * 3 + 0] * q[0] + M[r * 3 + 1] * q[1] + M[r * 3 + 2] * q[2]) / nq;
      double P[9];                                         // (I - q q^T / |q|^2) / |q|
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P[i * 3 + j] = ((i == j ? 1.0 : 0.0) - q[i] * q[j] / (nq * nq)) / nq;
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) {
          double acc = 0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += M[r * 3 + i] * P[i * 3 + j] * M[cc * 3 + j];
          H[r * 3 + cc] = acc;
        }
      return;
    }
    if (s.kind == SBM_SHAPE_COMPLEX2D) {
      double X = x[0], Y = x[1], sx = sin(kPi * X);
      double a = 1 - 0.75 * sx * sx;
      double ap = -0.75 * kPi * sin(2 * kPi * X);
      double app = -1.5 * kPi * kPi * cos(2 * kPi * X);
      double r2 = X * X + Y * Y;
      g[0] = ap * r2 + 2 * a * X;
      g[1] = 2 * a * Y;
      H[0] = app * r2 + 4 * ap * X + 2 * a;
      H[1] = H[2] = 2 * ap * Y;
      H[3] = 2 * a;
      return;
    }
    // disk / sphere
    double y[3] = {0, 0, 0}, r2 = 0;
    for (int k = 0; k < dim; ++k) {
      y[k] = x[k] - c[k];
      r2 += y[k] * y[k];
    }
    double r = sqrt(r2);
    for (int i = 0; i < dim; ++i) {
      g[i] = y[i] / r;
      for (int j = 0; j < dim; ++j) H[i * dim + j] = ((i == j) - y[i] * y[j] / r2) / r;
    }
  }
};

// Small dense solve with partial pivoting (n <= 4), in place on a copy.
SBM_HD inline bool small_solve(int n, const double* A_in, const double* b_in, double* x) {
  double A[16], b[4];
  for (int i = 0; i < n * n; ++i) A[i] = A_in[i];
  for (int i = 0; i < n; ++i) b[i] = b_in[i];
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
    if (A[piv * n + k] == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        const double t = A[k * n + j];
        A[k * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
      }
      const double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int j = i + 1; j < n; ++j) acc -= A[i * n + j] * x[j];
    x[i] = acc / A[i * n + i];
  }
  return true;
}


// Closest point on {phi = 0} (Sec. 4.2).  Disk/sphere and box: closed form.  Other shapes:
// Newton on F = [2(x - xt) + mu g; phi] (Eqs. 21-22) with Jacobian [[2I + mu H, g], [g^T, 0]]
// and backtracking on |F|, started from the nearest boundary sample (first on ties) with
// mu = 2 (xt - x).g / |g|^2.
SBM_HD inline bool closest_point(const Shape& sh, const double* samples, size_t n_samples, const double* xt,
                                 double* out) {
  const int dim = sh.dim;
  const double* c = sh.s.center;
  if (sh.s.kind == SBM_SHAPE_DISK) {
    double r2 = 0;
    for (int k = 0; k < dim; ++k) r2 += (xt[k] - c[k]) * (xt[k] - c[k]);
    double r = sqrt(r2);
    for (int k = 0; k < dim; ++k) out[k] = c[k] + sh.s.radius * (xt[k] - c[k]) / r;
    return true;
  }
  if (sh.s.kind == SBM_SHAPE_BOX) {
    double y[3], m = -1.0;
    int kmax = 0;
    for (int k = 0; k < dim; ++k) {
      y[k] = xt[k] - c[k];
      if (fabs(y[k]) > m) {
        m = fabs(y[k]);
        kmax = k;
      }
    }
    if (m <= sh.s.radius) {
      for (int k = 0; k < dim; ++k) out[k] = xt[k];
      out[kmax] = c[kmax] + (y[kmax] >= 0 ? sh.s.radius : -sh.s.radius);
    } else {
      for (int k = 0; k < dim; ++k) out[k] = c[k] + fmin(sh.s.radius, fmax(-sh.s.radius, y[k]));
    }
    return true;
  }
  const size_t ns = n_samples;
  size_t best = 0;
  double bd = 1e300;
  for (size_t k = 0; k < ns; ++k) {
    double d2 = 0;
    for (int m = 0; m < dim; ++m) {
      const double t = samples[k * dim + m] - xt[m];
      d2 += t * t;
    }
    if (d2 < bd) {
      bd = d2;
      best = k;
    }
  }
  double x[3], g[3], H[9];
  for (int k = 0; k < dim; ++k) x[k] = samples[best * dim + k];
  sh.grad_hess(x, g, H);
  double gg = 0, mu = 0;
  for (int k = 0; k < dim; ++k) {
    gg += g[k] * g[k];
    mu += (xt[k] - x[k]) * g[k];
  }
  mu = 2.0 * mu / gg;
  auto residual = [&](const double* xx, double mm, double* F, double* gx, double* Hx) {
    sh.grad_hess(xx, gx, Hx);
    double n2 = 0;
    for (int k = 0; k < dim; ++k) {
      F[k] = 2.0 * (xx[k] - xt[k]) + mm * gx[k];
      n2 += F[k] * F[k];
    }
    F[dim] = sh.phi(xx);
    n2 += F[dim] * F[dim];
    return sqrt(n2);
  };
  double F[4];
  double nF = residual(x, mu, F, g, H);
  for (int it = 0; it < 50 && nF > 1e-15; ++it) {
    const int m = dim + 1;
    double J[16] = {0}, rhs[4], del[4];
    for (int i = 0; i < dim; ++i) {
      for (int j = 0; j < dim; ++j) J[i * m + j] = (i == j ? 2.0 : 0.0) + mu * H[i * dim + j];
      J[i * m + dim] = g[i];
      J[dim * m + i] = g[i];
    }
    for (int i = 0; i < m; ++i) rhs[i] = -F[i];
    if (!small_solve(m, J, rhs, del)) return false;
    double t = 1.0, xn[3], mn = mu, Fn[4], gn[3], Hn[9], nFn = 0;
    while (true) {
      for (int k = 0; k < dim; ++k) xn[k] = x[k] + t * del[k];
      mn = mu + t * del[dim];
      nFn = residual(xn, mn, Fn, gn, Hn);
      if (nFn < (1.0 - 1e-4 * t) * nF || t < 1e-3) break;
      t *= 0.5;
    }
    double step = 0, xnorm = 0;
    for (int k = 0; k < dim; ++k) {
      step += t * del[k] * t * del[k];
      xnorm += xn[k] * xn[k];
      x[k] = xn[k];
    }
    mu = mn;
    for (int i = 0; i < 4; ++i) F[i] = Fn[i];
    for (int i = 0; i < 3; ++i) g[i] = gn[i];
    for (int i = 0; i < 9; ++i) H[i] = Hn[i];
    nF = nFn;
    if (sqrt(step) <= 1e-15 * fmax(1.0, sqrt(xnorm))) break;
  }
  if (!(nF <= 1e-10)) return false;
  for (int k = 0; k < dim; ++k) out[k] = x[k];
  return true;
}

}  // namespace sbm
