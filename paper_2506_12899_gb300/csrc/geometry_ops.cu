// Device set-up kernels (Sec. 2.1, Sec. 4.2): the volume fractions of the background cells from
// sub-cell sampling of the level set, and the closest points of the surrogate-face quadrature
// points on the true boundary by the Newton iteration on the Lagrangian stationarity system
// (Eqs. 19-22).  Both evaluate the shape with the code the host set-up uses (geometry.cuh), one
// thread per background cell, respectively per target point.  The host then builds the compact
// layout, the neighbour tables and the shift vectors from these results exactly as it does from
// its own.
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "geometry.cuh"
#include "ops.h"

namespace sbm {
namespace {

constexpr int kGeoThreads = 128;

// counts[lin] = number of the s^d sub-cell midpoints of background cell lin with phi < 0.
__global__ void __launch_bounds__(kGeoThreads) k_volume_counts(const sbm_shape shp, int dim, int n, double h,
                                                               double lo0, double lo1, double lo2, int s,
                                                               int* __restrict__ counts) {
  const long long nbg = dim == 2 ? (long long)n * n : (long long)n * n * n;
  const long long lin = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= nbg) return;
  const Shape sh{shp, dim};
  const int idx[3] = {(int)(lin % n), (int)((lin / n) % n), dim > 2 ? (int)(lin / ((long long)n * n)) : 0};
  const double lo[3] = {lo0, lo1, lo2};
  const int S = dim == 2 ? s * s : s * s * s;
  int count = 0;
  for (int q = 0; q < S; ++q) {
    double X[3] = {0.0, 0.0, 0.0};
    int qq = q;
    for (int k = 0; k < dim; ++k) {
      X[k] = lo[k] + h * (idx[k] + ((qq % s) + 0.5) / s);
      qq /= s;
    }
    count += sh.phi(X) < 0.0;
  }
  counts[lin] = count;
}

// C[i] = closest point on {phi = 0} to X[i] (rows of 3), ok[i] = 1 if the Newton iteration converged.
__global__ void __launch_bounds__(kGeoThreads) k_closest_points(const sbm_shape shp, int dim,
                                                                const double* __restrict__ samples, int ns,
                                                                const double* __restrict__ X, int m,
                                                                double* __restrict__ C, int* __restrict__ ok) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const Shape sh{shp, dim};
  double xt[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]}, out[3] = {0.0, 0.0, 0.0};
  ok[i] = closest_point(sh, samples, (size_t)ns, xt, out) ? 1 : 0;
  for (int k = 0; k < 3; ++k) C[3 * i + k] = k < dim ? out[k] : 0.0;
}

// Device buffer freed when it goes out of scope.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  explicit DevBuf(size_t n) {
    const cudaError_t e = cudaMalloc(&p, (n == 0 ? 1 : n) * sizeof(T));
    if (e != cudaSuccess) throw SetupError{SBM_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

void check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw SetupError{SBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

}  // namespace

void device_volume_counts(const sbm_setup_desc& d, int n, double h, int s, std::vector<int>& counts) {
  const size_t nbg = d.dim == 2 ? (size_t)n * n : (size_t)n * n * n;
  counts.assign(nbg, 0);
  if (nbg == 0) return;
  DevBuf<int> dc(nbg);
  const unsigned grid = (unsigned)((nbg + kGeoThreads - 1) / kGeoThreads);
  k_volume_counts<<<grid, kGeoThreads>>>(d.shape, d.dim, n, h, d.lo[0], d.lo[1], d.lo[2], s, dc.p);
  check(cudaGetLastError(), "volume-fraction kernel");
  check(cudaMemcpy(counts.data(), dc.p, nbg * sizeof(int), cudaMemcpyDeviceToHost), "volume-fraction copy");
  count_launches();
}

void device_closest_points(const sbm_setup_desc& d, const std::vector<double>& samples, const std::vector<double>& X,
                           std::vector<double>& C, std::vector<int>& ok) {
  const size_t m = X.size() / 3;
  C.assign(X.size(), 0.0);
  ok.assign(m, 0);
  if (m == 0) return;
  const int ns = (int)(samples.size() / d.dim);
  DevBuf<double> ds(samples.size()), dx(X.size()), dc(X.size());
  DevBuf<int> dok(m);
  if (!samples.empty())
    check(cudaMemcpy(ds.p, samples.data(), samples.size() * sizeof(double), cudaMemcpyHostToDevice), "samples copy");
  check(cudaMemcpy(dx.p, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice), "points copy");
  const unsigned grid = (unsigned)((m + kGeoThreads - 1) / kGeoThreads);
  k_closest_points<<<grid, kGeoThreads>>>(d.shape, d.dim, ds.p, ns, dx.p, (int)m, dc.p, dok.p);
  check(cudaGetLastError(), "closest-point kernel");
  check(cudaMemcpy(C.data(), dc.p, X.size() * sizeof(double), cudaMemcpyDeviceToHost), "closest-point copy");
  check(cudaMemcpy(ok.data(), dok.p, m * sizeof(int), cudaMemcpyDeviceToHost), "closest-point flags copy");
  count_launches();
}

}  // namespace sbm
