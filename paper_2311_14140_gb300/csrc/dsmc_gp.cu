// dsmc_gp.cu -- a Gaussian-process variant of the surrogate stage, not the paper's
// method (whose surrogates are Bayesian ridge regressions per flow case, Sec. 2.3): a GP
// over the (Kn, force) design of many DSMC runs predicts the slip coefficient and the
// stress correction of a new case, and the 1D CFD (Eq. 8 with Eq. 10) uses them.
//
// GP regression as in Rasmussen and Williams (2006), Ch. 2 and Sec. 5.4: squared-
// exponential covariance exp(-1/2 sum_d ((x_d - x'_d) / l_d)^2) over two inputs scaled to
// the unit square, noise variance s2 on the diagonal; each output column standardised
// (mean, standard deviation) and sharing the covariance.  All binary64 on the device:
//   k_gp_standardise  one thread per output column: mean and standard deviation;
//   k_gp_lml          one CTA per hyperparameter point: the covariance in shared memory,
//                     its Cholesky factor (right-looking), log|K|, and for every output
//                     column the forward solve L z = y and z^T z: the summed log marginal
//                     likelihood -1/2 sum_o z_o^T z_o - m sum log L_kk - n m/2 log 2 pi;
//   k_gp_alpha        one CTA: the factor at the chosen point and alpha = K^-1 y for every
//                     column (forward and back substitution);
//   k_gp_predict      one CTA per query point: k(x*, X) in shared memory, then every
//                     column's mean mu + sd (k* . alpha);
//   k_cfd_faces       the finite-volume solve of Eq. 8 with the stress correction given at
//                     the faces (Thomas algorithm), one thread per profile.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "dsmc.h"
#include "dsmc_internal.h"

namespace {

constexpr int kGpThreads = 256;
constexpr double kSqrtPi = 1.7724538509055160273;
constexpr double kLog2Pi = 1.8378770664093454836;

dsmc_status reject(dsmc_status s, const std::string& msg) {
  dsmc::set_last_error(msg);
  return s;
}

dsmc_status cuda_reject(cudaError_t e, const char* what) {
  return reject(DSMC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GP_CUDA(call, what)                            \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_reject(e_, what); \
  } while (0)

__device__ __forceinline__ double se_kernel(double ax, double ay, double bx, double by,
                                            double l1, double l2) {
  const double d1 = (ax - bx) / l1, d2 = (ay - by) / l2;
  return exp(-0.5 * (d1 * d1 + d2 * d2));
}

__global__ void k_gp_standardise(const double* __restrict__ Y, int n, int m,
                                 double* __restrict__ Ys, double* __restrict__ mu,
                                 double* __restrict__ sd) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= m) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += Y[(size_t)i * m + o];
  const double mean = s / n;
  double v = 0.0;
  for (int i = 0; i < n; ++i) {
    const double d = Y[(size_t)i * m + o] - mean;
    v += d * d;
  }
  double sdv = sqrt(v / n);
  if (!(sdv > 0.0)) sdv = 1.0;
  mu[o] = mean;
  sd[o] = sdv;
  for (int i = 0; i < n; ++i) Ys[(size_t)i * m + o] = (Y[(size_t)i * m + o] - mean) / sdv;
}

// Builds K = k(X, X) + s2 I in A (n x n, row-major, shared) and overwrites its lower
// triangle with the Cholesky factor.  Returns false (uniformly) if a pivot is not
// positive.
__device__ bool build_and_factor(double* A, const double* __restrict__ X, int n, double l1,
                                 double l2, double s2, int* bad) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double k = se_kernel(X[2 * i], X[2 * i + 1], X[2 * j], X[2 * j + 1], l1, l2);
    if (i == j) k += s2;
    A[e] = k;
  }
  if (threadIdx.x == 0) *bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[k * n + k];
      if (!(d > 0.0)) *bad = 1;
      A[k * n + k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double piv = A[k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + k] /= piv;
    __syncthreads();
    const int r = n - k - 1;  // trailing block (i, j), k < j <= i
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      const int i = k + 1 + e / r, j = k + 1 + e % r;
      if (j <= i) A[i * n + j] -= A[i * n + k] * A[j * n + k];
    }
    __syncthreads();
  }
  return *bad == 0;
}

__global__ void k_gp_lml(const double* __restrict__ X, const double* __restrict__ Ys, int n,
                         int m, const double* __restrict__ grid, double* __restrict__ lml) {
  extern __shared__ double A[];
  __shared__ int bad;
  __shared__ double part[kGpThreads];
  const double* g = grid + 3 * blockIdx.x;
  const bool ok = build_and_factor(A, X, n, g[0], g[1], g[2], &bad);
  double zz = 0.0;
  if (ok)
    for (int o = threadIdx.x; o < m; o += blockDim.x) {
      // forward substitution L z = y_o, z kept only as its running square sum; the
      // column's z values are recomputed from the rows already solved
      double zbuf[128];
      for (int i = 0; i < n; ++i) {
        double s = Ys[(size_t)i * m + o];
        for (int q = 0; q < i; ++q) s -= A[i * n + q] * zbuf[q];
        zbuf[i] = s / A[i * n + i];
        zz += zbuf[i] * zbuf[i];
      }
    }
  part[threadIdx.x] = zz;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (!ok) {
      lml[blockIdx.x] = -INFINITY;
      return;
    }
    double logdet = 0.0;
    for (int k = 0; k < n; ++k) logdet += log(A[k * n + k]);
    lml[blockIdx.x] = -0.5 * part[0] - m * logdet - 0.5 * (double)n * m * kLog2Pi;
  }
}

__global__ void k_gp_alpha(const double* __restrict__ X, const double* __restrict__ Ys, int n,
                           int m, double l1, double l2, double s2, double* __restrict__ alpha,
                           int* __restrict__ status) {
  extern __shared__ double A[];
  __shared__ int bad;
  const bool ok = build_and_factor(A, X, n, l1, l2, s2, &bad);
  if (threadIdx.x == 0) *status = ok ? 0 : 1;
  if (!ok) return;
  for (int o = threadIdx.x; o < m; o += blockDim.x) {
    double z[128];
    for (int i = 0; i < n; ++i) {  // L z = y
      double s = Ys[(size_t)i * m + o];
      for (int q = 0; q < i; ++q) s -= A[i * n + q] * z[q];
      z[i] = s / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T a = z
      double s = z[i];
      for (int q = i + 1; q < n; ++q) s -= A[q * n + i] * z[q];
      z[i] = s / A[i * n + i];
    }
    for (int i = 0; i < n; ++i) alpha[(size_t)i * m + o] = z[i];
  }
}

__global__ void k_gp_predict(const double* __restrict__ X, int n, int m,
                             const double* __restrict__ alpha, const double* __restrict__ mu,
                             const double* __restrict__ sd, double l1, double l2,
                             const double* __restrict__ Xs, double* __restrict__ out) {
  __shared__ double ks[128];
  const double* x = Xs + 2 * blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    ks[i] = se_kernel(x[0], x[1], X[2 * i], X[2 * i + 1], l1, l2);
  __syncthreads();
  for (int o = threadIdx.x; o < m; o += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += ks[i] * alpha[(size_t)i * m + o];
    out[(size_t)blockIdx.x * m + o] = mu[o] + sd[o] * s;
  }
}

__global__ void k_cfd_faces(double kn, double F, int n, int slip, double sigma_p,
                            const double* __restrict__ S, double* __restrict__ u,
                            double* __restrict__ cp) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double h = 1.0 / n;
  const double src = -h * kSqrtPi * F / kn;
  const double uw = slip ? sigma_p * F : 0.0;
  double cprev = 0.0, rprev = 0.0;
  for (int i = 0; i < n; ++i) {
    const double lo = (i > 0) ? 1.0 / h : 0.0;
    const double up = (i < n - 1) ? 1.0 / h : 0.0;
    const double d = -((i > 0) ? 1.0 / h : 2.0 / h) - ((i < n - 1) ? 1.0 / h : 2.0 / h);
    double r = src + S[i + 1] - S[i];
    if (i == 0) r -= 2.0 * uw / h;
    if (i == n - 1) r -= 2.0 * uw / h;
    const double den = d - lo * cprev;
    cprev = up / den;
    rprev = (r - lo * rprev) / den;
    cp[i] = cprev;
    u[i] = rprev;
  }
  for (int i = n - 2; i >= 0; --i) u[i] -= cp[i] * u[i + 1];
}

}  // namespace

struct dsmc_gp {
  int n = 0, m = 0;
  double l1 = 0, l2 = 0, s2 = 0;
  cudaStream_t stream = nullptr;
  double *X = nullptr, *alpha = nullptr, *mu = nullptr, *sd = nullptr;
};

extern "C" {

dsmc_status dsmc_gp_fit(const double* X, const double* Y, int n, int m, const double* grid,
                        int n_grid, void* stream, dsmc_gp_handle* out, double* lml,
                        int* best) {
  if (!out || !X || !Y || !grid) return reject(DSMC_E_INVAL, "gp: NULL argument");
  *out = nullptr;
  if (n < 2 || n > DSMC_GP_MAX_POINTS || m < 1 || n_grid < 1)
    return reject(DSMC_E_INVAL, "gp: 2 <= n <= 128 points, m >= 1 outputs, n_grid >= 1");
  for (int g = 0; g < n_grid; ++g)
    if (!(grid[3 * g] > 0.0) || !(grid[3 * g + 1] > 0.0) || !(grid[3 * g + 2] >= 0.0))
      return reject(DSMC_E_INVAL, "gp: length scales > 0 and noise >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  dsmc_gp* gp = new (std::nothrow) dsmc_gp();
  if (!gp) return reject(DSMC_E_NOMEM, "host allocation failed");
  gp->n = n;
  gp->m = m;
  gp->stream = st;
  double *Yd = nullptr, *Ys = nullptr, *gd = nullptr, *ld = nullptr;
  int* status = nullptr;
  auto fail = [&](dsmc_status s) {
    cudaFree(Yd);
    cudaFree(Ys);
    cudaFree(gd);
    cudaFree(ld);
    cudaFree(status);
    dsmc_gp_destroy(gp);
    return s;
  };
  const size_t nm = (size_t)n * m;
  cudaError_t e = cudaMalloc(&gp->X, 2 * (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&gp->alpha, nm * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&gp->mu, (size_t)m * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&gp->sd, (size_t)m * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Yd, nm * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&Ys, nm * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&gd, 3 * (size_t)n_grid * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ld, (size_t)n_grid * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e != cudaSuccess) return fail(cuda_reject(e, "gp allocation"));
  if ((e = cudaMemcpyAsync(gp->X, X, 2 * (size_t)n * sizeof(double), cudaMemcpyDefault, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(Yd, Y, nm * sizeof(double), cudaMemcpyDefault, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(gd, grid, 3 * (size_t)n_grid * sizeof(double), cudaMemcpyDefault,
                           st)) != cudaSuccess)
    return fail(cuda_reject(e, "gp copy"));
  const size_t smem = (size_t)n * n * sizeof(double);
  if ((e = cudaFuncSetAttribute(k_gp_lml, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gp_alpha, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem)) != cudaSuccess)
    return fail(cuda_reject(e, "gp shared memory"));
  k_gp_standardise<<<(m + 127) / 128, 128, 0, st>>>(Yd, n, m, Ys, gp->mu, gp->sd);
  k_gp_lml<<<n_grid, kGpThreads, smem, st>>>(gp->X, Ys, n, m, gd, ld);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(cuda_reject(e, "gp kernels"));
  std::vector<double> host((size_t)n_grid);
  if ((e = cudaMemcpyAsync(host.data(), ld, host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(cuda_reject(e, "gp marginal likelihoods"));
  int b = -1;
  for (int g = 0; g < n_grid; ++g)
    if (std::isfinite(host[g]) && (b < 0 || host[g] > host[b])) b = g;
  if (b < 0) return fail(reject(DSMC_E_STATE, "gp: no grid point gives a positive definite covariance"));
  gp->l1 = grid[3 * b];
  gp->l2 = grid[3 * b + 1];
  gp->s2 = grid[3 * b + 2];
  k_gp_alpha<<<1, kGpThreads, smem, st>>>(gp->X, Ys, n, m, gp->l1, gp->l2, gp->s2, gp->alpha,
                                           status);
  int sv = 1;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&sv, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(cuda_reject(e, "gp alpha"));
  if (sv != 0) return fail(reject(DSMC_E_STATE, "gp: covariance not positive definite"));
  if (lml)
    for (int g = 0; g < n_grid; ++g) lml[g] = host[g];
  if (best) *best = b;
  cudaFree(Yd);
  cudaFree(Ys);
  cudaFree(gd);
  cudaFree(ld);
  cudaFree(status);
  *out = gp;
  return DSMC_OK;
}

dsmc_status dsmc_gp_predict(dsmc_gp_handle gp, const double* Xs, int ns, double* out) {
  if (!gp || !Xs || !out) return reject(DSMC_E_INVAL, "gp: NULL argument");
  if (ns < 1) return reject(DSMC_E_INVAL, "gp: ns >= 1");
  cudaStream_t st = gp->stream;
  double *xd = nullptr, *od = nullptr;
  cudaError_t e = cudaMalloc(&xd, 2 * (size_t)ns * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&od, (size_t)ns * gp->m * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(xd, Xs, 2 * (size_t)ns * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_gp_predict<<<ns, kGpThreads, 0, st>>>(gp->X, gp->n, gp->m, gp->alpha, gp->mu, gp->sd,
                                             gp->l1, gp->l2, xd, od);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, od, (size_t)ns * gp->m * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(xd);
  cudaFree(od);
  if (e != cudaSuccess) return cuda_reject(e, "gp predict");
  return DSMC_OK;
}

dsmc_status dsmc_gp_hyper(dsmc_gp_handle gp, double* l1, double* l2, double* s2) {
  if (!gp) return reject(DSMC_E_INVAL, "gp: NULL");
  if (l1) *l1 = gp->l1;
  if (l2) *l2 = gp->l2;
  if (s2) *s2 = gp->s2;
  return DSMC_OK;
}

dsmc_status dsmc_gp_destroy(dsmc_gp_handle gp) {
  if (!gp) return DSMC_OK;
  cudaStreamSynchronize(gp->stream);
  cudaFree(gp->X);
  cudaFree(gp->alpha);
  cudaFree(gp->mu);
  cudaFree(gp->sd);
  delete gp;
  return DSMC_OK;
}

dsmc_status dsmc_cfd_faces(double Kn, double F, int n, int slip, double sigma_p,
                           const double* S_faces, double* u, void* stream) {
  if (!S_faces || !u) return reject(DSMC_E_INVAL, "cfd: NULL argument");
  if (!(Kn > 0.0) || n < 1) return reject(DSMC_E_INVAL, "cfd: Kn > 0, n >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  double *Sd = nullptr, *ud = nullptr;
  cudaError_t e = cudaMalloc(&Sd, ((size_t)n + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ud, 2 * (size_t)n * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Sd, S_faces, ((size_t)n + 1) * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_cfd_faces<<<1, 32, 0, st>>>(Kn, F, n, slip, sigma_p, Sd, ud, ud + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(u, ud, (size_t)n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(Sd);
  cudaFree(ud);
  if (e != cudaSuccess) return cuda_reject(e, "cfd");
  return DSMC_OK;
}

}  // extern "C"
