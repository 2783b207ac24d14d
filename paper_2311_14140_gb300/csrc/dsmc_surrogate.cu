// dsmc_surrogate.cu -- the surrogate stage of the Micro-Macro-Surrogate method
// (Sec. 2.3, Appendix A): training samples from DSMC moment windows, Bayesian ridge
// regression with evidence maximisation and model selection, and the corrected 1D
// macroscopic solve with Monte Carlo uncertainty bands.
//
// Device work (binary64):
//   k_window  one training sample per call: from a window's raw moment sums, the cell
//             velocities and shear stresses (Eq. 6 units), the constitutive targets
//             E_i = P_i + (2 Kn / sqrt(pi)) du/dy_i at the interior cells (Eq. 13, du/dy
//             by central differences) with their Appendix A basis rows, and the wall
//             velocities extrapolated linearly from the two nearest cells; it adds the
//             sample's sufficient statistics (Phi^T Phi, Phi^T t, t^T t, sum t, N) for
//             the boundary and constitutive models to running totals.  The moment sums
//             stay on the device: a run's accumulators are read in place.
//   k_trials  one thread per Monte Carlo trial: weights drawn from the selected
//             models' posteriors (w = m + L z, S = L L^T by Cholesky), the cell-centred
//             finite-volume system of Eq. 8 with Eqs. 9-10 solved by the Thomas
//             algorithm.
//   k_bands   per cell: mean and standard deviation over the trials.
// Host work: the evidence maximisation itself (MacKay's re-estimation of alpha and beta
// on 1x1 to 3x3 matrices, Bishop Sec. 3.5, Tipping App. A) and Eq. 17.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dsmc.h"
#include "dsmc_internal.h"

namespace {

constexpr int kStats = 20;  // sufficient statistics, layout below
// [0..8] Phi^T Phi (3x3, row-major) of the constitutive basis, [9..11] Phi^T t,
// [12] t^T t, [13] N (constitutive); [14] sum x t, [15] sum x^2, [16] t^T t, [17] N
// (boundary); [18] sum t (constitutive), [19] sum t (boundary).
constexpr int kThreads = 256;
constexpr double kAlphaMax = 1e30;  // weight precision above which weights are off
constexpr double kSqrtPi = 1.7724538509055160273;

// Table 1 of the paper: exponents b_1..b_3 at the tabulated Kn.
constexpr double kTableKn[7] = {0.01, 0.05, 0.1, 0.2, 0.5, 1.0, 5.0};
constexpr double kTableB[7][3] = {{130, 150, 200}, {30, 40, 70}, {20, 40, 10}, {20, 12, 8},
                                  {10, 7, 6},      {8, 6, 20},   {7, 6, 5}};

dsmc_status reject(dsmc_status s, const std::string& msg) {
  dsmc::set_last_error(msg);
  return s;
}

dsmc_status cuda_reject(cudaError_t e, const char* what) {
  return reject(DSMC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SUR_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_reject(e_, what); \
  } while (0)

struct WindowArgs {
  int n;           // cells
  double n_norm;   // steps * ppc: sampled count per cell at the initial density
  double kn, F;
  double b[3];
  double length;   // the run's extent in channel units (1: the whole channel)
  int last;        // last training cell (first is 1)
  int both;        // 1: both walls give boundary data (whole channel), 0: bottom only
};

__device__ __forceinline__ double cell_u(const double* acc, int i) {
  return acc[(size_t)i * dsmc::kNMom + 1] / acc[(size_t)i * dsmc::kNMom + 0];
}

__global__ void __launch_bounds__(kThreads) k_window(const double* __restrict__ acc,
                                                     WindowArgs a, double* __restrict__ stats) {
  __shared__ double red[16][kThreads];
  const int t = threadIdx.x;
  const double h = a.length / a.n;
  const double c = 2.0 * a.kn / kSqrtPi;
  double g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0, p0 = 0, p1 = 0, p2 = 0, tt = 0,
         st = 0, nn = 0;
  for (int i = 1 + t; i <= a.last; i += kThreads) {
    const double* r = acc + (size_t)i * dsmc::kNMom;
    const double N = r[0];
    const double ux = r[1] / N, uy = r[2] / N;
    const double P = 2.0 * (N / a.n_norm) * (r[7] / N - ux * uy);
    const double dudy = (cell_u(acc, i + 1) - cell_u(acc, i - 1)) / (2.0 * h);
    const double E = P + c * dudy;
    const double y = (i + 0.5) * h;
    const double f0 = c * (exp(-a.b[0] * y) - exp(-a.b[0] * (1.0 - y)));
    const double f1 = c * (exp(-a.b[1] * y) - exp(-a.b[1] * (1.0 - y)));
    const double f2 = c * (exp(-a.b[2] * y) - exp(-a.b[2] * (1.0 - y)));
    g00 += f0 * f0;
    g01 += f0 * f1;
    g02 += f0 * f2;
    g11 += f1 * f1;
    g12 += f1 * f2;
    g22 += f2 * f2;
    p0 += f0 * E;
    p1 += f1 * E;
    p2 += f2 * E;
    tt += E * E;
    st += E;
    nn += 1.0;
  }
  double v[12] = {g00, g01, g02, g11, g12, g22, p0, p1, p2, tt, st, nn};
#pragma unroll
  for (int k = 0; k < 12; ++k) red[k][t] = v[k];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (t < s)
#pragma unroll
      for (int k = 0; k < 12; ++k) red[k][t] += red[k][t + s];
    __syncthreads();
  }
  if (t == 0) {
    const double G[9] = {red[0][0], red[1][0], red[2][0], red[1][0], red[3][0],
                         red[4][0], red[2][0], red[4][0], red[5][0]};
    for (int k = 0; k < 9; ++k) stats[k] += G[k];
    stats[9] += red[6][0];
    stats[10] += red[7][0];
    stats[11] += red[8][0];
    stats[12] += red[9][0];
    stats[13] += red[11][0];
    stats[18] += red[10][0];
    // boundary models: x = -P(0) = F (and P(1) = F), t = wall velocities
    const int n = a.n;
    const double ub = 1.5 * cell_u(acc, 0) - 0.5 * cell_u(acc, 1);
    if (a.both) {
      const double ut = 1.5 * cell_u(acc, n - 1) - 0.5 * cell_u(acc, n - 2);
      stats[14] += a.F * ub + a.F * ut;
      stats[15] += a.F * a.F + a.F * a.F;
      stats[16] += ub * ub + ut * ut;
      stats[17] += 2.0;
      stats[19] += ub + ut;
    } else {
      stats[14] += a.F * ub;
      stats[15] += a.F * a.F;
      stats[16] += ub * ub;
      stats[17] += 1.0;
      stats[19] += ub;
    }
  }
}

// Posterior of one model as the trials need it.
struct TrialModels {
  int sel_v, k;  // slip selected; number of constitutive weights (0..3)
  double m_v, s_v;
  double m[3], S[9];
  double kn, F;
  double b[3];
  int n;  // CFD cells
};

__global__ void __launch_bounds__(128) k_trials(TrialModels tm, const double* __restrict__ z,
                                                int n_trials, double* __restrict__ u,
                                                double* __restrict__ cp) {
  const int tr = blockIdx.x * blockDim.x + threadIdx.x;
  if (tr >= n_trials) return;
  const double* zt = z + (size_t)tr * 4;
  double uw = 0.0;
  if (tm.sel_v) uw = (tm.m_v + sqrt(tm.s_v) * zt[0]) * tm.F;  // -sigma_P P(0) = sigma_P F
  double w[3] = {0.0, 0.0, 0.0};
  if (tm.k > 0) {
    // Cholesky S = L L^T (lower, k <= 3), then w = m + L z
    double L[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < tm.k; ++i)
      for (int j = 0; j <= i; ++j) {
        double s = tm.S[i * 3 + j];
        for (int q = 0; q < j; ++q) s -= L[i * 3 + q] * L[j * 3 + q];
        L[i * 3 + j] = (i == j) ? sqrt(s > 0.0 ? s : 0.0) : (L[j * 3 + j] > 0.0 ? s / L[j * 3 + j] : 0.0);
      }
    for (int i = 0; i < tm.k; ++i) {
      double s = tm.m[i];
      for (int j = 0; j <= i; ++j) s += L[i * 3 + j] * zt[1 + j];
      w[i] = s;
    }
  }
  const int n = tm.n;
  const double h = 1.0 / n;
  const double src = -h * kSqrtPi * tm.F / tm.kn;
  double* ut = u + (size_t)tr * n;
  double* ct = cp + (size_t)tr * n;
  // S at face f (y = f h)
  auto S = [&](int f) {
    const double y = f * h;
    double s = 0.0;
    for (int l = 0; l < tm.k; ++l) s += w[l] * (exp(-tm.b[l] * y) - exp(-tm.b[l] * (1.0 - y)));
    return s;
  };
  // Thomas algorithm: row i has sub 1/h (i > 0), super 1/h (i < n-1), diagonal -(sum of
  // face coefficients) with 2/h for a wall face, right side src + S_{i+1} - S_i minus
  // 2 uw / h per wall face.  Forward sweep keeps c' in cp and r' in u.
  double Sl = S(0);
  double cprev = 0.0, rprev = 0.0;
  for (int i = 0; i < n; ++i) {
    const double Su = S(i + 1);
    const double lo = (i > 0) ? 1.0 / h : 0.0;
    const double up = (i < n - 1) ? 1.0 / h : 0.0;
    double d = -((i > 0) ? 1.0 / h : 2.0 / h) - ((i < n - 1) ? 1.0 / h : 2.0 / h);
    double r = src + Su - Sl;
    if (i == 0) r -= 2.0 * uw / h;
    if (i == n - 1) r -= 2.0 * uw / h;
    const double den = d - lo * cprev;
    cprev = up / den;
    rprev = (r - lo * rprev) / den;
    ct[i] = cprev;
    ut[i] = rprev;
    Sl = Su;
  }
  for (int i = n - 2; i >= 0; --i) ut[i] -= ct[i] * ut[i + 1];
}

// S(y) of Eq. 14 with weights w (k of them) at the faces y = f / n, f = 0..n.
__global__ void k_correction(int k, double w0, double w1, double w2, double b0, double b1,
                             double b2, int n, double* __restrict__ S) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f > n) return;
  const double y = (double)f / n;
  const double w[3] = {w0, w1, w2}, b[3] = {b0, b1, b2};
  double s = 0.0;
  for (int l = 0; l < k; ++l) s += w[l] * (exp(-b[l] * y) - exp(-b[l] * (1.0 - y)));
  S[f] = s;
}

__global__ void k_bands(const double* __restrict__ u, int n_trials, int n,
                        double* __restrict__ mean, double* __restrict__ sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int t = 0; t < n_trials; ++t) s += u[(size_t)t * n + i];
  const double m = s / n_trials;
  double v = 0.0;
  for (int t = 0; t < n_trials; ++t) {
    const double d = u[(size_t)t * n + i] - m;
    v += d * d;
  }
  mean[i] = m;
  sd[i] = n_trials > 1 ? sqrt(v / (n_trials - 1)) : 0.0;
}

// ---------------------------------------------------------------------------
// Host linear algebra on k x k symmetric matrices (k <= 3).

// Cholesky A = L L^T; false if A is not positive definite.
bool cholesky(const double* A, int k, double* L) {
  for (int i = 0; i < 9; ++i) L[i] = 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[i * 3 + j];
      for (int q = 0; q < j; ++q) s -= L[i * 3 + q] * L[j * 3 + q];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i * 3 + i] = std::sqrt(s);
      } else {
        L[i * 3 + j] = s / L[j * 3 + j];
      }
    }
  return true;
}

// Inverse and log determinant of an SPD matrix through its Cholesky factor.
bool spd_inverse(const double* A, int k, double* inv, double* logdet) {
  double L[9];
  if (!cholesky(A, k, L)) return false;
  *logdet = 0.0;
  for (int i = 0; i < k; ++i) *logdet += 2.0 * std::log(L[i * 3 + i]);
  for (int c = 0; c < k; ++c) {  // solve A x = e_c
    double y[3] = {0, 0, 0}, x[3] = {0, 0, 0};
    for (int i = 0; i < k; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int q = 0; q < i; ++q) s -= L[i * 3 + q] * y[q];
      y[i] = s / L[i * 3 + i];
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = y[i];
      for (int q = i + 1; q < k; ++q) s -= L[q * 3 + i] * x[q];
      x[i] = s / L[i * 3 + i];
    }
    for (int i = 0; i < k; ++i) inv[i * 3 + c] = x[i];
  }
  return true;
}

// Eigenvalues of a symmetric k x k matrix by cyclic Jacobi rotations.
void sym_eigenvalues(const double* A0, int k, double* ev) {
  double A[9];
  std::memcpy(A, A0, sizeof(A));
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off += A[p * 3 + q] * A[p * 3 + q];
    if (off == 0.0) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = A[p * 3 + q];
        if (apq == 0.0) continue;
        const double theta = (A[q * 3 + q] - A[p * 3 + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < k; ++r) {  // A <- A J
          const double arp = A[r * 3 + p], arq = A[r * 3 + q];
          A[r * 3 + p] = c * arp - s * arq;
          A[r * 3 + q] = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {  // A <- J^T A
          const double apr = A[p * 3 + r], aqr = A[q * 3 + r];
          A[p * 3 + r] = c * apr - s * aqr;
          A[q * 3 + r] = s * apr + c * aqr;
        }
      }
  }
  for (int i = 0; i < k; ++i) ev[i] = A[i * 3 + i];
}

struct Fit {
  double m[3], S[9], alpha, beta, logev;
  int iterations;
};

// Evidence maximisation for a model with k weights from its sufficient statistics:
// G = Phi^T Phi (k x k block of a 3x3), pt = Phi^T t, tt = t^T t, st = sum t, N.
bool brr_stats(const double* G3, const double* pt, double tt, double st, double N, int k,
               Fit* f) {
  double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) G[i * 3 + j] = G3[i * 3 + j];
  double ev[3];
  sym_eigenvalues(G, k, ev);
  const double mean = st / N;
  double var = tt / N - mean * mean;
  double alpha = 1.0, beta = 1.0 / (var > 1e-300 ? var : 1e-300);
  double S[9], m[3], logdet = 0.0;
  auto posterior = [&](double al, double be) {
    double A[9];
    for (int i = 0; i < 9; ++i) A[i] = be * G[i];
    for (int i = 0; i < k; ++i) A[i * 3 + i] += al;
    if (!spd_inverse(A, k, S, &logdet)) return false;
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += S[i * 3 + j] * pt[j];
      m[i] = be * s;
    }
    return true;
  };
  auto resid = [&]() {  // |t - Phi m|^2 from the statistics
    double r = tt;
    for (int i = 0; i < k; ++i) {
      r -= 2.0 * m[i] * pt[i];
      for (int j = 0; j < k; ++j) r += m[i] * G[i * 3 + j] * m[j];
    }
    return r;
  };
  int it = 0;
  for (; it < 1000; ++it) {
    if (!posterior(alpha, beta)) return false;
    double gamma = 0.0;
    for (int i = 0; i < k; ++i) gamma += beta * ev[i] / (alpha + beta * ev[i]);
    double mm = 0.0;
    for (int i = 0; i < k; ++i) mm += m[i] * m[i];
    const double an = (mm <= gamma / kAlphaMax) ? kAlphaMax : gamma / mm;
    const double bn = (N - gamma) / resid();
    const bool done = std::fabs(an - alpha) <= 1e-12 * alpha && std::fabs(bn - beta) <= 1e-12 * beta;
    alpha = an;
    beta = bn;
    if (done) break;
  }
  if (!posterior(alpha, beta)) return false;
  double mm = 0.0;
  for (int i = 0; i < k; ++i) mm += m[i] * m[i];
  const double E = 0.5 * beta * resid() + 0.5 * alpha * mm;
  f->logev = 0.5 * k * std::log(alpha) + 0.5 * N * std::log(beta) - E - 0.5 * logdet -
             0.5 * N * std::log(2.0 * M_PI);
  std::memcpy(f->m, m, sizeof(m));
  std::memcpy(f->S, S, sizeof(S));
  f->alpha = alpha;
  f->beta = beta;
  f->iterations = it + 1;
  return true;
}

// Evidence of a model without weights: t ~ N(0, I / beta) at beta = N / t^T t.
double zero_evidence(double tt, double N, double* beta) {
  *beta = N / tt;
  return 0.5 * N * std::log(*beta) - 0.5 * N * std::log(2.0 * M_PI) - 0.5 * (*beta) * tt;
}

// Eq. 17's most probable model (equal priors), the simplest (lowest index) among models
// whose log evidences agree with the best to kTieRel: such ties are rounding noise, e.g.
// every extra weight shrunk to zero on data with no signal for it.
constexpr double kTieRel = 1e-9;

int select_model(const double* le, int n) {
  double top = le[0];
  for (int k = 1; k < n; ++k) top = std::max(top, le[k]);
  const double tol = kTieRel * std::max(1.0, std::fabs(top));
  for (int k = 0; k < n; ++k)
    if (le[k] >= top - tol) return k;
  return 0;
}

void probabilities(const double* le, int n, double* p) {
  double mx = le[0];
  for (int i = 1; i < n; ++i) mx = le[i] > mx ? le[i] : mx;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += (p[i] = std::exp(le[i] - mx));
  for (int i = 0; i < n; ++i) p[i] /= s;
}

}  // namespace

struct dsmc_surrogate {
  double Kn = 1.0, F = 0.0;
  int n_cells = 0, ppc = 0;
  double length = 1.0;  // extent of the runs in channel units
  int n_train = 0;      // cells of the training region (sub-domain runs)
  double b[3]{};
  cudaStream_t stream = nullptr;
  double* stats = nullptr;    // device, kStats
  double* window = nullptr;   // device, n_cells x 13 (host windows are copied here)
  double* trials = nullptr;   // device profiles and Thomas scratch
  size_t trials_cap = 0;
  long long n_samples = 0;
  dsmc_surrogate_fit fit{};
  bool fitted = false;
};

extern "C" {

dsmc_status dsmc_surrogate_exponents(double Kn, double* b) {
  if (!b || !(Kn > 0.0)) return reject(DSMC_E_INVAL, "surrogate: Kn > 0 and b non-NULL");
  int best = 0;
  for (int i = 1; i < 7; ++i)
    if (std::fabs(std::log(Kn) - std::log(kTableKn[i])) <
        std::fabs(std::log(Kn) - std::log(kTableKn[best])))
      best = i;
  for (int l = 0; l < 3; ++l) b[l] = kTableB[best][l];
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_create(double Kn, double F, int n_cells, int ppc, const double* b,
                                  void* stream, dsmc_surrogate_handle* out) {
  if (!out) return reject(DSMC_E_INVAL, "out: NULL");
  *out = nullptr;
  if (!(Kn > 0.0) || !std::isfinite(Kn) || !std::isfinite(F) || F == 0.0 || n_cells < 3 ||
      ppc < 1)
    return reject(DSMC_E_INVAL, "surrogate: finite Kn > 0, finite F != 0, n_cells >= 3, ppc >= 1");
  dsmc_surrogate* s = new (std::nothrow) dsmc_surrogate();
  if (!s) return reject(DSMC_E_NOMEM, "host allocation failed");
  s->Kn = Kn;
  s->F = F;
  s->n_cells = n_cells;
  s->ppc = ppc;
  s->stream = (cudaStream_t)stream;
  if (b)
    for (int l = 0; l < 3; ++l) s->b[l] = b[l];
  else
    dsmc_surrogate_exponents(Kn, s->b);
  cudaError_t e = cudaMalloc(&s->stats, kStats * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&s->window, (size_t)n_cells * dsmc::kNMom * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(s->stats, 0, kStats * sizeof(double), s->stream);
  if (e != cudaSuccess) {
    dsmc_surrogate_destroy(s);
    return cuda_reject(e, "surrogate allocation");
  }
  *out = s;
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_create_region(double Kn, double F, int n_cells, int ppc,
                                         double length, int n_train, const double* b,
                                         void* stream, dsmc_surrogate_handle* out) {
  if (!(length > 0.0 && length < 1.0) || n_train < 2 || n_train > n_cells - 1)
    return reject(DSMC_E_INVAL, "surrogate region: 0 < length < 1, 2 <= n_train <= n_cells - 1");
  dsmc_status st = dsmc_surrogate_create(Kn, F, n_cells, ppc, b, stream, out);
  if (st != DSMC_OK) return st;
  (*out)->length = length;
  (*out)->n_train = n_train;
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_destroy(dsmc_surrogate_handle s) {
  if (!s) return DSMC_OK;
  cudaStreamSynchronize(s->stream);
  cudaFree(s->stats);
  cudaFree(s->window);
  cudaFree(s->trials);
  delete s;
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_reset(dsmc_surrogate_handle s) {
  if (!s) return reject(DSMC_E_INVAL, "surrogate: NULL");
  SUR_CUDA(cudaMemsetAsync(s->stats, 0, kStats * sizeof(double), s->stream), "reset");
  s->n_samples = 0;
  s->fitted = false;
  return DSMC_OK;
}

// One window on the device (acc_dev: n_cells x 13 raw sums of n_steps sampled steps).
static dsmc_status add_device_window(dsmc_surrogate* s, const double* acc_dev, long long n_steps) {
  WindowArgs a;
  a.n = s->n_cells;
  a.n_norm = (double)n_steps * (double)s->ppc;
  a.kn = s->Kn;
  a.F = s->F;
  for (int l = 0; l < 3; ++l) a.b[l] = s->b[l];
  a.length = s->length;
  a.both = s->length == 1.0 ? 1 : 0;
  a.last = a.both ? s->n_cells - 2 : s->n_train - 1;
  k_window<<<1, kThreads, 0, s->stream>>>(acc_dev, a, s->stats);
  SUR_CUDA(cudaGetLastError(), "window kernel");
  s->n_samples += 1;
  s->fitted = false;
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_add_window(dsmc_surrogate_handle s, const double* acc,
                                      long long n_steps) {
  if (!s || !acc) return reject(DSMC_E_INVAL, "surrogate: NULL");
  if (n_steps < 1) return reject(DSMC_E_INVAL, "surrogate: n_steps >= 1");
  cudaPointerAttributes attr{};
  const bool on_device = cudaPointerGetAttributes(&attr, acc) == cudaSuccess &&
                         attr.type == cudaMemoryTypeDevice;
  cudaGetLastError();
  if (on_device) return add_device_window(s, acc, n_steps);
  SUR_CUDA(cudaMemcpyAsync(s->window, acc, (size_t)s->n_cells * dsmc::kNMom * sizeof(double),
                           cudaMemcpyDefault, s->stream),
           "copy window");
  return add_device_window(s, s->window, n_steps);
}

dsmc_status dsmc_surrogate_add_run(dsmc_surrogate_handle s, dsmc_handle h, int id) {
  if (!s || !h) return reject(DSMC_E_INVAL, "surrogate: NULL");
  dsmc_info info;
  dsmc_status st = dsmc_get_info_of(h, id, &info);
  if (st != DSMC_OK) return st;
  if (info.n_cells != s->n_cells || info.ppc != s->ppc)
    return reject(DSMC_E_INVAL, "surrogate: the run's n_cells and ppc differ from the surrogate's");
  if (info.n_samples < 1) return reject(DSMC_E_STATE, "surrogate: the run has no sampled steps");
  const double* acc = nullptr;
  if ((st = dsmc_device_moments_of(h, id, &acc)) != DSMC_OK) return st;
  // The run's work and the window kernel are ordered through the run's stream.
  if ((st = dsmc_sync(h)) != DSMC_OK) return st;
  if ((st = add_device_window(s, acc, info.n_samples)) != DSMC_OK) return st;
  SUR_CUDA(cudaStreamSynchronize(s->stream), "window");
  return dsmc_reset_samples_of(h, id);
}

dsmc_status dsmc_surrogate_train(dsmc_surrogate_handle s, dsmc_surrogate_fit* out) {
  if (!s || !out) return reject(DSMC_E_INVAL, "surrogate: NULL");
  if (s->n_samples < 1) return reject(DSMC_E_STATE, "surrogate: no training samples");
  double st[kStats];
  SUR_CUDA(cudaMemcpyAsync(st, s->stats, sizeof(st), cudaMemcpyDeviceToHost, s->stream), "stats");
  SUR_CUDA(cudaStreamSynchronize(s->stream), "stats");
  dsmc_surrogate_fit f;
  std::memset(&f, 0, sizeof(f));
  f.n_samples = s->n_samples;
  f.n_v = st[17];
  f.n_c = st[13];
  // Boundary models: no-slip (no weights) and slip (one weight, x = F).
  f.log_evidence_v[0] = zero_evidence(st[16], st[17], &f.beta_v[0]);
  {
    const double G[9] = {st[15], 0, 0, 0, 0, 0, 0, 0, 0};
    const double pt[3] = {st[14], 0, 0};
    Fit r;
    if (!brr_stats(G, pt, st[16], st[19], st[17], 1, &r))
      return reject(DSMC_E_STATE, "surrogate: slip model posterior not positive definite");
    f.log_evidence_v[1] = r.logev;
    f.alpha_v[1] = r.alpha;
    f.beta_v[1] = r.beta;
    f.sigma_p = r.m[0];
    f.sigma_p_var = r.S[0];
    f.iterations_v = r.iterations;
  }
  // Constitutive models C0..C3.
  f.log_evidence_c[0] = zero_evidence(st[12], st[13], &f.beta_c[0]);
  for (int k = 1; k <= 3; ++k) {
    Fit r;
    if (!brr_stats(st, st + 9, st[12], st[18], st[13], k, &r))
      return reject(DSMC_E_STATE, "surrogate: constitutive posterior not positive definite");
    f.log_evidence_c[k] = r.logev;
    f.alpha_c[k] = r.alpha;
    f.beta_c[k] = r.beta;
    for (int i = 0; i < 3; ++i) f.m_c[k][i] = r.m[i];
    for (int i = 0; i < 9; ++i) f.S_c[k][i] = r.S[i];
    f.iterations_c[k] = r.iterations;
  }
  probabilities(f.log_evidence_v, 2, f.prob_v);
  probabilities(f.log_evidence_c, 4, f.prob_c);
  f.sel_v = select_model(f.log_evidence_v, 2);
  f.sel_c = select_model(f.log_evidence_c, 4);
  for (int l = 0; l < 3; ++l) f.b[l] = s->b[l];
  s->fit = f;
  s->fitted = true;
  *out = f;
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_correction(const dsmc_surrogate_fit* fit, int n, double* S_faces,
                                      void* stream) {
  if (!fit || !S_faces) return reject(DSMC_E_INVAL, "surrogate: NULL");
  if (n < 1 || fit->sel_c < 0 || fit->sel_c > 3)
    return reject(DSMC_E_INVAL, "surrogate: n >= 1 and a selected model in C0..C3");
  cudaStream_t st = (cudaStream_t)stream;
  double* d = nullptr;
  SUR_CUDA(cudaMalloc(&d, ((size_t)n + 1) * sizeof(double)), "correction memory");
  const int k = fit->sel_c;
  const double* m = fit->m_c[k];
  k_correction<<<(n + 1 + 127) / 128, 128, 0, st>>>(k, m[0], m[1], m[2], fit->b[0], fit->b[1],
                                                    fit->b[2], n, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S_faces, d, ((size_t)n + 1) * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_reject(e, "correction");
  return DSMC_OK;
}

dsmc_status dsmc_surrogate_profile(dsmc_surrogate_handle s, const dsmc_surrogate_fit* fit,
                                   int n_cfd, const double* z, int n_trials, double* u_mean,
                                   double* u_std) {
  if (!s || !z || !u_mean) return reject(DSMC_E_INVAL, "surrogate: NULL");
  if (n_cfd < 1 || n_trials < 1) return reject(DSMC_E_INVAL, "surrogate: n_cfd, n_trials >= 1");
  if (!fit && !s->fitted) return reject(DSMC_E_STATE, "surrogate: no fit");
  const dsmc_surrogate_fit& f = fit ? *fit : s->fit;
  if (f.sel_v < 0 || f.sel_v > 1 || f.sel_c < 0 || f.sel_c > 3)
    return reject(DSMC_E_INVAL, "surrogate: selected models out of range");
  TrialModels tm{};
  tm.sel_v = f.sel_v;
  tm.k = f.sel_c;
  tm.m_v = f.sigma_p;
  tm.s_v = f.sigma_p_var;
  for (int i = 0; i < 3; ++i) tm.m[i] = f.m_c[f.sel_c][i];
  for (int i = 0; i < 9; ++i) tm.S[i] = f.S_c[f.sel_c][i];
  tm.kn = s->Kn;
  tm.F = s->F;
  for (int l = 0; l < 3; ++l) tm.b[l] = f.b[l];
  tm.n = n_cfd;
  // device space: z, profiles, Thomas scratch, mean, sd
  const size_t need = (size_t)n_trials * 4 + 2 * (size_t)n_trials * n_cfd + 2 * (size_t)n_cfd;
  if (need > s->trials_cap) {
    cudaFree(s->trials);
    s->trials = nullptr;
    s->trials_cap = 0;
    SUR_CUDA(cudaMalloc(&s->trials, need * sizeof(double)), "trial memory");
    s->trials_cap = need;
  }
  double* zd = s->trials;
  double* prof = zd + (size_t)n_trials * 4;
  double* scratch = prof + (size_t)n_trials * n_cfd;
  double* md = scratch + (size_t)n_trials * n_cfd;
  double* sd = md + n_cfd;
  SUR_CUDA(cudaMemcpyAsync(zd, z, (size_t)n_trials * 4 * sizeof(double), cudaMemcpyDefault,
                           s->stream),
           "copy z");
  k_trials<<<(n_trials + 127) / 128, 128, 0, s->stream>>>(tm, zd, n_trials, prof, scratch);
  SUR_CUDA(cudaGetLastError(), "trials kernel");
  k_bands<<<(n_cfd + 127) / 128, 128, 0, s->stream>>>(prof, n_trials, n_cfd, md, sd);
  SUR_CUDA(cudaGetLastError(), "bands kernel");
  SUR_CUDA(cudaMemcpyAsync(u_mean, md, n_cfd * sizeof(double), cudaMemcpyDefault, s->stream),
           "copy mean");
  if (u_std)
    SUR_CUDA(cudaMemcpyAsync(u_std, sd, n_cfd * sizeof(double), cudaMemcpyDefault, s->stream),
             "copy sd");
  SUR_CUDA(cudaStreamSynchronize(s->stream), "profile");
  return DSMC_OK;
}

}  // extern "C"
