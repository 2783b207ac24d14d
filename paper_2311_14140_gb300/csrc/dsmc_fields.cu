// dsmc_fields.cu -- cell fields from the raw moment sums: the last stage of the
// sampling (the paper's DSMC results are time averages of the sampled particles, Sec. 3,
// in the nondimensional units of Eq. 6).
//
// From the 13 raw sums S of a cell over n sampled steps of a run with ppc particles per
// cell at start (count, v_i, v_i v_j, v_i |v|^2, velocities in v0):
//   n    = S_0 / (n ppc)                  number density relative to the initial one
//   u_i  = S_i / S_0                      mean velocity (v0)
//   T    = (2/3) (<|v|^2> - |u|^2)        temperature (T0): m <|c|^2> / (3 k) with
//                                         v0^2 = 2 k T0 / m
//   Pxy  = 2 n (<vx vy> - ux uy)          shear stress (P0 = n0 k T0): rho / P0 = 2 / v0^2
//   q_i  = n <c_i |c|^2>                  heat flux (P0 v0), c = v - u, expanded in raw
//                                         moments: <v_i v^2> - 2 <v_i v_j> u_j - u_i <v^2>
//                                         + 2 u_i |u|^2
// All arithmetic binary64.  One function serves the host entry point and the kernel.
#include <cmath>

#include "dsmc.h"
#include "dsmc_internal.h"

namespace dsmc {

__host__ __device__ inline double quiet_nan() {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(0x7ff8000000000000LL);
#else
  return std::nan("");
#endif
}

__host__ __device__ inline void cell_fields(const double* S, double n_samples, double ppc,
                                            double* f) {
  const double N = S[0];
  if (!(N > 0.0)) {
    f[0] = 0.0;
    for (int k = 1; k < DSMC_NFIELD; ++k) f[k] = quiet_nan();
    return;
  }
  const double nhat = N / (n_samples * ppc);
  const double u[3] = {S[1] / N, S[2] / N, S[3] / N};
  // <v_i v_j>
  const double M[3][3] = {{S[4] / N, S[7] / N, S[8] / N},
                          {S[7] / N, S[5] / N, S[9] / N},
                          {S[8] / N, S[9] / N, S[6] / N}};
  const double vv = M[0][0] + M[1][1] + M[2][2];
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  f[0] = nhat;
  f[1] = u[0];
  f[2] = u[1];
  f[3] = u[2];
  f[4] = (2.0 / 3.0) * (vv - uu);
  f[5] = 2.0 * nhat * (M[0][1] - u[0] * u[1]);
  for (int i = 0; i < 3; ++i) {
    const double Mu = M[i][0] * u[0] + M[i][1] * u[1] + M[i][2] * u[2];
    f[6 + i] = nhat * (S[10 + i] / N - 2.0 * Mu - u[i] * vv + 2.0 * u[i] * uu);
  }
}

__global__ void k_cell_fields(const double* __restrict__ acc, int n_cells, double n_samples,
                              double ppc, double* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
    cell_fields(acc + (size_t)c * kNMom, n_samples, ppc, out + (size_t)c * DSMC_NFIELD);
}

cudaError_t launch_cell_fields(const double* acc, int n_cells, long long n_samples, int ppc,
                               double* out, cudaStream_t st) {
  const int blocks = (n_cells + 255) / 256;
  k_cell_fields<<<blocks, 256, 0, st>>>(acc, n_cells, (double)n_samples, (double)ppc, out);
  return cudaGetLastError();
}

}  // namespace dsmc

extern "C" dsmc_status dsmc_cell_fields(const double* sums, long long n_samples, int ppc,
                                        int n_cells, double* out) {
  if (!sums || !out) {
    dsmc::set_last_error("dsmc_cell_fields: NULL pointer");
    return DSMC_E_INVAL;
  }
  if (n_samples < 1 || ppc < 1 || n_cells < 1) {
    dsmc::set_last_error("dsmc_cell_fields: n_samples, ppc and n_cells must be >= 1");
    return DSMC_E_INVAL;
  }
  for (int c = 0; c < n_cells; ++c)
    dsmc::cell_fields(sums + (size_t)c * DSMC_NMOM, (double)n_samples, (double)ppc,
                      out + (size_t)c * DSMC_NFIELD);
  return DSMC_OK;
}
