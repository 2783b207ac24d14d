// dsmc_mms.cu -- the MMS hybrid (Sec. 2, Sec. 3.2) on the public C ABI: DSMC only in
// the Knudsen layer next to a wall, open to the CFD through a Chapman-Enskog interface,
// its data training the surrogates that correct the CFD, iterated.
//
// The DSMC sub-domain covers the training region (two mean free paths, Kn in channel
// units, rounded up to whole cells of width dy) plus `buffer` cells next to the
// interface; by the symmetry of the flow the layer at the bottom wall stands for both.
// In its own units the sub-domain has Kn / L_d and force F L_d.  Iteration k sets the
// interface from the current CFD profile (velocity at the face y = L_d, the mean of
// the two CFD cells next to it; stress P(L_d) = F (2 L_d - 1)), runs `steps` sampled
// steps (after `warmup` unsampled ones in the first iteration), adds one training
// sample per `window` steps (samples accumulate over iterations), retrains and solves
// the CFD with the selected models.  The first CFD profile is no-slip Navier-Stokes.
#include <cmath>
#include <string>
#include <vector>

#include "dsmc.h"
#include "dsmc_internal.h"

namespace {

dsmc_status reject(dsmc_status s, const std::string& msg) {
  dsmc::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" {

dsmc_status dsmc_default_mms_params(dsmc_mms_params* p) {
  if (!p) return reject(DSMC_E_INVAL, "mms params: NULL");
  *p = dsmc_mms_params{};
  p->gas.mass = 6.63e-26;
  p->gas.d_ref = 4.17e-10;
  p->gas.omega = 0.5;
  p->gas.T_ref = 273.0;
  p->wall_T = 273.0;
  p->dy = 0.005;
  p->ppc = 50;
  p->buffer = 5;
  p->iterations = 5;
  p->steps = 2000;
  p->window = 100;
  p->warmup = 1000;
  p->n_cfd = 200;
  p->group_size = 256;
  return DSMC_OK;
}

dsmc_status dsmc_mms_run(const dsmc_mms_params* p, void* stream, double* profile,
                         const double* z, int n_trials, double* band_sd,
                         dsmc_mms_result* out) {
  if (!p || !profile || !out) return reject(DSMC_E_INVAL, "mms: NULL argument");
  if (!(p->Kn > 0.0) || !std::isfinite(p->Kn) || !(p->dy > 0.0) || p->ppc < 1 ||
      p->buffer < 1 || p->iterations < 1 || p->iterations > DSMC_MMS_MAX_ITER ||
      p->window < 1 || p->steps < p->window || p->warmup < 0 || p->n_cfd < 4 ||
      !std::isfinite(p->body_force) || p->body_force == 0.0)
    return reject(DSMC_E_INVAL,
                  "mms: Kn > 0, dy > 0, ppc >= 1, buffer >= 1, 1 <= iterations <= 64, "
                  "steps >= window >= 1, warmup >= 0, n_cfd >= 4, F finite and != 0");
  if (z == nullptr && n_trials > 0) return reject(DSMC_E_INVAL, "mms: n_trials > 0 needs z");
  *out = dsmc_mms_result{};
  const int n_train = (int)std::ceil(2.0 * p->Kn / p->dy - 1e-9);
  const int n_sub = n_train + p->buffer;
  const double L_d = n_sub * p->dy;
  if (!(L_d < 0.5) || n_train < 2)
    return reject(DSMC_E_INVAL,
                  "mms: the Knudsen layers (2 lambda + buffer) must stay below half the channel "
                  "and hold at least 2 cells: run the whole channel instead");
  const double F = p->body_force;
  out->n_train = n_train;
  out->n_sub = n_sub;
  out->L_d = L_d;
  dsmc_surrogate_exponents(p->Kn, out->b);

  dsmc_options opt;
  dsmc_default_options(&opt);
  opt.stream = stream;
  opt.sample_start = 0;
  if (p->group_size) opt.group_size = p->group_size;
  dsmc_handle h = nullptr;
  dsmc_status st = dsmc_create_in(&p->gas, p->Kn / L_d, p->wall_T, F * L_d, n_sub, p->ppc,
                                  p->seed, &opt, nullptr, 0, &h);
  if (st != DSMC_OK) return st;
  dsmc_surrogate_handle s = nullptr;
  st = dsmc_surrogate_create_region(p->Kn, F, n_sub, p->ppc, L_d, n_train, out->b, stream, &s);
  if (st != DSMC_OK) {
    dsmc_destroy(h);
    return st;
  }
  std::vector<double> u(p->n_cfd);
  const double z0[4] = {0.0, 0.0, 0.0, 0.0};
  dsmc_surrogate_fit fit{};
  fit.sel_v = 0;
  fit.sel_c = 0;
  for (int l = 0; l < 3; ++l) fit.b[l] = out->b[l];
  auto done = [&](dsmc_status r) {
    dsmc_surrogate_destroy(s);
    dsmc_destroy(h);
    return r;
  };
  if ((st = dsmc_surrogate_profile(s, &fit, p->n_cfd, z0, 1, u.data(), nullptr)) != DSMC_OK)
    return done(st);
  const int face = (int)std::lround(L_d * p->n_cfd);
  for (int it = 0; it < p->iterations; ++it) {
    const double u_if = 0.5 * (u[face - 1] + u[face]);
    const double p_if = F * (2.0 * L_d - 1.0);
    if ((st = dsmc_set_open_top(h, 0, u_if, p_if)) != DSMC_OK) return done(st);
    out->u_interface[it] = (float)u_if;
    out->p_interface[it] = (float)p_if;
    if (it == 0 && p->warmup > 0 && (st = dsmc_step(h, p->warmup)) != DSMC_OK) return done(st);
    if ((st = dsmc_reset_samples(h)) != DSMC_OK) return done(st);
    for (int w = 0; w < p->steps / p->window; ++w) {
      if ((st = dsmc_step(h, p->window)) != DSMC_OK) return done(st);
      if ((st = dsmc_surrogate_add_run(s, h, 0)) != DSMC_OK) return done(st);
      out->samples += 1;
    }
    if ((st = dsmc_surrogate_train(s, &fit)) != DSMC_OK) return done(st);
    if ((st = dsmc_surrogate_profile(s, &fit, p->n_cfd, z0, 1, u.data(), nullptr)) != DSMC_OK)
      return done(st);
    out->iterations_done = it + 1;
  }
  out->fit = fit;
  for (int i = 0; i < p->n_cfd; ++i) profile[i] = u[i];
  if (n_trials > 0) {
    std::vector<double> mean(p->n_cfd);
    st = dsmc_surrogate_profile(s, &fit, p->n_cfd, z, n_trials, mean.data(), band_sd);
    if (st != DSMC_OK) return done(st);
  }
  if ((st = dsmc_sync(h)) != DSMC_OK) return done(st);
  return done(DSMC_OK);
}

}  // extern "C"
