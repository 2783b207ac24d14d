// dsmc_serve.cu -- request loop of micro-solves on a pool handle (continuous batching)
// and the same solve as a plain run of its own, on the public C ABI only.
//
// The paper's method asks its DSMC for many micro-solves at (Kn, force) points as the
// surrogate's training proceeds (Sec. 2.3-2.4); each is run until the channel-mean
// velocity is known to a relative standard error.  dsmc_serve takes such requests as
// they arrive, admits them into the pool while its device memory has room, advances
// every admitted instance together `epoch_steps` steps at a time, and retires each one
// whose error target is met, so that the next waiting requests can be admitted.
//
// Standard error: the channel sums of every instance are read after each epoch; the
// sampled epochs are split into `batches` consecutive batches of (nearly) equal length,
// each batch gives a channel-mean velocity (sum vx / count over its samples), and the
// standard error of the mean is the standard deviation of the batch means over
// sqrt(batches) (the method of batch means for correlated samples).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "dsmc.h"
#include "dsmc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

dsmc_status reject(dsmc_status s, const std::string& msg) {
  dsmc::set_last_error(msg);
  return s;
}

// Running statistics of one request: per-epoch increments of the channel sums.
struct Track {
  int req = -1;
  long long steps = 0;
  double last_n = 0.0, last_u = 0.0;
  std::vector<double> dn, du;  // sampled epochs only
};

// Batch-means estimate from the epochs of `t`; returns false with fewer epochs than
// batches.
bool batch_means(const Track& t, int batches, double* mean, double* se) {
  const int n = (int)t.dn.size();
  if (n < batches || batches < 2) return false;
  double tot_n = 0.0, tot_u = 0.0;
  for (int e = 0; e < n; ++e) {
    tot_n += t.dn[e];
    tot_u += t.du[e];
  }
  if (!(tot_n > 0.0)) return false;
  std::vector<double> means;
  means.reserve(batches);
  int e = 0;
  for (int b = 0; b < batches; ++b) {
    const int len = n / batches + (b < n % batches ? 1 : 0);
    double bn = 0.0, bu = 0.0;
    for (int k = 0; k < len; ++k, ++e) {
      bn += t.dn[e];
      bu += t.du[e];
    }
    if (!(bn > 0.0)) return false;
    means.push_back(bu / bn);
  }
  double m = 0.0;
  for (double x : means) m += x;
  m /= batches;
  double v = 0.0;
  for (double x : means) v += (x - m) * (x - m);
  v /= (batches - 1);
  *mean = tot_u / tot_n;
  *se = std::sqrt(v / batches);
  return true;
}

// Adds the epoch's increments to `t` from the channel sums (n, u); true when the request
// is done (target met or step limit), with the result filled in.
bool update(Track& t, double n, double u, const dsmc_request& r, const dsmc_serve_options& so,
            dsmc_request_result* res) {
  const double dn = n - t.last_n, du = u - t.last_u;
  t.last_n = n;
  t.last_u = u;
  if (dn > 0.0) {
    t.dn.push_back(dn);
    t.du.push_back(du);
  }
  double mean = 0.0, se = INFINITY;
  const bool have = batch_means(t, so.batches, &mean, &se);
  const bool met = have && mean != 0.0 && se <= r.target_se * std::fabs(mean);
  if (!met && t.steps < r.max_steps) return false;
  res->steps = t.steps;
  res->u_mean = n > 0.0 ? u / n : 0.0;
  res->u_se = have ? se : INFINITY;
  res->count = n;
  res->sum_vx = u;
  res->converged = met ? 1 : 0;
  return true;
}

dsmc_status check_requests(const dsmc_request* req, int n_req, const dsmc_serve_options* so) {
  if (!req || n_req < 1) return reject(DSMC_E_INVAL, "serve: requests NULL or n_requests < 1");
  if (!so || so->epoch_steps < 1 || so->batches < 2)
    return reject(DSMC_E_INVAL, "serve options: epoch_steps >= 1 and batches >= 2");
  for (int i = 0; i < n_req; ++i) {
    if (!(req[i].target_se > 0.0) || req[i].max_steps < 1 || !(req[i].arrival >= 0.0))
      return reject(DSMC_E_INVAL, "request " + std::to_string(i) +
                                      ": target_se > 0, max_steps >= 1, arrival >= 0");
    if (i > 0 && req[i].arrival < req[i - 1].arrival)
      return reject(DSMC_E_INVAL, "requests must be in order of arrival");
  }
  return DSMC_OK;
}

}  // namespace

extern "C" {

dsmc_status dsmc_default_serve_options(dsmc_serve_options* so) {
  if (!so) return reject(DSMC_E_INVAL, "serve options: NULL");
  so->epoch_steps = 32;
  so->batches = 16;
  so->max_active = 0;
  so->time_limit = 0.0;
  return DSMC_OK;
}

dsmc_status dsmc_serve(dsmc_handle pool, const dsmc_request* req, int n_req,
                       const dsmc_serve_options* so, dsmc_request_result* res) {
  if (!pool) return reject(DSMC_E_INVAL, "handle: NULL");
  if (!res) return reject(DSMC_E_INVAL, "results: NULL");
  dsmc_status st = check_requests(req, n_req, so);
  if (st != DSMC_OK) return st;
  if (dsmc_batch_size(pool) != 0) return reject(DSMC_E_STATE, "serve: the pool must be empty");
  for (int i = 0; i < n_req; ++i) {
    res[i] = dsmc_request_result{};
    res[i].admitted = res[i].finished = -1.0;
    res[i].id = -1;
  }
  const auto t0 = Clock::now();
  std::deque<int> waiting;
  std::vector<Track> active;  // by pool id
  std::vector<double> sums;
  int next = 0, done = 0, n_active = 0;
  while (done < n_req) {
    double now = seconds_since(t0);
    if (so->time_limit > 0.0 && now > so->time_limit) break;
    while (next < n_req && req[next].arrival <= now) waiting.push_back(next++);
    // Admit in order of arrival while the pool has room.
    while (!waiting.empty() && (so->max_active <= 0 || n_active < so->max_active)) {
      const int q = waiting.front();
      int id = -1;
      st = dsmc_pool_add(pool, &req[q].instance, &id);
      if (st == DSMC_E_NOMEM && n_active > 0) break;  // wait for room
      waiting.pop_front();
      if (st != DSMC_OK) {  // invalid, or larger than the empty pool: never runs
        res[q].finished = seconds_since(t0);
        res[q].converged = -1;
        ++done;
        continue;
      }
      if ((int)active.size() <= id) active.resize((size_t)id + 1);
      active[id] = Track{};
      active[id].req = q;
      res[q].admitted = seconds_since(t0);
      res[q].id = id;
      ++n_active;
    }
    if (n_active == 0) {
      if (next >= n_req) break;
      const double wait = req[next].arrival - seconds_since(t0);
      if (wait > 0.0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
      continue;
    }
    if ((st = dsmc_step(pool, so->epoch_steps)) != DSMC_OK) return st;
    sums.assign(2 * (size_t)dsmc_id_bound(pool), 0.0);
    if ((st = dsmc_channel_sums(pool, sums.data())) != DSMC_OK) return st;
    now = seconds_since(t0);
    for (int id = 0; id < (int)active.size(); ++id) {
      Track& t = active[id];
      if (t.req < 0) continue;
      t.steps += so->epoch_steps;
      dsmc_request_result* r = &res[t.req];
      if (update(t, sums[2 * id], sums[2 * id + 1], req[t.req], *so, r)) {
        r->finished = now;
        r->id = id;
        if ((st = dsmc_pool_remove(pool, id)) != DSMC_OK) return st;
        t.req = -1;
        --n_active;
        ++done;
      }
    }
  }
  // Time limit: what is still running or waiting is reported as not finished.
  for (auto& t : active)
    if (t.req >= 0) {
      res[t.req].steps = t.steps;
      dsmc_pool_remove(pool, res[t.req].id);
      t.req = -1;
    }
  return DSMC_OK;
}

dsmc_status dsmc_solve(const dsmc_request* req, const dsmc_options* opt,
                       const dsmc_serve_options* so, dsmc_request_result* res) {
  if (!res) return reject(DSMC_E_INVAL, "result: NULL");
  dsmc_status st = check_requests(req, 1, so);
  if (st != DSMC_OK) return st;
  *res = dsmc_request_result{};
  res->admitted = res->finished = -1.0;
  res->id = 0;
  const auto t0 = Clock::now();
  dsmc_handle h = nullptr;
  const dsmc_instance& d = req->instance;
  st = dsmc_create_in(&d.gas, d.Kn, d.wall_T, d.body_force, d.n_cells, d.ppc, d.seed, opt,
                      nullptr, 0, &h);
  if (st != DSMC_OK) return st;
  res->admitted = seconds_since(t0);
  Track t;
  t.req = 0;
  double sums[2];
  for (;;) {
    if ((st = dsmc_step(h, so->epoch_steps)) != DSMC_OK) break;
    if ((st = dsmc_channel_sums(h, sums)) != DSMC_OK) break;
    t.steps += so->epoch_steps;
    if (update(t, sums[0], sums[1], *req, *so, res)) break;
  }
  res->finished = seconds_since(t0);
  dsmc_destroy(h);
  return st;
}

}  // extern "C"
