// dsmc_capi.cu -- host side of the C ABI declared in include/dsmc.h: argument checks,
// the derived parameters of the method, device memory layout, the order of kernel
// launches within a step, synchronisation, the device error word and kernel timing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dsmc.h"
#include "dsmc_internal.h"

using namespace dsmc;

namespace {

thread_local std::string g_last_error;

dsmc_status fail(dsmc_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

dsmc_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return DSMC_E_CUDA;
}

#define DSMC_CUDA(call, what)                  \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

enum KernelId {
  K_INIT = 0,
  K_COLLIDE_MOVE,
  K_SCAN,
  K_OFFSETS,
  K_SCATTER_SPANS,
  K_INDEX_COUNT,
  K_INDEX_SCATTER,
  K_NUM
};
const char* const kKernelNames[K_NUM] = {"init",          "collide_move", "scan_hist",
                                         "cell_offsets",  "scatter_spans", "index_count",
                                         "index_scatter"};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Layout {
  int n_cap;
  SortPlan plan;  // fixed spans of slots for the stand-alone sort into cells
  int cps;        // cells per span of the step passes
  int n_spans;
  size_t st, hist, count, offset, smax, ncand, nacc, acc, err, total;
};

// Spans of the step: consecutive cells, enough of them that a span holds a few
// thousand particles at the initial density and that there are at most kMaxSpans.
void make_spans(int n_cells, int ppc, int* cps, int* n_spans) {
  const long long N = (long long)n_cells * ppc;
  long long target = (N + kMaxSpans - 1) / kMaxSpans;
  if (target < 2048) target = 2048;
  long long c = (target + ppc - 1) / ppc;
  if (c < (n_cells + kMaxSpans - 1) / kMaxSpans) c = (n_cells + kMaxSpans - 1) / kMaxSpans;
  if (c > kMaxCellsPerSpan) c = kMaxCellsPerSpan;
  if (c > n_cells) c = n_cells;
  if (c < 1) c = 1;
  *cps = (int)c;
  *n_spans = (int)((n_cells + c - 1) / c);
}

SortPlan make_plan(long long N, int n_cells) {
  long long w = (N + 255) / 256;
  if (w > kSortWarpsMax) w = kSortWarpsMax;
  if (w < 1) w = 1;
  long long span = (N + w - 1) / w;
  span = (span + 31) & ~31LL;
  if (span < 32) span = 32;
  w = (N + span - 1) / span;
  if (w < 1) w = 1;
  long long wpb = (long long)(kSortSmemMax / (sizeof(int) * (size_t)n_cells));
  if (wpb > kSortWarpsPerBlock) wpb = kSortWarpsPerBlock;
  if (wpb > w) wpb = w;
  if (wpb < 1) wpb = 1;
  return SortPlan{(int)w, (int)span, (int)wpb};
}

Layout make_layout(int n_cells, int ppc) {
  Layout L{};
  const long long N = (long long)n_cells * ppc;
  L.n_cap = (int)((N + 63) & ~63LL);
  L.plan = make_plan(N, n_cells);
  make_spans(n_cells, ppc, &L.cps, &L.n_spans);
  const size_t rows = (size_t)(L.plan.n_warps > L.n_spans ? L.plan.n_warps : L.n_spans);
  size_t o = 0;
  L.st = o;
  o += align256(8 * (size_t)L.n_cap * sizeof(float));
  L.hist = o;
  o += align256(rows * n_cells * sizeof(int));
  L.count = o;
  o += align256((size_t)n_cells * sizeof(int));
  L.offset = o;  // two arrays of n_cells + 1: current and next
  o += align256(2 * ((size_t)n_cells + 1) * sizeof(int));
  L.smax = o;
  o += align256(2 * (size_t)n_cells * sizeof(float));
  L.ncand = o;
  o += align256((size_t)n_cells * sizeof(unsigned long long));
  L.nacc = o;
  o += align256((size_t)n_cells * sizeof(unsigned long long));
  L.acc = o;
  o += align256((size_t)n_cells * kNMom * sizeof(double));
  L.err = o;
  o += 256;
  L.total = o;
  return L;
}

// Parameters of the method in binary64, rounded once to binary32 where the kernels
// use them.
struct Params {
  double nsig, dt;
  float dt_f, F_f, coef, cvhs, vexp, vinv, lncv, smax0;
};

// n sigma_ref H from Kn through mu0 v0 / (P0 H) = 2 Kn / sqrt(pi) (Eq. 7) and the
// first Chapman-Enskog viscosity of VHS molecules, mu = 15 sqrt(pi m k T) /
// (2 sigma (5 - 2 omega)(7 - 2 omega)) (Bird): n sigma H = 15 sqrt(2) pi /
// (4 (5 - 2 omega)(7 - 2 omega) Kn).  The equilibrium collision frequency is
// nu = n sigma <g>, <g> = 2 sqrt(2) / sqrt(pi).  VHS: sigma g / sigma_ref =
// 2^(omega - 1/2) / Gamma(5/2 - omega) g^(2 - 2 omega) in v0 units, which makes
// <sigma g> = sigma_ref <g> at the wall temperature.
bool derive_params(double omega, double Kn, double F, int ppc, const dsmc_options& o,
                   Params* p) {
  double nsig = 0.0;
  if (!std::isinf(Kn)) {
    const double top = 15.0 * std::sqrt(2.0) * M_PI;
    const double bottom = 4.0 * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega) * Kn;
    nsig = top / bottom;
  }
  const double mean_g = 2.0 * std::sqrt(2.0) / std::sqrt(M_PI);
  const double nu = nsig * mean_g;
  double dt;
  if (o.dt > 0.0)
    dt = o.dt;
  else if (nu > 0.0)
    dt = o.dt_factor / nu;
  else
    return false;
  const double cv = (omega == 0.5) ? 1.0 : std::pow(2.0, omega - 0.5) / std::tgamma(2.5 - omega);
  p->nsig = nsig;
  p->dt = dt;
  p->dt_f = (float)dt;
  p->F_f = (float)F;
  p->coef = (float)(nsig * dt / (2.0 * (double)ppc));
  p->cvhs = (float)cv;
  p->vexp = (float)(2.0 - 2.0 * omega);
  p->vinv = (omega < 1.0) ? (float)(1.0 / (2.0 - 2.0 * omega)) : 0.0f;
  p->lncv = (float)std::log(cv);
  p->smax0 = (float)(cv * std::pow(5.0, 2.0 - 2.0 * omega));
  return std::isfinite(dt) && dt > 0.0;
}

dsmc_status check_options(const dsmc_options* o) {
  if (!o) return fail(DSMC_E_INVAL, "options: NULL");
  if (!(o->dt_factor > 0.0) || !std::isfinite(o->dt_factor))
    return fail(DSMC_E_INVAL, "options: dt_factor must be finite and > 0");
  if (!(o->dt >= 0.0) || !std::isfinite(o->dt))
    return fail(DSMC_E_INVAL, "options: dt must be finite and >= 0");
  if (o->group_size < 2 || o->group_size > kMaxGroup || (o->group_size & 1))
    return fail(DSMC_E_INVAL, "options: group_size must be even, 2..512");
  return DSMC_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

void dsmc::set_last_error(const std::string& msg) { g_last_error = msg; }

struct dsmc_sim {
  int device = 0;
  int n_cells = 0, ppc = 0;
  long long N = 0;
  double omega = 0.5, Kn = 1.0, F = 0.0;
  Params p{};
  float ncf = 1.0f;
  uint64_t seed = 0;
  dsmc_options opt{};
  long long step = 0, n_samples = 0;
  Layout L{};
  void* ws = nullptr;
  bool owns = false;
  float4* P[2]{};  // particle records (y, vx, vy, vz), double-buffered for the sort
  int cur = 0;
  int *hist = nullptr, *count = nullptr, *err = nullptr;
  int* off[2]{};
  int ocur = 0;
  float* smax[2]{};
  int scur = 0;
  unsigned long long *ncand = nullptr, *nacc = nullptr;
  double* acc = nullptr;
  dsmc_status latched = DSMC_OK;
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kernel;
  size_t events_used = 0;
  double ktime[K_NUM] = {};
  long long kcount[K_NUM] = {};

  cudaStream_t stream() const { return (cudaStream_t)opt.stream; }
  uint32_t k0() const { return (uint32_t)(seed & 0xffffffffu); }
  uint32_t k1() const { return (uint32_t)(seed >> 32); }
};

namespace {

// Kernel timing: an event pair around a launch when profiling.
cudaError_t mark(dsmc_sim* h, int kernel) {
  if (!h->opt.profile) return cudaSuccess;
  if (h->events_used + 1 >= h->events.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      h->events.push_back(e);
      h->event_kernel.push_back(-1);
    }
  }
  h->event_kernel[h->events_used] = kernel;
  return cudaEventRecord(h->events[h->events_used++], h->stream());
}

template <typename Launch>
cudaError_t timed(dsmc_sim* h, int kernel, Launch&& launch) {
  cudaError_t e = mark(h, kernel);
  if (e != cudaSuccess) return e;
  e = launch();
  if (e != cudaSuccess) return e;
  return mark(h, -1);
}

dsmc_status collect_times(dsmc_sim* h) {
  if (h->events_used == 0) return DSMC_OK;
  DSMC_CUDA(cudaStreamSynchronize(h->stream()), "profile sync");
  for (size_t i = 0; i + 1 < h->events_used; i += 2) {
    float ms = 0.0f;
    DSMC_CUDA(cudaEventElapsedTime(&ms, h->events[i], h->events[i + 1]), "event time");
    const int k = h->event_kernel[i];
    if (k >= 0 && k < K_NUM) {
      h->ktime[k] += ms;
      h->kcount[k] += 1;
    }
  }
  h->events_used = 0;
  return DSMC_OK;
}

StepArgs step_args(const dsmc_sim* h, bool count_only) {
  const int G = h->opt.group_size;
  const bool sampling = h->step >= h->opt.sample_start;
  const bool collide = h->opt.collisions != 0 && h->p.nsig > 0.0;
  const int mode = (h->omega == 0.5) ? 0 : (h->omega == 1.0 ? 2 : 1);
  StepArgs a{};
  a.n_cells = h->n_cells;
  a.cps = h->L.cps;
  a.cap = G + G / 2 - 1;
  a.G = G;
  a.ncf = h->ncf;
  a.dt = h->p.dt_f;
  a.F = h->p.F_f;
  a.coef = h->p.coef;
  a.cvhs = h->p.cvhs;
  a.vexp = h->p.vexp;
  a.vinv = h->p.vinv;
  a.lncv = h->p.lncv;
  a.k0 = h->k0();
  a.k1 = h->k1();
  for (int r = 0; r < 10; ++r) {
    a.keys.k0[r] = a.k0 + (uint32_t)r * 0x9E3779B9u;
    a.keys.k1[r] = a.k1 + (uint32_t)r * 0xBB67AE85u;
  }
  a.step = (uint32_t)h->step;
  a.sample = (sampling && !count_only) ? 1 : 0;
  a.collide = (collide && !count_only) ? 1 : 0;
  a.mode = mode;
  a.count_only = count_only ? 1 : 0;
  return a;
}

// Sort into cells without moving (creation, state load).  off[ocur] must describe
// spans of slots (slot ranges per cell span); the records may be in any order within
// them.  Counting pass over the spans, prefix over spans and cells, stable scatter.
dsmc_status run_index(dsmc_sim* h) {
  cudaStream_t s = h->stream();
  const StepArgs a = step_args(h, /*count_only=*/true);
  int* off_cur = h->off[h->ocur];
  int* off_new = h->off[h->ocur ^ 1];
  DSMC_CUDA(timed(h, K_INDEX_COUNT, [&] {
              return launch_collide_move(h->P[h->cur], off_cur, h->smax[h->scur],
                                         h->smax[h->scur ^ 1], h->ncand, h->nacc, h->acc,
                                         h->hist, a, h->L.n_spans, h->err, s);
            }),
            "index_count");
  DSMC_CUDA(timed(h, K_SCAN,
                  [&] { return launch_scan_hist(h->hist, h->L.n_spans, h->n_cells, h->count, s); }),
            "scan_hist");
  DSMC_CUDA(timed(h, K_OFFSETS,
                  [&] { return launch_cell_offsets(h->count, h->n_cells, off_new, s); }),
            "cell_offsets");
  DSMC_CUDA(timed(h, K_INDEX_SCATTER, [&] {
              return launch_scatter_spans(h->P[h->cur], h->P[h->cur ^ 1], off_cur, off_new,
                                          h->hist, h->n_cells, h->L.cps, h->L.n_spans, h->ncf,
                                          (int)h->N, h->err, s);
            }),
            "index_scatter");
  h->cur ^= 1;
  h->ocur ^= 1;
  return DSMC_OK;
}

// Spans of slots for a sort of records in arbitrary order: cell span k covers slots
// [off[k cps], off[(k+1) cps]) with off[c] = floor(c N / n_cells).
dsmc_status set_uniform_offsets(dsmc_sim* h, std::vector<int>& host) {
  host.resize((size_t)h->n_cells + 1);
  for (int c = 0; c <= h->n_cells; ++c) host[c] = (int)((long long)c * h->N / h->n_cells);
  DSMC_CUDA(cudaMemcpyAsync(h->off[h->ocur], host.data(), host.size() * sizeof(int),
                            cudaMemcpyHostToDevice, h->stream()),
            "offsets");
  return DSMC_OK;
}

// One step: collide + sample + move + count (one pass over the records, in place),
// prefix over spans and cells, stable scatter into the other buffer.
dsmc_status run_step(dsmc_sim* h) {
  cudaStream_t s = h->stream();
  const StepArgs a = step_args(h, /*count_only=*/false);
  int* off_cur = h->off[h->ocur];
  int* off_new = h->off[h->ocur ^ 1];
  DSMC_CUDA(timed(h, K_COLLIDE_MOVE, [&] {
              return launch_collide_move(h->P[h->cur], off_cur, h->smax[h->scur],
                                         h->smax[h->scur ^ 1], h->ncand, h->nacc, h->acc,
                                         h->hist, a, h->L.n_spans, h->err, s);
            }),
            "collide_move");
  h->scur ^= 1;
  DSMC_CUDA(timed(h, K_SCAN,
                  [&] { return launch_scan_hist(h->hist, h->L.n_spans, h->n_cells, h->count, s); }),
            "scan_hist");
  DSMC_CUDA(timed(h, K_OFFSETS,
                  [&] { return launch_cell_offsets(h->count, h->n_cells, off_new, s); }),
            "cell_offsets");
  DSMC_CUDA(timed(h, K_SCATTER_SPANS, [&] {
              return launch_scatter_spans(h->P[h->cur], h->P[h->cur ^ 1], off_cur, off_new,
                                          h->hist, h->n_cells, h->L.cps, h->L.n_spans, h->ncf,
                                          (int)h->N, h->err, s);
            }),
            "scatter_spans");
  h->cur ^= 1;
  h->ocur ^= 1;
  return DSMC_OK;
}

// The collide/move pass must fit one CTA's shared memory for this group size.
bool step_fits(int n_cells, int cps, int G) {
  return step_smem_layout(n_cells, cps, G + G / 2 - 1).total <= kStepSmemMax;
}

dsmc_status read_error_word(dsmc_sim* h) {
  int v = 0;
  DSMC_CUDA(cudaMemcpyAsync(&v, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream()),
            "read error word");
  DSMC_CUDA(cudaStreamSynchronize(h->stream()), "stream sync");
  if (v != 0) {
    h->latched = DSMC_E_DEVICE_LIMIT;
    std::string what;
    if (v & kErrNormals) what += " gaussian-attempts";
    if (v & kErrBounces) what += " wall-bounces";
    if (v & kErrSphere) what += " scattering-attempts";
    if (v & kErrCandidates) what += " candidate-count";
    if (v & kErrSort) what += " sort-destination";
    if (v & kErrCopyTimeout) what += " bulk-copy-timeout";
    return fail(DSMC_E_DEVICE_LIMIT, "device limit reached:" + what);
  }
  return DSMC_OK;
}

dsmc_status check_handle(dsmc_sim* h) {
  if (!h) return fail(DSMC_E_INVAL, "handle: NULL");
  return DSMC_OK;
}

}  // namespace

extern "C" {

dsmc_status dsmc_default_options(dsmc_options* opt) {
  if (!opt) return fail(DSMC_E_INVAL, "options: NULL");
  opt->dt_factor = 0.2;
  opt->dt = 0.0;
  opt->sample_start = 0;
  opt->group_size = 256;
  opt->collisions = 1;
  opt->profile = 0;
  opt->stream = nullptr;
  return DSMC_OK;
}

size_t dsmc_workspace_bytes(int n_cells, int ppc) {
  if (n_cells < 1 || ppc < 1) return 0;
  return make_layout(n_cells, ppc).total;
}

dsmc_status dsmc_create_in(const dsmc_gas* gas, double Kn, double wall_T, double body_force,
                           int n_cells, int ppc, uint64_t seed, const dsmc_options* opt_in,
                           void* workspace, size_t workspace_bytes, dsmc_handle* out) {
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  *out = nullptr;
  if (!gas) return fail(DSMC_E_INVAL, "gas: NULL");
  if (!(gas->mass > 0.0) || !(gas->d_ref > 0.0) || !(gas->T_ref > 0.0))
    return fail(DSMC_E_INVAL, "gas: mass, d_ref and T_ref must be > 0");
  if (!(gas->omega >= 0.5 && gas->omega <= 1.0))
    return fail(DSMC_E_INVAL, "gas: omega must lie in [0.5, 1]");
  if (!(Kn > 0.0)) return fail(DSMC_E_INVAL, "Kn must be > 0 (or +inf)");
  if (!(wall_T > 0.0) || !std::isfinite(wall_T)) return fail(DSMC_E_INVAL, "wall_T must be > 0");
  if (!std::isfinite(body_force)) return fail(DSMC_E_INVAL, "body_force must be finite");
  if (n_cells < 1 || ppc < 1) return fail(DSMC_E_INVAL, "n_cells and ppc must be >= 1");
  const long long N = (long long)n_cells * ppc;
  if (N > kMaxParticles) return fail(DSMC_E_INVAL, "n_cells * ppc must be <= 2^31 - 2^24");
  if (n_cells > kMaxStepCells) return fail(DSMC_E_INVAL, "n_cells must be <= 16384");
  dsmc_options opt;
  dsmc_default_options(&opt);
  if (opt_in) opt = *opt_in;
  dsmc_status st = check_options(&opt);
  if (st != DSMC_OK) return st;
  Params p;
  if (!derive_params(gas->omega, Kn, body_force, ppc, opt, &p))
    return fail(DSMC_E_INVAL, "time step undefined: set options.dt for infinite Kn");
  {
    int cps, n_spans;
    make_spans(n_cells, ppc, &cps, &n_spans);
    if (!step_fits(n_cells, cps, opt.group_size))
      return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  }

  dsmc_sim* h = new (std::nothrow) dsmc_sim();
  if (!h) return fail(DSMC_E_NOMEM, "host allocation failed");
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce != cudaSuccess) {
    delete h;
    return cuda_fail(ce, "cudaGetDevice");
  }
  h->n_cells = n_cells;
  h->ppc = ppc;
  h->N = N;
  h->omega = gas->omega;
  h->Kn = Kn;
  h->F = body_force;
  h->p = p;
  h->ncf = (float)n_cells;
  h->seed = seed;
  h->opt = opt;
  h->L = make_layout(n_cells, ppc);
  if (workspace) {
    if (workspace_bytes < h->L.total || ((uintptr_t)workspace & 255u)) {
      delete h;
      return fail(DSMC_E_NOMEM, "workspace smaller than dsmc_workspace_bytes or not 256-byte aligned");
    }
    h->ws = workspace;
    h->owns = false;
  } else {
    ce = cudaMalloc(&h->ws, h->L.total);
    if (ce != cudaSuccess) {
      delete h;
      cudaGetLastError();
      return fail(DSMC_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(ce));
    }
    h->owns = true;
  }
  char* b = (char*)h->ws;
  h->P[0] = (float4*)(b + h->L.st);
  h->P[1] = h->P[0] + h->L.n_cap;
  h->hist = (int*)(b + h->L.hist);
  h->count = (int*)(b + h->L.count);
  h->off[0] = (int*)(b + h->L.offset);
  h->off[1] = h->off[0] + (n_cells + 1);
  h->smax[0] = (float*)(b + h->L.smax);
  h->smax[1] = h->smax[0] + n_cells;
  h->ncand = (unsigned long long*)(b + h->L.ncand);
  h->nacc = (unsigned long long*)(b + h->L.nacc);
  h->acc = (double*)(b + h->L.acc);
  h->err = (int*)(b + h->L.err);

  auto bail = [&](dsmc_status s) {
    dsmc_destroy(h);
    return s;
  };
  cudaStream_t s = h->stream();
  ce = set_step_smem_limits(kStepSmemMax, kStepSmemMax);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaFuncSetAttribute"));
  if ((ce = cudaMemsetAsync(h->acc, 0, (size_t)n_cells * kNMom * sizeof(double), s)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->ncand, 0, (size_t)n_cells * 8, s)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->nacc, 0, (size_t)n_cells * 8, s)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->err, 0, sizeof(int), s)) != cudaSuccess)
    return bail(cuda_fail(ce, "cudaMemsetAsync"));
  std::vector<float> smax0((size_t)n_cells, p.smax0);
  ce = cudaMemcpyAsync(h->smax[0], smax0.data(), (size_t)n_cells * sizeof(float),
                       cudaMemcpyHostToDevice, s);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemcpyAsync"));
  ce = timed(h, K_INIT,
             [&] { return launch_init(h->P[0], (int)N, ppc, h->ncf, h->k0(), h->k1(), h->err, s); });
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "init"));
  // Particle p was drawn in cell p / ppc: slot spans of whole cells.
  std::vector<int> off0((size_t)n_cells + 1);
  for (int c = 0; c <= n_cells; ++c) off0[c] = c * ppc;
  ce = cudaMemcpyAsync(h->off[h->ocur], off0.data(), off0.size() * sizeof(int),
                       cudaMemcpyHostToDevice, s);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemcpyAsync"));
  st = run_index(h);
  if (st != DSMC_OK) return bail(st);
  ce = cudaStreamSynchronize(s);  // smax0 host buffer must outlive the copy
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "stream sync"));
  st = collect_times(h);
  if (st != DSMC_OK) return bail(st);
  st = read_error_word(h);
  if (st != DSMC_OK) return bail(st);
  *out = h;
  return DSMC_OK;
}

dsmc_status dsmc_create(const dsmc_gas* gas, double Kn, double wall_T, double body_force,
                        int n_cells, int ppc, uint64_t seed, dsmc_handle* out) {
  return dsmc_create_in(gas, Kn, wall_T, body_force, n_cells, ppc, seed, nullptr, nullptr, 0,
                        out);
}

dsmc_status dsmc_set_options(dsmc_handle h, const dsmc_options* opt) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  s = check_options(opt);
  if (s != DSMC_OK) return s;
  Params p;
  if (!derive_params(h->omega, h->Kn, h->F, h->ppc, *opt, &p))
    return fail(DSMC_E_INVAL, "time step undefined: set options.dt for infinite Kn");
  if (!step_fits(h->n_cells, h->L.cps, opt->group_size))
    return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  if (h->events_used) {
    s = collect_times(h);
    if (s != DSMC_OK) return s;
  }
  h->opt = *opt;
  h->p = p;
  return DSMC_OK;
}

dsmc_status dsmc_step(dsmc_handle h, int n_steps) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (n_steps < 0) return fail(DSMC_E_INVAL, "n_steps must be >= 0");
  if (h->latched != DSMC_OK) return fail(h->latched, "an earlier step reached a device limit");
  DeviceGuard guard(h->device);
  for (int it = 0; it < n_steps; ++it) {
    h->step += 1;
    if (h->step >= h->opt.sample_start) h->n_samples += 1;
    s = run_step(h);
    if (s != DSMC_OK) return s;
  }
  if (h->opt.profile) return collect_times(h);
  return DSMC_OK;
}

dsmc_status dsmc_sync(dsmc_handle h) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  s = collect_times(h);
  if (s != DSMC_OK) return s;
  return read_error_word(h);
}

dsmc_status dsmc_sample_moments(dsmc_handle h, double* out, long long* n_samples) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  DSMC_CUDA(cudaMemcpyAsync(out, h->acc, (size_t)h->n_cells * kNMom * sizeof(double),
                            cudaMemcpyDefault, h->stream()),
            "copy moments");
  if (n_samples) *n_samples = h->n_samples;
  return dsmc_sync(h);
}

dsmc_status dsmc_reset_samples(dsmc_handle h) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  DSMC_CUDA(cudaMemsetAsync(h->acc, 0, (size_t)h->n_cells * kNMom * sizeof(double), st), "reset");
  DSMC_CUDA(cudaMemsetAsync(h->ncand, 0, (size_t)h->n_cells * 8, st), "reset");
  DSMC_CUDA(cudaMemsetAsync(h->nacc, 0, (size_t)h->n_cells * 8, st), "reset");
  h->n_samples = 0;
  return DSMC_OK;
}

dsmc_status dsmc_copy_state(dsmc_handle h, float* y, float* vx, float* vy, float* vz) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  // Unpack the records into four arrays in the idle sort buffer, then copy out.
  float* tmp = reinterpret_cast<float*>(h->P[h->cur ^ 1]);
  const size_t n = (size_t)h->N;
  float* arr[4] = {tmp, tmp + n, tmp + 2 * n, tmp + 3 * n};
  DSMC_CUDA(launch_unpack(h->P[h->cur], arr[0], arr[1], arr[2], arr[3], (int)h->N, st), "unpack");
  float* dst[4] = {y, vx, vy, vz};
  for (int k = 0; k < 4; ++k)
    if (dst[k])
      DSMC_CUDA(cudaMemcpyAsync(dst[k], arr[k], n * sizeof(float), cudaMemcpyDefault, st),
                "copy state");
  return dsmc_sync(h);
}

dsmc_status dsmc_copy_cells(dsmc_handle h, int* offset, float* smax, unsigned long long* ncand,
                            unsigned long long* nacc) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  const size_t nc = (size_t)h->n_cells;
  if (offset)
    DSMC_CUDA(cudaMemcpyAsync(offset, h->off[h->ocur], (nc + 1) * sizeof(int), cudaMemcpyDefault,
                              st),
              "copy cells");
  if (smax)
    DSMC_CUDA(cudaMemcpyAsync(smax, h->smax[h->scur], nc * sizeof(float), cudaMemcpyDefault, st), "copy cells");
  if (ncand) DSMC_CUDA(cudaMemcpyAsync(ncand, h->ncand, nc * 8, cudaMemcpyDefault, st), "copy cells");
  if (nacc) DSMC_CUDA(cudaMemcpyAsync(nacc, h->nacc, nc * 8, cudaMemcpyDefault, st), "copy cells");
  return dsmc_sync(h);
}

dsmc_status dsmc_load_state(dsmc_handle h, const float* y, const float* vx, const float* vy,
                            const float* vz, const float* smax, long long step) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!y || !vx || !vy || !vz) return fail(DSMC_E_INVAL, "state arrays must not be NULL");
  if (step < 0) return fail(DSMC_E_INVAL, "step must be >= 0");
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  float* tmp = reinterpret_cast<float*>(h->P[h->cur ^ 1]);
  const size_t n = (size_t)h->N;
  const float* src[4] = {y, vx, vy, vz};
  for (int k = 0; k < 4; ++k)
    DSMC_CUDA(cudaMemcpyAsync(tmp + k * n, src[k], n * sizeof(float), cudaMemcpyDefault, st),
              "load state");
  DSMC_CUDA(launch_pack(tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, h->P[h->cur], (int)h->N, st),
            "pack");
  if (smax)
    DSMC_CUDA(cudaMemcpyAsync(h->smax[h->scur], smax, (size_t)h->n_cells * sizeof(float),
                              cudaMemcpyDefault, st),
              "load smax");
  h->step = step;
  std::vector<int> host;
  s = set_uniform_offsets(h, host);
  if (s != DSMC_OK) return s;
  s = run_index(h);
  if (s != DSMC_OK) return s;
  return dsmc_sync(h);  // also keeps `host` alive until its copy has run
}

dsmc_status dsmc_get_info(dsmc_handle h, dsmc_info* info) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!info) return fail(DSMC_E_INVAL, "info: NULL");
  info->n_particles = h->N;
  info->n_cells = h->n_cells;
  info->ppc = h->ppc;
  info->step = h->step;
  info->n_samples = h->n_samples;
  info->Kn = h->Kn;
  info->omega = h->omega;
  info->body_force = h->F;
  info->nsigma = h->p.nsig;
  info->dt = h->p.dt;
  info->dt_f = h->p.dt_f;
  info->F_f = h->p.F_f;
  info->coef = h->p.coef;
  info->cvhs = h->p.cvhs;
  info->vexp = h->p.vexp;
  info->vinv = h->p.vinv;
  info->lncv = h->p.lncv;
  info->smax0 = h->p.smax0;
  info->device_bytes = h->L.total;
  info->sort_warps = h->L.plan.n_warps;
  info->sort_span = h->L.plan.span;
  info->cells_per_span = h->L.cps;
  info->n_spans = h->L.n_spans;
  return DSMC_OK;
}

int dsmc_kernel_count(void) { return K_NUM; }

const char* dsmc_kernel_name(int k) { return (k >= 0 && k < K_NUM) ? kKernelNames[k] : ""; }

dsmc_status dsmc_kernel_times(dsmc_handle h, double* total_ms, long long* launches) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  s = collect_times(h);
  if (s != DSMC_OK) return s;
  for (int k = 0; k < K_NUM; ++k) {
    if (total_ms) total_ms[k] = h->ktime[k];
    if (launches) launches[k] = h->kcount[k];
  }
  return DSMC_OK;
}

dsmc_status dsmc_reset_kernel_times(dsmc_handle h) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  s = collect_times(h);
  for (int k = 0; k < K_NUM; ++k) {
    h->ktime[k] = 0.0;
    h->kcount[k] = 0;
  }
  return s;
}

dsmc_status dsmc_destroy(dsmc_handle h) {
  if (!h) return DSMC_OK;
  DeviceGuard guard(h->device);
  cudaStreamSynchronize(h->stream());
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  if (h->owns && h->ws) cudaFree(h->ws);
  delete h;
  return DSMC_OK;
}

const char* dsmc_last_error(void) { return g_last_error.c_str(); }

const char* dsmc_status_string(dsmc_status s) {
  switch (s) {
    case DSMC_OK: return "ok";
    case DSMC_E_INVAL: return "invalid argument";
    case DSMC_E_NOMEM: return "out of memory";
    case DSMC_E_CUDA: return "CUDA error";
    case DSMC_E_DEVICE_LIMIT: return "device limit reached";
    case DSMC_E_STATE: return "invalid state";
  }
  return "unknown status";
}

}  // extern "C"
