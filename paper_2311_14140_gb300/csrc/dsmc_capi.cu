// dsmc_capi.cu -- host side of the C ABI declared in include/dsmc.h: argument checks,
// the derived parameters of the method, the device memory layout of a run (one or
// more independent instances), the order of kernel launches within a step, the span
// partition of the step passes and its tuner, CUDA-graph replay, synchronisation,
// the device error word and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
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

constexpr int kDefaultSpanParticles = 2048;
constexpr int kMinSpanParticles = 1024;
constexpr int kMaxSpanParticles = 1 << 24;
constexpr int kMaxInstances = 65535;  // grid y of the per-instance prefix pass
constexpr int kGraphSteps = 16;       // steps per replay of the captured graph (even)

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Spans of the step passes: consecutive cells holding about `target` particles at
// the initial density, at most kMaxSpans spans and kMaxCellsPerSpan cells per span.
// Only the work split depends on the spans: collision groups, random-number counters
// and the sort order do not, so every partition gives the same results.
void make_spans(int n_cells, int ppc, int target, int* cps, int* n_spans) {
  const long long N = (long long)n_cells * ppc;
  long long t = (N + kMaxSpans - 1) / kMaxSpans;
  if (t < target) t = target;
  long long c = (t + ppc - 1) / ppc;
  if (c < (n_cells + kMaxSpans - 1) / kMaxSpans) c = (n_cells + kMaxSpans - 1) / kMaxSpans;
  if (c > kMaxCellsPerSpan) c = kMaxCellsPerSpan;
  if (c > n_cells) c = n_cells;
  if (c < 1) c = 1;
  *cps = (int)c;
  *n_spans = (int)((n_cells + c - 1) / c);
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
  if (o->span_particles != 0 &&
      (o->span_particles < kMinSpanParticles || o->span_particles > kMaxSpanParticles))
    return fail(DSMC_E_INVAL, "options: span_particles must be 0 or 1024..2^24");
  if (o->graph && o->stream == nullptr)
    return fail(DSMC_E_INVAL, "options: graph replay needs a stream other than the legacy default");
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

// One instance of a run: its definition, derived parameters, place in the
// concatenated device arrays, span partition and counters.
struct Inst {
  double omega = 0.5, Kn = 1.0, wall_T = 273.0, F = 0.0;
  int n_cells = 0, ppc = 0;
  long long N = 0;
  uint64_t seed = 0;
  Params p{};
  int max_spans = 0;  // rows of the sort matrix reserved (finest partition)
  int part_base = 0, cell_base = 0, off_base = 0;
  long long hist_base = 0;
  int cps = 0, n_spans = 0, span_base = 0;  // partition in use
  long long step = 0, n_samples = 0;
};

// Byte offsets of the arrays in the device workspace.
struct Layout {
  long long n_slots = 0, hist_ints = 0;
  int cells = 0, offs = 0, max_spans = 0, max_cells = 0;
  size_t st, hist, count, offset, smax, ncand, nacc, acc, tab, span_inst, err, total;
};

// Concatenates the instances: slots (each instance padded to 64), cells, cell
// offsets (n_cells + 1 each) and sort-matrix rows, and sizes the workspace.
Layout place(std::vector<Inst>& v) {
  Layout L{};
  for (size_t i = 0; i < v.size(); ++i) {
    Inst& x = v[i];
    int cps, ns;
    make_spans(x.n_cells, x.ppc, kMinSpanParticles, &cps, &ns);
    x.max_spans = ns;
    x.part_base = (int)L.n_slots;
    x.cell_base = L.cells;
    x.off_base = L.offs;
    x.hist_base = L.hist_ints;
    L.n_slots += (x.N + 63) & ~63LL;
    L.cells += x.n_cells;
    L.offs += x.n_cells + 1;
    L.hist_ints += (long long)ns * x.n_cells;
    L.max_spans += ns;
    L.max_cells = std::max(L.max_cells, x.n_cells);
  }
  size_t o = 0;
  L.st = o;
  o += align256(2 * (size_t)L.n_slots * sizeof(float4));
  L.hist = o;
  o += align256((size_t)L.hist_ints * sizeof(int));
  L.count = o;
  o += align256((size_t)L.cells * sizeof(int));
  L.offset = o;  // two arrays: current and next
  o += align256(2 * (size_t)L.offs * sizeof(int));
  L.smax = o;
  o += align256(2 * (size_t)L.cells * sizeof(float));
  L.ncand = o;
  o += align256((size_t)L.cells * sizeof(unsigned long long));
  L.nacc = o;
  o += align256((size_t)L.cells * sizeof(unsigned long long));
  L.acc = o;
  o += align256((size_t)L.cells * kNMom * sizeof(double));
  L.tab = o;
  o += align256(v.size() * sizeof(InstParams));
  L.span_inst = o;
  o += align256((size_t)L.max_spans * sizeof(int));
  L.err = o;
  o += 256;
  L.total = o;
  return L;
}

// Checks one instance definition; the message names the instance in a batch.
dsmc_status check_instance(const dsmc_instance& d, int index, int n_inst) {
  const std::string at = n_inst > 1 ? "instance " + std::to_string(index) + ": " : "";
  if (!(d.gas.mass > 0.0) || !(d.gas.d_ref > 0.0) || !(d.gas.T_ref > 0.0))
    return fail(DSMC_E_INVAL, at + "gas: mass, d_ref and T_ref must be > 0");
  if (!(d.gas.omega >= 0.5 && d.gas.omega <= 1.0))
    return fail(DSMC_E_INVAL, at + "gas: omega must lie in [0.5, 1]");
  if (!(d.Kn > 0.0)) return fail(DSMC_E_INVAL, at + "Kn must be > 0 (or +inf)");
  if (!(d.wall_T > 0.0) || !std::isfinite(d.wall_T))
    return fail(DSMC_E_INVAL, at + "wall_T must be > 0");
  if (!std::isfinite(d.body_force)) return fail(DSMC_E_INVAL, at + "body_force must be finite");
  if (d.n_cells < 1 || d.ppc < 1) return fail(DSMC_E_INVAL, at + "n_cells and ppc must be >= 1");
  if ((long long)d.n_cells * d.ppc > kMaxParticles)
    return fail(DSMC_E_INVAL, at + "n_cells * ppc must be <= 2^31 - 2^24");
  if (d.n_cells > kMaxStepCells) return fail(DSMC_E_INVAL, at + "n_cells must be <= 16384");
  return DSMC_OK;
}

int collision_mode(double omega) { return omega == 0.5 ? 0 : (omega == 1.0 ? 2 : 1); }

}  // namespace

void dsmc::set_last_error(const std::string& msg) { g_last_error = msg; }

struct dsmc_sim {
  int device = 0;
  dsmc_options opt{};
  std::vector<Inst> inst;
  long long gstep = 0;  // steps this handle has launched
  int span_target = kDefaultSpanParticles;
  int spans = 0, max_cps = 0;  // partition in use
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
  InstParams* tab_dev = nullptr;
  int* span_inst_dev = nullptr;
  std::vector<InstParams> tab;
  std::vector<int> span_inst;
  bool tab_dirty = true, spans_dirty = true;
  // CUDA graph of kGraphSteps consecutive steps, replayed by dsmc_step when
  // options.graph is set.  Its kernels read the global step from gstep_dev, which the
  // last prefix kernel of each step advances.
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false, capturing = false;
  int graph_parity = 0;  // buffer parities (cur, ocur, scur) the graph starts from
  long long* gstep_dev = nullptr;
  dsmc_status latched = DSMC_OK;
  std::vector<cudaEvent_t> events;
  std::vector<int> event_kernel;
  size_t events_used = 0;
  double ktime[K_NUM] = {};
  long long kcount[K_NUM] = {};

  cudaStream_t stream() const { return (cudaStream_t)opt.stream; }
  int n_inst() const { return (int)inst.size(); }
  int cap() const { return opt.group_size + opt.group_size / 2 - 1; }
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

// The step passes must fit one CTA's shared memory with this partition and group size.
bool step_fits(int max_cells, int max_cps, int G) {
  return step_smem_layout(max_cells, max_cps, G + G / 2 - 1).total <= kStepSmemMax;
}

// The largest cells-per-span any instance would use with `target` particles per span.
int partition_max_cps(const dsmc_sim* h, int target) {
  int m = 1;
  for (const Inst& x : h->inst) {
    int cps, ns;
    make_spans(x.n_cells, x.ppc, target, &cps, &ns);
    m = std::max(m, cps);
  }
  return m;
}

// Assigns spans with `target` particles per span to every instance.
void set_partition(dsmc_sim* h, int target) {
  h->span_target = target;
  h->span_inst.clear();
  int base = 0, m = 1;
  for (int i = 0; i < h->n_inst(); ++i) {
    Inst& x = h->inst[i];
    make_spans(x.n_cells, x.ppc, target, &x.cps, &x.n_spans);
    x.span_base = base;
    base += x.n_spans;
    m = std::max(m, x.cps);
    h->span_inst.insert(h->span_inst.end(), (size_t)x.n_spans, i);
  }
  h->spans = base;
  h->max_cps = m;
  h->tab_dirty = h->spans_dirty = true;
  h->graph_valid = false;
}

InstParams instance_params(const dsmc_sim* h, const Inst& x) {
  InstParams a{};
  a.n_cells = x.n_cells;
  a.cell_base = x.cell_base;
  a.off_base = x.off_base;
  a.span_base = x.span_base;
  a.n_spans = x.n_spans;
  a.cps = x.cps;
  a.part_base = x.part_base;
  a.n_part = (int)x.N;
  a.hist_base = x.hist_base;
  a.G = h->opt.group_size;
  a.cap = h->cap();
  a.ncf = (float)x.n_cells;
  a.dt = x.p.dt_f;
  a.F = x.p.F_f;
  a.coef = x.p.coef;
  a.cvhs = x.p.cvhs;
  a.vexp = x.p.vexp;
  a.vinv = x.p.vinv;
  a.lncv = x.p.lncv;
  a.k0 = (uint32_t)(x.seed & 0xffffffffu);
  a.k1 = (uint32_t)(x.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    a.keys.k0[r] = a.k0 + (uint32_t)r * 0x9E3779B9u;
    a.keys.k1[r] = a.k1 + (uint32_t)r * 0xBB67AE85u;
  }
  a.step0 = h->gstep - x.step;  // the instance's step = global step - step0
  a.sample_start = h->opt.sample_start;
  a.collide = (h->opt.collisions != 0 && x.p.nsig > 0.0) ? 1 : 0;
  a.mode = collision_mode(x.omega);
  return a;
}

// Rebuilds the instance table after a change and, for a batch, enqueues its copy to
// the device (ordered on the stream before the next launch).  The copies read
// pageable host memory, which CUDA stages before the call returns.
dsmc_status upload_tables(dsmc_sim* h) {
  if (h->tab_dirty) {
    h->tab.resize(h->inst.size());
    for (int i = 0; i < h->n_inst(); ++i) h->tab[i] = instance_params(h, h->inst[i]);
    if (h->n_inst() > 1)
      DSMC_CUDA(cudaMemcpyAsync(h->tab_dev, h->tab.data(), h->tab.size() * sizeof(InstParams),
                                cudaMemcpyHostToDevice, h->stream()),
                "instance table");
    h->tab_dirty = false;
    if (h->n_inst() == 1) h->graph_valid = false;  // the captured launches hold tab[0]
  }
  if (h->spans_dirty) {
    if (h->n_inst() > 1)
      DSMC_CUDA(cudaMemcpyAsync(h->span_inst_dev, h->span_inst.data(),
                                h->span_inst.size() * sizeof(int), cudaMemcpyHostToDevice,
                                h->stream()),
                "span table");
    h->spans_dirty = false;
  }
  return DSMC_OK;
}

StepLaunch step_launch(const dsmc_sim* h, bool count_only) {
  StepLaunch L{};
  L.n_inst = h->n_inst();
  L.tab = h->tab_dev;
  L.span_inst = h->span_inst_dev;
  L.n_spans_total = h->spans;
  L.max_cells = h->L.max_cells;
  L.max_cps = h->max_cps;
  L.max_cap = h->cap();
  L.gstep = h->gstep;
  L.gstep_dev = h->capturing ? h->gstep_dev : nullptr;
  L.count_only = count_only ? 1 : 0;
  return L;
}

// The launches of one pass over the records: collide + sample + move + count (or
// count only), prefix over spans, cell offsets, stable scatter into the other buffer.
dsmc_status run_pass(dsmc_sim* h, bool count_only) {
  cudaStream_t s = h->stream();
  const StepLaunch SL = step_launch(h, count_only);
  const InstParams& one = h->tab[0];
  int* off_cur = h->off[h->ocur];
  int* off_new = h->off[h->ocur ^ 1];
  DSMC_CUDA(timed(h, count_only ? K_INDEX_COUNT : K_COLLIDE_MOVE, [&] {
              return launch_collide_move(h->P[h->cur], off_cur, h->smax[h->scur],
                                         h->smax[h->scur ^ 1], h->ncand, h->nacc, h->acc,
                                         h->hist, one, SL, h->err, s);
            }),
            count_only ? "index_count" : "collide_move");
  if (!count_only) h->scur ^= 1;
  DSMC_CUDA(timed(h, K_SCAN, [&] { return launch_scan_spans(h->hist, h->count, one, SL, s); }),
            "scan_hist");
  DSMC_CUDA(timed(h, K_OFFSETS,
                  [&] { return launch_offsets_cells(h->count, off_new, one, SL, s); }),
            "cell_offsets");
  DSMC_CUDA(timed(h, count_only ? K_INDEX_SCATTER : K_SCATTER_SPANS, [&] {
              return launch_scatter_spans(h->P[h->cur], h->P[h->cur ^ 1], off_cur, off_new,
                                          h->hist, one, SL, h->err, s);
            }),
            count_only ? "index_scatter" : "scatter_spans");
  h->cur ^= 1;
  h->ocur ^= 1;
  return DSMC_OK;
}

// Sort into cells without moving (creation, state load).  The current offsets must
// describe slot ranges per cell span; records may be in any order within them.
dsmc_status run_index(dsmc_sim* h) {
  dsmc_status s = upload_tables(h);
  if (s != DSMC_OK) return s;
  return run_pass(h, /*count_only=*/true);
}

// Advances every instance's counters for one step.
void count_step(dsmc_sim* h) {
  h->gstep += 1;
  for (Inst& x : h->inst) {
    x.step += 1;
    if (x.step >= h->opt.sample_start) x.n_samples += 1;
  }
}

// Slot ranges for a sort of instance i's records in arbitrary order: cell span k
// covers [off[k cps], off[(k+1) cps]) with off[c] = part_base + floor(c N / n_cells).
dsmc_status set_uniform_offsets(dsmc_sim* h, int i, std::vector<int>& host) {
  const Inst& x = h->inst[i];
  host.resize((size_t)x.n_cells + 1);
  for (int c = 0; c <= x.n_cells; ++c)
    host[c] = x.part_base + (int)((long long)c * x.N / x.n_cells);
  DSMC_CUDA(cudaMemcpyAsync(h->off[h->ocur] + x.off_base, host.data(), host.size() * sizeof(int),
                            cudaMemcpyHostToDevice, h->stream()),
            "offsets");
  return DSMC_OK;
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

dsmc_status check_index(dsmc_sim* h, int i) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (i < 0 || i >= h->n_inst()) return fail(DSMC_E_INVAL, "instance index out of range");
  return DSMC_OK;
}

void drop_graph(dsmc_sim* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_valid = false;
}

int parity(const dsmc_sim* h) { return h->cur | (h->ocur << 1) | (h->scur << 2); }

// Captures the launches of kGraphSteps steps into a graph.  Capture only records:
// the host-side buffer parities are restored afterwards (an even step count returns
// them to the same values after each replay).
dsmc_status capture_graph(dsmc_sim* h) {
  cudaStream_t s = h->stream();
  const int c0 = h->cur, o0 = h->ocur, s0 = h->scur;
  cudaGraph_t g = nullptr;
  DSMC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  h->capturing = true;
  dsmc_status st = DSMC_OK;
  for (int k = 0; k < kGraphSteps && st == DSMC_OK; ++k) st = run_pass(h, false);
  h->capturing = false;
  const cudaError_t e_end = cudaStreamEndCapture(s, &g);
  h->cur = c0;
  h->ocur = o0;
  h->scur = s0;
  if (st != DSMC_OK || e_end != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st != DSMC_OK ? st : cuda_fail(e_end, "stream capture");
  }
  drop_graph(h);
  const cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  h->graph_parity = parity(h);
  h->graph_valid = true;
  return DSMC_OK;
}

dsmc_status step_once(dsmc_sim* h) {
  count_step(h);
  dsmc_status s = upload_tables(h);
  if (s != DSMC_OK) return s;
  return run_pass(h, false);
}

dsmc_status step_n(dsmc_sim* h, int n_steps) {
  dsmc_status s;
  int it = 0;
  if (h->opt.graph && !h->opt.profile) {
    while (n_steps - it >= kGraphSteps) {
      if ((s = upload_tables(h)) != DSMC_OK) return s;
      if (!h->graph_valid || h->graph_parity != parity(h))
        if ((s = capture_graph(h)) != DSMC_OK) return s;
      // The graph's first step runs at global step gstep + 1.
      DSMC_CUDA(launch_set_counter(h->gstep_dev, h->gstep + 1, h->stream()), "set step");
      DSMC_CUDA(cudaGraphLaunch(h->graph, h->stream()), "graph launch");
      for (int k = 0; k < kGraphSteps; ++k) count_step(h);
      it += kGraphSteps;
    }
  }
  for (; it < n_steps; ++it)
    if ((s = step_once(h)) != DSMC_OK) return s;
  return DSMC_OK;
}

dsmc_status create_run(const dsmc_instance* defs, int n_inst, const dsmc_options* opt_in,
                       void* workspace, size_t workspace_bytes, dsmc_handle* out) {
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  *out = nullptr;
  if (!defs) return fail(DSMC_E_INVAL, "instances: NULL");
  if (n_inst < 1 || n_inst > kMaxInstances)
    return fail(DSMC_E_INVAL, "n_instances must be 1..65535");
  dsmc_options opt;
  dsmc_default_options(&opt);
  if (opt_in) opt = *opt_in;
  dsmc_status st = check_options(&opt);
  if (st != DSMC_OK) return st;
  std::vector<Inst> v((size_t)n_inst);
  long long slots = 0;
  for (int i = 0; i < n_inst; ++i) {
    const dsmc_instance& d = defs[i];
    if ((st = check_instance(d, i, n_inst)) != DSMC_OK) return st;
    Inst& x = v[i];
    x.omega = d.gas.omega;
    x.Kn = d.Kn;
    x.wall_T = d.wall_T;
    x.F = d.body_force;
    x.n_cells = d.n_cells;
    x.ppc = d.ppc;
    x.N = (long long)d.n_cells * d.ppc;
    x.seed = d.seed;
    if (!derive_params(x.omega, x.Kn, x.F, x.ppc, opt, &x.p))
      return fail(DSMC_E_INVAL, (n_inst > 1 ? "instance " + std::to_string(i) + ": " : "") +
                                    "time step undefined: set options.dt for infinite Kn");
    slots += (x.N + 63) & ~63LL;
  }
  if (slots > kMaxParticles)
    return fail(DSMC_E_INVAL, "the instances' particles (each padded to 64) must total <= 2^31 - 2^24");

  dsmc_sim* h = new (std::nothrow) dsmc_sim();
  if (!h) return fail(DSMC_E_NOMEM, "host allocation failed");
  h->inst = std::move(v);
  h->opt = opt;
  h->L = place(h->inst);
  set_partition(h, opt.span_particles ? opt.span_particles : kDefaultSpanParticles);
  if (!step_fits(h->L.max_cells, h->max_cps, opt.group_size)) {
    delete h;
    return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  }
  cudaError_t ce = cudaGetDevice(&h->device);
  if (ce != cudaSuccess) {
    delete h;
    return cuda_fail(ce, "cudaGetDevice");
  }
  if (workspace) {
    if (workspace_bytes < h->L.total || ((uintptr_t)workspace & 255u)) {
      delete h;
      return fail(DSMC_E_NOMEM, "workspace smaller than the workspace size or not 256-byte aligned");
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
  const Layout& L = h->L;
  char* b = (char*)h->ws;
  h->P[0] = (float4*)(b + L.st);
  h->P[1] = h->P[0] + L.n_slots;
  h->hist = (int*)(b + L.hist);
  h->count = (int*)(b + L.count);
  h->off[0] = (int*)(b + L.offset);
  h->off[1] = h->off[0] + L.offs;
  h->smax[0] = (float*)(b + L.smax);
  h->smax[1] = h->smax[0] + L.cells;
  h->ncand = (unsigned long long*)(b + L.ncand);
  h->nacc = (unsigned long long*)(b + L.nacc);
  h->acc = (double*)(b + L.acc);
  h->tab_dev = (InstParams*)(b + L.tab);
  h->span_inst_dev = (int*)(b + L.span_inst);
  h->err = (int*)(b + L.err);
  h->gstep_dev = (long long*)(b + L.err + 8);

  auto bail = [&](dsmc_status s) {
    dsmc_destroy(h);
    return s;
  };
  cudaStream_t s = h->stream();
  ce = set_step_smem_limits(kStepSmemMax, kStepSmemMax);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaFuncSetAttribute"));
  const size_t nc = (size_t)L.cells;
  if ((ce = cudaMemsetAsync(h->acc, 0, nc * kNMom * sizeof(double), s)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->ncand, 0, nc * 8, s)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->nacc, 0, nc * 8, s)) != cudaSuccess ||
      (ce = cudaMemsetAsync(h->err, 0, sizeof(int), s)) != cudaSuccess)
    return bail(cuda_fail(ce, "cudaMemsetAsync"));
  // Initial (sigma g)_max per cell and slot ranges of whole cells (particle p of an
  // instance is drawn in its cell p / ppc).
  std::vector<float> smax0(nc);
  std::vector<int> off0((size_t)L.offs);
  for (const Inst& x : h->inst) {
    std::fill(smax0.begin() + x.cell_base, smax0.begin() + x.cell_base + x.n_cells, x.p.smax0);
    for (int c = 0; c <= x.n_cells; ++c) off0[(size_t)x.off_base + c] = x.part_base + c * x.ppc;
  }
  ce = cudaMemcpyAsync(h->smax[0], smax0.data(), nc * sizeof(float), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(h->off[h->ocur], off0.data(), off0.size() * sizeof(int),
                         cudaMemcpyHostToDevice, s);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaMemcpyAsync"));
  for (const Inst& x : h->inst) {
    ce = timed(h, K_INIT, [&] {
      return launch_init(h->P[0] + x.part_base, (int)x.N, x.ppc, (float)x.n_cells,
                         (uint32_t)(x.seed & 0xffffffffu), (uint32_t)(x.seed >> 32), h->err, s);
    });
    if (ce != cudaSuccess) return bail(cuda_fail(ce, "init"));
  }
  st = run_index(h);
  if (st != DSMC_OK) return bail(st);
  ce = cudaStreamSynchronize(s);  // the host buffers must outlive their copies
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "stream sync"));
  st = collect_times(h);
  if (st != DSMC_OK) return bail(st);
  st = read_error_word(h);
  if (st != DSMC_OK) return bail(st);
  *out = h;
  return DSMC_OK;
}

dsmc_instance make_instance(const dsmc_gas* gas, double Kn, double wall_T, double body_force,
                            int n_cells, int ppc, uint64_t seed) {
  dsmc_instance d{};
  if (gas) d.gas = *gas;
  d.Kn = Kn;
  d.wall_T = wall_T;
  d.body_force = body_force;
  d.n_cells = n_cells;
  d.ppc = ppc;
  d.seed = seed;
  return d;
}

}  // namespace

extern "C" {

dsmc_status dsmc_default_options(dsmc_options* opt) {
  if (!opt) return fail(DSMC_E_INVAL, "options: NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->dt_factor = 0.2;
  opt->dt = 0.0;
  opt->sample_start = 0;
  opt->group_size = 256;
  opt->collisions = 1;
  opt->profile = 0;
  opt->span_particles = 0;
  opt->graph = 0;
  opt->stream = nullptr;
  return DSMC_OK;
}

size_t dsmc_batch_workspace_bytes(const dsmc_instance* inst, int n_inst) {
  if (!inst || n_inst < 1 || n_inst > kMaxInstances) return 0;
  std::vector<Inst> v((size_t)n_inst);
  for (int i = 0; i < n_inst; ++i) {
    if (inst[i].n_cells < 1 || inst[i].ppc < 1 || inst[i].n_cells > kMaxStepCells) return 0;
    v[i].n_cells = inst[i].n_cells;
    v[i].ppc = inst[i].ppc;
    v[i].N = (long long)inst[i].n_cells * inst[i].ppc;
  }
  return place(v).total;
}

size_t dsmc_workspace_bytes(int n_cells, int ppc) {
  dsmc_instance d{};
  d.n_cells = n_cells;
  d.ppc = ppc;
  return dsmc_batch_workspace_bytes(&d, 1);
}

dsmc_status dsmc_create_in(const dsmc_gas* gas, double Kn, double wall_T, double body_force,
                           int n_cells, int ppc, uint64_t seed, const dsmc_options* opt_in,
                           void* workspace, size_t workspace_bytes, dsmc_handle* out) {
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  *out = nullptr;
  if (!gas) return fail(DSMC_E_INVAL, "gas: NULL");
  const dsmc_instance d = make_instance(gas, Kn, wall_T, body_force, n_cells, ppc, seed);
  return create_run(&d, 1, opt_in, workspace, workspace_bytes, out);
}

dsmc_status dsmc_create(const dsmc_gas* gas, double Kn, double wall_T, double body_force,
                        int n_cells, int ppc, uint64_t seed, dsmc_handle* out) {
  return dsmc_create_in(gas, Kn, wall_T, body_force, n_cells, ppc, seed, nullptr, nullptr, 0,
                        out);
}

dsmc_status dsmc_create_batch(const dsmc_instance* inst, int n_inst, const dsmc_options* opt,
                              void* workspace, size_t workspace_bytes, dsmc_handle* out) {
  return create_run(inst, n_inst, opt, workspace, workspace_bytes, out);
}

int dsmc_batch_size(dsmc_handle h) { return h ? h->n_inst() : 0; }

dsmc_status dsmc_set_options(dsmc_handle h, const dsmc_options* opt) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  s = check_options(opt);
  if (s != DSMC_OK) return s;
  std::vector<Params> ps(h->inst.size());
  for (int i = 0; i < h->n_inst(); ++i) {
    const Inst& x = h->inst[i];
    if (!derive_params(x.omega, x.Kn, x.F, x.ppc, *opt, &ps[i]))
      return fail(DSMC_E_INVAL, "time step undefined: set options.dt for infinite Kn");
  }
  // span_particles = 0 keeps the partition in use (default or tuned).
  const int target_use = opt->span_particles ? opt->span_particles : h->span_target;
  if (!step_fits(h->L.max_cells, partition_max_cps(h, target_use), opt->group_size))
    return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  if (h->events_used) {
    s = collect_times(h);
    if (s != DSMC_OK) return s;
  }
  h->opt = *opt;
  for (int i = 0; i < h->n_inst(); ++i) h->inst[i].p = ps[i];
  if (target_use != h->span_target) set_partition(h, target_use);
  h->tab_dirty = true;
  drop_graph(h);  // launch shapes or the stream may have changed
  return DSMC_OK;
}

dsmc_status dsmc_step(dsmc_handle h, int n_steps) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (n_steps < 0) return fail(DSMC_E_INVAL, "n_steps must be >= 0");
  if (h->latched != DSMC_OK) return fail(h->latched, "an earlier step reached a device limit");
  DeviceGuard guard(h->device);
  s = step_n(h, n_steps);
  if (s != DSMC_OK) return s;
  if (h->opt.profile) return collect_times(h);
  return DSMC_OK;
}

dsmc_status dsmc_autotune(dsmc_handle h, int steps_per_trial, int* best_span_particles,
                          double* best_ms_per_step) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (steps_per_trial < 1) return fail(DSMC_E_INVAL, "steps_per_trial must be >= 1");
  if (h->latched != DSMC_OK) return fail(h->latched, "an earlier step reached a device limit");
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  cudaEvent_t e0, e1;
  DSMC_CUDA(cudaEventCreate(&e0), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(DSMC_E_CUDA, "event");
  }
  int best = h->span_target;
  double best_ms = -1.0;
  int last_cps = -1;
  dsmc_status r = DSMC_OK;
  for (int target = kMinSpanParticles; target <= (1 << 17) && r == DSMC_OK; target *= 2) {
    const int mc = partition_max_cps(h, target);
    if (!step_fits(h->L.max_cells, mc, h->opt.group_size)) break;
    // Skip targets that give the same partition as the last one.
    int sig = 0;
    for (const Inst& x : h->inst) {
      int cps, ns;
      make_spans(x.n_cells, x.ppc, target, &cps, &ns);
      sig = sig * 31 + cps;
    }
    if (sig == last_cps) continue;
    last_cps = sig;
    set_partition(h, target);
    // one untimed step with the new partition, then the timed trial
    if ((r = step_n(h, 1)) != DSMC_OK) break;
    if (cudaEventRecord(e0, st) != cudaSuccess) { r = fail(DSMC_E_CUDA, "event record"); break; }
    if ((r = step_n(h, steps_per_trial)) != DSMC_OK) break;
    if (cudaEventRecord(e1, st) != cudaSuccess) { r = fail(DSMC_E_CUDA, "event record"); break; }
    if (cudaEventSynchronize(e1) != cudaSuccess) { r = fail(DSMC_E_CUDA, "event sync"); break; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / steps_per_trial;
    if (best_ms < 0.0 || per < best_ms) {
      best_ms = per;
      best = target;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != DSMC_OK) return r;
  set_partition(h, best);
  h->opt.span_particles = best;
  if (best_span_particles) *best_span_particles = best;
  if (best_ms_per_step) *best_ms_per_step = best_ms;
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

dsmc_status dsmc_sample_moments_of(dsmc_handle h, int i, double* out, long long* n_samples) {
  dsmc_status s = check_index(h, i);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  const Inst& x = h->inst[i];
  DSMC_CUDA(cudaMemcpyAsync(out, h->acc + (size_t)x.cell_base * kNMom,
                            (size_t)x.n_cells * kNMom * sizeof(double), cudaMemcpyDefault,
                            h->stream()),
            "copy moments");
  if (n_samples) *n_samples = x.n_samples;
  return dsmc_sync(h);
}

dsmc_status dsmc_sample_moments(dsmc_handle h, double* out, long long* n_samples) {
  return dsmc_sample_moments_of(h, 0, out, n_samples);
}

dsmc_status dsmc_sample_moments_all(dsmc_handle h, double* out, long long* n_samples) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  DSMC_CUDA(cudaMemcpyAsync(out, h->acc, (size_t)h->L.cells * kNMom * sizeof(double),
                            cudaMemcpyDefault, h->stream()),
            "copy moments");
  if (n_samples)
    for (int i = 0; i < h->n_inst(); ++i) n_samples[i] = h->inst[i].n_samples;
  return dsmc_sync(h);
}

dsmc_status dsmc_reset_samples_of(dsmc_handle h, int i) {
  dsmc_status s = check_index(h, i);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  Inst& x = h->inst[i];
  const size_t c0 = (size_t)x.cell_base, nc = (size_t)x.n_cells;
  DSMC_CUDA(cudaMemsetAsync(h->acc + c0 * kNMom, 0, nc * kNMom * sizeof(double), st), "reset");
  DSMC_CUDA(cudaMemsetAsync(h->ncand + c0, 0, nc * 8, st), "reset");
  DSMC_CUDA(cudaMemsetAsync(h->nacc + c0, 0, nc * 8, st), "reset");
  x.n_samples = 0;
  return DSMC_OK;
}

dsmc_status dsmc_reset_samples(dsmc_handle h) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  const size_t nc = (size_t)h->L.cells;
  DSMC_CUDA(cudaMemsetAsync(h->acc, 0, nc * kNMom * sizeof(double), st), "reset");
  DSMC_CUDA(cudaMemsetAsync(h->ncand, 0, nc * 8, st), "reset");
  DSMC_CUDA(cudaMemsetAsync(h->nacc, 0, nc * 8, st), "reset");
  for (Inst& x : h->inst) x.n_samples = 0;
  return DSMC_OK;
}

dsmc_status dsmc_copy_state_of(dsmc_handle h, int i, float* y, float* vx, float* vy,
                               float* vz) {
  dsmc_status s = check_index(h, i);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  const Inst& x = h->inst[i];
  // Unpack the records into four arrays in the instance's part of the idle sort
  // buffer, then copy out.
  float* tmp = reinterpret_cast<float*>(h->P[h->cur ^ 1] + x.part_base);
  const size_t n = (size_t)x.N;
  float* arr[4] = {tmp, tmp + n, tmp + 2 * n, tmp + 3 * n};
  DSMC_CUDA(launch_unpack(h->P[h->cur] + x.part_base, arr[0], arr[1], arr[2], arr[3], (int)x.N,
                          st),
            "unpack");
  float* dst[4] = {y, vx, vy, vz};
  for (int k = 0; k < 4; ++k)
    if (dst[k])
      DSMC_CUDA(cudaMemcpyAsync(dst[k], arr[k], n * sizeof(float), cudaMemcpyDefault, st),
                "copy state");
  return dsmc_sync(h);
}

dsmc_status dsmc_copy_state(dsmc_handle h, float* y, float* vx, float* vy, float* vz) {
  return dsmc_copy_state_of(h, 0, y, vx, vy, vz);
}

dsmc_status dsmc_copy_cells_of(dsmc_handle h, int i, int* offset, float* smax,
                               unsigned long long* ncand, unsigned long long* nacc) {
  dsmc_status s = check_index(h, i);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  const Inst& x = h->inst[i];
  const size_t c0 = (size_t)x.cell_base, nc = (size_t)x.n_cells;
  if (offset) {
    // Offsets relative to the instance's first slot (as for a run of its own).
    std::vector<int> host(nc + 1);
    DSMC_CUDA(cudaMemcpyAsync(host.data(), h->off[h->ocur] + x.off_base, (nc + 1) * sizeof(int),
                              cudaMemcpyDeviceToHost, st),
              "copy cells");
    DSMC_CUDA(cudaStreamSynchronize(st), "stream sync");
    for (int& o : host) o -= x.part_base;
    DSMC_CUDA(cudaMemcpyAsync(offset, host.data(), (nc + 1) * sizeof(int), cudaMemcpyDefault, st),
              "copy cells");
    DSMC_CUDA(cudaStreamSynchronize(st), "stream sync");
  }
  if (smax)
    DSMC_CUDA(cudaMemcpyAsync(smax, h->smax[h->scur] + c0, nc * sizeof(float), cudaMemcpyDefault,
                              st),
              "copy cells");
  if (ncand)
    DSMC_CUDA(cudaMemcpyAsync(ncand, h->ncand + c0, nc * 8, cudaMemcpyDefault, st), "copy cells");
  if (nacc)
    DSMC_CUDA(cudaMemcpyAsync(nacc, h->nacc + c0, nc * 8, cudaMemcpyDefault, st), "copy cells");
  return dsmc_sync(h);
}

dsmc_status dsmc_copy_cells(dsmc_handle h, int* offset, float* smax, unsigned long long* ncand,
                            unsigned long long* nacc) {
  return dsmc_copy_cells_of(h, 0, offset, smax, ncand, nacc);
}

dsmc_status dsmc_load_state_of(dsmc_handle h, int i, const float* y, const float* vx,
                               const float* vy, const float* vz, const float* smax,
                               long long step) {
  dsmc_status s = check_index(h, i);
  if (s != DSMC_OK) return s;
  if (!y || !vx || !vy || !vz) return fail(DSMC_E_INVAL, "state arrays must not be NULL");
  if (step < 0) return fail(DSMC_E_INVAL, "step must be >= 0");
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  Inst& x = h->inst[i];
  float* tmp = reinterpret_cast<float*>(h->P[h->cur ^ 1] + x.part_base);
  const size_t n = (size_t)x.N;
  const float* src[4] = {y, vx, vy, vz};
  for (int k = 0; k < 4; ++k)
    DSMC_CUDA(cudaMemcpyAsync(tmp + k * n, src[k], n * sizeof(float), cudaMemcpyDefault, st),
              "load state");
  DSMC_CUDA(launch_pack(tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, h->P[h->cur] + x.part_base,
                        (int)x.N, st),
            "pack");
  if (smax)
    DSMC_CUDA(cudaMemcpyAsync(h->smax[h->scur] + x.cell_base, smax,
                              (size_t)x.n_cells * sizeof(float), cudaMemcpyDefault, st),
              "load smax");
  x.step = step;
  h->tab_dirty = true;
  std::vector<int> host;
  s = set_uniform_offsets(h, i, host);
  if (s != DSMC_OK) return s;
  // The sort pass runs over every instance: for the others, already in cell order,
  // the stable sort leaves records and offsets unchanged.
  s = run_index(h);
  if (s != DSMC_OK) return s;
  return dsmc_sync(h);  // also keeps `host` alive until its copy has run
}

dsmc_status dsmc_load_state(dsmc_handle h, const float* y, const float* vx, const float* vy,
                            const float* vz, const float* smax, long long step) {
  return dsmc_load_state_of(h, 0, y, vx, vy, vz, smax, step);
}

dsmc_status dsmc_get_info_of(dsmc_handle h, int i, dsmc_info* info) {
  dsmc_status s = check_index(h, i);
  if (s != DSMC_OK) return s;
  if (!info) return fail(DSMC_E_INVAL, "info: NULL");
  const Inst& x = h->inst[i];
  info->n_particles = x.N;
  info->n_cells = x.n_cells;
  info->ppc = x.ppc;
  info->step = x.step;
  info->n_samples = x.n_samples;
  info->Kn = x.Kn;
  info->omega = x.omega;
  info->body_force = x.F;
  info->nsigma = x.p.nsig;
  info->dt = x.p.dt;
  info->dt_f = x.p.dt_f;
  info->F_f = x.p.F_f;
  info->coef = x.p.coef;
  info->cvhs = x.p.cvhs;
  info->vexp = x.p.vexp;
  info->vinv = x.p.vinv;
  info->lncv = x.p.lncv;
  info->smax0 = x.p.smax0;
  info->device_bytes = h->L.total;
  info->n_instances = h->n_inst();
  info->span_particles = h->span_target;
  info->cells_per_span = x.cps;
  info->n_spans = x.n_spans;
  info->total_spans = h->spans;
  info->first_slot = x.part_base;
  return DSMC_OK;
}

dsmc_status dsmc_get_info(dsmc_handle h, dsmc_info* info) { return dsmc_get_info_of(h, 0, info); }

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
  drop_graph(h);
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
