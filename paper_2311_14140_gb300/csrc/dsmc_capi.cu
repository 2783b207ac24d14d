// dsmc_capi.cu -- host side of the C ABI declared in include/dsmc.h: argument checks,
// the derived parameters of the method, the device memory layout of a run (one or
// more independent instances), the order of kernel launches within a step, the span
// partition of the step passes and its tuner, CUDA-graph replay, synchronisation,
// the device error word and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
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

constexpr int kDefaultSpanParticles = 4096;
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
  if (o->cta_warps != 0 && o->cta_warps != kAWarps && o->cta_warps != kAWarpsSmall)
    return fail(DSMC_E_INVAL, "options: cta_warps must be 0, 4 or 8");
  if (o->span_rows < 0 || o->span_rows > kMaxSpanRows)
    return fail(DSMC_E_INVAL, "options: span_rows must be 0, 1 or 2");
  if (o->graph && o->stream == nullptr)
    return fail(DSMC_E_INVAL, "options: graph replay needs a stream other than the legacy default");
  if (o->accum != DSMC_ACCUM_FP32 && o->accum != DSMC_ACCUM_FP64)
    return fail(DSMC_E_INVAL, "options: accum must be DSMC_ACCUM_FP32 or DSMC_ACCUM_FP64");
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

// First-fit allocator of index ranges [0, capacity) (slots, cells, cell offsets and
// sort-matrix entries of the instances of a handle).
class Extents {
 public:
  void reset(long long capacity) {
    free_.clear();
    if (capacity > 0) free_[0] = capacity;
  }
  long long alloc(long long n) {
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        const long long s = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[s + n] = len - n;
        return s;
      }
    return -1;
  }
  void release(long long s, long long n) {
    auto it = free_.emplace(s, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<long long, long long> free_;
};

// One instance of a run: its definition, derived parameters, place in the device
// arrays, span partition and counters.
struct Inst {
  bool active = false;
  bool fresh = false;  // added, not yet initialised on the device
  double omega = 0.5, Kn = 1.0, wall_T = 273.0, F = 0.0;
  int n_cells = 0, ppc = 0;
  long long N = 0;
  uint64_t seed = 0;
  Params p{};
  int max_spans = 0;  // rows of the sort matrix reserved (finest partition)
  long long slot_len = 0;
  int part_base = 0, cell_base = 0, off_base = 0;
  long long hist_base = 0;
  int cps = 0, n_spans = 0, span_base = 0;  // partition in use
  long long step = 0, n_samples = 0;
  int open_top = 0;  // y = 1 an open Chapman-Enskog interface
  float u_top = 0.0f, p_top = 0.0f;
};

// Sizes of the device arrays of a handle.
struct Capacity {
  long long slots = 0, hist_ints = 0;
  int cells = 0, offs = 0, spans = 0, inst = 0;
};

// Byte offsets of the arrays in the device workspace.
struct Layout {
  size_t st, hist, count, offset, smax, ncand, nacc, acc, fields, tab, span_inst, chan, err,
      total;
};

long long padded_slots(long long N) { return (N + 63) & ~63LL; }

int reserved_spans(int n_cells, int ppc) {
  int cps, ns;
  make_spans(n_cells, ppc, kMinSpanParticles, &cps, &ns);
  return ns;
}

// Workspace layout for a capacity: two record buffers, the sort matrix, per-cell
// arrays, two instance tables, two span tables (the step's and the admission pass's)
// and the step's span order, the channel sums and the error word.
Layout layout_of(const Capacity& C) {
  Layout L{};
  size_t o = 0;
  L.st = o;
  o += align256(2 * (size_t)C.slots * sizeof(float4));
  L.hist = o;
  o += align256((size_t)C.hist_ints * sizeof(int));
  L.count = o;
  o += align256((size_t)C.cells * sizeof(int));
  L.offset = o;
  o += align256(2 * (size_t)C.offs * sizeof(int));
  L.smax = o;
  o += align256(2 * (size_t)C.cells * sizeof(float));
  L.ncand = o;
  o += align256((size_t)C.cells * sizeof(unsigned long long));
  L.nacc = o;
  o += align256((size_t)C.cells * sizeof(unsigned long long));
  L.acc = o;
  o += align256((size_t)C.cells * kNMom * sizeof(double));
  L.fields = o;
  o += align256((size_t)C.cells * DSMC_NFIELD * sizeof(double));
  L.tab = o;
  o += align256(2 * (size_t)C.inst * sizeof(InstParams));
  L.span_inst = o;
  o += align256(3 * (size_t)C.spans * sizeof(int));
  L.chan = o;
  o += align256(2 * (size_t)C.inst * sizeof(double));
  L.err = o;
  o += 256;
  L.total = o;
  return L;
}

// The capacity that holds exactly these instances, placed one after another.
Capacity capacity_of(const dsmc_instance* d, int n) {
  Capacity C{};
  for (int i = 0; i < n; ++i) {
    const long long N = (long long)d[i].n_cells * d[i].ppc;
    const int rows = reserved_spans(d[i].n_cells, d[i].ppc);
    C.slots += padded_slots(N);
    C.cells += d[i].n_cells;
    C.offs += d[i].n_cells + 1;
    C.hist_ints += (long long)rows * kMaxSpanRows * d[i].n_cells;
    C.spans += rows;
  }
  C.inst = n;
  return C;
}

// The capacity of a pool: every instance of `lim` fits as long as the totals do (up to
// fragmentation of the free ranges).
dsmc_status capacity_of_pool(const dsmc_pool_limits* lim, Capacity* C) {
  if (!lim) return fail(DSMC_E_INVAL, "pool limits: NULL");
  if (lim->max_particles < 1 || lim->max_particles > kMaxParticles || lim->max_cells < 1 ||
      lim->max_instances < 1 || lim->max_instances > kMaxInstances ||
      lim->max_cells_per_instance < 1 || lim->max_cells_per_instance > kMaxStepCells ||
      lim->max_cells_per_instance > lim->max_cells)
    return fail(DSMC_E_INVAL,
                "pool limits: max_particles 1..2^31 - 2^24, max_instances 1..65535, "
                "1 <= max_cells_per_instance <= min(16384, max_cells)");
  Capacity c{};
  c.slots = lim->max_particles;
  c.cells = lim->max_cells;
  c.offs = lim->max_cells + lim->max_instances;
  c.inst = lim->max_instances;
  // An instance of N particles reserves at most N / 1024 + 1 sort-matrix rows.
  const long long rows = lim->max_particles / kMinSpanParticles + lim->max_instances;
  c.spans = (int)std::min<long long>(rows, INT_MAX / 2);
  c.hist_ints = rows * kMaxSpanRows * (long long)lim->max_cells_per_instance;
  *C = c;
  return DSMC_OK;
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
  bool pool = false;  // instances may be added and removed
  dsmc_options opt{};
  std::vector<Inst> inst;  // by id
  std::vector<int> order;  // active ids in table order
  long long gstep = 0;     // steps this handle has launched
  int span_target = kDefaultSpanParticles;
  int cta_warps = kAWarps;  // warps per CTA of the collide/move pass
  int span_rows = 1;        // sort-matrix rows per span
  int spans = 0, max_cps = 1, max_cells = 1, max_spans = 1;  // partition in use
  long long part_total = 0;  // particles of the active instances
  int spans_reserved = 0;
  Capacity C{};
  Layout L{};
  Extents ex_slots, ex_cells, ex_offs, ex_hist;
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
  double* fields = nullptr;  // dsmc_cell_fields_of's output on the device
  InstParams* tab_dev = nullptr;  // [0, C.inst): the step's; [C.inst, 2 C.inst): admission
  int* span_inst_dev = nullptr;   // likewise with C.spans entries each, then the order
  int* span_order_dev = nullptr;  // the span each collide/move CTA takes (C.spans entries)
  double* chan_dev = nullptr;
  std::vector<InstParams> tab, adm_tab;
  std::vector<int> span_inst, adm_span, span_order;
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
  int n_inst() const { return (int)order.size(); }
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

// The step passes must fit one CTA's shared memory with this partition, group size and
// CTA shape.
bool step_fits(int max_cells, int max_cps, int G, int warps = kAWarps, int rows = 1) {
  return step_smem_layout(max_cells, max_cps, G + G / 2 - 1, warps, rows).total <= kStepSmemMax;
}

// The largest cells-per-span any active instance (and `extra`, if given) would use
// with `target` particles per span, and the largest cell count.
void partition_extent(const dsmc_sim* h, int target, const Inst* extra, int* max_cps,
                      int* max_cells) {
  int m = 1, mc = 1;
  auto visit = [&](const Inst& x) {
    int cps, ns;
    make_spans(x.n_cells, x.ppc, target, &cps, &ns);
    m = std::max(m, cps);
    mc = std::max(mc, x.n_cells);
  };
  for (int id : h->order) visit(h->inst[id]);
  if (extra) visit(*extra);
  *max_cps = m;
  *max_cells = mc;
}

// Launch order of the collide/move CTAs: the spans by estimated cost, heaviest first, so
// that the pass does not end on a few slow CTAs started last (the spans at the top wall of
// a run started in cell order ran about twice as long as the rest and left most SMs idle
// for the last sixth of the pass).  A span's cost is taken as its particles times
// (1 + 2.2 h), h the expected wall hits per particle and step: with normal velocity
// components of variance 1/2 (v0 units), a particle at distance d from a wall reaches it
// within dt with probability erfc(d / dt) / 2, evaluated at the span's centre for both
// walls; 2.2 is the measured extra cost of a hit relative to a particle's other work in the
// step (a batch at Kn = 10, about one hit per particle and step, costs 3.2 times one at
// Kn = 0.1).  The order changes which CTA takes a span, never a result.
void set_span_order(dsmc_sim* h) {
  std::vector<std::pair<double, int>> cost;
  cost.reserve((size_t)h->spans);
  for (int t = 0; t < h->n_inst(); ++t) {
    const Inst& x = h->inst[h->order[t]];
    const double dt = x.p.dt;
    for (int k = 0; k < x.n_spans; ++k) {
      const int c0 = k * x.cps, c1 = std::min(c0 + x.cps, x.n_cells);
      const double yc = 0.5 * (c0 + c1) / x.n_cells;
      const double hits = dt > 0.0 ? 0.5 * (std::erfc(yc / dt) + std::erfc((1.0 - yc) / dt)) : 0.0;
      cost.emplace_back(-(double)(c1 - c0) * x.ppc * (1.0 + 2.2 * hits), x.span_base + k);
    }
  }
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
                     return a.first < b.first;
                   });
  h->span_order.resize(cost.size());
  for (size_t i = 0; i < cost.size(); ++i) h->span_order[i] = cost[i].second;
}

// Assigns spans with `target` particles per span to every active instance.
void set_partition(dsmc_sim* h, int target) {
  h->span_target = target;
  h->span_inst.clear();
  int base = 0, m = 1, mc = 1, ms = 1;
  long long np = 0;
  for (int t = 0; t < h->n_inst(); ++t) {
    Inst& x = h->inst[h->order[t]];
    np += x.N;
    make_spans(x.n_cells, x.ppc, target, &x.cps, &x.n_spans);
    x.span_base = base;
    base += x.n_spans;
    m = std::max(m, x.cps);
    mc = std::max(mc, x.n_cells);
    ms = std::max(ms, x.n_spans);
    h->span_inst.insert(h->span_inst.end(), (size_t)x.n_spans, t);
  }
  h->spans = base;
  h->max_cps = m;
  h->max_cells = mc;
  h->max_spans = ms;
  h->part_total = np;
  set_span_order(h);
  h->tab_dirty = h->spans_dirty = true;
  h->graph_valid = false;
}

InstParams instance_params(const dsmc_sim* h, int id, int span_base) {
  const Inst& x = h->inst[id];
  InstParams a{};
  a.n_cells = x.n_cells;
  a.cell_base = x.cell_base;
  a.off_base = x.off_base;
  a.span_base = span_base;
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
  a.lg2cv = (float)std::log2((double)x.p.cvhs);
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
  a.id = id;
  a.smax0 = x.p.smax0;
  a.open_top = x.open_top;
  a.u_top = x.u_top;
  a.p_top = x.p_top;
  return a;
}

// Rebuilds the instance table after a change and, for a batch, enqueues its copy to
// the device (ordered on the stream before the next launch).  The copies read
// pageable host memory, which CUDA stages before the call returns.
dsmc_status upload_tables(dsmc_sim* h) {
  if (h->tab_dirty) {
    h->tab.resize(h->order.size());
    for (int t = 0; t < h->n_inst(); ++t)
      h->tab[t] = instance_params(h, h->order[t], h->inst[h->order[t]].span_base);
    if (!h->tab.empty())
      DSMC_CUDA(cudaMemcpyAsync(h->tab_dev, h->tab.data(), h->tab.size() * sizeof(InstParams),
                                cudaMemcpyHostToDevice, h->stream()),
                "instance table");
    h->tab_dirty = false;
    if (h->n_inst() == 1) h->graph_valid = false;  // the captured launches hold tab[0]
  }
  if (h->spans_dirty) {
    if (!h->span_inst.empty())
      DSMC_CUDA(cudaMemcpyAsync(h->span_inst_dev, h->span_inst.data(),
                                h->span_inst.size() * sizeof(int), cudaMemcpyHostToDevice,
                                h->stream()),
                "span table");
    if (!h->span_order.empty())
      DSMC_CUDA(cudaMemcpyAsync(h->span_order_dev, h->span_order.data(),
                                h->span_order.size() * sizeof(int), cudaMemcpyHostToDevice,
                                h->stream()),
                "span order");
    h->spans_dirty = false;
  }
  return DSMC_OK;
}

StepLaunch step_launch(const dsmc_sim* h, bool count_only) {
  StepLaunch L{};
  L.n_inst = h->n_inst();
  L.tab = h->tab_dev;
  L.span_inst = h->span_inst_dev;
  L.span_order = h->span_order.empty() ? nullptr : h->span_order_dev;
  L.n_spans_total = h->spans;
  L.max_cells = h->max_cells;
  L.max_spans = h->max_spans;
  L.n_part_total = h->part_total;
  L.max_cps = h->max_cps;
  L.max_cap = h->cap();
  L.warps = h->cta_warps;
  L.rows = h->span_rows;
  L.gstep = h->gstep;
  L.gstep_dev = h->capturing ? h->gstep_dev : nullptr;
  L.count_only = count_only ? 1 : 0;
  L.accum = h->opt.accum;
  return L;
}

// The launches of one pass over the records from buffer `src` to buffer src ^ 1:
// collide + sample + move + count (or count only), prefix over spans, cell offsets,
// stable scatter.
dsmc_status launch_pass(dsmc_sim* h, bool count_only, const StepLaunch& SL,
                        const InstParams& one, int src, int osrc) {
  cudaStream_t s = h->stream();
  int* off_cur = h->off[osrc];
  int* off_new = h->off[osrc ^ 1];
  DSMC_CUDA(timed(h, count_only ? K_INDEX_COUNT : K_COLLIDE_MOVE, [&] {
              return launch_collide_move(h->P[src], off_cur, h->smax[h->scur],
                                         h->smax[h->scur ^ 1], h->ncand, h->nacc, h->acc,
                                         h->hist, one, SL, h->err, s);
            }),
            count_only ? "index_count" : "collide_move");
  if (prefix_small_fits(SL)) {  // both prefix passes in one launch (timed as the scan)
    DSMC_CUDA(timed(h, K_SCAN, [&] { return launch_prefix_small(h->hist, off_new, one, SL, s); }),
              "prefix");
  } else {
    DSMC_CUDA(timed(h, K_SCAN, [&] { return launch_scan_spans(h->hist, h->count, one, SL, s); }),
              "scan_hist");
    DSMC_CUDA(timed(h, K_OFFSETS,
                    [&] { return launch_offsets_cells(h->count, off_new, one, SL, s); }),
              "cell_offsets");
  }
  DSMC_CUDA(timed(h, count_only ? K_INDEX_SCATTER : K_SCATTER_SPANS, [&] {
              return launch_scatter_spans(h->P[src], h->P[src ^ 1], off_cur, off_new, h->hist,
                                          one, SL, h->err, s);
            }),
            count_only ? "index_scatter" : "scatter_spans");
  return DSMC_OK;
}

// One pass over every active instance from the current buffers to the other ones.
dsmc_status run_pass(dsmc_sim* h, bool count_only) {
  if (h->n_inst() == 0) return DSMC_OK;
  const StepLaunch SL = step_launch(h, count_only);
  dsmc_status s = launch_pass(h, count_only, SL, h->tab[0], h->cur, h->ocur);
  if (s != DSMC_OK) return s;
  if (!count_only) h->scur ^= 1;
  h->cur ^= 1;
  h->ocur ^= 1;
  return DSMC_OK;
}

// Sort into cells without moving (state load).  The current offsets must describe
// slot ranges per cell span; records may be in any order within them.
dsmc_status run_index(dsmc_sim* h) {
  dsmc_status s = upload_tables(h);
  if (s != DSMC_OK) return s;
  return run_pass(h, /*count_only=*/true);
}

// Device initialisation of the instances added since the last step: particles drawn
// into the idle record buffer with offsets of whole cells, per-cell arrays reset, then
// a sort into cells of those instances alone into the current buffers (the other
// instances are not touched).
dsmc_status admit_fresh(dsmc_sim* h) {
  std::vector<int> ids;
  for (int id : h->order)
    if (h->inst[id].fresh) ids.push_back(id);
  if (ids.empty()) return DSMC_OK;
  cudaStream_t s = h->stream();
  const int idle = h->cur ^ 1, oidle = h->ocur ^ 1;
  h->adm_tab.clear();
  h->adm_span.clear();
  int base = 0, m = 1, mc = 1, ms = 1;
  long long np = 0;
  for (size_t k = 0; k < ids.size(); ++k) {
    const Inst& x = h->inst[ids[k]];
    np += x.N;
    h->adm_tab.push_back(instance_params(h, ids[k], base));
    h->adm_span.insert(h->adm_span.end(), (size_t)x.n_spans, (int)k);
    base += x.n_spans;
    m = std::max(m, x.cps);
    mc = std::max(mc, x.n_cells);
    ms = std::max(ms, x.n_spans);
    DSMC_CUDA(timed(h, K_INIT, [&] {
                return launch_init(h->P[idle] + x.part_base, (int)x.N, x.ppc, (float)x.n_cells,
                                   (uint32_t)(x.seed & 0xffffffffu), (uint32_t)(x.seed >> 32),
                                   h->err, s);
              }),
              "init");
  }
  InstParams* adm_tab_dev = h->tab_dev + h->C.inst;
  int* adm_span_dev = h->span_inst_dev + h->C.spans;
  DSMC_CUDA(cudaMemcpyAsync(adm_tab_dev, h->adm_tab.data(), h->adm_tab.size() * sizeof(InstParams),
                            cudaMemcpyHostToDevice, s),
            "admission table");
  DSMC_CUDA(cudaMemcpyAsync(adm_span_dev, h->adm_span.data(), h->adm_span.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s),
            "admission span table");
  DSMC_CUDA(launch_admit_cells(adm_tab_dev, (int)ids.size(), h->off[oidle], h->smax[h->scur],
                               h->ncand, h->nacc, h->acc, s),
            "admit cells");
  StepLaunch SL{};
  SL.n_inst = (int)ids.size();
  SL.tab = adm_tab_dev;
  SL.span_inst = adm_span_dev;
  SL.n_spans_total = base;
  SL.max_cells = mc;
  SL.max_spans = ms;
  SL.n_part_total = np;
  SL.max_cps = m;
  SL.max_cap = h->cap();
  SL.warps = h->cta_warps;
  SL.rows = h->span_rows;
  SL.gstep = h->gstep;
  SL.gstep_dev = nullptr;
  SL.count_only = 1;
  dsmc_status st = launch_pass(h, true, SL, h->adm_tab[0], idle, oidle);
  if (st != DSMC_OK) return st;
  for (int id : ids) h->inst[id].fresh = false;
  return DSMC_OK;
}

// Advances every active instance's counters for one step.
void count_step(dsmc_sim* h) {
  h->gstep += 1;
  for (int id : h->order) {
    Inst& x = h->inst[id];
    x.step += 1;
    if (x.step >= h->opt.sample_start) x.n_samples += 1;
  }
}

// Slot ranges for a sort of instance id's records in arbitrary order: cell span k
// covers [off[k cps], off[(k+1) cps]) with off[c] = part_base + floor(c N / n_cells).
dsmc_status set_uniform_offsets(dsmc_sim* h, int id, std::vector<int>& host) {
  const Inst& x = h->inst[id];
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
    if (v & kErrInflow) what += " inflow-attempts";
    if (v & kErrMoments) what += " moment-range";
    return fail(DSMC_E_DEVICE_LIMIT, "device limit reached:" + what);
  }
  return DSMC_OK;
}

dsmc_status check_handle(dsmc_sim* h) {
  if (!h) return fail(DSMC_E_INVAL, "handle: NULL");
  return DSMC_OK;
}

dsmc_status check_index(dsmc_sim* h, int id) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (id < 0 || id >= (int)h->inst.size() || !h->inst[id].active)
    return fail(DSMC_E_INVAL, "instance index out of range or not active");
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
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  int it = 0;
  if (h->opt.graph && !h->opt.profile && h->n_inst() > 0) {
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

// Adds an instance (extents, parameters, counters); its device data is set up by the
// next step or synchronising call.  *id gets its id.
dsmc_status add_instance(dsmc_sim* h, const dsmc_instance& d, int index, int n_def, int* id) {
  dsmc_status st = check_instance(d, index, n_def);
  if (st != DSMC_OK) return st;
  Inst x;
  x.omega = d.gas.omega;
  x.Kn = d.Kn;
  x.wall_T = d.wall_T;
  x.F = d.body_force;
  x.n_cells = d.n_cells;
  x.ppc = d.ppc;
  x.N = (long long)d.n_cells * d.ppc;
  x.seed = d.seed;
  if (!derive_params(x.omega, x.Kn, x.F, x.ppc, h->opt, &x.p))
    return fail(DSMC_E_INVAL, (n_def > 1 ? "instance " + std::to_string(index) + ": " : "") +
                                  "time step undefined: set options.dt for infinite Kn");
  int mcps, mcells;
  partition_extent(h, h->span_target, &x, &mcps, &mcells);
  if (!step_fits(mcells, mcps, h->opt.group_size, h->cta_warps, h->span_rows))
    return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  // Find a free id and room in every array.
  int new_id = -1;
  for (int i = 0; i < (int)h->inst.size(); ++i)
    if (!h->inst[i].active) {
      new_id = i;
      break;
    }
  if (new_id < 0 && (int)h->inst.size() >= h->C.inst)
    return fail(DSMC_E_NOMEM, "no room: instance table full");
  x.max_spans = reserved_spans(x.n_cells, x.ppc);
  if (h->spans_reserved + x.max_spans > h->C.spans)
    return fail(DSMC_E_NOMEM, "no room: span table full");
  x.slot_len = padded_slots(x.N);
  const long long ps = h->ex_slots.alloc(x.slot_len);
  const long long cb = ps < 0 ? -1 : h->ex_cells.alloc(x.n_cells);
  const long long ob = cb < 0 ? -1 : h->ex_offs.alloc(x.n_cells + 1);
  const long long hb =
      ob < 0 ? -1 : h->ex_hist.alloc((long long)x.max_spans * kMaxSpanRows * x.n_cells);
  if (hb < 0) {
    if (ob >= 0) h->ex_offs.release(ob, x.n_cells + 1);
    if (cb >= 0) h->ex_cells.release(cb, x.n_cells);
    if (ps >= 0) h->ex_slots.release(ps, x.slot_len);
    return fail(DSMC_E_NOMEM, "no room: device memory of the handle is taken");
  }
  x.part_base = (int)ps;
  x.cell_base = (int)cb;
  x.off_base = (int)ob;
  x.hist_base = hb;
  x.active = true;
  x.fresh = true;
  if (new_id < 0) {
    new_id = (int)h->inst.size();
    h->inst.push_back(x);
  } else {
    h->inst[new_id] = x;
  }
  h->order.push_back(new_id);
  h->spans_reserved += x.max_spans;
  set_partition(h, h->span_target);
  *id = new_id;
  return DSMC_OK;
}

// Default particles per span for a handle of n particles: 4,096, or fewer for a small run
// so that its step passes still spread over two CTAs per SM (a 20,000-particle run: 17
// spans of 1,024 particles instead of 5 of 4,096), never below the finest partition its
// sort matrix is sized for.
int default_span_particles(long long n) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    sms = 152;
  const long long t = n / (2LL * sms);
  return (int)std::max<long long>(kMinSpanParticles,
                                  std::min<long long>(kDefaultSpanParticles, t));
}

// Allocates the handle and its device workspace for capacity C.
dsmc_status new_handle(const Capacity& C, const dsmc_options& opt, bool pool, void* workspace,
                       size_t workspace_bytes, dsmc_sim** out) {
  dsmc_sim* h = new (std::nothrow) dsmc_sim();
  if (!h) return fail(DSMC_E_NOMEM, "host allocation failed");
  h->pool = pool;
  h->opt = opt;
  h->C = C;
  h->L = layout_of(C);
  h->span_target = opt.span_particles ? opt.span_particles : default_span_particles(C.slots);
  // A pool holds many small instances whose membership changes too often to tune live;
  // 4-warp CTAs are what dsmc_autotune picks for such batches (8 % more micro-solves/s
  // than 8-warp CTAs in the request loop).
  h->cta_warps = opt.cta_warps ? opt.cta_warps : (pool ? kAWarpsSmall : kAWarps);
  h->span_rows = opt.span_rows ? opt.span_rows : 1;
  h->ex_slots.reset(C.slots);
  h->ex_cells.reset(C.cells);
  h->ex_offs.reset(C.offs);
  h->ex_hist.reset(C.hist_ints);
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
  h->P[1] = h->P[0] + C.slots;
  h->hist = (int*)(b + L.hist);
  h->count = (int*)(b + L.count);
  h->off[0] = (int*)(b + L.offset);
  h->off[1] = h->off[0] + C.offs;
  h->smax[0] = (float*)(b + L.smax);
  h->smax[1] = h->smax[0] + C.cells;
  h->ncand = (unsigned long long*)(b + L.ncand);
  h->nacc = (unsigned long long*)(b + L.nacc);
  h->acc = (double*)(b + L.acc);
  h->fields = (double*)(b + L.fields);
  h->tab_dev = (InstParams*)(b + L.tab);
  h->span_inst_dev = (int*)(b + L.span_inst);
  h->span_order_dev = h->span_inst_dev + 2 * (size_t)h->C.spans;
  h->chan_dev = (double*)(b + L.chan);
  h->err = (int*)(b + L.err);
  h->gstep_dev = (long long*)(b + L.err + 8);
  ce = set_step_smem_limits(kStepSmemMax, kStepSmemMax);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream());
  if (ce != cudaSuccess) {
    dsmc_status s = cuda_fail(ce, "handle setup");
    dsmc_destroy(h);
    return s;
  }
  *out = h;
  return DSMC_OK;
}

// Sets up fresh instances on the device and checks for errors (synchronises).
dsmc_status settle(dsmc_sim* h) {
  dsmc_status st = admit_fresh(h);
  if (st != DSMC_OK) return st;
  st = collect_times(h);
  if (st != DSMC_OK) return st;
  return read_error_word(h);
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
  for (int i = 0; i < n_inst; ++i)
    if ((st = check_instance(defs[i], i, n_inst)) != DSMC_OK) return st;
  long long slots = 0;
  for (int i = 0; i < n_inst; ++i) slots += padded_slots((long long)defs[i].n_cells * defs[i].ppc);
  if (slots > kMaxParticles)
    return fail(DSMC_E_INVAL, "the instances' particles (each padded to 64) must total <= 2^31 - 2^24");
  // Parameters and shared-memory fit before any device work.
  {
    int mcps = 1, mcells = 1;
    const int target = opt.span_particles ? opt.span_particles : kDefaultSpanParticles;
    for (int i = 0; i < n_inst; ++i) {
      Params p;
      if (!derive_params(defs[i].gas.omega, defs[i].Kn, defs[i].body_force, defs[i].ppc, opt, &p))
        return fail(DSMC_E_INVAL, (n_inst > 1 ? "instance " + std::to_string(i) + ": " : "") +
                                      "time step undefined: set options.dt for infinite Kn");
      int cps, ns;
      make_spans(defs[i].n_cells, defs[i].ppc, target, &cps, &ns);
      mcps = std::max(mcps, cps);
      mcells = std::max(mcells, defs[i].n_cells);
    }
    if (!step_fits(mcells, mcps, opt.group_size, opt.cta_warps ? opt.cta_warps : kAWarps,
                   opt.span_rows ? opt.span_rows : 1))
      return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  }
  dsmc_sim* h = nullptr;
  st = new_handle(capacity_of(defs, n_inst), opt, false, workspace, workspace_bytes, &h);
  if (st != DSMC_OK) return st;
  for (int i = 0; i < n_inst; ++i) {
    int id = -1;
    st = add_instance(h, defs[i], i, n_inst, &id);
    if (st != DSMC_OK) {
      dsmc_destroy(h);
      return st;
    }
  }
  st = settle(h);
  if (st != DSMC_OK) {
    dsmc_destroy(h);
    return st;
  }
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
  opt->cta_warps = 0;
  opt->span_rows = 0;
  opt->graph = 0;
  opt->accum = DSMC_ACCUM_FP32;
  opt->stream = nullptr;
  return DSMC_OK;
}

size_t dsmc_batch_workspace_bytes(const dsmc_instance* inst, int n_inst) {
  if (!inst || n_inst < 1 || n_inst > kMaxInstances) return 0;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].n_cells < 1 || inst[i].ppc < 1 || inst[i].n_cells > kMaxStepCells) return 0;
  return layout_of(capacity_of(inst, n_inst)).total;
}

size_t dsmc_workspace_bytes(int n_cells, int ppc) {
  dsmc_instance d{};
  d.n_cells = n_cells;
  d.ppc = ppc;
  return dsmc_batch_workspace_bytes(&d, 1);
}

size_t dsmc_pool_workspace_bytes(const dsmc_pool_limits* limits) {
  Capacity C;
  const std::string saved = g_last_error;
  if (capacity_of_pool(limits, &C) != DSMC_OK) {
    g_last_error = saved;
    return 0;
  }
  return layout_of(C).total;
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

dsmc_status dsmc_pool_create(const dsmc_pool_limits* limits, const dsmc_options* opt_in,
                             void* workspace, size_t workspace_bytes, dsmc_handle* out) {
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  *out = nullptr;
  Capacity C;
  dsmc_status st = capacity_of_pool(limits, &C);
  if (st != DSMC_OK) return st;
  dsmc_options opt;
  dsmc_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if ((st = check_options(&opt)) != DSMC_OK) return st;
  dsmc_sim* h = nullptr;
  st = new_handle(C, opt, true, workspace, workspace_bytes, &h);
  if (st != DSMC_OK) return st;
  *out = h;
  return DSMC_OK;
}

dsmc_status dsmc_pool_add(dsmc_handle h, const dsmc_instance* inst, int* id) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!inst || !id) return fail(DSMC_E_INVAL, "instance and id must not be NULL");
  if (!h->pool) return fail(DSMC_E_STATE, "dsmc_pool_add needs a handle from dsmc_pool_create");
  *id = -1;
  return add_instance(h, *inst, 0, 1, id);
}

dsmc_status dsmc_pool_remove(dsmc_handle h, int id) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!h->pool) return fail(DSMC_E_STATE, "dsmc_pool_remove needs a handle from dsmc_pool_create");
  Inst& x = h->inst[id];
  // Work already enqueued on the stream still reads these ranges; anything that reuses
  // them is enqueued after it.
  h->ex_slots.release(x.part_base, x.slot_len);
  h->ex_cells.release(x.cell_base, x.n_cells);
  h->ex_offs.release(x.off_base, x.n_cells + 1);
  h->ex_hist.release(x.hist_base, (long long)x.max_spans * kMaxSpanRows * x.n_cells);
  h->spans_reserved -= x.max_spans;
  x.active = false;
  x.fresh = false;
  h->order.erase(std::find(h->order.begin(), h->order.end(), id));
  set_partition(h, h->span_target);
  return DSMC_OK;
}

dsmc_status dsmc_channel_sums(dsmc_handle h, double* out) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  if ((s = upload_tables(h)) != DSMC_OK) return s;
  const size_t n_ids = h->inst.size();
  if (h->n_inst() > 0)
    DSMC_CUDA(launch_channel_sums(h->tab_dev, h->n_inst(), h->acc, h->chan_dev, h->stream()),
              "channel sums");
  if (n_ids > 0)
    DSMC_CUDA(cudaMemcpyAsync(out, h->chan_dev, 2 * n_ids * sizeof(double), cudaMemcpyDefault,
                              h->stream()),
              "copy channel sums");
  s = dsmc_sync(h);
  if (s != DSMC_OK) return s;
  for (size_t i = 0; i < n_ids; ++i)
    if (!h->inst[i].active) out[2 * i] = out[2 * i + 1] = 0.0;
  return DSMC_OK;
}

dsmc_status dsmc_device_moments_of(dsmc_handle h, int id, const double** acc) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!acc) return fail(DSMC_E_INVAL, "acc: NULL");
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  *acc = h->acc + (size_t)h->inst[id].cell_base * kNMom;
  return DSMC_OK;
}

dsmc_status dsmc_set_open_top(dsmc_handle h, int id, double u, double P) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!std::isfinite(u) || !std::isfinite(P) || std::fabs(P) > 0.25)
    return fail(DSMC_E_INVAL, "open boundary: finite u and |P| <= 0.25");
  Inst& x = h->inst[id];
  x.open_top = 1;
  x.u_top = (float)u;
  x.p_top = (float)P;
  h->tab_dirty = true;
  return DSMC_OK;
}

int dsmc_batch_size(dsmc_handle h) { return h ? h->n_inst() : 0; }

int dsmc_id_bound(dsmc_handle h) { return h ? (int)h->inst.size() : 0; }

dsmc_status dsmc_set_options(dsmc_handle h, const dsmc_options* opt) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  s = check_options(opt);
  if (s != DSMC_OK) return s;
  std::vector<Params> ps(h->inst.size());
  for (int id : h->order) {
    const Inst& x = h->inst[id];
    if (!derive_params(x.omega, x.Kn, x.F, x.ppc, *opt, &ps[id]))
      return fail(DSMC_E_INVAL, "time step undefined: set options.dt for infinite Kn");
  }
  // span_particles = 0 and cta_warps = 0 keep the partition and CTA shape in use.
  const int target_use = opt->span_particles ? opt->span_particles : h->span_target;
  const int warps_use = opt->cta_warps ? opt->cta_warps : h->cta_warps;
  const int rows_use = opt->span_rows ? opt->span_rows : h->span_rows;
  int mcps, mcells;
  partition_extent(h, target_use, nullptr, &mcps, &mcells);
  if (!step_fits(mcells, mcps, opt->group_size, warps_use, rows_use))
    return fail(DSMC_E_INVAL, "n_cells and group_size exceed the step's shared memory");
  if (h->events_used) {
    s = collect_times(h);
    if (s != DSMC_OK) return s;
  }
  h->opt = *opt;
  for (int id : h->order) h->inst[id].p = ps[id];
  h->cta_warps = warps_use;
  h->span_rows = rows_use;
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
  if (h->n_inst() == 0) return fail(DSMC_E_STATE, "no instances to tune on");
  DeviceGuard guard(h->device);
  cudaStream_t st = h->stream();
  cudaEvent_t e0, e1;
  DSMC_CUDA(cudaEventCreate(&e0), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(DSMC_E_CUDA, "event");
  }
  int best = h->span_target, best_warps = h->cta_warps, best_rows = h->span_rows;
  double best_ms = -1.0;
  dsmc_status r = DSMC_OK;
  const int shapes[4][2] = {{kAWarps, 1}, {kAWarps, 2}, {kAWarpsSmall, 1}, {kAWarpsSmall, 2}};
  for (const auto& shape : shapes) {
    const int w = shape[0], rows = shape[1];
    long long last_sig = -1;
    for (int target = kMinSpanParticles; target <= (1 << 17) && r == DSMC_OK; target *= 2) {
      int mcps, mcells;
      partition_extent(h, target, nullptr, &mcps, &mcells);
      if (!step_fits(mcells, mcps, h->opt.group_size, w, rows)) break;
      // Skip targets that give the same partition as the last one.
      long long sig = 0;
      for (int id : h->order) {
        int cps, ns;
        make_spans(h->inst[id].n_cells, h->inst[id].ppc, target, &cps, &ns);
        sig = (sig * 1000003 + cps) & 0x3fffffffffffLL;
      }
      if (sig == last_sig) continue;
      last_sig = sig;
      h->cta_warps = w;
      h->span_rows = rows;
      set_partition(h, target);
      // one untimed step with the new shape, then the timed trial
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
        best_warps = w;
        best_rows = rows;
      }
    }
    if (r != DSMC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != DSMC_OK) return r;
  h->cta_warps = best_warps;
  h->span_rows = best_rows;
  set_partition(h, best);
  h->opt.span_particles = best;
  h->opt.cta_warps = best_warps;
  h->opt.span_rows = best_rows;
  if (best_span_particles) *best_span_particles = best;
  if (best_ms_per_step) *best_ms_per_step = best_ms;
  if (h->opt.profile) return collect_times(h);
  return DSMC_OK;
}

dsmc_status dsmc_sync(dsmc_handle h) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  return settle(h);
}

dsmc_status dsmc_sample_moments_of(dsmc_handle h, int id, double* out, long long* n_samples) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  const Inst& x = h->inst[id];
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

dsmc_status dsmc_cell_fields_of(dsmc_handle h, int id, double* out) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  const Inst& x = h->inst[id];
  if (x.n_samples < 1) return fail(DSMC_E_STATE, "cell fields: no sampled steps yet");
  double* f = h->fields + (size_t)x.cell_base * DSMC_NFIELD;
  DSMC_CUDA(launch_cell_fields(h->acc + (size_t)x.cell_base * kNMom, x.n_cells, x.n_samples,
                               x.ppc, f, h->stream()),
            "cell fields");
  DSMC_CUDA(cudaMemcpyAsync(out, f, (size_t)x.n_cells * DSMC_NFIELD * sizeof(double),
                            cudaMemcpyDefault, h->stream()),
            "copy cell fields");
  return dsmc_sync(h);
}

dsmc_status dsmc_sample_moments_all(dsmc_handle h, double* out, long long* n_samples) {
  dsmc_status s = check_handle(h);
  if (s != DSMC_OK) return s;
  if (!out) return fail(DSMC_E_INVAL, "out: NULL");
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  DSMC_CUDA(cudaMemcpyAsync(out, h->acc, (size_t)h->C.cells * kNMom * sizeof(double),
                            cudaMemcpyDefault, h->stream()),
            "copy moments");
  if (n_samples)
    for (size_t i = 0; i < h->inst.size(); ++i)
      n_samples[i] = h->inst[i].active ? h->inst[i].n_samples : 0;
  return dsmc_sync(h);
}

dsmc_status dsmc_reset_samples_of(dsmc_handle h, int id) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  cudaStream_t st = h->stream();
  Inst& x = h->inst[id];
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
  for (int id : h->order)
    if ((s = dsmc_reset_samples_of(h, id)) != DSMC_OK) return s;
  return DSMC_OK;
}

dsmc_status dsmc_copy_state_of(dsmc_handle h, int id, float* y, float* vx, float* vy,
                               float* vz) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  cudaStream_t st = h->stream();
  const Inst& x = h->inst[id];
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

dsmc_status dsmc_copy_cells_of(dsmc_handle h, int id, int* offset, float* smax,
                               unsigned long long* ncand, unsigned long long* nacc) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  cudaStream_t st = h->stream();
  const Inst& x = h->inst[id];
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

dsmc_status dsmc_load_state_of(dsmc_handle h, int id, const float* y, const float* vx,
                               const float* vy, const float* vz, const float* smax,
                               long long step) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!y || !vx || !vy || !vz) return fail(DSMC_E_INVAL, "state arrays must not be NULL");
  if (step < 0) return fail(DSMC_E_INVAL, "step must be >= 0");
  DeviceGuard guard(h->device);
  if ((s = admit_fresh(h)) != DSMC_OK) return s;
  cudaStream_t st = h->stream();
  Inst& x = h->inst[id];
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
  s = set_uniform_offsets(h, id, host);
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

dsmc_status dsmc_get_info_of(dsmc_handle h, int id, dsmc_info* info) {
  dsmc_status s = check_index(h, id);
  if (s != DSMC_OK) return s;
  if (!info) return fail(DSMC_E_INVAL, "info: NULL");
  const Inst& x = h->inst[id];
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
  info->cta_warps = h->cta_warps;
  info->span_rows = h->span_rows;
  info->cells_per_span = x.cps;
  info->n_spans = x.n_spans;
  info->total_spans = h->spans;
  info->first_slot = x.part_base;
  info->first_cell = x.cell_base;
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
