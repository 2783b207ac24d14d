// dsmc_step.cu -- the two state passes of one DSMC step (Bird's method, which the
// paper cites for its micro model; problem of Sec. 2.1, units of Eq. 6).
//
// The resident particle state is an array of float4 records (y, vx, vy, vz): one
// 16-byte load or store moves a whole particle, so the sort's scattered writes cost
// one L2 sector per particle instead of four.
//
//   k_collide_move   one CTA per span of consecutive cells, the heaviest spans launched
//                    first (an order the host estimates).  Its warps take the span's
//                    collision groups one after another (a shared counter hands them
//                    out) and for each group
//                      1. load the group's records, keep them in shared memory and add
//                         their moment sums before the collisions,
//                      2. draw every NTC candidate's pair, acceptance threshold and
//                         scattering direction up front (one Philox draw per candidate,
//                         32 candidates at a time, one per lane), then apply the
//                         candidates in conflict-free rounds that reproduce the
//                         sequential order exactly,
//                      3. per particle: add the moment sums after the collisions, fly
//                         with the body force and diffuse walls, store the record back
//                         in place and count its new cell in the CTA's histogram.
//                    The histogram becomes the span's row of the sort matrix.  Per-cell
//                    (sigma g)_max, collision counters and moment sums are written by
//                    the one CTA that owns the cell.  With `count_only` the pass just
//                    counts cells of the span's slots (the sort into cells at creation
//                    and after a state load).
//   k_scatter_spans  one warp per span: re-reads the records in slot order, 16 per lane
//                    in flight, ranks each record among the same-cell records before it
//                    and scatters it stably into the other buffer from the span's row of
//                    the prefix-summed matrix plus the new cell offsets.
//   k_scatter_coop   the same scatter with a CTA per span (up to 1,365 cells): all its
//                    warps rank one round of 256 (or 512) records at a time.
//
// Between them, k_scan_spans (or k_scan_cols for instances of few spans) and
// k_offsets_cells (below) turn the matrix into per-span bases and the new cell offsets;
// for a small single run k_prefix_small does both in one launch.
#include <climits>
#include <type_traits>

#include "dsmc_device.cuh"
#include "dsmc_internal.h"

namespace dsmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// sin(2 pi v) and cos(2 pi v) for v in [0, 1], binary32: 4 v = n + r with n the nearest
// integer (4 v, n and r exact), theta = r pi/2 in [-pi/4, pi/4], the Taylor series of
// sin theta through theta^9 and of cos theta through theta^10 (truncation below 2e-9 on
// that range) by Horner's rule, then n quarter turns (selects, not branches: lanes of a
// warp fall in different quadrants).
__device__ __forceinline__ void sincos_turn(float v, float& sn, float& cs) {
  const float t = fmul(4.0f, v);
  const float n = floorf(fadd(t, 0.5f));
  const float r = fsub(t, n);
  const float th = fmul(r, 0x1.921fb6p+0f);  // pi/2
  const float t2 = fmul(th, th);
  float ps = 0x1.71de3ap-19f;                  // 1/9!
  ps = fsub(fmul(ps, t2), 0x1.a01a02p-13f);    // 1/7!
  ps = fadd(fmul(ps, t2), 0x1.111112p-7f);     // 1/5!
  ps = fsub(fmul(ps, t2), 0x1.555556p-3f);     // 1/3!
  ps = fmul(ps, t2);
  const float s = fadd(th, fmul(th, ps));
  float pc = -0x1.27e4fcp-22f;                 // -1/10!
  pc = fadd(fmul(pc, t2), 0x1.a01a02p-16f);    // 1/8!
  pc = fsub(fmul(pc, t2), 0x1.6c16c2p-10f);    // 1/6!
  pc = fadd(fmul(pc, t2), 0x1.555556p-5f);     // 1/4!
  pc = fsub(fmul(pc, t2), 0.5f);
  const float c = fadd(1.0f, fmul(t2, pc));
  const int q = ((int)n) & 3;  // quarter turns: swap for odd q, signs by quadrant
  const float a = (q & 1) ? c : s, b = (q & 1) ? s : c;
  sn = (q & 2) ? -a : a;
  cs = ((q + 1) & 2) ? -b : b;
}

// VHS acceptance threshold on the relative speed (sigma g > u (sigma g)_max written as
// g > thr): thr = exp((ln(u smax) - ln cvhs) / (2 - 2 omega)), with the library's own
// binary32 ln and exp; this value decides.
__device__ __forceinline__ float vhs_threshold(float us, float vinv, float lncv) {
  return exp32(fmul(vinv, fsub(ln32(us), lncv)));
}

// The same threshold from the hardware's base-2 approximations: within 3e-5 relative of
// vhs_threshold (the approximations' own errors, the binary32 rounding of an argument of
// magnitude below 70, and the 2-ulp error of ln32 and exp32).  [t (1 - 2^-10),
// t (1 + 2^-10)] therefore brackets the deciding value; a relative speed outside the
// bracket is decided without it.
constexpr float kThrLo = 1.0f - 0x1p-10f;
constexpr float kThrHi = 1.0f + 0x1p-10f;

__device__ __forceinline__ float vhs_threshold_approx(float us, float vinv, float lg2cv) {
  float l, t;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(us));
  const float x = fmul(vinv, fsub(l, lg2cv));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}

// Isotropic scattering direction from two uniform words by the cylindrical (Archimedes)
// map: n_z = 2 u(w0) - 1 and azimuth 2 pi u(w1), independent and uniform, give
// n = (sqrt(1 - n_z^2) cos, sqrt(1 - n_z^2) sin, n_z), uniform on the sphere.  No
// rejection, so every candidate of a warp takes the same two draws.
__device__ __forceinline__ void direction_of(uint32_t w0, uint32_t w1, float& nx, float& ny,
                                             float& nz) {
  nz = s11(w0);
  const float rho = fsqrt(fsub(1.0f, fmul(nz, nz)));
  float sn, cs;
  sincos_turn(u01(w1), sn, cs);
  nx = fmul(rho, cs);
  ny = fmul(rho, sn);
}

// Per-lane sums of the 12 velocity moments of a group's particles (the count is the
// cell's particle number and needs no sum): v, v_i v_j (six), v_i |v|^2 (three).
// LaneSums<float>: the products of the binary32 velocities summed in binary32, the
// second and third moments by fused multiply-add (one rounding per term).
// LaneSums<double>: every product rounded to binary32 exactly as the oracle forms it,
// then added in binary64.
template <typename T>
struct LaneSums;

template <>
struct LaneSums<float> {
  float2 a, b, c, d, e, f;  // (vx, vy) (vz, vz2) (vx2, vy2) (vxvy, vxvz) (vyvz, vz v2) (vx v2, vy v2)
  __device__ __forceinline__ void zero() {
    a = b = c = d = e = f = make_float2(0.0f, 0.0f);
  }
  __device__ __forceinline__ void add(float x, float y, float z) {
    const float2 xy = make_float2(x, y);
    const float2 sq = __fmul2_rn(xy, xy);
    const float zz = fmul(z, z);
    const float v2 = fadd(fadd(sq.x, sq.y), zz);
    a = __fadd2_rn(a, xy);
    b = __fadd2_rn(b, make_float2(z, zz));
    c = __fadd2_rn(c, sq);
    d = __ffma2_rn(make_float2(x, x), make_float2(y, z), d);
    e = __ffma2_rn(make_float2(y, z), make_float2(z, v2), e);
    f = __ffma2_rn(xy, make_float2(v2, v2), f);
  }
  // moment k = 1..12 in the order of the raw sums (1 vx, 2 vy, 3 vz, 4 vx2, 5 vy2, 6 vz2,
  // 7 vxvy, 8 vxvz, 9 vyvz, 10 vx v2, 11 vy v2, 12 vz v2); 0 for the padding slots
  __device__ __forceinline__ float get(int k) const {
    switch (k) {
      case 1: return a.x;
      case 2: return a.y;
      case 3: return b.x;
      case 4: return c.x;
      case 5: return c.y;
      case 6: return b.y;
      case 7: return d.x;
      case 8: return d.y;
      case 9: return e.x;
      case 10: return f.x;
      case 11: return f.y;
      case 12: return e.y;
      default: return 0.0f;
    }
  }
};

template <>
struct LaneSums<double> {
  double m[12];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 12; ++k) m[k] = 0.0;
  }
  __device__ __forceinline__ void add(float x, float y, float z) {
    const float v2 = fadd(fadd(fmul(x, x), fmul(y, y)), fmul(z, z));
    const float p[12] = {x,          y,          z,          fmul(x, x), fmul(y, y), fmul(z, z),
                         fmul(x, y), fmul(x, z), fmul(y, z), fmul(x, v2), fmul(y, v2),
                         fmul(z, v2)};
#pragma unroll
    for (int k = 0; k < 12; ++k) m[k] = __dadd_rn(m[k], (double)p[k]);
  }
  __device__ __forceinline__ double get(int k) const {
    double r = 0.0;
#pragma unroll
    for (int j = 0; j < 12; ++j)
      if (k == j + 1) r = m[j];
    return r;
  }
};

// Warp sum of a group's lane sums by a transposing butterfly over 16 slots (moments
// 1..12 and zero padding): each exchange halves the values a lane carries, so 16
// shuffles leave the total of moment moment_of_lane(lane) on lanes 2i and 2i+1.
__device__ __forceinline__ int moment_of_lane(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

template <typename T>
__device__ __forceinline__ T group_total(const LaneSums<T>& m, int lane) {
  T v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = m.get(k);
#pragma unroll
  for (int half = 8, mask = 16; half >= 1; half >>= 1, mask >>= 1) {
    const bool upper = (lane & mask) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const T send = upper ? v[k] : v[k + half];
      const T keep = upper ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(kFull, send, mask);
    }
  }
  return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

// Exact, order-independent combination of group totals.  A cell's group totals are
// rounded to integer multiples of a grid 2^-(41 - e), e = bit length of the cell's
// particle count nc, and the integers added in 64 bits: integer addition does not
// depend on the order in which warps finish their groups, so a step's cell sums are a
// pure function of the state.  With |v| <= 101 (|each product| <= 2^20) a group total is
// at most 2 n_g 2^20 in magnitude and the cell's integer sum stays below 2^62.  The
// rounding adds at most 2^-(42 - e) per group total.
__device__ __forceinline__ int grid_exponent(int nc) { return 41 - (32 - __clz(nc)); }

__device__ __forceinline__ long long fixed_of(float t, int gexp) {
  return __float2ll_rn(fmul(t, __int_as_float((127 + gexp) << 23)));
}
__device__ __forceinline__ long long fixed_of(double t, int gexp) {
  return __double2ll_rn(__dmul_rn(t, __longlong_as_double((long long)(1023 + gexp) << 52)));
}

// Adds a group's results into the CTA's slots of its cell: the 12 moment totals as
// fixed-point integers (lanes 2i of the butterfly), the largest relative speed, the
// candidate and accepted-collision counts.  Returns false when a total exceeds the
// magnitude the fixed-point range allows for the group's size.
template <typename T>
__device__ __forceinline__ bool add_group(const LaneSums<T>& m, bool sample, int gn, int nc,
                                          float gmax, uint32_t M, unsigned accn,
                                          unsigned long long* cfix, unsigned* cgmax,
                                          unsigned long long* ccand,
                                          unsigned long long* caccn, int lane) {
  bool ok = true;
  if (sample) {
    const T tot = group_total(m, lane);
    const int k = moment_of_lane(lane);
    if ((lane & 1) == 0 && k >= 1 && k <= 12) {
      const int ge = grid_exponent(nc);
      const long long q = fixed_of(tot, ge);
      // |q| <= 2 gn 2^20 2^ge holds for |products| <= 2^20
      const long long lim = (long long)(2 * gn) << (20 + ge);
      if (q > lim || q < -lim) ok = false;
      atomicAdd(&cfix[k], (unsigned long long)q);
    }
  }
  const unsigned gbits = __reduce_max_sync(kFull, __float_as_uint(gmax));  // gmax >= 0
  const unsigned nacc = __reduce_add_sync(kFull, accn);
  if (lane == 0) {
    atomicMax(cgmax, gbits);
    atomicAdd(ccand, (unsigned long long)M);
    atomicAdd(caccn, (unsigned long long)nacc);
  }
  return ok;
}

}  // namespace

// The parameters of the instance a span belongs to: the kernel argument for a
// single-instance run, else the entry of the run's instance table.
template <bool kBatch>
__device__ __forceinline__ const InstParams& instance_of(const InstParams& one,
                                                         const StepLaunch& SL, int span) {
  if constexpr (kBatch)
    return SL.tab[SL.span_inst[span]];
  else
    return one;
}

// Copies the CTA's instance entry into shared memory (one read of the table per CTA,
// then broadcast reads); returns the copy, or the kernel argument for one instance.
template <bool kBatch>
__device__ __forceinline__ const InstParams& stage_instance(const InstParams& one,
                                                            const StepLaunch& SL, int span,
                                                            InstParams* sh) {
  if constexpr (kBatch) {
    static_assert(sizeof(InstParams) % 4 == 0, "InstParams is copied as words");
    const int* src = reinterpret_cast<const int*>(&SL.tab[SL.span_inst[span]]);
    int* dst = reinterpret_cast<int*>(sh);
    for (int i = threadIdx.x; i < (int)(sizeof(InstParams) / 4); i += blockDim.x)
      dst[i] = src[i];
    __syncthreads();
    return *sh;
  } else {
    return one;
  }
}

// Collision models (a.mode): 0 hard spheres, 1 VHS with 0.5 < omega < 1, 2 omega = 1
// (sigma g independent of g).  CTAs per SM the register budget is set for: 3 of 8 warps,
// 6 of 4 warps; the batched 4-warp kernel reads its parameters from shared memory and
// spills at 6 (85 registers), so it is given 5 (no spills, 10 % faster on the
// 256-instance batch).  The binary64 moment sums (kF64) hold twelve binary64 values per
// lane and get half the CTAs per SM.
template <bool kBatch, int kWarps, bool kF64>
constexpr int collide_ctas_per_sm() {
  return (kWarps == kAWarps ? 3 : (kBatch ? 5 : 6)) / (kF64 ? 2 : 1);
}

template <bool kBatch, int kWarps, bool kF64>
__global__ void __launch_bounds__(kWarps * 32, (collide_ctas_per_sm<kBatch, kWarps, kF64>()))
    k_collide_move(float4* __restrict__ P, const int* __restrict__ off_all,
                   const float* __restrict__ smax_in_all, float* __restrict__ smax_out_all,
                   unsigned long long* __restrict__ ncand_all,
                   unsigned long long* __restrict__ nacc_all, double* __restrict__ acc_all,
                   int* __restrict__ hist, const InstParams one, const StepLaunch SL,
                   int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ InstParams sh_inst;
  // unrolling the per-particle loops helps the single run; the batched kernel, which
  // already spills, was 16 % slower with it
  constexpr int kMoveUnroll = kBatch ? 1 : 4;
  // the global span of this CTA: the launch takes spans heaviest first
  const int gspan = SL.span_order ? SL.span_order[blockIdx.x] : (int)blockIdx.x;
  const InstParams& a = stage_instance<kBatch>(one, SL, gspan, &sh_inst);
  const int* __restrict__ off = off_all + a.off_base;
  const float* __restrict__ smax_in = smax_in_all + a.cell_base;
  float* __restrict__ smax_out = smax_out_all + a.cell_base;
  unsigned long long* __restrict__ ncand = ncand_all + a.cell_base;
  unsigned long long* __restrict__ nacc = nacc_all + a.cell_base;
  double* __restrict__ acc = acc_all + (size_t)a.cell_base * kNMom;
  // the instance's step number
  const long long istep = (SL.gstep_dev ? *SL.gstep_dev : SL.gstep) - a.step0;
  const uint32_t step = (uint32_t)istep;
  const bool count_only = SL.count_only != 0;
  const bool sample = !count_only && istep >= a.sample_start;
  const bool collide = !count_only && a.collide != 0;
  const int mode = a.mode;
  const int n_cells = a.n_cells;
  const int cps = a.cps;
  const int cap = a.cap;
  const int G = a.G;
  const int R = SL.rows;
  const StepSmem L = step_smem_layout(n_cells, cps, cap, kWarps, R);
  using Acc = typename std::conditional<kF64, double, float>::type;
  int* h = reinterpret_cast<int*>(smem + L.hist);  // the span's rows x n_cells counts
  // per local cell: fixed-point moment sums (slot 0 unused), in a cell's grid
  unsigned long long* cfix = reinterpret_cast<unsigned long long*>(smem + L.cell_acc);
  unsigned long long* ccand = reinterpret_cast<unsigned long long*>(smem + L.cell_cand);
  unsigned long long* caccn = reinterpret_cast<unsigned long long*>(smem + L.cell_accn);
  unsigned* cgmax = reinterpret_cast<unsigned*>(smem + L.cell_gmax);
  int* gfirst = reinterpret_cast<int*>(smem + L.cell_groups);  // cps + 1 group prefix
  int* next_group = gfirst + cps + 1;
  int* cstart = reinterpret_cast<int*>(smem + L.cell_start);     // cps + 1 cell starts
  float* csmax = reinterpret_cast<float*>(smem + L.cell_smax);   // cps (sigma g)_max
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* wmem = smem + L.warps + (size_t)wib * L.per_warp;
  float4* rec = reinterpret_cast<float4*>(wmem + L.w_rec);  // (y, vx, vy, vz) per particle
  // Per particle of the staged group: during a batch of candidates, the lanes whose
  // candidates touch it (bit mask); zero between batches.  Also the queue of wall hits
  // (then restored to zero).
  unsigned* touch = reinterpret_cast<unsigned*>(wmem + L.w_own);
  uint64_t* bar = reinterpret_cast<uint64_t*>(wmem + L.w_bar);

  const int span = gspan - a.span_base;  // the instance's span
  const int c0 = span * cps;
  const int c1 = min(c0 + cps, n_cells);
  const unsigned lt = (1u << lane) - 1u;
  // rows (span R + r) of the sort matrix; row r counts the r-th half of the slots
  int* row = hist + a.hist_base + (size_t)span * R * n_cells;
  const int sb0 = off[c0], sb1 = off[c1];
  const int mid = (R > 1) ? sb0 + ((sb1 - sb0) >> 1) : sb1;  // first slot of the second row
  for (int i = threadIdx.x; i < R * n_cells; i += blockDim.x) h[i] = 0;
  // count one particle of slot p in new cell cn
  auto count_cell = [&](int p, int cn) { atomicAdd(&h[(p >= mid ? n_cells : 0) + cn], 1); };
  auto write_rows = [&]() {
    for (int e = threadIdx.x; e < R * n_cells; e += blockDim.x) row[e] = h[e];
  };

  if (count_only) {  // sort into cells: count the cells of the span's slots
    __syncthreads();
    for (int p = sb0 + threadIdx.x; p < sb1; p += blockDim.x)
      count_cell(p, cell_of(P[p].x, n_cells, a.ncf));
    __syncthreads();
    write_rows();
    return;
  }

  for (int i = threadIdx.x; i < cps * kNMom; i += blockDim.x) cfix[i] = 0ull;
  for (int i = threadIdx.x; i < cps; i += blockDim.x) {
    ccand[i] = 0;
    caccn[i] = 0;
    cgmax[i] = 0u;
  }
  if (wib == 0) {  // group prefix over the span's cells, 32 cells at a time
    int base = 0;
    for (int i0 = 0; i0 < c1 - c0; i0 += 32) {
      const int i = i0 + lane;
      int g = 0;
      if (i < c1 - c0) {
        const int s0 = off[c0 + i], s1 = off[c0 + i + 1];
        g = group_count(s1 - s0, G);
        cstart[i] = s0;
        csmax[i] = smax_in[c0 + i];
      }
      int incl = g;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
      }
      if (i < c1 - c0) gfirst[i] = base + incl - g;
      base += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) {
      gfirst[c1 - c0] = base;
      cstart[c1 - c0] = off[c1];
      *next_group = 0;
    }
  }
  for (int i = lane; i < cap; i += 32) touch[i] = 0u;
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int n_groups = gfirst[c1 - c0];

  bool bad_bounce = false, cand_fail = false, timeout = false;
  bool inflow_fail = false, mom_range = false;
  uint32_t parity = 0;
  // Groups are handed out by a counter.  Each warp reserves its next group when it
  // starts one, prefetches the next group's records into L2, and issues their bulk copy
  // into its buffer as soon as the current group's records have been read for the last
  // time.  A group is described from shared memory alone (cell starts and group prefix).
  auto cell_of_group = [&](int q, int from) {
    int l = from;
    while (gfirst[l + 1] <= q) ++l;
    return l;
  };
  auto group_slots = [&](int q, int l, int& gs_, int& gn_) {
    const int gi_ = q - gfirst[l];
    const int nc_ = cstart[l + 1] - cstart[l];
    gs_ = cstart[l] + gi_ * G;
    gn_ = (gi_ == gfirst[l + 1] - gfirst[l] - 1) ? nc_ - gi_ * G : G;
  };
  auto issue_copy = [&](int gs_, int gn_) {
    fence_proxy_async_smem();  // earlier generic accesses to rec before the async write
    __syncwarp();
    if (lane == 0) {
      mbar_arrive_expect_tx(bar, (uint32_t)gn_ * 16u);
      bulk_load(rec, P + gs_, (uint32_t)gn_ * 16u, bar);
    }
  };
  int q_next = 0;
  if (lane == 0) q_next = atomicAdd(next_group, 1);
  q_next = __shfl_sync(kFull, q_next, 0);
  int l_next = 0;
  if (q_next < n_groups) {
    int s_, n_;
    l_next = cell_of_group(q_next, 0);
    group_slots(q_next, l_next, s_, n_);
    issue_copy(s_, n_);
  }
  for (;;) {
    const int q = q_next;
    if (q >= n_groups) break;
    const int lc = l_next;
    const int c = c0 + lc;
    const int gi = q - gfirst[lc];
    const int nc = cstart[lc + 1] - cstart[lc];
    int gs, gn;
    group_slots(q, lc, gs, gn);
    if (lane == 0) q_next = atomicAdd(next_group, 1);
    q_next = __shfl_sync(kFull, q_next, 0);
    int gs_next = 0, gn_next = 0;
    if (q_next < n_groups) {
      l_next = cell_of_group(q_next, lc);
      group_slots(q_next, l_next, gs_next, gn_next);
      if (lane == 0) bulk_prefetch_l2(P + gs_next, (uint32_t)gn_next * 16u);
    }

    // 1. The group's records in shared memory (bulk copy issued beforehand).
    const float smax = csmax[lc];
    if (!mbar_wait(bar, parity)) {
      timeout = true;
      mbar_wait(bar, parity);  // give the copy one more bounded chance to land
      break;
    }
    parity ^= 1u;

    // 2. Moments before the collisions.
    float gmax = 0.0f;
    unsigned laccn = 0;
    uint32_t M = 0;
    LaneSums<Acc> m;
    m.zero();
    if (sample)
#pragma unroll kMoveUnroll
      for (int i = lane; i < gn; i += 32) {
        const float4 r = rec[i];
        m.add(r.y, r.z, r.w);
      }

    // 3. NTC candidates of the group.
    if (collide && gn >= 2) {
      const uint32_t c3 = (kStreamColl << 24) | ((uint32_t)gi << 4);
      const float t1 = fmul((float)(gn - 1), (float)nc);
      const float mf = fmul(fmul(t1, a.coef), smax);
      const float fl = floorf(mf);
      const float frac = fsub(mf, fl);
      const bool mbad = !(mf <= kMaxCandidates);
      if (mbad) cand_fail = true;
      // M is floor(mf) or floor(mf) + 1 by the count-rounding draw (candidate counter
      // 0xffffffff).  Batch 0 draws it on lane 31 beside candidates 0..30 on lanes
      // 0..30; later batches hold candidates 31 + 32 b + lane.
      for (uint32_t kb = 0, first = 1;; first = 0) {
        const uint32_t k =
            first ? (lane == 31 ? 0xffffffffu : (uint32_t)lane) : kb + (uint32_t)lane;
        U4 w{};
        if (first) {
          w = philox_rk(k, (uint32_t)c, step, c3, a.keys);
          const float ur = __shfl_sync(kFull, u01(w.x), 31);
          M = mbad ? 0u : (uint32_t)fl + (ur < frac ? 1u : 0u);
        }
        bool pend = first ? (lane < 31 && (uint32_t)lane < M) : (k < M);
        if (M == 0u) break;
        int i = 0, j = 0;
        // acceptance: g > thr; thr_lo <= thr <= thr_hi, equal unless the VHS threshold
        // was bracketed by the fast approximation (thr itself is then formed only for
        // a relative speed inside the bracket)
        float us = 0.0f, thr_lo = 0.0f, thr_hi = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;
        if (pend) {
          // one draw per candidate: word 0 the pair (multiply-shift: i from the high
          // half of w0 gn, j from the low half times gn - 1), word 1 the acceptance
          // uniform, words 2 and 3 the scattering direction
          if (!first) w = philox_rk(k, (uint32_t)c, step, c3, a.keys);
          const unsigned long long pij = (unsigned long long)w.x * (unsigned long long)gn;
          i = (int)(pij >> 32);
          j = (int)__umulhi((uint32_t)pij, (uint32_t)(gn - 1));
          j += (j >= i) ? 1 : 0;
          us = fmul(u01(w.y), smax);
          if (mode == 0) {
            thr_lo = thr_hi = us;
          } else if (mode == 1) {
            const float t = vhs_threshold_approx(us, a.vinv, a.lg2cv);
            if (t > 0x1p-100f && t < 0x1p100f) {
              thr_lo = fmul(t, kThrLo);
              thr_hi = fmul(t, kThrHi);
            } else {
              thr_lo = thr_hi = vhs_threshold(us, a.vinv, a.lncv);
            }
          } else {
            thr_lo = thr_hi = (us < a.cvhs) ? -1.0f : __int_as_float(0x7f800000);
          }
          direction_of(w.z, w.w, nx, ny, nz);
        }
        // Earlier candidates of the batch that share a particle with this one: the
        // candidate may be applied once none of them is pending any more, which gives
        // exactly the result of applying the candidates in order.
        if (pend) {
          atomicOr(&touch[i], 1u << lane);
          atomicOr(&touch[j], 1u << lane);
        }
        __syncwarp();
        const unsigned before = pend ? ((touch[i] | touch[j]) & lt) : 0u;
        __syncwarp();
        if (pend) {
          touch[i] = 0u;
          touch[j] = 0u;
        }
        for (;;) {
          const unsigned waiting = __ballot_sync(kFull, pend);
          if (waiting == 0u) break;
          const bool ready = pend && (before & waiting) == 0u;
          if (ready) {
            const float4 ri = rec[i], rj = rec[j];
            const float gx = fsub(ri.y, rj.y), gy = fsub(ri.z, rj.z), gz = fsub(ri.w, rj.w);
            const float g = fsqrt(fadd(fadd(fmul(gx, gx), fmul(gy, gy)), fmul(gz, gz)));
            gmax = fmaxf(gmax, g);
            bool accept = g > thr_hi;
            if (!accept && g > thr_lo) accept = g > vhs_threshold(us, a.vinv, a.lncv);
            if (accept) {
              const float hg = fmul(0.5f, g);
              const float cx = fmul(fadd(ri.y, rj.y), 0.5f);
              const float cy = fmul(fadd(ri.z, rj.z), 0.5f);
              const float cz = fmul(fadd(ri.w, rj.w), 0.5f);
              const float dx = fmul(hg, nx), dy = fmul(hg, ny), dz = fmul(hg, nz);
              rec[i] = make_float4(ri.x, fadd(cx, dx), fadd(cy, dy), fadd(cz, dz));
              rec[j] = make_float4(rj.x, fsub(cx, dx), fsub(cy, dy), fsub(cz, dz));
              laccn += 1;
            }
            pend = false;
          }
          __syncwarp();
        }
        kb = first ? 31u : kb + 32u;
        if (kb >= M) break;
      }
    }
    __syncwarp();

    // 4. Moments after the collisions, free flight, store, count the new cell.
    //    A particle whose flight reaches a wall is queued and flown afterwards, all such
    //    particles of the group together (the free flight is exactly the first leg of
    //    the full flight, so the result is the same).
    int n_wall = 0;
#pragma unroll kMoveUnroll
    for (int b = 0; b < gn; b += 32) {
      const int i = b + lane;
      bool hits = false;
      if (i < gn) {
        const float4 r = rec[i];
        if (sample) m.add(r.y, r.z, r.w);
        const float ynew = fadd(r.x, fmul(r.z, a.dt));
        hits = (ynew < 0.0f) || (ynew > 1.0f);
        if (!hits) {
          const float xx = fadd(r.y, fmul(a.F, a.dt));
          P[gs + i] = make_float4(ynew, xx, r.z, r.w);
          count_cell(gs + i, cell_of(ynew, n_cells, a.ncf));
        }
      }
      const unsigned q = __ballot_sync(kFull, hits);
      if (hits) touch[n_wall + __popc(q & lt)] = (unsigned)i;
      n_wall += __popc(q);
    }
    __syncwarp();
    for (int b = 0; b < n_wall; b += 32) {
      if (b + lane < n_wall) {
        const int i = (int)touch[b + lane];
        const int p = gs + i;
        const float4 r = rec[i];
        float yy = r.x, xx = r.y, uy = r.z, zz = r.w;
        if (!fly(yy, xx, uy, zz, a.dt, a.F, a.keys, step, (uint32_t)(p - a.part_base),
                 a.open_top, a.u_top, a.p_top, inflow_fail))
          bad_bounce = true;
        P[p] = make_float4(yy, xx, uy, zz);
        count_cell(p, cell_of(yy, n_cells, a.ncf));
      }
    }
    __syncwarp();
    for (int i = lane; i < n_wall; i += 32) touch[i] = 0u;
    // the records are read for the last time: bring in the next group's
    if (q_next < n_groups) issue_copy(gs_next, gn_next);
    if (!add_group(m, sample, gn, nc, gmax, M, laccn, cfix + (size_t)lc * kNMom, &cgmax[lc],
                   &ccand[lc], &caccn[lc], lane))
      mom_range = true;
    __syncwarp();
  }
  if (bad_bounce) atomicOr(err, kErrBounces);
  if (cand_fail && lane == 0) atomicOr(err, kErrCandidates);
  if (timeout && lane == 0) atomicOr(err, kErrCopyTimeout);
  if (inflow_fail) atomicOr(err, kErrInflow);
  if (mom_range) atomicOr(err, kErrMoments);
  __syncthreads();

  write_rows();
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int lc = c - c0;
    const float gm = __uint_as_float(cgmax[lc]);
    const float sg = (mode == 0) ? gm : fmul(a.cvhs, pow32(gm, a.vexp));
    smax_out[c] = fmaxf(smax_in[c], sg);
    ncand[c] += ccand[lc];
    nacc[c] += caccn[lc];
    if (sample) {
      // count: half before and half after the collisions of every particle of the cell
      const int nc = off[c + 1] - off[c];
      acc[(size_t)c * kNMom] += (double)nc;
      const double grid = __longlong_as_double((long long)(1023 - grid_exponent(nc > 0 ? nc : 1)) << 52);
      for (int k = 1; k < kNMom; ++k)
        acc[(size_t)c * kNMom + k] +=
            0.5 * grid * (double)(long long)cfix[(size_t)lc * kNMom + k];
    }
  }
}

// One warp per span: stable scatter of the span's records into the other buffer.  Slots
// are taken 256 at a time (8 per lane); the loads of the next 256 are issued before the
// current ones are placed, so each lane keeps 8 to 16 records in flight.
//
// A record's place is its cell's running slot (run[]) plus the number of lanes before
// it in its 32-record slice that go to the same cell.  Those "peer" lanes come from a
// small per-warp table of lane masks: each lane ORs its bit into entry (cell mod 256)
// and reads the entry back.  While a slice's cells lie within 256 consecutive values,
// which holds unless a particle crosses more than 255 cells in one step, two cells never
// share an entry and the mask is exactly the set of same-cell lanes; otherwise the slice
// falls back to __match_any_sync.  The table costs a few shared-memory operations per
// slice, where __match_any_sync on ~25 distinct values of 32 (2,000 cells, particles
// crossing ~20 cells a step) was the scatter's bottleneck.  With few warps per SM the
// longer chain of one warp matters more, and the launcher keeps __match_any_sync
// (place_batch_match); both give the same places.
namespace {

constexpr int kScatterUnroll = 8;
constexpr int kMaskSlots = 256;  // entries of the per-warp mask table (a power of two)
constexpr int kMaskWarpsPerSm = 4;

__device__ __forceinline__ void load_batch(float4 (&r)[kScatterUnroll],
                                           const float4* __restrict__ P, int base, int b1,
                                           int lane) {
#pragma unroll
  for (int u = 0; u < kScatterUnroll; ++u) {
    const int p = base + u * 32 + lane;
    if (p < b1) r[u] = P[p];
  }
}

__device__ __forceinline__ bool place_batch_mask(const float4 (&r)[kScatterUnroll],
                                            float4* __restrict__ P2, int* run, unsigned* msk,
                                            int base, int b1,
                                            int n_cells, float ncf, int lo, int hi, int lane,
                                            unsigned lt) {
  int cell[kScatterUnroll];
  unsigned peers[kScatterUnroll];
#pragma unroll
  for (int u = 0; u < kScatterUnroll; ++u) {
    const int p = base + u * 32 + lane;
    cell[u] = (p < b1) ? cell_of(r[u].x, n_cells, ncf) : -1;  // -1: no record
  }
  // lanes of each slice bound for the same cell
#pragma unroll
  for (int u = 0; u < kScatterUnroll; ++u) {
    const int cmin = __reduce_min_sync(kFull, cell[u] >= 0 ? cell[u] : INT_MAX);
    const int cmax = __reduce_max_sync(kFull, cell[u]);
    if (cmax - cmin < kMaskSlots) {  // no two cells share a slot of the mask table
      const int slot = cell[u] & (kMaskSlots - 1);
      if (cell[u] >= 0) atomicOr(&msk[slot], 1u << lane);
      __syncwarp();
      peers[u] = (cell[u] >= 0) ? msk[slot] : 0u;
      __syncwarp();
      if (cell[u] >= 0) msk[slot] = 0u;  // the table is all zero between slices
      __syncwarp();
    } else {
      peers[u] = __match_any_sync(kFull, cell[u]);
    }
  }
  // slots, slice after slice: the first lane of each peer group advances the run
  int d[kScatterUnroll];
#pragma unroll
  for (int u = 0; u < kScatterUnroll; ++u) {
    const bool act = cell[u] >= 0;
    const int first = act ? run[cell[u]] : 0;
    __syncwarp();
    if (act && (peers[u] & lt) == 0) run[cell[u]] = first + __popc(peers[u]);
    __syncwarp();
    d[u] = first + __popc(peers[u] & lt);
  }
  bool bad = false;
#pragma unroll
  for (int u = 0; u < kScatterUnroll; ++u) {
    if (cell[u] >= 0) {
      if (d[u] >= lo && d[u] < hi)
        P2[d[u]] = r[u];
      else
        bad = true;
    }
  }
  return bad;
}

// Ranking with __match_any_sync, slice after slice (fewer instructions in the chain of
// one warp: the better choice when few warps share an SM).
__device__ __forceinline__ bool place_batch_match(const float4 (&r)[kScatterUnroll],
                                                  float4* __restrict__ P2, int* run, int base,
                                                  int b1, int n_cells, float ncf, int lo, int hi,
                                                  int lane, unsigned lt) {
  bool bad = false;
#pragma unroll
  for (int u = 0; u < kScatterUnroll; ++u) {
    const int p = base + u * 32 + lane;
    const bool act = p < b1;
    const int cell = act ? cell_of(r[u].x, n_cells, ncf) : -1;
    const unsigned peers = __match_any_sync(kFull, cell);
    const int first = act ? run[cell] : 0;
    __syncwarp();
    if (act && (peers & lt) == 0) run[cell] = first + __popc(peers);
    __syncwarp();
    if (act) {
      const int d = first + __popc(peers & lt);
      if (d >= lo && d < hi)
        P2[d] = r[u];
      else
        bad = true;
    }
  }
  return bad;
}

}  // namespace

template <bool kBatch, bool kMask>
__global__ void __launch_bounds__(kBWarpsMax * 32)
    k_scatter_spans(const float4* __restrict__ P, float4* __restrict__ P2,
                    const int* __restrict__ off_cur_all, const int* __restrict__ off_new_all,
                    const int* __restrict__ hist, const InstParams one, const StepLaunch SL,
                    int* __restrict__ err) {
  constexpr int kBatch2 = 32 * kScatterUnroll;
  extern __shared__ int sh_run[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int unit = blockIdx.x * (blockDim.x >> 5) + wib;  // (span, row of the span)
  const int R = SL.rows;
  const int gspan = unit / R, sub = unit - gspan * R;
  if (gspan >= SL.n_spans_total) return;
  const InstParams& a = instance_of<kBatch>(one, SL, gspan);
  const int n_cells = a.n_cells;
  const int span = gspan - a.span_base;
  const int* __restrict__ off_cur = off_cur_all + a.off_base;
  const int* __restrict__ off_new = off_new_all + a.off_base;
  int* run = sh_run + (size_t)wib * (SL.max_cells + kMaskSlots);
  unsigned* msk = reinterpret_cast<unsigned*>(run + SL.max_cells);
  for (int i = lane; i < kMaskSlots; i += 32) msk[i] = 0u;
  const int* row = hist + a.hist_base + ((size_t)span * R + sub) * n_cells;
  for (int c = lane; c < n_cells; c += 32) run[c] = off_new[c] + row[c];
  __syncwarp();
  const int c0 = span * a.cps;
  const int c1 = min(c0 + a.cps, n_cells);
  const int sb0 = off_cur[c0], sb1 = off_cur[c1];
  const int mid = (R > 1) ? sb0 + ((sb1 - sb0) >> 1) : sb1;
  const int b0 = (sub == 0) ? sb0 : mid;
  const int b1 = (sub == 0) ? mid : sb1;
  const int lo = a.part_base, hi = a.part_base + a.n_part;  // the instance's slots
  const unsigned lt = (1u << lane) - 1u;
  bool bad = false;
  float4 ra[kScatterUnroll], rb[kScatterUnroll];
  load_batch(ra, P, b0, b1, lane);
  for (int base = b0; base < b1; base += 2 * kBatch2) {
    load_batch(rb, P, base + kBatch2, b1, lane);
    bad |= kMask ? place_batch_mask(ra, P2, run, msk, base, b1, n_cells, a.ncf, lo, hi, lane, lt)
                 : place_batch_match(ra, P2, run, base, b1, n_cells, a.ncf, lo, hi, lane, lt);
    if (base + kBatch2 >= b1) break;
    load_batch(ra, P, base + 2 * kBatch2, b1, lane);
    bad |= kMask ? place_batch_mask(rb, P2, run, msk, base + kBatch2, b1, n_cells, a.ncf, lo, hi,
                                    lane, lt)
                 : place_batch_match(rb, P2, run, base + kBatch2, b1, n_cells, a.ncf, lo, hi,
                                     lane, lt);
  }
  if (bad) atomicOr(err, kErrSort);
}

// One CTA of kCoopWarps warps per (span, row): the stable scatter of the row's records
// into the other buffer, kCoopWarps * 64 records per round.  In a round warp w takes the
// 64 consecutive records [base + 64 w, base + 64 w + 64) as two 32-record slices; a
// record's place is
//   run[cell]                      the cell's next slot after the earlier rounds,
// + sum over warps w' < w of       the round's records of w' bound for the same cell,
// + its rank among its warp's records bound for the same cell (__match_any_sync within
//   its slice, plus the first slice's count for a record of the second).
// Each warp publishes its per-cell counts in its own row of a table tagged with the
// round number (no clearing between rounds); after the places are taken, every warp
// adds its counts into run[].  All warps of the CTA work on one span at once: for
// short spans of small instances (a batch) this beats a warp per span, whose time is
// its span's ranking chain plus a pass over all of the instance's cells to set up run[].
// Shared memory: run[n_cells] and the table kCoopWarps x n_cells, so it is used while
// that leaves room for 4 CTAs per SM.
constexpr int kCoopWarps = 8;
constexpr size_t kCoopSmemMax = 48 * 1024;

template <bool kBatch, int kSlices>
__global__ void __launch_bounds__(kCoopWarps * 32)
    k_scatter_coop(const float4* __restrict__ P, float4* __restrict__ P2,
                   const int* __restrict__ off_cur_all, const int* __restrict__ off_new_all,
                   const int* __restrict__ hist, const InstParams one, const StepLaunch SL,
                   int* __restrict__ err) {
  extern __shared__ int sh_coop[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int R = SL.rows;
  const int gspan = blockIdx.x / R, sub = blockIdx.x - gspan * R;
  const InstParams& a = instance_of<kBatch>(one, SL, gspan);
  const int n_cells = a.n_cells;
  const int span = gspan - a.span_base;
  const int* __restrict__ off_cur = off_cur_all + a.off_base;
  const int* __restrict__ off_new = off_new_all + a.off_base;
  int* run = sh_coop;
  int* tab = sh_coop + n_cells;  // tab[w' * n_cells + c] = (round << 8) | count
  const int* row = hist + a.hist_base + ((size_t)span * R + sub) * n_cells;
  for (int c = threadIdx.x; c < n_cells; c += blockDim.x) run[c] = off_new[c] + row[c];
  for (int i = threadIdx.x; i < kCoopWarps * n_cells; i += blockDim.x) tab[i] = -1;
  const int c0 = span * a.cps;
  const int c1 = min(c0 + a.cps, n_cells);
  const int sb0 = off_cur[c0], sb1 = off_cur[c1];
  const int mid = (R > 1) ? sb0 + ((sb1 - sb0) >> 1) : sb1;
  const int b0 = (sub == 0) ? sb0 : mid;
  const int b1 = (sub == 0) ? mid : sb1;
  const int lo = a.part_base, hi = a.part_base + a.n_part;  // the instance's slots
  const unsigned lt = (1u << lane) - 1u;
  // A round: warp w takes the 32 kSlices records [base + 32 kSlices w, ...) as kSlices
  // slices of 32 (one record per lane each); two barriers per round.
  static_assert(kSlices == 1 || kSlices == 2, "one or two slices per warp and round");
  constexpr int kWarpRecs = 32 * kSlices;
  constexpr int kRound = kCoopWarps * kWarpRecs;
  constexpr int kAhead = 6 / kSlices;  // rounds of records in flight per lane (6 records)
  float4 r[kAhead][kSlices];
#pragma unroll
  for (int u = 0; u < kAhead; ++u)
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) {
      const int p = b0 + u * kRound + w * kWarpRecs + sl * 32 + lane;
      if (p < b1) r[u][sl] = P[p];
    }
  bool bad = false;
  int* tw = tab + w * n_cells;  // this warp's counts of the round, per cell
  __syncthreads();
  int round = 0;
  for (int base = b0; base < b1; base += kAhead * kRound) {
#pragma unroll
    for (int u = 0; u < kAhead; ++u, ++round) {
      const int rb = base + u * kRound;
      if (rb >= b1) break;  // uniform across the CTA
      const int pw = rb + w * kWarpRecs + lane;
      float4 rec[kSlices];
      int cell[kSlices], prev[kSlices];
      unsigned peers[kSlices];
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        const int p = pw + 32 * sl;
        rec[sl] = r[u][sl];
        // the record kAhead rounds later into this register
        if (p + kAhead * kRound < b1) r[u][sl] = P[p + kAhead * kRound];
        cell[sl] = (p < b1) ? cell_of(rec[sl].x, n_cells, a.ncf) : -1;
        peers[sl] = __match_any_sync(kFull, cell[sl]);
      }
      const int tag = round << 8;
      // the warp's count per cell, slice after slice: a slice's lanes find how many of the
      // earlier slices precede them in their cell, and its leaders store the running count
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        prev[sl] = 0;
        if (sl > 0) {
          __syncwarp();
          if (cell[sl] >= 0) {
            const int e = tw[cell[sl]];
            prev[sl] = ((e >> 8) == round) ? (e & 0xff) : 0;
          }
          __syncwarp();
        }
        if (cell[sl] >= 0 && (peers[sl] & lt) == 0u)
          tw[cell[sl]] = tag | (prev[sl] + __popc(peers[sl]));
      }
      __syncthreads();
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) {
        if (cell[sl] < 0) continue;
        int before = prev[sl] + __popc(peers[sl] & lt);
#pragma unroll
        for (int v = 0; v < kCoopWarps - 1; ++v) {
          if (v < w) {
            const int e = tab[v * n_cells + cell[sl]];
            if ((e >> 8) == round) before += e & 0xff;
          }
        }
        const int d = run[cell[sl]] + before;
        if (d >= lo && d < hi)
          P2[d] = rec[sl];
        else
          bad = true;
      }
      __syncthreads();
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl)
        if (cell[sl] >= 0 && (peers[sl] & lt) == 0u) atomicAdd(&run[cell[sl]], __popc(peers[sl]));
    }
  }
  if (bad) atomicOr(err, kErrSort);
}

// Per instance and cell c: row r of the sort matrix <- sum over rows r' < r (the spans
// before), count[c] <- total.  Block (32, 32): x = cell within a chunk of 32, y = one of
// 32 contiguous row segments; grid (cell chunks, instances).
template <bool kBatch>
__global__ void __launch_bounds__(1024)
    k_scan_spans(int* __restrict__ hist, int* __restrict__ count_all, const InstParams one,
                 const StepLaunch SL) {
  __shared__ int seg_tot[32][33];
  const InstParams& a = kBatch ? SL.tab[blockIdx.y] : one;
  const int n_cells = a.n_cells;
  if ((int)blockIdx.x * 32 >= n_cells) return;
  const int n_rows = a.n_spans * SL.rows;
  int* __restrict__ m = hist + a.hist_base;
  int* __restrict__ count = count_all + a.cell_base;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.x * 32 + tx;
  const int seg = (n_rows + 31) / 32;
  const int r0 = min(n_rows, ty * seg);
  const int r1 = min(n_rows, r0 + seg);
  int s = 0;
  if (c < n_cells) {
    int r = r0;
    for (; r + 8 <= r1; r += 8) {
      int v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = m[(size_t)(r + u) * n_cells + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; r < r1; ++r) s += m[(size_t)r * n_cells + c];
  }
  seg_tot[ty][tx] = s;
  __syncthreads();
  if (ty == 0) {
    int run = 0;
    for (int k = 0; k < 32; ++k) {
      const int v = seg_tot[k][tx];
      seg_tot[k][tx] = run;
      run += v;
    }
    if (c < n_cells) count[c] = run;
  }
  __syncthreads();
  if (c < n_cells) {
    int run = seg_tot[ty][tx];
    int r = r0;
    for (; r + 8 <= r1; r += 8) {
      int v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = m[(size_t)(r + u) * n_cells + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        m[(size_t)(r + u) * n_cells + c] = run;
        run += v[u];
      }
    }
    for (; r < r1; ++r) {
      const size_t i = (size_t)r * n_cells + c;
      const int v = m[i];
      m[i] = run;
      run += v;
    }
  }
}

// The same prefix for runs whose instances have at most kScanColsMaxRows rows (batches
// and pools of small instances): one thread per cell walks its column of the matrix, 32
// rows of loads in flight at a time; blocks of 64 cells, grid (cell chunks, instances).
// The block-per-32-cells kernel above would spend most of its 1,024 threads and its two
// CTA barriers on a handful of rows per instance (0.049 against 0.022 ms per step on the
// 256-instance batch).
constexpr int kScanColsMaxRows = 256;
constexpr int kScanColsCells = 64;
constexpr int kScanColsDepth = 32;

template <bool kBatch>
__global__ void __launch_bounds__(kScanColsCells)
    k_scan_cols(int* __restrict__ hist, int* __restrict__ count_all, const InstParams one,
                const StepLaunch SL) {
  const InstParams& a = kBatch ? SL.tab[blockIdx.y] : one;
  const int n_cells = a.n_cells;
  const int c = blockIdx.x * kScanColsCells + threadIdx.x;
  if (c >= n_cells) return;
  const int n_rows = a.n_spans * SL.rows;
  int* __restrict__ m = hist + a.hist_base + c;  // m[r n_cells]: row r of this column
  int run = 0;
  for (int r = 0; r < n_rows; r += kScanColsDepth) {
    int v[kScanColsDepth];
#pragma unroll
    for (int u = 0; u < kScanColsDepth; ++u)
      if (r + u < n_rows) v[u] = m[(size_t)(r + u) * n_cells];
#pragma unroll
    for (int u = 0; u < kScanColsDepth; ++u)
      if (r + u < n_rows) {
        m[(size_t)(r + u) * n_cells] = run;
        run += v[u];
      }
  }
  count_all[a.cell_base + c] = run;
}

// Per instance (one CTA each): off_new[c] = first global slot of cell c,
// off_new[n_cells] = end of the instance's slots.
template <bool kBatch>
__global__ void __launch_bounds__(1024)
    k_offsets_cells(const int* __restrict__ count_all, int* __restrict__ off_new_all,
                    const InstParams one, const StepLaunch SL) {
  __shared__ int part[1024];
  const InstParams& a = kBatch ? SL.tab[blockIdx.x] : one;
  const int n_cells = a.n_cells;
  const int* __restrict__ count = count_all + a.cell_base;
  int* __restrict__ offset = off_new_all + a.off_base;
  const int t = threadIdx.x;
  const int per = (n_cells + 1023) / 1024;
  const int cb = t * per;
  const int ce = min(n_cells, cb + per);
  int s = 0;
  for (int c = cb; c < ce; ++c) s += count[c];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {  // inclusive Hillis-Steele scan
    const int v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = a.part_base + (t > 0 ? part[t - 1] : 0);
  for (int c = cb; c < ce; ++c) {
    offset[c] = run;
    run += count[c];
  }
  if (t == 1023) offset[n_cells] = a.part_base + part[1023];
  // Graph replay: the step's collide/move pass has finished reading the step number.
  if (SL.gstep_dev != nullptr && blockIdx.x == 0 && t == 0) *SL.gstep_dev += 1;
}

// Both prefix passes in one launch for a single instance of at most kPrefixSmallCells
// cells and kScanColsMaxRows sort rows (a small run, whose step is launch-bound): one
// CTA, thread c walks cell c's column of the matrix (its exclusive prefix over the spans,
// 8 rows of loads in flight), then the CTA scans the cells' totals into the new offsets.
// (For a batch, a CTA per instance this way was slower than the two launches.)
constexpr int kPrefixSmallCells = 1024;

__global__ void __launch_bounds__(kPrefixSmallCells, 2)
    k_prefix_small(int* __restrict__ hist, int* __restrict__ off_new_all, const InstParams a,
                   const StepLaunch SL) {
  __shared__ int wsum[kPrefixSmallCells / 32];
  const int n_cells = a.n_cells;
  const int c = threadIdx.x;
  const int n_rows = a.n_spans * SL.rows;
  int run = 0;  // cell c's particles over all rows
  if (c < n_cells) {
    int* __restrict__ m = hist + a.hist_base + c;  // m[r n_cells]: row r of this column
    for (int r = 0; r < n_rows; r += 8) {
      int v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (r + u < n_rows) v[u] = m[(size_t)(r + u) * n_cells];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (r + u < n_rows) {
          m[(size_t)(r + u) * n_cells] = run;
          run += v[u];
        }
    }
  }
  // exclusive prefix of the totals over the cells: within each warp, then over warps
  const int lane = c & 31, w = c >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    const int x = wsum[lane];
    int y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, y, o);
      if (lane >= o) y += t;
    }
    wsum[lane] = y - x;
  }
  __syncthreads();
  const int excl = wsum[w] + incl - run;
  int* __restrict__ offset = off_new_all + a.off_base;
  if (c < n_cells) offset[c] = a.part_base + excl;
  if (c == n_cells - 1) offset[n_cells] = a.part_base + excl + run;
  // Graph replay: the step's collide/move pass has finished reading the step number.
  if (SL.gstep_dev != nullptr && c == 0) *SL.gstep_dev += 1;
}

bool prefix_small_fits(const StepLaunch& L) {
  return L.n_inst == 1 && L.max_cells <= kPrefixSmallCells &&
         (long long)L.max_spans * L.rows <= kScanColsMaxRows;
}

cudaError_t launch_prefix_small(int* hist, int* off_new, const InstParams& one,
                                const StepLaunch& L, cudaStream_t st) {
  k_prefix_small<<<1, kPrefixSmallCells, 0, st>>>(hist, off_new, one, L);
  return cudaGetLastError();
}

__global__ void k_set_counter(long long* counter, long long value) { *counter = value; }

__global__ void __launch_bounds__(256)
    k_admit_cells(const InstParams* __restrict__ tab, int* __restrict__ off_all,
                  float* __restrict__ smax_all, unsigned long long* __restrict__ ncand_all,
                  unsigned long long* __restrict__ nacc_all, double* __restrict__ acc_all) {
  const InstParams& a = tab[blockIdx.x];
  const int n_cells = a.n_cells;
  const int ppc = a.n_part / n_cells;
  int* off = off_all + a.off_base;
  for (int c = threadIdx.x; c <= n_cells; c += blockDim.x) off[c] = a.part_base + c * ppc;
  for (int c = threadIdx.x; c < n_cells; c += blockDim.x) {
    smax_all[a.cell_base + c] = a.smax0;
    ncand_all[a.cell_base + c] = 0ull;
    nacc_all[a.cell_base + c] = 0ull;
  }
  double* acc = acc_all + (size_t)a.cell_base * kNMom;
  for (int i = threadIdx.x; i < n_cells * kNMom; i += blockDim.x) acc[i] = 0.0;
}

__global__ void __launch_bounds__(256)
    k_channel_sums(const InstParams* __restrict__ tab, const double* __restrict__ acc_all,
                   double* __restrict__ out) {
  __shared__ double part[2][8];
  const InstParams& a = tab[blockIdx.x];
  const double* acc = acc_all + (size_t)a.cell_base * kNMom;
  double n = 0.0, u = 0.0;
  for (int c = threadIdx.x; c < a.n_cells; c += blockDim.x) {
    n += acc[(size_t)c * kNMom + 0];
    u += acc[(size_t)c * kNMom + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    u += __shfl_xor_sync(0xffffffffu, u, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    part[0][w] = n;
    part[1][w] = u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sn = 0.0, su = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      sn += part[0][k];
      su += part[1][k];
    }
    out[2 * a.id] = sn;
    out[2 * a.id + 1] = su;
  }
}

// Records <-> four arrays (y, vx, vy, vz), for the state accessors.
__global__ void k_unpack(const float4* __restrict__ P, float* __restrict__ y,
                         float* __restrict__ vx, float* __restrict__ vy, float* __restrict__ vz,
                         int N) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const float4 r = P[p];
    y[p] = r.x;
    vx[p] = r.y;
    vy[p] = r.z;
    vz[p] = r.w;
  }
}

// Pack four arrays into records; y is moved onto the nearest wall if outside [0, 1].
__global__ void k_pack(const float* __restrict__ y, const float* __restrict__ vx,
                       const float* __restrict__ vy, const float* __restrict__ vz,
                       float4* __restrict__ P, int N) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const float v = y[p];
    const float yc = (v >= 0.0f) ? ((v <= 1.0f) ? v : 1.0f) : 0.0f;
    P[p] = make_float4(yc, vx[p], vy[p], vz[p]);
  }
}

// ---------------------------------------------------------------------------

cudaError_t launch_collide_move(float4* P, const int* off, const float* smax_in,
                                float* smax_out, unsigned long long* ncand,
                                unsigned long long* nacc, double* acc, int* hist,
                                const InstParams& one, const StepLaunch& L, int* err,
                                cudaStream_t st) {
  const bool small = L.warps == kAWarpsSmall;
  const int warps = small ? kAWarpsSmall : kAWarps;
  const StepSmem S = step_smem_layout(L.max_cells, L.max_cps, L.max_cap, warps, L.rows);
  const dim3 block(warps * 32);
#define DSMC_COLLIDE(B, W, D)                                                       \
  k_collide_move<B, W, D><<<L.n_spans_total, block, S.total, st>>>(               \
      P, off, smax_in, smax_out, ncand, nacc, acc, hist, one, L, err)
#define DSMC_COLLIDE_SHAPE(B, D)   \
  do {                             \
    if (small)                     \
      DSMC_COLLIDE(B, kAWarpsSmall, D); \
    else                           \
      DSMC_COLLIDE(B, kAWarps, D); \
  } while (0)
  const bool f64 = L.accum == DSMC_ACCUM_FP64;
  if (L.n_inst == 1) {
    if (f64)
      DSMC_COLLIDE_SHAPE(false, true);
    else
      DSMC_COLLIDE_SHAPE(false, false);
  } else {
    if (f64)
      DSMC_COLLIDE_SHAPE(true, true);
    else
      DSMC_COLLIDE_SHAPE(true, false);
  }
#undef DSMC_COLLIDE_SHAPE
#undef DSMC_COLLIDE
  return cudaGetLastError();
}

int scatter_spans_warps(int n_cells) {
  size_t w = kStepSmemMax / ((size_t)(n_cells + kMaskSlots) * sizeof(int));
  if (w > (size_t)kBWarpsMax) w = kBWarpsMax;
  return w < 1 ? 1 : (int)w;
}

size_t scatter_coop_smem(int max_cells) {
  return (size_t)(kCoopWarps + 1) * (size_t)max_cells * sizeof(int);
}

cudaError_t launch_scatter_spans(const float4* P, float4* P2, const int* off_cur,
                                 const int* off_new, const int* hist, const InstParams& one,
                                 const StepLaunch& L, int* err, cudaStream_t st) {
  const size_t coop = scatter_coop_smem(L.max_cells);
  if (coop <= kCoopSmemMax) {  // a CTA per (span, row)
    const int units = L.n_spans_total * L.rows;
    // two slices per warp and round once the rows average 4,096 records (the batch's
    // tuned spans: 0.328 -> 0.30 ms); one for shorter rows (small runs' 1,024-particle
    // spans, where fewer, longer rounds were slower)
    const bool two = L.n_part_total >= 4096LL * units;
#define DSMC_COOP(B, S)                                                                  \
  k_scatter_coop<B, S><<<units, kCoopWarps * 32, coop, st>>>(P, P2, off_cur, off_new, hist, \
                                                             one, L, err)
    if (L.n_inst == 1) {
      if (two) DSMC_COOP(false, 2); else DSMC_COOP(false, 1);
    } else {
      if (two) DSMC_COOP(true, 2); else DSMC_COOP(true, 1);
    }
#undef DSMC_COOP
    return cudaGetLastError();
  }
  const int wpb = scatter_spans_warps(L.max_cells);
  const size_t smem = (size_t)wpb * (L.max_cells + kMaskSlots) * sizeof(int);
  const int units = L.n_spans_total * L.rows;
  const int blocks = (units + wpb - 1) / wpb;
  // the mask-table ranking once at least kMaskWarpsPerSm scatter warps share an SM
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool mask = units >= kMaskWarpsPerSm * sms;
#define DSMC_SCATTER(B, M)                                                                   \
  k_scatter_spans<B, M><<<blocks, wpb * 32, smem, st>>>(P, P2, off_cur, off_new, hist, one, L, \
                                                        err)
  if (L.n_inst == 1) {
    if (mask)
      DSMC_SCATTER(false, true);
    else
      DSMC_SCATTER(false, false);
  } else {
    if (mask)
      DSMC_SCATTER(true, true);
    else
      DSMC_SCATTER(true, false);
  }
#undef DSMC_SCATTER
  return cudaGetLastError();
}

cudaError_t launch_scan_spans(int* hist, int* count, const InstParams& one, const StepLaunch& L,
                              cudaStream_t st) {
  if ((long long)L.max_spans * L.rows <= kScanColsMaxRows) {
    const dim3 grid((L.max_cells + kScanColsCells - 1) / kScanColsCells, L.n_inst);
    if (L.n_inst == 1)
      k_scan_cols<false><<<grid, kScanColsCells, 0, st>>>(hist, count, one, L);
    else
      k_scan_cols<true><<<grid, kScanColsCells, 0, st>>>(hist, count, one, L);
    return cudaGetLastError();
  }
  const dim3 grid((L.max_cells + 31) / 32, L.n_inst);
  if (L.n_inst == 1)
    k_scan_spans<false><<<grid, dim3(32, 32), 0, st>>>(hist, count, one, L);
  else
    k_scan_spans<true><<<grid, dim3(32, 32), 0, st>>>(hist, count, one, L);
  return cudaGetLastError();
}

cudaError_t launch_offsets_cells(const int* count, int* off_new, const InstParams& one,
                                 const StepLaunch& L, cudaStream_t st) {
  if (L.n_inst == 1)
    k_offsets_cells<false><<<1, 1024, 0, st>>>(count, off_new, one, L);
  else
    k_offsets_cells<true><<<L.n_inst, 1024, 0, st>>>(count, off_new, one, L);
  return cudaGetLastError();
}

cudaError_t launch_set_counter(long long* counter, long long value, cudaStream_t st) {
  k_set_counter<<<1, 1, 0, st>>>(counter, value);
  return cudaGetLastError();
}

cudaError_t launch_admit_cells(const InstParams* tab, int n, int* off, float* smax,
                               unsigned long long* ncand, unsigned long long* nacc,
                               double* acc, cudaStream_t st) {
  k_admit_cells<<<n, 256, 0, st>>>(tab, off, smax, ncand, nacc, acc);
  return cudaGetLastError();
}

cudaError_t launch_channel_sums(const InstParams* tab, int n, const double* acc, double* out,
                                cudaStream_t st) {
  k_channel_sums<<<n, 256, 0, st>>>(tab, acc, out);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const float4* P, float* y, float* vx, float* vy, float* vz, int N,
                          cudaStream_t st) {
  const int blocks = (N + 255) / 256;
  k_unpack<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(P, y, vx, vy, vz, N);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* y, const float* vx, const float* vy, const float* vz,
                        float4* P, int N, cudaStream_t st) {
  const int blocks = (N + 255) / 256;
  k_pack<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(y, vx, vy, vz, P, N);
  return cudaGetLastError();
}

cudaError_t set_step_smem_limits(size_t a_bytes, size_t b_bytes) {
  const void* collide[8] = {(const void*)k_collide_move<false, kAWarps, false>,
                            (const void*)k_collide_move<true, kAWarps, false>,
                            (const void*)k_collide_move<false, kAWarpsSmall, false>,
                            (const void*)k_collide_move<true, kAWarpsSmall, false>,
                            (const void*)k_collide_move<false, kAWarps, true>,
                            (const void*)k_collide_move<true, kAWarps, true>,
                            (const void*)k_collide_move<false, kAWarpsSmall, true>,
                            (const void*)k_collide_move<true, kAWarpsSmall, true>};
  for (const void* f : collide) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)a_bytes);
    if (e != cudaSuccess) return e;
  }
  const void* scatter[8] = {(const void*)k_scatter_spans<false, false>,
                            (const void*)k_scatter_spans<false, true>,
                            (const void*)k_scatter_spans<true, false>,
                            (const void*)k_scatter_spans<true, true>,
                            (const void*)k_scatter_coop<false, 1>,
                            (const void*)k_scatter_coop<true, 1>,
                            (const void*)k_scatter_coop<false, 2>,
                            (const void*)k_scatter_coop<true, 2>};
  for (const void* f : scatter) {
    const cudaError_t e =
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b_bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dsmc
