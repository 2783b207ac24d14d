// dsmc_internal.h -- declarations shared by the kernel file and the C-ABI host file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dsmc.h"

#include <string>

namespace dsmc {

constexpr int kNMom = 13;          // raw moment sums per cell
constexpr int kMaxGroup = 512;     // largest collision group size G
constexpr int kAWarps = 8;         // warps per CTA of the collide/move pass (default)
constexpr int kAWarpsSmall = 4;    // the other CTA shape the tuner may choose
constexpr int kMaxSpanRows = 2;    // rows of the sort matrix per span (halves of its slots)
// Warps (spans) per CTA of the span scatter.  Small CTAs spread the spans evenly over the
// SMs: 2,000 one-warp spans as 4-warp CTAs leave 44 SMs with 16 warps and the rest with
// 12, and the SMs with 16 set the kernel's time (0.355 ms against 0.339 ms with 2-warp CTAs).
constexpr int kBWarpsMax = 2;
constexpr int kMaxStepCells = 16384;
constexpr int kMaxSpans = 152 * 16;   // rows of the per-step sort matrix, at most
// At most 24 cells per span: the CTA's per-cell slots stay small (at 4,096-particle spans
// the batch of small instances keeps 5 CTAs per SM), 4 % faster than 256 on the batch.
constexpr int kMaxCellsPerSpan = 24;
constexpr size_t kStepSmemMax = 220 * 1024;
constexpr int kSortWarpsMax = 152 * 16;
constexpr int kSortWarpsPerBlock = 8;
constexpr size_t kSortSmemMax = 200 * 1024;

// Device error word bits.
constexpr int kErrNormals = 1;  // Gaussian attempts ran out
constexpr int kErrBounces = 2;  // wall bounce limit
constexpr int kErrSphere = 4;   // reserved (the post-collision direction draw cannot fail)
constexpr int kErrCandidates = 8;  // a group's candidate count exceeded kMaxCandidates
constexpr int kErrSort = 16;       // a scatter destination fell outside [0, N)
constexpr int kErrCopyTimeout = 32;  // a bulk copy into shared memory did not complete
constexpr int kErrInflow = 64;       // an open-boundary emission ran out of attempts
constexpr int kErrMoments = 128;     // a group's moment total exceeded the fixed-point range

// Largest NTC candidate count of one group in one step (about 80 on the largest
// workload): anything above means corrupted (sigma g)_max and is skipped.
constexpr float kMaxCandidates = 1.0e7f;
// Particle count limit: keeps every slot index and loop bound inside int.
constexpr long long kMaxParticles = (1LL << 31) - (1LL << 24);

struct DevState {
  float* y;
  float* vx;
  float* vy;
  float* vz;
};

// Partition of the slots for the two sort passes: warp w owns
// [w * span, min(N, (w+1) * span)); wpb warps per CTA.
struct SortPlan {
  int n_warps;
  int span;
  int wpb;
};

struct MoveArgs {
  float dt;
  float F;
  uint32_t k0, k1;  // Philox key (seed)
  uint32_t step;
  int do_move;
};

// The round keys of Philox4x32-10 for one key: round r uses (k0 + r W0, k1 + r W1).
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

// One simulation instance as the step kernels see it.  A run holds one or more
// instances; their particles, cells, spans and sort matrices are concatenated, and the
// fields below place instance i in those arrays.  Random numbers are keyed on the
// instance's own seed, step, local cell and local slot, so an instance evolves the
// same alone and in a batch.
struct InstParams {
  // placement in the concatenated arrays
  int n_cells;
  int cell_base;   // first index of the instance in per-cell arrays
  int off_base;    // first index in the cell-offset arrays (n_cells + 1 entries)
  int span_base;   // first global span
  int n_spans;
  int cps;         // cells per span (one collide/move CTA each)
  int part_base;   // first global slot of the instance's particles
  int n_part;
  long long hist_base;  // first entry of the instance's sort matrix (n_spans x n_cells)
  // method parameters, binary32 as the kernels use them
  int G;
  int cap;  // largest group: G + G/2 - 1
  float ncf;
  float dt, F;
  float coef;              // n sigma_ref dt / (2 ppc)
  float cvhs, vexp, vinv;  // VHS factor, exponent 2 - 2 omega and its inverse
  float lncv;              // ln cvhs
  float lg2cv;             // log2 cvhs (for the bracketing approximation of the threshold)
  uint32_t k0, k1;         // Philox key (seed)
  PhiloxKeys keys;         // the ten round keys of that key
  long long step0;         // the instance's step k runs at global step step0 + k
  long long sample_start;  // instance steps >= sample_start are sampled
  int collide;
  int mode;     // 0 hard spheres, 1 VHS (0.5 < omega < 1), 2 omega = 1
  int id;       // the instance's id in its handle
  float smax0;  // initial (sigma g)_max / sigma_ref of every cell
  int open_top;        // 1: y = 1 is an open Chapman-Enskog interface
  float u_top, p_top;  // its bulk velocity and shear stress
};

// Dynamic shared memory of one collide/move CTA (byte offsets).
struct StepSmem {
  size_t hist, cell_acc, cell_cand, cell_accn, cell_gmax, cell_groups, cell_start, cell_smax,
      warps, per_warp, total;
  size_t w_rec, w_own, w_bar;  // offsets inside one warp's area
};

__host__ __device__ inline size_t step_align(size_t o, size_t a) { return (o + a - 1) / a * a; }

__host__ __device__ inline StepSmem step_smem_layout(int n_cells, int cps, int cap,
                                                     int warps = kAWarps, int rows = 1) {
  StepSmem L;
  size_t o = 0;
  L.hist = o;
  o = step_align(o + (size_t)rows * n_cells * 4, 8);
  L.cell_acc = o;
  o += (size_t)cps * kNMom * 8;
  L.cell_cand = o;
  o += (size_t)cps * 8;
  L.cell_accn = o;
  o += (size_t)cps * 8;
  L.cell_gmax = o;
  o += (size_t)cps * 4;
  L.cell_groups = o;  // group prefix of the span's cells (cps + 1) and a counter
  o += ((size_t)cps + 2) * 4;
  L.cell_start = o;  // first slot of each of the span's cells and the end (cps + 1)
  o += ((size_t)cps + 1) * 4;
  L.cell_smax = o;  // (sigma g)_max of the span's cells at the step's start
  o = step_align(o + (size_t)cps * 4, 128);
  // per warp: the group's records (cap float4, written by a bulk copy), an owner word
  // per particle (reused as the queue of wall hits), and an mbarrier
  size_t w = 0;
  L.w_rec = w;
  w += (size_t)cap * 16;
  L.w_own = w;
  w = step_align(w + (size_t)cap * 4, 8);
  L.w_bar = w;
  w += 8;
  L.per_warp = step_align(w, 128);
  L.warps = o;
  o += (size_t)warps * L.per_warp;
  L.total = o;
  return L;
}

cudaError_t launch_init(float4* P, int N, int ppc, float ncf, uint32_t k0, uint32_t k1,
                        int* err, cudaStream_t st);
int scatter_spans_warps(int n_cells);

// Sort into cells over fixed spans of slots, four separate arrays (the
// allocation-free sort); the prefix kernels are also used by every step.
cudaError_t launch_move_count(const DevState& s, int N, const SortPlan& sp, int n_cells,
                              float ncf, const MoveArgs& m, int* hist, int* err,
                              cudaStream_t st);
cudaError_t launch_scan_hist(int* hist, int n_warps, int n_cells, int* count, cudaStream_t st);
cudaError_t launch_cell_offsets(const int* count, int n_cells, int* offset, cudaStream_t st);
cudaError_t launch_scatter(const DevState& from, const DevState& to, int N, const SortPlan& sp,
                           int n_cells, float ncf, const int* hist, const int* offset,
                           int* err, cudaStream_t st);
cudaError_t set_kernel_smem_limits(size_t sort_bytes);

// The two state passes of a step (float4 records).  With one instance the
// parameters travel as a kernel argument; with several, kernels read the run's
// instance table in device memory, finding a span's instance through span_inst.
struct StepLaunch {
  int n_inst;
  const InstParams* tab;  // device, n_inst entries (batched launches)
  const int* span_inst;   // device, one entry per global span (batched launches)
  const int* span_order;  // device or NULL: collide/move CTA b takes span span_order[b]
  int n_spans_total;
  int max_cells;         // largest n_cells of the instances
  int max_spans;         // largest n_spans of the instances
  long long n_part_total;  // particles of all the launch's instances
  int max_cps;
  int max_cap;
  int warps;             // warps per CTA of the collide/move pass (kAWarps or kAWarpsSmall)
  int rows;              // sort-matrix rows per span, 1 or kMaxSpanRows: row r counts the
                         // particles of the r-th half of the span's slots, and the scatter
                         // gives each row its own warp
  long long gstep;       // global step number
  long long* gstep_dev;  // non-NULL (graph replay): read the step number here instead;
                         // the cell-offset kernel advances it at the end of the step
  int count_only;
  int accum;  // DSMC_ACCUM_FP32 or DSMC_ACCUM_FP64: per-lane moment sums
};
cudaError_t launch_cell_fields(const double* acc, int n_cells, long long n_samples, int ppc,
                               double* out, cudaStream_t st);
cudaError_t launch_collide_move(float4* P, const int* off, const float* smax_in,
                                float* smax_out, unsigned long long* ncand,
                                unsigned long long* nacc, double* acc, int* hist,
                                const InstParams& one, const StepLaunch& L, int* err,
                                cudaStream_t st);
cudaError_t launch_scatter_spans(const float4* P, float4* P2, const int* off_cur,
                                 const int* off_new, const int* hist, const InstParams& one,
                                 const StepLaunch& L, int* err, cudaStream_t st);
cudaError_t launch_scan_spans(int* hist, int* count, const InstParams& one, const StepLaunch& L,
                              cudaStream_t st);
cudaError_t launch_offsets_cells(const int* count, int* off_new, const InstParams& one,
                                 const StepLaunch& L, cudaStream_t st);
// Both prefix passes as one launch, when prefix_small_fits(L) (one instance, few cells
// and rows).
bool prefix_small_fits(const StepLaunch& L);
cudaError_t launch_prefix_small(int* hist, int* off_new, const InstParams& one,
                                const StepLaunch& L, cudaStream_t st);
cudaError_t launch_set_counter(long long* counter, long long value, cudaStream_t st);
// Per-cell arrays of newly added instances (table `tab`, n of them): moment sums and
// collision counters zeroed, (sigma g)_max set to smax0, and cell offsets of whole
// cells of ppc = n_part / n_cells particles starting at part_base.
cudaError_t launch_admit_cells(const InstParams* tab, int n, int* off, float* smax,
                               unsigned long long* ncand, unsigned long long* nacc,
                               double* acc, cudaStream_t st);
// Per instance of `tab` (n of them): the sums over its cells of the sampled particle
// count and of vx, into out[2 id] and out[2 id + 1].
cudaError_t launch_channel_sums(const InstParams* tab, int n, const double* acc, double* out,
                                cudaStream_t st);
cudaError_t launch_unpack(const float4* P, float* y, float* vx, float* vy, float* vz, int N,
                          cudaStream_t st);
cudaError_t launch_pack(const float* y, const float* vx, const float* vy, const float* vz,
                        float4* P, int N, cudaStream_t st);
cudaError_t set_step_smem_limits(size_t a_bytes, size_t b_bytes);

// Sets the message dsmc_last_error() returns on the calling thread.
void set_last_error(const std::string& msg);

}  // namespace dsmc
