// dsmc_internal.h -- declarations shared by the kernel file and the C-ABI host file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace dsmc {

constexpr int kNMom = 13;          // raw moment sums per cell
constexpr int kCollideWarps = 4;   // warps (concurrent groups) per collision CTA
constexpr int kMaxGroup = 512;     // largest collision group size G
constexpr int kSortWarpsMax = 152 * 16;
constexpr int kSortWarpsPerBlock = 8;
constexpr size_t kSortSmemMax = 200 * 1024;

// Device error word bits.
constexpr int kErrNormals = 1;  // Gaussian attempts ran out
constexpr int kErrBounces = 2;  // wall bounce limit
constexpr int kErrSphere = 4;   // post-collision direction attempts ran out
constexpr int kErrCandidates = 8;  // a group's candidate count exceeded kMaxCandidates
constexpr int kErrSort = 16;       // a scatter destination fell outside [0, N)

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

struct CollideArgs {
  int G;
  int cap;  // largest group: G + G/2 - 1
  float coef;
  float cvhs;
  float vexp;
  uint32_t k0, k1;
  uint32_t step;
  int sample;
  int collide;
};

cudaError_t launch_init(const DevState& s, int N, int ppc, float ncf, uint32_t k0, uint32_t k1,
                        int* err, cudaStream_t st);
cudaError_t launch_move_count(const DevState& s, int N, const SortPlan& sp, int n_cells,
                              float ncf, const MoveArgs& m, int* hist, int* err,
                              cudaStream_t st);
cudaError_t launch_scan_hist(int* hist, int n_warps, int n_cells, int* count, cudaStream_t st);
cudaError_t launch_cell_offsets(const int* count, int n_cells, int* offset, cudaStream_t st);
cudaError_t launch_scatter(const DevState& from, const DevState& to, int N, const SortPlan& sp,
                           int n_cells, float ncf, const int* hist, const int* offset,
                           int* err, cudaStream_t st);
size_t collide_smem_bytes(int cap);
cudaError_t launch_collide_sample(const DevState& s, int n_cells, const int* offset,
                                  const float* smax_in, float* smax_out,
                                  unsigned long long* ncand, unsigned long long* nacc,
                                  double* acc, const CollideArgs& a, bool vhs, int* err,
                                  cudaStream_t st);
cudaError_t launch_clamp_y(float* y, int N, cudaStream_t st);
cudaError_t set_kernel_smem_limits(size_t sort_bytes, size_t collide_bytes);

// Sets the message dsmc_last_error() returns on the calling thread.
void set_last_error(const std::string& msg);

}  // namespace dsmc
