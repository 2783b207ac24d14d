// dsmc_noalloc.cu -- a stable sort of particles into cells that never allocates.
//
// Some callers cannot allocate device memory at the moment they need this sort:
// code embedded in a host application or runtime that owns all device memory and
// hands its plug-ins no allocator, and latency-sensitive loops that must not call
// cudaMalloc/cudaFree, whose implicit device-wide synchronisation would stall every
// other stream.  dsmc_sort_cells_static serves them: the caller passes the input
// state, the output state and the cell offsets (all device memory), and the scratch
// the sort needs lives in a fixed array compiled into this library.
//
// The scratch array is file-scope device memory of kStaticScratchBytes (8 MiB).  Every
// GPU that loads the library holds it until the process exits, and every call on that
// GPU uses the same array: calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on it and give wrong results.
//
// Host code cannot use the array's name as a device address (on the host it is only a
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current, and later calls reuse it.  That
// first call should come before any stream capture on that device.
//
// A destination outside [0, n_particles) (which only inputs changing while the sort runs,
// such as an overlapping call, can produce) is never written: the scatter records it in
// the scratch's error word, and a last one-thread kernel turns a non-zero error word into
// offset_out[n_cells] = -1, which the caller reads with the outputs.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "dsmc.h"
#include "dsmc_internal.h"

constexpr size_t kStaticScratchBytes = 8u << 20;  // 8 MiB
constexpr size_t kStaticScratchInts = kStaticScratchBytes / sizeof(int);

// Layout of the scratch: [0, 64) error word and padding, [64, 64 + n_cells) per-cell
// totals, then the sort-partition histogram (n_warps x n_cells).
static __device__ __align__(256) int g_static_scratch[kStaticScratchInts];

// offset_out[n_cells] = -1 when a kernel of this sort recorded an error.
__global__ void k_flag_sort_error(const int* __restrict__ err, int* __restrict__ offset_out,
                                  int n_cells) {
  if (*err != 0) offset_out[n_cells] = -1;
}

namespace {

constexpr int kMaxDevices = 64;

// Do the byte ranges [a, a + na) and [b, b + nb) share a byte?
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

std::mutex g_setup_mutex;
int* g_scratch_addr[kMaxDevices] = {};

// The address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(int device, int** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[device] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<int*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

dsmc_status reject(dsmc_status s, const std::string& msg) {
  dsmc::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" dsmc_status dsmc_sort_cells_static(const float* y, const float* vx, const float* vy,
                                              const float* vz, float* y_out, float* vx_out,
                                              float* vy_out, float* vz_out, int* offset_out,
                                              int n_particles, int n_cells, void* stream) {
  using namespace dsmc;
  if (!y || !vx || !vy || !vz || !y_out || !vx_out || !vy_out || !vz_out || !offset_out)
    return reject(DSMC_E_INVAL, "dsmc_sort_cells_static: NULL pointer");
  if (n_particles < 1 || n_cells < 1)
    return reject(DSMC_E_INVAL, "dsmc_sort_cells_static: n_particles and n_cells must be >= 1");
  if ((long long)n_particles > kMaxParticles)
    return reject(DSMC_E_INVAL, "dsmc_sort_cells_static: n_particles must be <= 2^31 - 2^24");
  if ((size_t)n_cells * sizeof(int) > kSortSmemMax)
    return reject(DSMC_E_INVAL, "dsmc_sort_cells_static: n_cells must be <= 51200");
  // Every output must be disjoint from every input and from the other outputs: the
  // scatter writes outputs while other warps still read inputs.
  {
    const size_t fb = (size_t)n_particles * sizeof(float);
    const void* in[4] = {y, vx, vy, vz};
    const void* outp[5] = {y_out, vx_out, vy_out, vz_out, offset_out};
    const size_t outb[5] = {fb, fb, fb, fb, ((size_t)n_cells + 1) * sizeof(int)};
    for (int o = 0; o < 5; ++o) {
      for (int i = 0; i < 4; ++i)
        if (overlap(outp[o], outb[o], in[i], fb))
          return reject(DSMC_E_INVAL,
                        "dsmc_sort_cells_static: an output overlaps an input array");
      for (int o2 = 0; o2 < o; ++o2)
        if (overlap(outp[o], outb[o], outp[o2], outb[o2]))
          return reject(DSMC_E_INVAL,
                        "dsmc_sort_cells_static: two output arrays overlap");
    }
  }
  // Partition of the particles into warp spans: as many spans as the scratch holds
  // histogram rows for, at most the library's usual count.
  const size_t rows_fit = (kStaticScratchInts - 64 - (size_t)n_cells) / (size_t)n_cells;
  if (rows_fit < 1)
    return reject(DSMC_E_INVAL, "dsmc_sort_cells_static: n_cells exceeds the 8 MiB scratch");
  const long long N = n_particles;
  long long w = (N + 255) / 256;
  if (w > kSortWarpsMax) w = kSortWarpsMax;
  if (w > (long long)rows_fit) w = (long long)rows_fit;
  long long span = (N + w - 1) / w;
  span = (span + 31) & ~31LL;
  w = (N + span - 1) / span;
  long long wpb = (long long)(kSortSmemMax / (sizeof(int) * (size_t)n_cells));
  if (wpb > kSortWarpsPerBlock) wpb = kSortWarpsPerBlock;
  if (wpb > w) wpb = w;
  const SortPlan plan{(int)w, (int)span, (int)wpb};

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess)
    return reject(DSMC_E_CUDA, std::string("dsmc_sort_cells_static: cudaGetDevice: ") +
                              cudaGetErrorString(e));
  if (device < 0 || device >= kMaxDevices)
    return reject(DSMC_E_CUDA, "dsmc_sort_cells_static: device index " +
                                   std::to_string(device) + " is beyond the " +
                                   std::to_string(kMaxDevices) + " devices it keeps scratch "
                                   "addresses for");
  int* scratch = nullptr;
  e = scratch_address(device, &scratch);
  if (e != cudaSuccess)
    return reject(DSMC_E_CUDA, std::string("dsmc_sort_cells_static: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e));
  int* err = scratch;
  int* count = scratch + 64;
  int* hist = count + n_cells;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const float ncf = (float)n_cells;
  // The error word must start at zero; the histogram and totals are fully rewritten.
  e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = set_kernel_smem_limits(kSortSmemMax);
  const MoveArgs no_move{0.0f, 0.0f, 0u, 0u, 0u, 0};
  const DevState in{const_cast<float*>(y), const_cast<float*>(vx), const_cast<float*>(vy),
                    const_cast<float*>(vz)};
  const DevState out{y_out, vx_out, vy_out, vz_out};
  if (e == cudaSuccess)
    e = launch_move_count(in, n_particles, plan, n_cells, ncf, no_move, hist, err, st);
  if (e == cudaSuccess) e = launch_scan_hist(hist, plan.n_warps, n_cells, count, st);
  if (e == cudaSuccess) e = launch_cell_offsets(count, n_cells, offset_out, st);
  if (e == cudaSuccess)
    e = launch_scatter(in, out, n_particles, plan, n_cells, ncf, hist, offset_out, err, st);
  if (e == cudaSuccess) {
    k_flag_sort_error<<<1, 1, 0, st>>>(err, offset_out, n_cells);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return reject(DSMC_E_CUDA, std::string("dsmc_sort_cells_static: ") + cudaGetErrorString(e));
  return DSMC_OK;
}
