// dsmc_kernels.cu -- initial state and the stand-alone sort into cells of the DSMC of
// force-driven flow between parallel plates (arXiv 2311.14140, Sec. 2.1 problem,
// Bird's DSMC):
//
//   k_init            initial state: ppc particles per cell, uniform in the cell,
//                     velocity components N(0, 1/2) (gas at rest at the wall
//                     temperature, Sec. 2.1, units of Eq. 6)
//   k_move_count      (optional free flight,) new cell, warp-private histogram over
//                     fixed spans of slots
//   k_scan_hist       per cell, exclusive prefix of the histogram over partitions
//   k_cell_offsets    exclusive prefix over cells -> first slot of each cell
//   k_scatter         stable counting-sort scatter into the other buffer
// The two state passes of a step are in dsmc_step.cu.
//
// The resident state of a run is an array of float4 records (y, vx, vy, vz),
// double-buffered for the sort; k_init writes records.  k_move_count, k_scan_hist,
// k_cell_offsets and k_scatter serve only the allocation-free sort, whose caller owns
// four binary32 arrays (y, vx, vy, vz).  Kernel launches live in the host file;
// declarations are in dsmc_internal.h.
#include <climits>

#include "dsmc_device.cuh"
#include "dsmc_internal.h"

namespace dsmc {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Initial state, as float4 records (y, vx, vy, vz).
__global__ void k_init(float4* __restrict__ P, int N, int ppc, float ncf, uint32_t k0,
                       uint32_t k1, int* __restrict__ err) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int c = p / ppc;
    const uint32_t c3 = kStreamInit << 24;
    U4 w = philox((uint32_t)p, 0u, 0u, c3, k0, k1);
    const float y = fdiv(fadd((float)c, u01(w.x)), ncf);
    float z[3];
    int have = 0;
    for (int a = 0; a < kNormalAttempts && have < 3; ++a) {
      if ((a & 1) == 0) w = philox((uint32_t)p, 1u + (uint32_t)(a >> 1), 0u, c3, k0, k1);
      float z0, z1;
      const bool ok = (a & 1) ? polar_pair(w.z, w.w, z0, z1) : polar_pair(w.x, w.y, z0, z1);
      if (!ok) continue;
      z[have++] = z0;
      if (have < 3) z[have++] = z1;
    }
    if (have < 3) {
      atomicOr(err, kErrNormals);
      for (int i = have; i < 3; ++i) z[i] = 0.0f;
    }
    P[p] = make_float4(y, z[0], z[1], z[2]);
  }
}

// Flight (optional), cell index and a warp-private histogram over the warp's span of
// slots [w * span, (w+1) * span).  Dynamic shared memory: n_cells ints per warp.
__global__ void k_move_count(float* __restrict__ y, float* __restrict__ vx,
                             float* __restrict__ vy, float* __restrict__ vz, int N, int span,
                             int n_warps, int n_cells, float ncf, MoveArgs m,
                             int* __restrict__ hist, int* __restrict__ err) {
  extern __shared__ int sh_hist[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  if (gw >= n_warps) return;
  int* h = sh_hist + (size_t)wib * n_cells;
  for (int c = lane; c < n_cells; c += 32) h[c] = 0;
  __syncwarp();
  const int begin = gw * span;
  const int end = (int)min((long long)N, (long long)begin + span);
  bool bad = false;
  for (int base = begin; base < end; base += 32) {
    const int p = base + lane;
    const bool act = p < end;
    int cell = -1;
    if (act) {
      float yy = y[p];
      if (m.do_move) {
        float xx = vx[p], uy = vy[p], zz = vz[p];
        if (!fly(yy, xx, uy, zz, m.dt, m.F, m.k0, m.k1, m.step, (uint32_t)p)) bad = true;
        y[p] = yy;
        vx[p] = xx;
        vy[p] = uy;
        vz[p] = zz;
      }
      cell = cell_of(yy, n_cells, ncf);
    }
    const unsigned peers = __match_any_sync(kFull, cell);
    if (act && lane == __ffs(peers) - 1) h[cell] += __popc(peers);
    __syncwarp();
  }
  if (bad) atomicOr(err, kErrBounces);
  __syncwarp();
  int* out = hist + (size_t)gw * n_cells;
  for (int c = lane; c < n_cells; c += 32) out[c] = h[c];
}

// For each cell c: hist[w][c] <- sum_{w' < w} hist[w'][c]; count[c] <- total.
// Block (32, 32): x = cell within a chunk of 32 cells, y = one of 32 contiguous row
// segments; each pass keeps eight independent loads per thread in flight.
constexpr int kScanSegs = 32;
__global__ void __launch_bounds__(32 * kScanSegs)
    k_scan_hist(int* __restrict__ hist, int n_warps, int n_cells, int* __restrict__ count) {
  __shared__ int seg_tot[kScanSegs][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.x * 32 + tx;
  const int seg = (n_warps + kScanSegs - 1) / kScanSegs;
  const int r0 = min(n_warps, ty * seg);
  const int r1 = min(n_warps, r0 + seg);
  int s = 0;
  if (c < n_cells) {
    int r = r0;
    for (; r + 8 <= r1; r += 8) {
      int v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = hist[(size_t)(r + u) * n_cells + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; r < r1; ++r) s += hist[(size_t)r * n_cells + c];
  }
  seg_tot[ty][tx] = s;
  __syncthreads();
  if (ty == 0) {
    int run = 0;
    for (int k = 0; k < kScanSegs; ++k) {
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
      for (int u = 0; u < 8; ++u) v[u] = hist[(size_t)(r + u) * n_cells + c];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        hist[(size_t)(r + u) * n_cells + c] = run;
        run += v[u];
      }
    }
    for (; r < r1; ++r) {
      const size_t i = (size_t)r * n_cells + c;
      const int v = hist[i];
      hist[i] = run;
      run += v;
    }
  }
}

// offset[c] = sum_{c' < c} count[c'], offset[n_cells] = N.  One CTA of 1024 threads.
__global__ void k_cell_offsets(const int* __restrict__ count, int n_cells,
                               int* __restrict__ offset) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n_cells + 1023) / 1024;
  const int c0 = t * per;
  const int c1 = min(n_cells, c0 + per);
  int s = 0;
  for (int c = c0; c < c1; ++c) s += count[c];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {  // inclusive Hillis-Steele scan
    const int v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = t > 0 ? part[t - 1] : 0;
  for (int c = c0; c < c1; ++c) {
    offset[c] = run;
    run += count[c];
  }
  if (t == 1023) offset[n_cells] = part[1023];
}

// Stable scatter: slot p of the warp's span goes to offset[cell] + (particles of the
// same cell in earlier spans) + (earlier particles of the same cell in this span).
__global__ void k_scatter(const float* __restrict__ y, const float* __restrict__ vx,
                          const float* __restrict__ vy, const float* __restrict__ vz,
                          float* __restrict__ y2, float* __restrict__ vx2,
                          float* __restrict__ vy2, float* __restrict__ vz2, int N, int span,
                          int n_warps, int n_cells, float ncf, const int* __restrict__ hist,
                          const int* __restrict__ offset, int* __restrict__ err) {
  extern __shared__ int sh_run[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
  if (gw >= n_warps) return;
  int* run = sh_run + (size_t)wib * n_cells;
  const int* base_row = hist + (size_t)gw * n_cells;
  for (int c = lane; c < n_cells; c += 32) run[c] = offset[c] + base_row[c];
  __syncwarp();
  const int begin = gw * span;
  const int end = (int)min((long long)N, (long long)begin + span);
  const unsigned lt = (1u << lane) - 1u;
  for (int b = begin; b < end; b += 32) {
    const int p = b + lane;
    const bool act = p < end;
    float yy = 0.f, xx = 0.f, uy = 0.f, zz = 0.f;
    int cell = -1;
    if (act) {
      yy = y[p];
      xx = vx[p];
      uy = vy[p];
      zz = vz[p];
      cell = cell_of(yy, n_cells, ncf);
    }
    const unsigned peers = __match_any_sync(kFull, cell);
    const int first = act ? run[cell] : 0;
    __syncwarp();
    if (act && lane == __ffs(peers) - 1) run[cell] = first + __popc(peers);
    __syncwarp();
    if (act) {
      const int d = first + __popc(peers & lt);
      if (d >= 0 && d < N) {
        y2[d] = yy;
        vx2[d] = xx;
        vy2[d] = uy;
        vz2[d] = zz;
      } else {
        atomicOr(err, kErrSort);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers.

cudaError_t launch_init(float4* P, int N, int ppc, float ncf, uint32_t k0, uint32_t k1,
                        int* err, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (N + threads - 1) / threads;
  k_init<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(P, N, ppc, ncf, k0, k1, err);
  return cudaGetLastError();
}

cudaError_t launch_move_count(const DevState& s, int N, const SortPlan& sp, int n_cells,
                              float ncf, const MoveArgs& m, int* hist, int* err,
                              cudaStream_t st) {
  const size_t smem = (size_t)sp.wpb * n_cells * sizeof(int);
  const int blocks = (sp.n_warps + sp.wpb - 1) / sp.wpb;
  k_move_count<<<blocks, sp.wpb * 32, smem, st>>>(s.y, s.vx, s.vy, s.vz, N, sp.span,
                                                  sp.n_warps, n_cells, ncf, m, hist, err);
  return cudaGetLastError();
}

cudaError_t launch_scan_hist(int* hist, int n_warps, int n_cells, int* count, cudaStream_t st) {
  const int blocks = (n_cells + 31) / 32;
  k_scan_hist<<<blocks, dim3(32, kScanSegs), 0, st>>>(hist, n_warps, n_cells, count);
  return cudaGetLastError();
}

cudaError_t launch_cell_offsets(const int* count, int n_cells, int* offset, cudaStream_t st) {
  k_cell_offsets<<<1, 1024, 0, st>>>(count, n_cells, offset);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const DevState& from, const DevState& to, int N, const SortPlan& sp,
                           int n_cells, float ncf, const int* hist, const int* offset,
                           int* err, cudaStream_t st) {
  const size_t smem = (size_t)sp.wpb * n_cells * sizeof(int);
  const int blocks = (sp.n_warps + sp.wpb - 1) / sp.wpb;
  k_scatter<<<blocks, sp.wpb * 32, smem, st>>>(from.y, from.vx, from.vy, from.vz, to.y, to.vx,
                                               to.vy, to.vz, N, sp.span, sp.n_warps, n_cells,
                                               ncf, hist, offset, err);
  return cudaGetLastError();
}

cudaError_t set_kernel_smem_limits(size_t sort_bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_move_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sort_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sort_bytes);
}

}  // namespace dsmc
