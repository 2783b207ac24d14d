// dsmc_step.cu -- the two state passes of one DSMC step (Bird's method, which the
// paper cites for its micro model; problem of Sec. 2.1, units of Eq. 5):
//
//   k_collide_move   one CTA per span of consecutive cells.  Each warp takes the
//                    span's collision groups in turn, stages a group's velocities in
//                    shared memory and
//                      1. adds the group's moment sums taken before the collisions,
//                      2. draws every NTC candidate's pair, acceptance threshold and
//                         scattering direction up front (32 candidates at a time,
//                         one per lane), then applies the candidates in conflict-free
//                         rounds that reproduce the sequential order exactly,
//                      3. adds the moment sums taken after the collisions,
//                      4. moves each particle (body force, diffuse walls) and counts
//                         its new cell into the CTA's histogram,
//                    writing the moved state back in place.  The histogram becomes the
//                    span's row of the sort matrix; per-cell (sigma g)_max, collision
//                    counters and moment sums are written by the one CTA that owns
//                    the cell.
//   k_scatter_spans  one warp per span: re-reads the moved state in slot order and
//                    scatters it, stably, into the other buffer, using the span's row
//                    of the prefix-summed matrix plus the new cell offsets.
//
// Between them, k_scan_hist and k_cell_offsets (dsmc_kernels.cu) turn the matrix into
// per-span bases and the new cell offsets.
#include <climits>

#include "dsmc_device.cuh"
#include "dsmc_internal.h"

namespace dsmc {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFlushEvery = 4;  // groups per lane-accumulator flush (bounds FP32 chains)

// Scattering direction from one polar attempt (Marsaglia 1972): (a0, a1) uniform in
// the unit disc gives n = (2 a0 sqrt(1-s), 2 a1 sqrt(1-s), 1 - 2 s), uniform on the
// sphere.
__device__ __forceinline__ bool sphere(uint32_t w0, uint32_t w1, float& nx, float& ny,
                                       float& nz) {
  const float a0 = s11(w0);
  const float a1 = s11(w1);
  const float sq = fadd(fmul(a0, a0), fmul(a1, a1));
  if (sq >= 1.0f) return false;
  const float q = fmul(2.0f, fsqrt(fsub(1.0f, sq)));
  nx = fmul(a0, q);
  ny = fmul(a1, q);
  nz = fsub(1.0f, fmul(2.0f, sq));
  return true;
}

// Add one group's 13 raw moment sums (products in binary32, as the oracle forms them)
// to this lane's column of the warp's accumulators.
__device__ __forceinline__ void sample_group(float* lacc, const float* sx, const float* sy,
                                             const float* sz, int gn, int lane) {
  float m[kNMom];
#pragma unroll
  for (int k = 0; k < kNMom; ++k) m[k] = 0.0f;
  for (int i = lane; i < gn; i += 32) {
    const float x = sx[i], y = sy[i], z = sz[i];
    const float xx = fmul(x, x), yy = fmul(y, y), zz = fmul(z, z);
    const float v2 = fadd(fadd(xx, yy), zz);
    m[0] += 1.0f;
    m[1] += x;
    m[2] += y;
    m[3] += z;
    m[4] += xx;
    m[5] += yy;
    m[6] += zz;
    m[7] += fmul(x, y);
    m[8] += fmul(x, z);
    m[9] += fmul(y, z);
    m[10] += fmul(x, v2);
    m[11] += fmul(y, v2);
    m[12] += fmul(z, v2);
  }
#pragma unroll
  for (int k = 0; k < kNMom; ++k) lacc[k * 32 + lane] += m[k];
}

// Warp sum of the lane accumulators, added (times 1/2: half a sample before and half
// after the collisions) to the CTA's binary64 sums of one cell; accumulators cleared.
__device__ __forceinline__ void flush_moments(float* lacc, double* cell_acc, int lane) {
#pragma unroll
  for (int k = 0; k < kNMom; ++k) {
    float v = lacc[k * 32 + lane];
    lacc[k * 32 + lane] = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) atomicAdd(&cell_acc[k], 0.5 * (double)v);
  }
}

}  // namespace

// Modes of the collision model: 0 hard spheres, 1 VHS with 0.5 < omega < 1,
// 2 omega = 1 (sigma g independent of g).
template <int kMode>
__global__ void __launch_bounds__(kAWarps * 32, 2)
    k_collide_move(float* __restrict__ y, float* __restrict__ vx, float* __restrict__ vy,
                   float* __restrict__ vz, const int* __restrict__ off,
                   const float* __restrict__ smax_in, float* __restrict__ smax_out,
                   unsigned long long* __restrict__ ncand, unsigned long long* __restrict__ nacc,
                   double* __restrict__ acc, int* __restrict__ hist, StepArgs a,
                   int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_cells = a.n_cells;
  const int cps = a.cps;
  const int cap = a.cap;
  const int G = a.G;
  const StepSmem L = step_smem_layout(n_cells, cps, cap);
  int* h = reinterpret_cast<int*>(smem + L.hist);
  double* cacc = reinterpret_cast<double*>(smem + L.cell_acc);
  unsigned long long* ccand = reinterpret_cast<unsigned long long*>(smem + L.cell_cand);
  unsigned long long* caccn = reinterpret_cast<unsigned long long*>(smem + L.cell_accn);
  unsigned* cgmax = reinterpret_cast<unsigned*>(smem + L.cell_gmax);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* wmem = smem + L.warps + (size_t)wib * L.per_warp;
  float* sx = reinterpret_cast<float*>(wmem);
  float* sy = sx + cap;
  float* sz = sy + cap;
  int* own = reinterpret_cast<int*>(sz + cap);
  float* lacc = reinterpret_cast<float*>(own + cap);  // kNMom x 32

  const int span = blockIdx.x;
  const int c0 = span * cps;
  const int c1 = min(c0 + cps, n_cells);
  for (int i = threadIdx.x; i < n_cells; i += blockDim.x) h[i] = 0;
  for (int i = threadIdx.x; i < cps * kNMom; i += blockDim.x) cacc[i] = 0.0;
  for (int i = threadIdx.x; i < cps; i += blockDim.x) {
    ccand[i] = 0;
    caccn[i] = 0;
    cgmax[i] = 0u;
  }
  for (int k = 0; k < kNMom; ++k) lacc[k * 32 + lane] = 0.0f;
  __syncthreads();

  bool bad_bounce = false, sphere_fail = false, cand_fail = false;
  const unsigned lt = (1u << lane) - 1u;
  int qbase = 0;  // groups of the span before cell c
  for (int c = c0; c < c1; ++c) {
    const int start = off[c];
    const int nc = off[c + 1] - start;
    const int ng = group_count(nc, G);
    const float smax = smax_in[c];
    float gmax = 0.0f;
    unsigned long long lcand = 0, laccn = 0;
    int pending_flush = 0;
    // This warp takes the groups q of the span with q = wib (mod kAWarps).
    const int gi0 = ((wib - qbase) % kAWarps + kAWarps) % kAWarps;
    for (int gi = gi0; gi < ng; gi += kAWarps) {
      const int gs = start + gi * G;
      const int gn = (gi == ng - 1) ? nc - gi * G : G;
      for (int i = lane; i < gn; i += 32) {
        sx[i] = vx[gs + i];
        sy[i] = vy[gs + i];
        sz[i] = vz[gs + i];
        own[i] = INT_MAX;
      }
      __syncwarp();
      if (a.sample) sample_group(lacc, sx, sy, sz, gn, lane);

      if (a.collide && gn >= 2) {
        const uint32_t c3 = (kStreamColl << 24) | ((uint32_t)gi << 4);
        const float t1 = fmul((float)(gn - 1), (float)nc);
        const float mf = fmul(fmul(t1, a.coef), smax);
        const float fl = floorf(mf);
        const float frac = fsub(mf, fl);
        uint32_t M = (uint32_t)fl;
        const U4 r = philox(0xffffffffu, (uint32_t)c, a.step, c3, a.k0, a.k1);
        if (u01(r.x) < frac) M += 1;
        if (!(mf <= kMaxCandidates)) {
          M = 0;
          cand_fail = true;
        }
        lcand += M;
        for (uint32_t kb = 0; kb < M; kb += 32) {
          const uint32_t k = kb + (uint32_t)lane;
          bool pend = k < M;
          int i = 0, j = 0;
          float thr = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;
          bool have_dir = false;
          if (pend) {
            const U4 w = philox(k, (uint32_t)c, a.step, c3, a.k0, a.k1);
            i = (int)__umulhi(w.x, (uint32_t)gn);
            j = (int)__umulhi(w.y, (uint32_t)(gn - 1));
            j += (j >= i) ? 1 : 0;
            const float us = fmul(u01(w.z), smax);
            if (kMode == 0)
              thr = us;
            else if (kMode == 1)
              thr = exp32(fmul(a.vinv, ln32(fdiv(us, a.cvhs))));
            else
              thr = (us < a.cvhs) ? -1.0f : __int_as_float(0x7f800000);
            const U4 d = philox(k, (uint32_t)c, a.step, c3 | 1u, a.k0, a.k1);
            have_dir = sphere(d.x, d.y, nx, ny, nz) || sphere(d.z, d.w, nx, ny, nz);
          }
          if (__any_sync(kFull, pend && !have_dir)) {
            // Rare: both attempts of the first draw fell outside the disc.
            for (int at = 2; at < kNormalAttempts && pend && !have_dir; at += 2) {
              const U4 d = philox(k, (uint32_t)c, a.step, c3 | (1u + (uint32_t)(at >> 1)),
                                  a.k0, a.k1);
              have_dir = sphere(d.x, d.y, nx, ny, nz) || sphere(d.z, d.w, nx, ny, nz);
            }
          }
          while (__any_sync(kFull, pend)) {
            if (pend) {
              atomicMin(&own[i], lane);
              atomicMin(&own[j], lane);
            }
            __syncwarp();
            const bool ready = pend && own[i] == lane && own[j] == lane;
            __syncwarp();
            if (pend) {
              own[i] = INT_MAX;
              own[j] = INT_MAX;
            }
            if (ready) {
              const float xi = sx[i], yi = sy[i], zi = sz[i];
              const float xj = sx[j], yj = sy[j], zj = sz[j];
              const float gx = fsub(xi, xj), gy = fsub(yi, yj), gz = fsub(zi, zj);
              const float g = fsqrt(fadd(fadd(fmul(gx, gx), fmul(gy, gy)), fmul(gz, gz)));
              gmax = fmaxf(gmax, g);
              if (g > thr) {
                if (have_dir) {
                  const float hg = fmul(0.5f, g);
                  const float cx = fmul(fadd(xi, xj), 0.5f);
                  const float cy = fmul(fadd(yi, yj), 0.5f);
                  const float cz = fmul(fadd(zi, zj), 0.5f);
                  const float dx = fmul(hg, nx), dy = fmul(hg, ny), dz = fmul(hg, nz);
                  sx[i] = fadd(cx, dx);
                  sy[i] = fadd(cy, dy);
                  sz[i] = fadd(cz, dz);
                  sx[j] = fsub(cx, dx);
                  sy[j] = fsub(cy, dy);
                  sz[j] = fsub(cz, dz);
                  laccn += 1;
                } else {
                  sphere_fail = true;
                }
              }
              pend = false;
            }
            __syncwarp();
          }
        }
      }
      __syncwarp();
      if (a.sample) {
        sample_group(lacc, sx, sy, sz, gn, lane);
        if (++pending_flush == kFlushEvery) {
          __syncwarp();
          flush_moments(lacc, cacc + (size_t)(c - c0) * kNMom, lane);
          pending_flush = 0;
        }
      }
      // Free flight and the count of the new cell; the state goes back in place.
      for (int b = 0; b < gn; b += 32) {
        const int i = b + lane;
        const bool act = i < gn;
        int cell = -1;
        if (act) {
          const int p = gs + i;
          float yy = y[p], xx = sx[i], uy = sy[i], zz = sz[i];
          if (!fly(yy, xx, uy, zz, a.dt, a.F, a.k0, a.k1, a.step, (uint32_t)p)) bad_bounce = true;
          y[p] = yy;
          vx[p] = xx;
          vy[p] = uy;
          vz[p] = zz;
          cell = cell_of(yy, n_cells, a.ncf);
        }
        const unsigned peers = __match_any_sync(kFull, cell);
        if (act && (peers & lt) == 0) atomicAdd(&h[cell], __popc(peers));
      }
      __syncwarp();
    }
    if (a.sample && pending_flush > 0) {
      __syncwarp();
      flush_moments(lacc, cacc + (size_t)(c - c0) * kNMom, lane);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gmax = fmaxf(gmax, __shfl_xor_sync(kFull, gmax, o));
      laccn += __shfl_xor_sync(kFull, laccn, o);
    }
    if (lane == 0) {  // lcand is the same on every lane: the sum of the groups' M
      atomicMax(&cgmax[c - c0], __float_as_uint(gmax));  // gmax >= 0: bits order as values
      atomicAdd(&ccand[c - c0], lcand);
      atomicAdd(&caccn[c - c0], laccn);
    }
    qbase += ng;
  }
  if (bad_bounce) atomicOr(err, kErrBounces);
  if (sphere_fail) atomicOr(err, kErrSphere);
  if (cand_fail && lane == 0) atomicOr(err, kErrCandidates);
  __syncthreads();

  int* row = hist + (size_t)span * n_cells;
  for (int i = threadIdx.x; i < n_cells; i += blockDim.x) row[i] = h[i];
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const int lc = c - c0;
    const float gm = __uint_as_float(cgmax[lc]);
    const float sg = (kMode == 0) ? gm : fmul(a.cvhs, pow32(gm, a.vexp));
    smax_out[c] = fmaxf(smax_in[c], sg);
    ncand[c] += ccand[lc];
    nacc[c] += caccn[lc];
    if (a.sample)
      for (int k = 0; k < kNMom; ++k) acc[(size_t)c * kNMom + k] += cacc[lc * kNMom + k];
  }
}

// One warp per span: stable scatter of the span's slots into the other buffer.  Eight
// groups of 32 slots are loaded before any is placed, so each lane keeps 32 loads in
// flight.
__global__ void __launch_bounds__(kBWarpsMax * 32)
    k_scatter_spans(const float* __restrict__ y, const float* __restrict__ vx,
                    const float* __restrict__ vy, const float* __restrict__ vz,
                    float* __restrict__ y2, float* __restrict__ vx2, float* __restrict__ vy2,
                    float* __restrict__ vz2, const int* __restrict__ off_cur,
                    const int* __restrict__ off_new, const int* __restrict__ hist, int n_cells,
                    int cps, int n_spans, float ncf, int N, int* __restrict__ err) {
  constexpr int kUnroll = 8;
  extern __shared__ int sh_run[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int span = blockIdx.x * (blockDim.x >> 5) + wib;
  if (span >= n_spans) return;
  int* run = sh_run + (size_t)wib * n_cells;
  const int* row = hist + (size_t)span * n_cells;
  for (int c = lane; c < n_cells; c += 32) run[c] = off_new[c] + row[c];
  __syncwarp();
  const int c0 = span * cps;
  const int c1 = min(c0 + cps, n_cells);
  const int b0 = off_cur[c0];
  const int b1 = off_cur[c1];
  const unsigned lt = (1u << lane) - 1u;
  bool bad = false;
  for (int base = b0; base < b1; base += 32 * kUnroll) {
    float ry[kUnroll], rx[kUnroll], rv[kUnroll], rz[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int p = base + u * 32 + lane;
      if (p < b1) {
        ry[u] = y[p];
        rx[u] = vx[p];
        rv[u] = vy[p];
        rz[u] = vz[p];
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int p = base + u * 32 + lane;
      const bool act = p < b1;
      const int cell = act ? cell_of(ry[u], n_cells, ncf) : -1;
      const unsigned peers = __match_any_sync(kFull, cell);
      const int first = act ? run[cell] : 0;
      __syncwarp();
      if (act && (peers & lt) == 0) run[cell] = first + __popc(peers);
      __syncwarp();
      if (act) {
        const int d = first + __popc(peers & lt);
        if (d >= 0 && d < N) {
          y2[d] = ry[u];
          vx2[d] = rx[u];
          vy2[d] = rv[u];
          vz2[d] = rz[u];
        } else {
          bad = true;
        }
      }
    }
  }
  if (bad) atomicOr(err, kErrSort);
}

// ---------------------------------------------------------------------------

cudaError_t launch_collide_move(const DevState& s, const int* off, const float* smax_in,
                                float* smax_out, unsigned long long* ncand,
                                unsigned long long* nacc, double* acc, int* hist,
                                const StepArgs& a, int n_spans, int* err, cudaStream_t st) {
  const StepSmem L = step_smem_layout(a.n_cells, a.cps, a.cap);
  const dim3 block(kAWarps * 32);
  switch (a.mode) {
    case 0:
      k_collide_move<0><<<n_spans, block, L.total, st>>>(s.y, s.vx, s.vy, s.vz, off, smax_in,
                                                          smax_out, ncand, nacc, acc, hist, a,
                                                          err);
      break;
    case 1:
      k_collide_move<1><<<n_spans, block, L.total, st>>>(s.y, s.vx, s.vy, s.vz, off, smax_in,
                                                          smax_out, ncand, nacc, acc, hist, a,
                                                          err);
      break;
    default:
      k_collide_move<2><<<n_spans, block, L.total, st>>>(s.y, s.vx, s.vy, s.vz, off, smax_in,
                                                          smax_out, ncand, nacc, acc, hist, a,
                                                          err);
  }
  return cudaGetLastError();
}

int scatter_spans_warps(int n_cells) {
  size_t w = kStepSmemMax / ((size_t)n_cells * sizeof(int));
  if (w > (size_t)kBWarpsMax) w = kBWarpsMax;
  return w < 1 ? 1 : (int)w;
}

cudaError_t launch_scatter_spans(const DevState& from, const DevState& to, const int* off_cur,
                                 const int* off_new, const int* hist, int n_cells, int cps,
                                 int n_spans, float ncf, int N, int* err, cudaStream_t st) {
  const int wpb = scatter_spans_warps(n_cells);
  const size_t smem = (size_t)wpb * n_cells * sizeof(int);
  const int blocks = (n_spans + wpb - 1) / wpb;
  k_scatter_spans<<<blocks, wpb * 32, smem, st>>>(from.y, from.vx, from.vy, from.vz, to.y,
                                                     to.vx, to.vy, to.vz, off_cur, off_new,
                                                     hist, n_cells, cps, n_spans, ncf, N, err);
  return cudaGetLastError();
}

cudaError_t set_step_smem_limits(size_t a_bytes, size_t b_bytes) {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_collide_move<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)a_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_collide_move<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)a_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_collide_move<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)a_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_scatter_spans, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)b_bytes);
}

}  // namespace dsmc
