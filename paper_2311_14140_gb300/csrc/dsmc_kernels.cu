// dsmc_kernels.cu -- the sm_103a kernels of one DSMC step for force-driven flow
// between parallel plates (arXiv 2311.14140, Sec. 2.1 problem, Bird's DSMC):
//
//   k_init            initial state: ppc particles per cell, uniform in the cell,
//                     velocity components N(0, 1/2) (gas at rest at the wall
//                     temperature, Sec. 2.1, units of Eq. 5)
//   k_collide_sample  per cell (one CTA), groups of <= G sorted particles staged in
//                     shared memory, one warp per group: symmetric moment sample,
//                     NTC candidates applied in order through conflict-free rounds,
//                     write-back; per-cell (sigma g)_max, counters and moment sums
//   k_move_count      free flight with the body force and diffuse walls (Philox keyed
//                     on step, slot and bounce), new cell, warp-private histogram
//   k_scan_hist       per cell, exclusive prefix of the histogram over partitions
//   k_cell_offsets    exclusive prefix over cells -> first slot of each cell
//   k_scatter         stable counting-sort scatter into the other buffer
//
// The state is structure-of-arrays binary32 (y, vx, vy, vz), double-buffered for
// the sort.  Kernel launches live in the host file; declarations are in
// dsmc_internal.h.
#include <climits>

#include "dsmc_device.cuh"
#include "dsmc_internal.h"

namespace dsmc {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Initial state.
__global__ void k_init(float* __restrict__ y, float* __restrict__ vx, float* __restrict__ vy,
                       float* __restrict__ vz, int N, int ppc, float ncf, uint32_t k0,
                       uint32_t k1, int* __restrict__ err) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const int c = p / ppc;
    const uint32_t c3 = kStreamInit << 24;
    U4 w = philox((uint32_t)p, 0u, 0u, c3, k0, k1);
    y[p] = fdiv(fadd((float)c, u01(w.x)), ncf);
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
    vx[p] = z[0];
    vy[p] = z[1];
    vz[p] = z[2];
  }
}

// ---------------------------------------------------------------------------
// Free flight of one particle over dt with the body force along x and fully
// diffuse walls at the wall temperature.  Returns false at the bounce limit.
__device__ __forceinline__ bool fly(float& y, float& vx, float& vy, float& vz, float dt,
                                    float F, uint32_t k0, uint32_t k1, uint32_t step,
                                    uint32_t slot) {
  float t = dt;
  bool ok = true;
  for (int b = 0;; ++b) {
    const float ynew = fadd(y, fmul(vy, t));
    float thit, wall;
    if (ynew < 0.0f) {
      thit = fdiv(y, -vy);
      wall = 0.0f;
    } else if (ynew > 1.0f) {
      thit = fdiv(fsub(1.0f, y), vy);
      wall = 1.0f;
    } else {
      y = ynew;
      vx = fadd(vx, fmul(F, t));
      return ok;
    }
    if (b >= kMaxBounces) {  // leave the particle on the wall
      y = wall;
      return false;
    }
    if (thit > t) thit = t;
    t = fsub(t, thit);
    const uint32_t c1 = (uint32_t)b << 8;
    const uint32_t c3 = kStreamMove << 24;
    U4 w = philox(slot, c1, step, c3, k0, k1);
    const float speed = fsqrt(-ln32(u01(w.x)));
    float z0 = 0.0f, z1 = 0.0f;
    bool got = false;
    for (int a = 0; a < kNormalAttempts && !got; ++a) {
      if ((a & 1) == 0) w = philox(slot, c1 | (1u + (uint32_t)(a >> 1)), step, c3, k0, k1);
      got = (a & 1) ? polar_pair(w.z, w.w, z0, z1) : polar_pair(w.x, w.y, z0, z1);
    }
    if (!got) {
      z0 = 0.0f;
      z1 = 0.0f;
      ok = false;
    }
    vx = z0;
    vz = z1;
    vy = (wall == 0.0f) ? speed : -speed;
    y = wall;
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
// Block (32, 8): x = cell within a chunk of 32, y = one of 8 contiguous row segments.
__global__ void k_scan_hist(int* __restrict__ hist, int n_warps, int n_cells,
                            int* __restrict__ count) {
  __shared__ int seg_tot[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.x * 32 + tx;
  const int seg = (n_warps + 7) / 8;
  const int r0 = ty * seg;
  const int r1 = min(n_warps, r0 + seg);
  int s = 0;
  if (c < n_cells)
    for (int r = r0; r < r1; ++r) s += hist[(size_t)r * n_cells + c];
  seg_tot[ty][tx] = s;
  __syncthreads();
  if (ty == 0) {
    int run = 0;
    for (int k = 0; k < 8; ++k) {
      const int v = seg_tot[k][tx];
      seg_tot[k][tx] = run;
      run += v;
    }
    if (c < n_cells) count[c] = run;
  }
  __syncthreads();
  if (c < n_cells) {
    int run = seg_tot[ty][tx];
    for (int r = r0; r < r1; ++r) {
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
// Collisions and sampling.

// Warp-wide sum of the 13 raw moments of the staged group, added with weight 1/2
// into lane 0's binary64 accumulators.  Products in binary32; the per-lane and the
// shuffle-tree sums are binary32 over at most 767 particles.
__device__ __forceinline__ void sample_group(const float* sx, const float* sy, const float* sz,
                                             int gn, int lane, double* acc) {
  float m[kNMom];
#pragma unroll
  for (int k = 0; k < kNMom; ++k) m[k] = 0.0f;
  for (int i = lane; i < gn; i += 32) {
    const float x = sx[i], y = sy[i], z = sz[i];
    const float v2 = fadd(fadd(fmul(x, x), fmul(y, y)), fmul(z, z));
    m[0] += 1.0f;
    m[1] += x;
    m[2] += y;
    m[3] += z;
    m[4] += fmul(x, x);
    m[5] += fmul(y, y);
    m[6] += fmul(z, z);
    m[7] += fmul(x, y);
    m[8] += fmul(x, z);
    m[9] += fmul(y, z);
    m[10] += fmul(x, v2);
    m[11] += fmul(y, v2);
    m[12] += fmul(z, v2);
  }
#pragma unroll
  for (int k = 0; k < kNMom; ++k) {
    float v = m[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    m[k] = v;
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNMom; ++k) acc[k] += 0.5 * (double)m[k];
  }
}

// Post-collision velocities of an accepted pair: relative speed kept, direction
// uniform on the sphere (Marsaglia 1972) from the candidate's sub-draws 1..15.
__device__ __forceinline__ bool scatter_pair(float& xi, float& yi, float& zi, float& xj,
                                             float& yj, float& zj, float g, uint32_t k,
                                             uint32_t cell, uint32_t step, uint32_t c3,
                                             uint32_t k0, uint32_t k1) {
  U4 w{0, 0, 0, 0};
  for (int a = 0; a < kNormalAttempts; ++a) {
    if ((a & 1) == 0) w = philox(k, cell, step, c3 | (1u + (uint32_t)(a >> 1)), k0, k1);
    const float a0 = s11((a & 1) ? w.z : w.x);
    const float a1 = s11((a & 1) ? w.w : w.y);
    const float sq = fadd(fmul(a0, a0), fmul(a1, a1));
    if (sq >= 1.0f) continue;
    const float q = fmul(2.0f, fsqrt(fsub(1.0f, sq)));
    const float nx = fmul(a0, q);
    const float ny = fmul(a1, q);
    const float nz = fsub(1.0f, fmul(2.0f, sq));
    const float hg = fmul(0.5f, g);
    const float cx = fmul(fadd(xi, xj), 0.5f);
    const float cy = fmul(fadd(yi, yj), 0.5f);
    const float cz = fmul(fadd(zi, zj), 0.5f);
    const float dx = fmul(hg, nx), dy = fmul(hg, ny), dz = fmul(hg, nz);
    xi = fadd(cx, dx);
    yi = fadd(cy, dy);
    zi = fadd(cz, dz);
    xj = fsub(cx, dx);
    yj = fsub(cy, dy);
    zj = fsub(cz, dz);
    return true;
  }
  return false;
}

// One CTA per cell.  Warp w stages groups w, w + W, ... of the cell in shared memory
// (vx, vy, vz and an owner word per particle), samples, collides, samples, writes
// back.  NTC candidates k = 0..M-1 of a group are drawn 32 at a time; a candidate is
// applied in a round once no earlier pending candidate of its batch touches either
// of its particles, which gives exactly the result of applying them in order.
template <bool kVHS>
__global__ void __launch_bounds__(kCollideWarps * 32)
    k_collide_sample(const int* __restrict__ offset, float* __restrict__ vx,
                     float* __restrict__ vy, float* __restrict__ vz,
                     const float* __restrict__ smax_in, float* __restrict__ smax_out,
                     unsigned long long* __restrict__ ncand,
                     unsigned long long* __restrict__ nacc, double* __restrict__ acc,
                     CollideArgs a, int* __restrict__ err) {
  extern __shared__ float sh[];
  __shared__ double red_acc[kCollideWarps][kNMom];
  __shared__ float red_max[kCollideWarps];
  __shared__ unsigned long long red_cand[kCollideWarps], red_acc_n[kCollideWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int c = blockIdx.x;
  const int start = offset[c];
  const int nc = offset[c + 1] - start;
  const int G = a.G;
  const int ng = group_count(nc, G);
  const int cap = a.cap;
  float* sx = sh + (size_t)wib * 4 * cap;
  float* sy = sx + cap;
  float* sz = sy + cap;
  int* own = reinterpret_cast<int*>(sz + cap);
  const float smax = smax_in[c];
  double dacc[kNMom];
#pragma unroll
  for (int k = 0; k < kNMom; ++k) dacc[k] = 0.0;
  float lmax = 0.0f;
  unsigned long long lcand = 0, lacc = 0;
  bool sphere_fail = false, cand_fail = false;

  for (int gi = wib; gi < ng; gi += kCollideWarps) {
    const int gs = start + gi * G;
    const int gn = (gi == ng - 1) ? nc - gi * G : G;
    for (int i = lane; i < gn; i += 32) {
      sx[i] = vx[gs + i];
      sy[i] = vy[gs + i];
      sz[i] = vz[gs + i];
      own[i] = INT_MAX;
    }
    __syncwarp();
    if (a.sample) sample_group(sx, sy, sz, gn, lane, dacc);
    const bool collide = a.collide && gn >= 2;
    if (collide) {
      const uint32_t c3 = (kStreamColl << 24) | ((uint32_t)gi << 4);
      const float t1 = fmul((float)(gn - 1), (float)nc);
      const float mf = fmul(fmul(t1, a.coef), smax);
      const float fl = floorf(mf);
      const float frac = fsub(mf, fl);
      uint32_t M = (uint32_t)fl;
      const U4 r = philox(0xffffffffu, (uint32_t)c, a.step, c3, a.k0, a.k1);
      if (u01(r.x) < frac) M += 1;
      if (!(mf <= kMaxCandidates)) {  // also catches NaN
        M = 0;
        cand_fail = true;
      }
      if (lane == 0) lcand += M;
      for (uint32_t kb = 0; kb < M; kb += 32) {
        const uint32_t k = kb + (uint32_t)lane;
        bool pend = k < M;
        int i = 0, j = 0;
        float ua = 0.0f;
        if (pend) {
          const U4 w = philox(k, (uint32_t)c, a.step, c3, a.k0, a.k1);
          i = (int)__umulhi(w.x, (uint32_t)gn);
          j = (int)__umulhi(w.y, (uint32_t)(gn - 1));
          j += (j >= i) ? 1 : 0;
          ua = u01(w.z);
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
            float xi = sx[i], yi = sy[i], zi = sz[i];
            float xj = sx[j], yj = sy[j], zj = sz[j];
            const float gx = fsub(xi, xj), gy = fsub(yi, yj), gz = fsub(zi, zj);
            const float g = fsqrt(fadd(fadd(fmul(gx, gx), fmul(gy, gy)), fmul(gz, gz)));
            const float sg = kVHS ? fmul(a.cvhs, pow32(g, a.vexp)) : g;
            lmax = fmaxf(lmax, sg);
            if (fmul(ua, smax) < sg) {
              if (scatter_pair(xi, yi, zi, xj, yj, zj, g, k, (uint32_t)c, a.step, c3, a.k0,
                               a.k1)) {
                sx[i] = xi;
                sy[i] = yi;
                sz[i] = zi;
                sx[j] = xj;
                sy[j] = yj;
                sz[j] = zj;
                lacc += 1;
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
    if (a.sample) sample_group(sx, sy, sz, gn, lane, dacc);
    if (collide) {
      for (int i = lane; i < gn; i += 32) {
        vx[gs + i] = sx[i];
        vy[gs + i] = sy[i];
        vz[gs + i] = sz[i];
      }
    }
    __syncwarp();
  }
  if (sphere_fail) atomicOr(err, kErrSphere);
  if (cand_fail && lane == 0) atomicOr(err, kErrCandidates);

  // Block totals in a fixed order (warp 0, 1, ...): one writer per cell.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lmax = fmaxf(lmax, __shfl_xor_sync(kFull, lmax, o));
    lacc += __shfl_xor_sync(kFull, lacc, o);
  }
  if (lane == 0) {
    red_max[wib] = lmax;
    red_cand[wib] = lcand;
    red_acc_n[wib] = lacc;
#pragma unroll
    for (int k = 0; k < kNMom; ++k) red_acc[wib][k] = dacc[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float mx = smax;
    unsigned long long tc = 0, ta = 0;
    for (int w = 0; w < kCollideWarps; ++w) {
      mx = fmaxf(mx, red_max[w]);
      tc += red_cand[w];
      ta += red_acc_n[w];
    }
    smax_out[c] = mx;
    ncand[c] += tc;
    nacc[c] += ta;
  }
  if (a.sample && threadIdx.x < kNMom) {
    double s = 0.0;
    for (int w = 0; w < kCollideWarps; ++w) s += red_acc[w][threadIdx.x];
    acc[(size_t)c * kNMom + threadIdx.x] += s;
  }
}

__global__ void k_clamp_y(float* __restrict__ y, int N) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const float v = y[p];
    y[p] = (v >= 0.0f) ? ((v <= 1.0f) ? v : 1.0f) : 0.0f;
  }
}

// ---------------------------------------------------------------------------
// Launchers.

cudaError_t launch_init(const DevState& s, int N, int ppc, float ncf, uint32_t k0, uint32_t k1,
                        int* err, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (N + threads - 1) / threads;
  k_init<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(s.y, s.vx, s.vy, s.vz, N, ppc, ncf, k0,
                                                      k1, err);
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
  k_scan_hist<<<blocks, dim3(32, 8), 0, st>>>(hist, n_warps, n_cells, count);
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

size_t collide_smem_bytes(int cap) { return (size_t)kCollideWarps * 4 * cap * sizeof(float); }

cudaError_t launch_collide_sample(const DevState& s, int n_cells, const int* offset,
                                  const float* smax_in, float* smax_out,
                                  unsigned long long* ncand, unsigned long long* nacc,
                                  double* acc, const CollideArgs& a, bool vhs, int* err,
                                  cudaStream_t st) {
  const size_t smem = collide_smem_bytes(a.cap);
  if (vhs)
    k_collide_sample<true><<<n_cells, kCollideWarps * 32, smem, st>>>(
        offset, s.vx, s.vy, s.vz, smax_in, smax_out, ncand, nacc, acc, a, err);
  else
    k_collide_sample<false><<<n_cells, kCollideWarps * 32, smem, st>>>(
        offset, s.vx, s.vy, s.vz, smax_in, smax_out, ncand, nacc, acc, a, err);
  return cudaGetLastError();
}

cudaError_t launch_clamp_y(float* y, int N, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (N + threads - 1) / threads;
  k_clamp_y<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(y, N);
  return cudaGetLastError();
}

cudaError_t set_kernel_smem_limits(size_t sort_bytes, size_t collide_bytes) {
  cudaError_t e;
  e = cudaFuncSetAttribute(k_move_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sort_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sort_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_collide_sample<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)collide_bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_collide_sample<false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)collide_bytes);
}

}  // namespace dsmc
