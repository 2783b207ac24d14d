// dsmc_device.cuh -- device arithmetic shared by the DSMC kernels: the Philox
// generator, the uniform and Gaussian maps, the binary32 logarithm and exponential,
// and the cell index.  Every floating-point operation that decides a trajectory is
// written with an explicit round-to-nearest intrinsic (__fmul_rn, __fadd_rn, ...)
// so that no contraction into FMA can happen, whatever the compile flags: a run is
// then a deterministic function of its inputs, operation for operation.
#pragma once

#include <stdint.h>

#include "dsmc_internal.h"

namespace dsmc {

// Random-number streams: the top byte of the last counter word.
constexpr uint32_t kStreamInit = 1u;
constexpr uint32_t kStreamMove = 2u;
constexpr uint32_t kStreamColl = 3u;

constexpr int kNormalAttempts = 30;  // sub-draws 1..15, two attempts per draw
constexpr int kInflowAttempts = 30;  // open-boundary emission: sub-draws 16..45
constexpr int kMaxBounces = 64;


__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

struct U4 {
  uint32_t x, y, z, w;
};

// Philox4x32-10 (Salmon et al., SC'11): ten rounds; round r uses the key plus r
// Weyl increments.  The two 32x32 products give hi/lo halves.
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit multiply gives both halves of each product
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ (k0 + (uint32_t)r * 0x9E3779B9u);
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ (k1 + (uint32_t)r * 0xBB67AE85u);
    c0 = n0;
    c1 = (uint32_t)p1;
    c2 = n2;
    c3 = (uint32_t)p0;
  }
  return U4{c0, c1, c2, c3};
}

// The same generator with the round keys precomputed (kernel arguments), so a round
// is two wide multiplies and two three-input XORs.
__device__ __forceinline__ U4 philox_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const PhiloxKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk.k1[r];
    c0 = n0;
    c1 = (uint32_t)p1;
    c2 = n2;
    c3 = (uint32_t)p0;
  }
  return U4{c0, c1, c2, c3};
}

// Uniform in (0,1) from the top 23 bits: (m + 1/2) 2^-23, exact in binary32.
__device__ __forceinline__ float u01(uint32_t x) {
  return fmul(fadd((float)(x >> 9), 0.5f), 0x1p-23f);
}

// Uniform in (-1,1), never 0: 2u - 1 (exact).
__device__ __forceinline__ float s11(uint32_t x) { return fsub(fmul(2.0f, u01(x)), 1.0f); }

// ln x for finite x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)];
// ln m = 2 artanh(s), s = (m-1)/(m+1), by its odd power series through s^9;
// ln 2 as a 17-bit head (e * head exact) plus a tail.
__device__ __forceinline__ float ln32(float x) {
  uint32_t b = __float_as_uint(x);
  int e = 0;
  if (b < 0x00800000u) {
    b = __float_as_uint(fmul(x, 0x1p24f));
    e = -24;
  }
  e += (int)(b >> 23) - 127;
  float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = fmul(m, 0.5f);
    e += 1;
  }
  const float f = fsub(m, 1.0f);
  const float s = fdiv(f, fadd(2.0f, f));
  const float z = fmul(s, s);
  float p = fmul(0x1.c71c72p-4f, z);  // z/9
  p = fmul(fadd(p, 0x1.24924ap-3f), z);
  p = fmul(fadd(p, 0x1.99999ap-3f), z);
  p = fmul(fadd(p, 0x1.555556p-2f), z);
  const float t = fadd(fmul(s, p), s);
  const float lnm = fadd(t, t);
  const float ef = (float)e;
  return fadd(fadd(fmul(ef, 0x1.7f7d1cp-20f), lnm), fmul(ef, 0x1.62e4p-1f));
}

// e^x: x = k ln2 + r, k = floor(x / ln2 + 1/2); Taylor polynomial of e^r through
// r^7 (Horner); scale by 2^k through the exponent field.  0 below -87.
__device__ __forceinline__ float exp32(float x) {
  if (x < -87.0f) return 0.0f;
  if (x > 88.0f) x = 88.0f;
  const float kf = floorf(fadd(fmul(x, 0x1.715476p+0f), 0.5f));
  float r = fsub(x, fmul(kf, 0x1.62e4p-1f));
  r = fsub(r, fmul(kf, 0x1.7f7d1cp-20f));
  float p = fmul(0x1.a01a02p-13f, r);
  p = fmul(fadd(p, 0x1.6c16c2p-10f), r);
  p = fmul(fadd(p, 0x1.111112p-7f), r);
  p = fmul(fadd(p, 0x1.555556p-5f), r);
  p = fmul(fadd(p, 0x1.555556p-3f), r);
  p = fmul(fadd(p, 0.5f), r);
  p = fmul(fadd(p, 1.0f), r);
  p = fadd(p, 1.0f);
  const int k = (int)kf;
  return fmul(p, __uint_as_float((uint32_t)(k + 127) << 23));
}

// g^a for g >= 0 (0 at g = 0).
__device__ __forceinline__ float pow32(float g, float a) {
  if (g == 0.0f) return 0.0f;
  return exp32(fmul(a, ln32(g)));
}

// The two N(0,1/2) deviates of an accepted polar (Marsaglia-Bray) attempt (a0, a1) with
// s = a0^2 + a1^2 < 1.
__device__ __forceinline__ void polar_scale(float a0, float a1, float s, float& z0, float& z1) {
  const float fac = fsqrt(fdiv(-ln32(s), s));
  z0 = fmul(a0, fac);
  z1 = fmul(a1, fac);
}

// One polar attempt: two N(0,1/2) deviates or a rejection.
__device__ __forceinline__ bool polar_pair(uint32_t w0, uint32_t w1, float& z0, float& z1) {
  const float a0 = s11(w0);
  const float a1 = s11(w1);
  const float s = fadd(fmul(a0, a0), fmul(a1, a1));
  if (s >= 1.0f) return false;
  polar_scale(a0, a1, s, z0, z1);
  return true;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory, completing on an
// mbarrier.  Waits are bounded: a copy that never lands is reported, not waited for
// forever.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// Makes mbarrier initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later
// asynchronous-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also expects `bytes` of bulk-copy completion on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// to shared memory, signalled on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Asynchronous prefetch of `bytes` (a multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the barrier phase with the given parity to complete, giving up after
// kMaxWaitPolls polls (each poll itself may suspend the thread for a while).
constexpr int kMaxWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int i = 0; i < kMaxWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Cell of y in [0,1]: truncation of y * n_cells, clamped to the last cell.
__device__ __forceinline__ int cell_of(float y, int n_cells, float ncf) {
  int c = (int)fmul(y, ncf);
  c = c < n_cells ? c : n_cells - 1;
  return c > 0 ? c : 0;
}

// Groups of a cell with nc particles (runs of G; a remainder below G/2 joins the
// previous run).
__device__ __forceinline__ int group_count(int nc, int G) {
  int ng = nc / G;
  const int r = nc - ng * G;
  if (r > 0 && (ng == 0 || r >= G / 2)) ng += 1;
  return ng;
}

// Re-emission below an open boundary at y = 1 facing a gas in the first-order
// Chapman-Enskog state of a shear flow (the MMS hybrid's DSMC-CFD interface): velocity
// distribution exp(-c^2) (1 + 2 P c_x c_y) of the peculiar velocity c in the units of
// Eq. 6, flux weight |c_y|, c_y < 0.  Attempt a (sub-draw 16 + a of the bounce's
// counter) proposes c_y = -sqrt(-ln u(w0)) and (c_x, c_z) from one polar attempt on
// (w1, w2), accepted when u(w3) (1 + 16 |P|) < 1 + 2 P c_x c_y.  Returns false when the
// attempts ran out (the last proposal is kept).
template <class Gen>
__device__ __forceinline__ bool inflow_emission(float& vx, float& vy, float& vz, int b,
                                                uint32_t step, uint32_t slot, float u_top,
                                                float p_top, Gen gen) {
  const float gmax = fadd(1.0f, fmul(16.0f, fabsf(p_top)));
  const uint32_t c3 = kStreamMove << 24;
  float cx = 0.0f, cy = 0.0f, cz = 0.0f;
  for (int a = 0; a < kInflowAttempts; ++a) {
    const U4 w = gen(slot, ((uint32_t)b << 8) | (16u + (uint32_t)a), step, c3);
    cy = -fsqrt(-ln32(u01(w.x)));
    float z0, z1;
    if (!polar_pair(w.y, w.z, z0, z1)) continue;
    cx = z0;
    cz = z1;
    const float gam = fadd(1.0f, fmul(fmul(fmul(2.0f, p_top), cx), cy));
    if (fmul(u01(w.w), gmax) < gam) {
      vx = fadd(u_top, cx);
      vy = cy;
      vz = cz;
      return true;
    }
  }
  vx = fadd(u_top, cx);
  vy = cy;
  vz = cz;
  return false;
}

// Free flight of one particle over dt with the body force along x and fully diffuse
// walls at the wall temperature; with open_top the boundary at y = 1 is the open
// Chapman-Enskog interface above.  Returns false at the bounce limit; inflow_fail is
// set when an inflow emission ran out of attempts.
// `gen(c0, c1, c2, c3)` is the Philox4x32-10 generator of the run's key.
template <class Gen>
__device__ __forceinline__ bool fly_with(float& y, float& vx, float& vy, float& vz, float dt,
                                         float F, uint32_t step, uint32_t slot, Gen gen,
                                         int open_top, float u_top, float p_top,
                                         bool& inflow_fail) {
  float t = dt;
  bool ok = true;
  for (int b = 0;; ++b) {
    const float ynew = fadd(y, fmul(vy, t));
    if (!(ynew < 0.0f) && !(ynew > 1.0f)) {
      y = ynew;
      vx = fadd(vx, fmul(F, t));
      return ok;
    }
    // time to the wall reached, one division for lanes bound for either wall
    const bool bottom = ynew < 0.0f;
    float thit = fdiv(bottom ? y : fsub(1.0f, y), bottom ? -vy : vy);
    const float wall = bottom ? 0.0f : 1.0f;
    if (b >= kMaxBounces) {  // leave the particle on the wall
      y = wall;
      return false;
    }
    if (thit > t) thit = t;
    t = fsub(t, thit);
    if (open_top && wall == 1.0f) {
      if (!inflow_emission(vx, vy, vz, b, step, slot, u_top, p_top, gen)) inflow_fail = true;
      y = wall;
      continue;
    }
    const uint32_t c1 = (uint32_t)b << 8;
    const uint32_t c3 = kStreamMove << 24;
    U4 w = gen(slot, c1, step, c3);
    const float speed = fsqrt(-ln32(u01(w.x)));
    // polar attempts until one falls inside the unit disc; the logarithm, division and
    // square root of the accepted attempt once after the loop (the lanes of a warp need
    // different numbers of attempts, so inside it they would run once per attempt)
    float a0 = 0.0f, a1 = 0.0f, sacc = 0.0f;
    bool got = false;
    for (int a = 0; a < kNormalAttempts && !got; ++a) {
      if ((a & 1) == 0) w = gen(slot, c1 | (1u + (uint32_t)(a >> 1)), step, c3);
      const float t0 = s11((a & 1) ? w.z : w.x);
      const float t1 = s11((a & 1) ? w.w : w.y);
      const float sq = fadd(fmul(t0, t0), fmul(t1, t1));
      if (sq < 1.0f) {
        a0 = t0;
        a1 = t1;
        sacc = sq;
        got = true;
      }
    }
    float z0 = 0.0f, z1 = 0.0f;
    if (got) {
      polar_scale(a0, a1, sacc, z0, z1);
    } else {
      ok = false;
    }
    vx = z0;
    vz = z1;
    vy = (wall == 0.0f) ? speed : -speed;
    y = wall;
  }
}

__device__ __forceinline__ bool fly(float& y, float& vx, float& vy, float& vz, float dt,
                                    float F, uint32_t k0, uint32_t k1, uint32_t step,
                                    uint32_t slot) {
  bool unused = false;
  return fly_with(
      y, vx, vy, vz, dt, F, step, slot,
      [=](uint32_t a, uint32_t b, uint32_t c, uint32_t d) { return philox(a, b, c, d, k0, k1); },
      0, 0.0f, 0.0f, unused);
}

// The same with the key's round keys precomputed and the run's upper boundary.
__device__ __forceinline__ bool fly(float& y, float& vx, float& vy, float& vz, float dt,
                                    float F, const PhiloxKeys& rk, uint32_t step,
                                    uint32_t slot, int open_top, float u_top, float p_top,
                                    bool& inflow_fail) {
  return fly_with(
      y, vx, vy, vz, dt, F, step, slot,
      [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d) { return philox_rk(a, b, c, d, rk); },
      open_top, u_top, p_top, inflow_fail);
}

}  // namespace dsmc
