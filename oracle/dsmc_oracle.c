/*
 * dsmc_oracle.c -- plain, slow, single-threaded CPU DSMC of force-driven rarefied
 * flow between two parallel plates.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is checked
 * against.  Only the test suite, the smoke check of the package entry module and the
 * CPU-baseline leg of the benchmark may build, load or call it.  The product path
 * never does.  It shares no code with the CUDA library: every routine here (the
 * Philox generator, the logarithm, the Gaussian sampler, the collision, the sort) is
 * written separately from its published definition.
 *
 * What it follows (sections and equations of arXiv 2311.14140, "A DSMC-CFD coupling
 * method using surrogate modelling for low-speed rarefied gas flows"):
 *   - the problem: monatomic gas between two plates at a constant temperature, driven
 *     by a small external acceleration parallel to the plates (Sec. 2.1);
 *   - the nondimensionalisation: lengths in H, speeds in v0 = sqrt(2 k T0 / m), body
 *     force F = F' H / v0^2, stress in P0 (Eq. 6);
 *   - the Knudsen number through the viscosity, mu0 v0 / (P0 H) = 2 Kn / sqrt(pi)
 *     (Eq. 7 against Eq. 2);
 *   - the DSMC cell size and particles per cell as free inputs, and sampling by time
 *     averaging (Sec. 3);
 *   - the DSMC method itself, which the paper takes from Bird (cited in Sec. 1 and
 *     Sec. 2): free flight with the body force, fully diffuse isothermal walls, a
 *     stable counting sort into cells, no-time-counter (NTC) collisions of hard-sphere
 *     (HS) or variable-hard-sphere (VHS) molecules, and cell moments.
 *
 * The paper does not describe its DSMC at all; every step below is the textbook
 * algorithm with the readings recorded in the design notes (collision groups,
 * stochastic rounding of the candidate count, counter-based random numbers keyed on
 * step, cell and candidate, and the order of floating-point operations).
 *
 * Arithmetic: particle state and kinematics in IEEE binary32 with every operation
 * rounded once (this file must be compiled with -ffp-contract=off and without
 * fast-math); moment sums in binary64, one particle at a time.
 *
 * Sampling is symmetric about the collision phase (half before, half after): the
 * cell moments after the collisions alone under-read the momentum flux by O(nu dt)
 * (about 9 percent at dt = 0.2 mean collision times), because collisions relax the
 * stress that the free flight builds up; the symmetric sample is the trapezoidal
 * average over each flight and satisfies the momentum balance of Eq. 1.
 *
 * Parity status of each part (what pins it; see tests/test_oracle_*.py):
 *   philox4x32_10     pinned: cuRAND's host Philox4_32_10 generator and the
 *                     Random123 known-answer vectors (Salmon et al., SC'11).
 *   or_ln / or_exp    pinned: error against binary64 libm over all binary32 inputs
 *                     of the range used.
 *   Gaussian / wall   pinned: moments and Kolmogorov-Smirnov against N(0,1/2) and the
 *                     flux-weighted half-Maxwellian.
 *   collision         pinned: momentum and energy conservation per collision,
 *                     isotropy of the post-collision direction, HS and VHS collision
 *                     rate N(N-1) sigma <g> dt / (2V) at equilibrium, acceptance
 *                     probability sigma g / (sigma g)_max against its definition.
 *   move + walls      pinned: collisionless transient closed form (1D quadrature).
 *   sort              pinned: brute-force stable sort by (cell, previous slot).
 *   whole step        pinned: Maxwellian preservation, momentum balance
 *                     dP_xy/dy = 2F (Eq. 1), near-continuum parabola curvature
 *                     -sqrt(pi) F / Kn (Eq. 8 with S = 0).
 *   slip value        parity unpinned beyond a band: the paper prints no sigma_P.
 *   transition-regime profiles (Kn 0.1 to 5)
 *                     parity unpinned: the paper's figures carry no data.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11).  Ten rounds of the 4x32 Philox S-box with the published
 * multipliers and Weyl key increments. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

OR_EXPORT void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ x1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ x3 ^ k1;
    uint32_t n3 = lo0;
    x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Random-number streams.  The counter's top byte names the stream. */
#define TAG_INIT 1u
#define TAG_MOVE 2u
#define TAG_COLL 3u
#define MAX_NORMAL_ATTEMPTS 30 /* sub-draws 1..15, two attempts each */
#define MAX_BOUNCES 64

/* Error bits (same meaning as the library's device error word). */
#define OR_ERR_NORMAL_ATTEMPTS 1
#define OR_ERR_BOUNCES 2
#define OR_ERR_SPHERE_ATTEMPTS 4 /* kept for the bit layout; the direction draw cannot fail */
#define OR_ERR_CANDIDATES 8
#define OR_ERR_INFLOW_ATTEMPTS 64
#define MAX_INFLOW_ATTEMPTS 30 /* sub-draws 16..45 */

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* 32-bit word -> uniform in the open interval (0,1): the top 23 bits plus one half,
 * scaled by 2^-23, so u lies in [2^-24, 1 - 2^-24].  Every step is exact in binary32
 * (with 24 bits the largest value, 2^24 - 1/2, would round up to 1), and so is
 * 2u - 1, which is never 0. */
OR_EXPORT float or_u01(uint32_t x) {
  return ((float)(x >> 9) + 0.5f) * 0x1p-23f;
}

/* Natural logarithm in binary32 from the series
 *   ln m = 2 artanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9 + ...),  s = (m-1)/(m+1),
 * after splitting x = m 2^e with m in [sqrt(1/2), sqrt(2)], and ln 2 split into a
 * 17-bit head and a tail so that e * head is exact.  |s| <= 0.1716, so the first
 * dropped term is below 2^-30 relative.  Defined for finite x > 0. */
OR_EXPORT float or_ln(float x) {
  uint32_t bits;
  memcpy(&bits, &x, 4);
  int e = 0;
  if (bits < 0x00800000u) { /* subnormal: scale by 2^24 first */
    float xs = x * 0x1p24f;
    memcpy(&bits, &xs, 4);
    e = -24;
  }
  e += (int)(bits >> 23) - 127;
  uint32_t mbits = (bits & 0x007fffffu) | 0x3f800000u;
  float m;
  memcpy(&m, &mbits, 4);
  if (m > 0x1.6a09e6p+0f) { /* m > sqrt(2) */
    m = m * 0.5f;
    e = e + 1;
  }
  float f = m - 1.0f;
  float s = f / (2.0f + f);
  float z = s * s;
  float p = 0x1.c71c72p-4f; /* 1/9 */
  p = p * z;
  p = p + 0x1.24924ap-3f; /* 1/7 */
  p = p * z;
  p = p + 0x1.99999ap-3f; /* 1/5 */
  p = p * z;
  p = p + 0x1.555556p-2f; /* 1/3 */
  p = p * z;
  float t = s * p;
  t = t + s;
  float lnm = t + t;
  float ef = (float)e;
  float r = ef * 0x1.7f7d1cp-20f; /* tail of ln 2 */
  r = r + lnm;
  r = r + ef * 0x1.62e4p-1f; /* head of ln 2 */
  return r;
}

/* Exponential in binary32: x = k ln2 + r with k = floor(x/ln2 + 1/2) and
 * |r| <= ln2/2, then the Taylor polynomial of e^r to degree 7 (first dropped term
 * below 2^-27) and a scale by 2^k.  Returns 0 below -87 (not reached by the VHS
 * exponent on this path). */
OR_EXPORT float or_exp(float x) {
  if (x < -87.0f) return 0.0f;
  if (x > 88.0f) x = 88.0f;
  float kf = floorf(x * 0x1.715476p+0f + 0.5f);
  float r = x - kf * 0x1.62e4p-1f;
  r = r - kf * 0x1.7f7d1cp-20f;
  float p = 0x1.a01a02p-13f; /* 1/7! */
  p = p * r;
  p = p + 0x1.6c16c2p-10f; /* 1/6! */
  p = p * r;
  p = p + 0x1.111112p-7f; /* 1/5! */
  p = p * r;
  p = p + 0x1.555556p-5f; /* 1/4! */
  p = p * r;
  p = p + 0x1.555556p-3f; /* 1/3! */
  p = p * r;
  p = p + 0.5f;
  p = p * r;
  p = p + 1.0f;
  p = p * r;
  p = p + 1.0f;
  int k = (int)kf;
  uint32_t sb = (uint32_t)(k + 127) << 23;
  float scale;
  memcpy(&scale, &sb, 4);
  return p * scale;
}

/* g^a for g >= 0 and 0 <= a <= 1 (the VHS factor); 0 for g == 0. */
OR_EXPORT float or_pow(float g, float a) {
  if (g == 0.0f) return 0.0f;
  return or_exp(a * or_ln(g));
}

/* One attempt of the Marsaglia-Bray polar method: two words -> two independent
 * N(0, 1/2) deviates, or a rejection (returns 0).  The variance 1/2 is the
 * Maxwellian at the wall temperature in v0 units (Eq. 6). */
OR_EXPORT int or_normal_pair(uint32_t w0, uint32_t w1, float* z0, float* z1) {
  float a0 = 2.0f * or_u01(w0) - 1.0f;
  float a1 = 2.0f * or_u01(w1) - 1.0f;
  float s = a0 * a0 + a1 * a1;
  if (s >= 1.0f) return 0;
  float fac = sqrtf(-or_ln(s) / s);
  *z0 = a0 * fac;
  *z1 = a1 * fac;
  return 1;
}

/* Normal attempt number a of a draw family: sub-draw 1 + a/2, words (0,1) for even
 * a and (2,3) for odd a.  fam[] holds the counter with c1 or c3 carrying the
 * sub-draw as described by the caller through `sub_in_c1`. */
typedef struct {
  uint64_t seed;
  uint32_t c0, c1, c2, c3;
  int sub_in_c1; /* 1: sub-draw is or-ed into c1; 0: into c3 */
} family;

static void family_draw(const family* f, uint32_t sub, uint32_t out[4]) {
  if (f->sub_in_c1)
    draw(f->seed, f->c0, f->c1 | sub, f->c2, f->c3, out);
  else
    draw(f->seed, f->c0, f->c1, f->c2, f->c3 | sub, out);
}

/* Fill `n` N(0,1/2) deviates from the attempts of one family; returns 0 when the
 * attempts ran out (the deviates left are set to zero and an error bit is raised). */
static int family_normals(const family* f, float* z, int n) {
  int have = 0;
  for (int a = 0; a < MAX_NORMAL_ATTEMPTS && have < n; ++a) {
    uint32_t w[4];
    family_draw(f, 1u + (uint32_t)(a >> 1), w);
    float z0, z1;
    int ok = (a & 1) ? or_normal_pair(w[2], w[3], &z0, &z1)
                     : or_normal_pair(w[0], w[1], &z0, &z1);
    if (!ok) continue;
    z[have++] = z0;
    if (have < n) z[have++] = z1;
  }
  if (have < n) {
    for (int i = have; i < n; ++i) z[i] = 0.0f;
    return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------- */
/* Simulation parameters (host arithmetic in binary64, rounded once to binary32). */

/* Number density times reference cross-section, in 1/H, from the viscosity
 * definition of Kn: mu0 v0 / (P0 H) = 2 Kn / sqrt(pi) (Eq. 7 with Eq. 2) and the
 * first Chapman-Enskog viscosity of VHS molecules,
 *   mu = 15 sqrt(pi m k T) / (2 sigma (5 - 2w)(7 - 2w))      (Bird),
 * which together give n sigma H = 15 sqrt(2) pi / (4 (5-2w)(7-2w) Kn).
 * Kn = +inf gives 0 (collisionless). */
OR_EXPORT double or_nsigma(double omega, double Kn) {
  if (isinf(Kn)) return 0.0;
  double num = 15.0 * sqrt(2.0) * M_PI;
  double den = 4.0 * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega) * Kn;
  return num / den;
}

typedef struct {
  /* inputs */
  double omega, Kn, F_d, dt_factor, dt_in;
  int n_cells, ppc, G, collisions;
  long long sample_start;
  uint64_t seed;
  /* derived */
  int N;
  double nsig, dt_d;
  float dt, F, coef, cvhs, vexp, vinv, lncv, smax0, ncf;
  /* state: sorted by cell */
  float *y, *vx, *vy, *vz;
  float *ty, *tvx, *tvy, *tvz; /* sort scratch */
  int* cell;                   /* per slot */
  int* offset;                 /* n_cells + 1 */
  float* smax;                 /* (sigma g)_max per cell, units sigma_ref v0 */
  float* gmax_obs;              /* largest candidate relative speed of the step */
  unsigned long long *ncand, *nacc;
  double* acc;  /* n_cells x 13 raw sums */
  double* aacc; /* n_cells x 13 sums of absolute values (error bounds of other
                   summation orders) */
  long long n_samples;
  long long step;
  int err;
  /* open boundary at y = 1 (Chapman-Enskog reservoir), off by default */
  int open_top;
  float u_top, p_top;
} osim;

#define NMOM 13

/* Cell of a position: truncation of y * n_cells, clamped to the last cell (y = 1
 * lies on the top wall). */
OR_EXPORT int or_cell_of(float y, int n_cells) {
  int c = (int)(y * (float)n_cells);
  if (c >= n_cells) c = n_cells - 1;
  if (c < 0) c = 0;
  return c;
}

/* Stable counting sort of slots by cell: perm[k] is the previous slot of the
 * particle that lands in slot k; slots in one cell keep their previous order. */
OR_EXPORT void or_stable_cell_sort(const int* cell, int n, int n_cells, int* perm,
                                   int* offset) {
  int* cnt = (int*)calloc((size_t)n_cells + 1, sizeof(int));
  for (int p = 0; p < n; ++p) cnt[cell[p] + 1] += 1;
  for (int c = 0; c < n_cells; ++c) cnt[c + 1] += cnt[c];
  if (offset) memcpy(offset, cnt, sizeof(int) * ((size_t)n_cells + 1));
  for (int p = 0; p < n; ++p) perm[cnt[cell[p]]++] = p;
  free(cnt);
}

static void index_cells(osim* s) {
  int n = s->N;
  int* perm = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int p = 0; p < n; ++p) s->cell[p] = or_cell_of(s->y[p], s->n_cells);
  or_stable_cell_sort(s->cell, n, s->n_cells, perm, s->offset);
  for (int k = 0; k < n; ++k) {
    int p = perm[k];
    s->ty[k] = s->y[p];
    s->tvx[k] = s->vx[p];
    s->tvy[k] = s->vy[p];
    s->tvz[k] = s->vz[p];
  }
  float* t;
  t = s->y; s->y = s->ty; s->ty = t;
  t = s->vx; s->vx = s->tvx; s->tvx = t;
  t = s->vy; s->vy = s->tvy; s->tvy = t;
  t = s->vz; s->vz = s->tvz; s->tvz = t;
  for (int c = 0; c < s->n_cells; ++c)
    for (int k = s->offset[c]; k < s->offset[c + 1]; ++k) s->cell[k] = c;
  free(perm);
}

/* Initial state: the gas at rest at the wall temperature (Sec. 2.1), `ppc`
 * particles per cell, each placed uniformly inside its cell, each velocity
 * component N(0, 1/2). */
static void init_particles(osim* s) {
  for (int p = 0; p < s->N; ++p) {
    int c = p / s->ppc;
    family f = {s->seed, (uint32_t)p, 0u, 0u, TAG_INIT << 24, 1};
    uint32_t w[4];
    family_draw(&f, 0u, w);
    s->y[p] = ((float)c + or_u01(w[0])) / s->ncf;
    float z[3];
    if (!family_normals(&f, z, 3)) s->err |= OR_ERR_NORMAL_ATTEMPTS;
    s->vx[p] = z[0];
    s->vy[p] = z[1];
    s->vz[p] = z[2];
  }
}

/* Re-emission into the gas below an open boundary at y = 1 that faces a gas in the
 * first-order Chapman-Enskog state of a shear flow (the MMS hybrid's DSMC-CFD interface,
 * Sec. 2 and Sec. 3.2: the CFD's velocity u and shear stress P there).  In units of
 * Eq. 6 the velocity distribution is the Maxwellian of the peculiar velocity c times
 * Gamma(c) = 1 + 2 P c_x c_y (this normalisation makes 2 <c_x c_y> = P, the stress
 * estimator of the sampling), and particles enter with the flux weight |c_y|, c_y < 0.
 * Attempt a (sub-draw 16 + a of the bounce's counter) proposes c_y = -sqrt(-ln u(w0)),
 * (c_x, c_z) from one polar attempt on (w1, w2), and accepts when
 * u(w3) (1 + 16 |P|) < Gamma(c) (rejection against the bound of Gamma for
 * |c_x c_y| <= 8).  Returns 0 when the attempts ran out (then the last proposal, or the
 * Maxwellian flux without shear, is used). */
static int inflow_emission(uint64_t seed, uint32_t slot, uint32_t step, int b, float u_top,
                           float p_top, float* vx, float* vy, float* vz) {
  const float gmax = 1.0f + 16.0f * fabsf(p_top);
  float cx = 0.0f, cy = 0.0f, cz = 0.0f;
  for (int a = 0; a < MAX_INFLOW_ATTEMPTS; ++a) {
    uint32_t w[4];
    draw(seed, slot, ((uint32_t)b << 8) | (16u + (uint32_t)a), step, TAG_MOVE << 24, w);
    cy = -sqrtf(-or_ln(or_u01(w[0])));
    float z0, z1;
    if (!or_normal_pair(w[1], w[2], &z0, &z1)) continue;
    cx = z0;
    cz = z1;
    float gam = 1.0f + 2.0f * p_top * cx * cy;
    if (or_u01(w[3]) * gmax < gam) {
      *vx = u_top + cx;
      *vy = cy;
      *vz = cz;
      return 1;
    }
  }
  *vx = u_top + cx;
  *vy = cy;
  *vz = cz;
  return 0;
}

/* Free flight over one time step with the body force along x and fully diffuse
 * walls at the wall temperature (Sec. 2.1: plates at constant temperature, external
 * acceleration parallel to the plates).  A particle that crosses a wall is moved to
 * the wall after the fraction of the remaining time it needs, re-emitted with
 * |vy| = sqrt(-ln u) (flux-weighted half-Maxwellian) into the gas and vx, vz drawn
 * from N(0, 1/2), and flies on for the time left.  With open_top the boundary at y = 1
 * is a Chapman-Enskog reservoir instead (inflow_emission).  Returns 0 when the
 * bounce limit is hit; *err gets the error bits. */
static int move_general(float* py, float* pvx, float* pvy, float* pvz, float dt, float F,
                        uint64_t seed, uint32_t step, uint32_t slot, int open_top,
                        float u_top, float p_top, int* err) {
  float y = *py, vx = *pvx, vy = *pvy, vz = *pvz;
  float t = dt;
  int ok = 1;
  for (int b = 0;; ++b) {
    float ynew = y + vy * t;
    float thit;
    float wall;
    if (ynew < 0.0f) {
      thit = y / (-vy);
      wall = 0.0f;
    } else if (ynew > 1.0f) {
      thit = (1.0f - y) / vy;
      wall = 1.0f;
    } else {
      y = ynew;
      vx = vx + F * t;
      break;
    }
    if (b >= MAX_BOUNCES) { /* leave the particle on the wall */
      y = wall;
      ok = 0;
      *err |= OR_ERR_BOUNCES;
      break;
    }
    if (thit > t) thit = t;
    t = t - thit;
    if (open_top && wall == 1.0f) {
      if (!inflow_emission(seed, slot, step, b, u_top, p_top, &vx, &vy, &vz))
        *err |= OR_ERR_INFLOW_ATTEMPTS;
      y = wall;
      continue;
    }
    family f = {seed, slot, (uint32_t)b << 8, step, TAG_MOVE << 24, 1};
    uint32_t w[4];
    family_draw(&f, 0u, w);
    float speed = sqrtf(-or_ln(or_u01(w[0])));
    float z[2];
    if (!family_normals(&f, z, 2)) {
      ok = 0;
      *err |= OR_ERR_NORMAL_ATTEMPTS;
    }
    vx = z[0];
    vz = z[1];
    vy = (wall == 0.0f) ? speed : -speed;
    y = wall;
  }
  *py = y; *pvx = vx; *pvy = vy; *pvz = vz;
  return ok;
}

OR_EXPORT int or_move_particle(float* py, float* pvx, float* pvy, float* pvz,
                               float dt, float F, uint64_t seed, uint32_t step,
                               uint32_t slot) {
  int err = 0;
  int ok = move_general(py, pvx, pvy, pvz, dt, F, seed, step, slot, 0, 0.0f, 0.0f, &err);
  return ok && !(err & OR_ERR_NORMAL_ATTEMPTS);
}

/* The same flight with the open boundary at y = 1; returns the error bits (0: none). */
OR_EXPORT int or_move_particle_open(float* py, float* pvx, float* pvy, float* pvz, float dt,
                                    float F, uint64_t seed, uint32_t step, uint32_t slot,
                                    float u_top, float p_top) {
  int err = 0;
  move_general(py, pvx, pvy, pvz, dt, F, seed, step, slot, 1, u_top, p_top, &err);
  return err;
}

/* The pair i != j of a candidate among a group's ng particles, from one word by
 * multiply-shift: i = floor(w0 ng / 2^32); the low half of that product, spread evenly
 * over [0, 2^32) within each i, gives j = floor(lo (ng - 1) / 2^32), moved past i.
 * Each ordered pair receives floor or ceil of 2^32 / (ng (ng - 1)) words, so within
 * ng^2 / 2^32 (3.4e-5 at ng = 383) of uniform. */
OR_EXPORT void or_pair_choice(uint32_t w0, int ng, uint32_t* i, uint32_t* j) {
  uint64_t p = (uint64_t)w0 * (uint64_t)ng;
  uint32_t a = (uint32_t)(p >> 32);
  uint32_t b = (uint32_t)(((uint64_t)(uint32_t)p * (uint64_t)(ng - 1)) >> 32);
  if (b >= a) b += 1;
  *i = a;
  *j = b;
}

/* sigma(g) g in units of sigma_ref v0: g for hard spheres, cvhs g^(2-2w) for VHS. */
static float sigma_g(const osim* s, float g) {
  if (s->omega == 0.5) return g;
  return s->cvhs * or_pow(g, s->vexp);
}

/* NTC acceptance, sigma(g) g > u (sigma g)_max (probability sigma g / (sigma g)_max),
 * written as a threshold on the relative speed, g > thr:
 *   hard spheres:  thr = u (sigma g)_max;
 *   VHS, w < 1:    thr = (u (sigma g)_max / cvhs)^(1/(2-2w))
 *                      = exp((ln(u (sigma g)_max) - ln cvhs) / (2-2w)),
 *                  since sigma g grows monotonically with g (ln cvhs is a run
 *                  constant, so no division per candidate);
 *   w = 1:         sigma g = cvhs for every g: thr = -1 (accept) when
 *                  u (sigma g)_max < cvhs, else +inf (reject). */
static float accept_threshold(const osim* s, float u, float smax) {
  float us = u * smax;
  if (s->omega == 0.5) return us;
  if (s->omega == 1.0) return (us < s->cvhs) ? -1.0f : INFINITY;
  float t = or_ln(us) - s->lncv;
  return or_exp(s->vinv * t);
}

/* sin(2 pi v) and cos(2 pi v) for v in [0, 1], binary32.  4 v = n + r with n the
 * nearest integer (4 v, n and r are exact), theta = r pi/2 in [-pi/4, pi/4], the Taylor
 * series of sin theta through theta^9 and of cos theta through theta^10 (truncation
 * below 2e-9 on that range) by Horner's rule, then n quarter turns:
 * (cos, sin)(theta + n pi/2) = (c, s), (-s, c), (-c, -s), (s, -c) for n mod 4 = 0..3. */
OR_EXPORT void or_sincos_turn(float v, float* sn, float* cs) {
  float t = 4.0f * v;
  float n = floorf(t + 0.5f);
  float r = t - n;
  float th = r * 0x1.921fb6p+0f; /* pi/2 */
  float t2 = th * th;
  float ps = 0x1.71de3ap-19f;    /* 1/9! */
  ps = ps * t2 - 0x1.a01a02p-13f; /* 1/7! */
  ps = ps * t2 + 0x1.111112p-7f;  /* 1/5! */
  ps = ps * t2 - 0x1.555556p-3f;  /* 1/3! */
  ps = ps * t2;
  float s = th + th * ps;
  float pc = -0x1.27e4fcp-22f;   /* -1/10! */
  pc = pc * t2 + 0x1.a01a02p-16f; /* 1/8! */
  pc = pc * t2 - 0x1.6c16c2p-10f; /* 1/6! */
  pc = pc * t2 + 0x1.555556p-5f;  /* 1/4! */
  pc = pc * t2 - 0.5f;
  float c = 1.0f + t2 * pc;
  switch (((int)n) & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

/* Post-collision velocities of an accepted pair (isotropic scattering, which both
 * HS and VHS share): the relative speed g is kept, its direction is drawn uniformly
 * on the sphere, and the centre-of-mass velocity is unchanged.  The direction comes
 * from the words w2, w3 of the candidate's draw by the cylindrical (Archimedes) map:
 * n_z = 2 u(w2) - 1 and azimuth 2 pi u(w3) are independent and uniform, so
 * n = (sqrt(1 - n_z^2) cos, sqrt(1 - n_z^2) sin, n_z) is uniform on the sphere
 * (the area between two heights is proportional to their distance).  Always succeeds
 * (returns 1). */
static int scatter_pair(float* vi, float* vj, float g, uint32_t w2, uint32_t w3) {
  float nz = 2.0f * or_u01(w2) - 1.0f;
  float rho = sqrtf(1.0f - nz * nz);
  float sn, cs;
  or_sincos_turn(or_u01(w3), &sn, &cs);
  float nx = rho * cs;
  float ny = rho * sn;
  float hg = 0.5f * g;
  float cx = (vi[0] + vj[0]) * 0.5f;
  float cy = (vi[1] + vj[1]) * 0.5f;
  float cz = (vi[2] + vj[2]) * 0.5f;
  float dx = hg * nx, dy = hg * ny, dz = hg * nz;
  vi[0] = cx + dx; vi[1] = cy + dy; vi[2] = cz + dz;
  vj[0] = cx - dx; vj[1] = cy - dy; vj[2] = cz - dz;
  return 1;
}

/* Exposed for the conservation pins: collide vi with vj as an accepted candidate of
 * family (seed, k, cell, step, group) would. */
OR_EXPORT int or_scatter_pair(float* vi, float* vj, uint64_t seed, uint32_t k,
                              uint32_t cell, uint32_t step, uint32_t group) {
  float gx = vi[0] - vj[0], gy = vi[1] - vj[1], gz = vi[2] - vj[2];
  float g = sqrtf(gx * gx + gy * gy + gz * gz);
  uint32_t w[4];
  draw(seed, k, cell, step, (TAG_COLL << 24) | (group << 4), w);
  return scatter_pair(vi, vj, g, w[2], w[3]);
}

/* Exposed for the acceptance pin. */
OR_EXPORT float or_accept_threshold(const osim* s, float u, float smax) {
  return accept_threshold(s, u, smax);
}

/* Collision groups of a cell holding nc particles: consecutive runs of G sorted
 * particles, the last run taking the remainder, and a remainder below G/2 merged into
 * the run before it, so every group but a lone one has at least G/2 particles. */
OR_EXPORT int or_group_count(int nc, int G) {
  int ng = nc / G;
  int r = nc - ng * G;
  if (r > 0 && (ng == 0 || r >= G / 2)) ng += 1;
  return ng;
}

/* NTC collisions of one group (Bird's no-time-counter scheme applied to a group of
 * ng of the nc particles of cell c, with the group volume ng/nc of the cell's):
 *   M = (ng - 1) nc (n sigma_ref) dt / (2 ppc) * (sigma g)_max,
 * rounded stochastically; each candidate picks i != j uniformly and is accepted with
 * probability sigma g / (sigma g)_max (accept_threshold).  Candidates are applied in
 * order.  The largest relative speed among the candidates is kept for the update of
 * (sigma g)_max after the step. */
static void collide_group(osim* s, int c, int nc, int gic, int start, int ng) {
  if (ng < 2) return;
  float smax = s->smax[c];
  uint32_t st = (uint32_t)s->step;
  uint32_t c3 = (TAG_COLL << 24) | ((uint32_t)gic << 4);
  float t1 = (float)(ng - 1) * (float)nc;
  float t2 = t1 * s->coef;
  float mf = t2 * smax;
  float fl = floorf(mf);
  float frac = mf - fl;
  uint32_t M = (uint32_t)fl;
  uint32_t w[4];
  draw(s->seed, 0xffffffffu, (uint32_t)c, st, c3, w);
  if (or_u01(w[0]) < frac) M += 1;
  if (!(mf <= 1.0e7f)) { /* corrupted (sigma g)_max: skip the group, report */
    M = 0;
    s->err |= OR_ERR_CANDIDATES;
  }
  s->ncand[c] += M;
  float* vx = s->vx + start;
  float* vy = s->vy + start;
  float* vz = s->vz + start;
  for (uint32_t k = 0; k < M; ++k) {
    draw(s->seed, k, (uint32_t)c, st, c3, w);
    uint32_t i, j;
    or_pair_choice(w[0], ng, &i, &j);
    float gx = vx[i] - vx[j];
    float gy = vy[i] - vy[j];
    float gz = vz[i] - vz[j];
    float g = sqrtf(gx * gx + gy * gy + gz * gz);
    if (g > s->gmax_obs[c]) s->gmax_obs[c] = g;
    if (g > accept_threshold(s, or_u01(w[1]), smax)) {
      float vi[3] = {vx[i], vy[i], vz[i]};
      float vj[3] = {vx[j], vy[j], vz[j]};
      if (!scatter_pair(vi, vj, g, w[2], w[3])) {
        s->err |= OR_ERR_SPHERE_ATTEMPTS;
        continue;
      }
      vx[i] = vi[0]; vy[i] = vi[1]; vz[i] = vi[2];
      vx[j] = vj[0]; vy[j] = vj[1]; vz[j] = vj[2];
      s->nacc[c] += 1;
    }
  }
}

static void collide_all(osim* s) {
  for (int c = 0; c < s->n_cells; ++c) s->gmax_obs[c] = 0.0f;
  for (int c = 0; c < s->n_cells; ++c) {
    int start = s->offset[c];
    int nc = s->offset[c + 1] - start;
    int ngroups = or_group_count(nc, s->G);
    for (int g = 0; g < ngroups; ++g) {
      int gs = start + g * s->G;
      int gn = (g == ngroups - 1) ? nc - g * s->G : s->G;
      collide_group(s, c, nc, g, gs, gn);
    }
  }
  /* (sigma g)_max is raised after the step to sigma g of the largest candidate
   * relative speed, so it never depends on group order. */
  for (int c = 0; c < s->n_cells; ++c) {
    float sg = sigma_g(s, s->gmax_obs[c]);
    if (sg > s->smax[c]) s->smax[c] = sg;
  }
}

/* Raw moment sums per cell (Sec. 3: DSMC results are time averages): count,
 * sum v, sum v_i v_j (six), sum v_i |v|^2 (three); products in binary32, sums in
 * binary64.  Each sampled step adds half of these sums taken just before the
 * collisions and half taken just after them (`w` = 1/2 each time), i.e. the
 * trapezoidal average over the free flights between collision phases. */
static void sample_all(osim* s, double w) {
  for (int c = 0; c < s->n_cells; ++c) {
    double* a = s->acc + (size_t)c * NMOM;
    double* b = s->aacc + (size_t)c * NMOM;
    for (int k = s->offset[c]; k < s->offset[c + 1]; ++k) {
      float x = s->vx[k], y = s->vy[k], z = s->vz[k];
      float v2 = x * x + y * y + z * z;
      float pr[NMOM] = {1.0f, x, y, z, x * x, y * y, z * z, x * y, x * z, y * z,
                        x * v2, y * v2, z * v2};
      for (int m = 0; m < NMOM; ++m) b[m] += w * fabs((double)pr[m]);
      a[0] += w;
      a[1] += w * (double)x;
      a[2] += w * (double)y;
      a[3] += w * (double)z;
      a[4] += w * (double)(x * x);
      a[5] += w * (double)(y * y);
      a[6] += w * (double)(z * z);
      a[7] += w * (double)(x * y);
      a[8] += w * (double)(x * z);
      a[9] += w * (double)(y * z);
      a[10] += w * (double)(x * v2);
      a[11] += w * (double)(y * v2);
      a[12] += w * (double)(z * v2);
    }
  }
}

static void move_all(osim* s) {
  for (int p = 0; p < s->N; ++p)
    move_general(&s->y[p], &s->vx[p], &s->vy[p], &s->vz[p], s->dt, s->F, s->seed,
                 (uint32_t)s->step, (uint32_t)p, s->open_top, s->u_top, s->p_top, &s->err);
}

/* ------------------------------------------------------------------------- */
/* Public API (ctypes). */

/* Makes the boundary at y = 1 an open Chapman-Enskog reservoir with bulk velocity u
 * and shear stress P (rounded once to binary32), from the next step on. */
OR_EXPORT void or_set_open_top(osim* s, double u, double P) {
  s->open_top = 1;
  s->u_top = (float)u;
  s->p_top = (float)P;
}

OR_EXPORT void or_destroy(osim* s) {
  if (!s) return;
  free(s->y); free(s->vx); free(s->vy); free(s->vz);
  free(s->ty); free(s->tvx); free(s->tvy); free(s->tvz);
  free(s->cell); free(s->offset); free(s->smax); free(s->gmax_obs);
  free(s->ncand); free(s->nacc); free(s->acc); free(s->aacc);
  free(s);
}

/* omega: VHS viscosity index (0.5 = hard sphere); Kn: Knudsen number on the plate
 * gap (+inf = collisionless); F: body force in v0^2/H; dt_factor: time step as a
 * fraction of the equilibrium mean collision time 1/nu, nu = n sigma_ref <g>,
 * <g> = 2 sqrt(2/pi); dt > 0 overrides it.  Returns NULL on bad arguments. */
OR_EXPORT osim* or_create(double omega, double Kn, double F, int n_cells, int ppc,
                          uint64_t seed, int G, double dt_factor, double dt,
                          long long sample_start, int collisions) {
  if (!(Kn > 0.0) || n_cells < 1 || ppc < 1 || G < 2 || (G & 1)) return NULL;
  if (!(omega >= 0.5 && omega <= 1.0)) return NULL;
  if ((long long)n_cells * ppc > 0x7fffffffLL) return NULL;
  osim* s = (osim*)calloc(1, sizeof(osim));
  s->omega = omega; s->Kn = Kn; s->F_d = F; s->dt_factor = dt_factor; s->dt_in = dt;
  s->n_cells = n_cells; s->ppc = ppc; s->G = G; s->collisions = collisions;
  s->sample_start = sample_start; s->seed = seed;
  s->N = n_cells * ppc;
  s->nsig = or_nsigma(omega, Kn);
  double gbar = 2.0 * sqrt(2.0) / sqrt(M_PI);
  double nu = s->nsig * gbar;
  if (dt > 0.0)
    s->dt_d = dt;
  else if (nu > 0.0)
    s->dt_d = dt_factor / nu;
  else {
    free(s);
    return NULL;
  }
  s->dt = (float)s->dt_d;
  s->F = (float)F;
  s->coef = (float)(s->nsig * s->dt_d / (2.0 * (double)ppc));
  double cv = (omega == 0.5) ? 1.0 : pow(2.0, omega - 0.5) / tgamma(2.5 - omega);
  s->cvhs = (float)cv;
  s->vexp = (float)(2.0 - 2.0 * omega);
  s->vinv = (omega < 1.0) ? (float)(1.0 / (2.0 - 2.0 * omega)) : 0.0f;
  s->lncv = (float)log(cv);
  s->smax0 = (float)(cv * pow(5.0, 2.0 - 2.0 * omega));
  s->ncf = (float)n_cells;
  size_t n = (size_t)s->N, nb = n ? n : 1;
  s->y = malloc(nb * 4); s->vx = malloc(nb * 4); s->vy = malloc(nb * 4); s->vz = malloc(nb * 4);
  s->ty = malloc(nb * 4); s->tvx = malloc(nb * 4); s->tvy = malloc(nb * 4); s->tvz = malloc(nb * 4);
  s->cell = malloc(nb * sizeof(int));
  s->offset = calloc((size_t)n_cells + 1, sizeof(int));
  s->smax = malloc((size_t)n_cells * 4);
  s->gmax_obs = malloc((size_t)n_cells * 4);
  s->ncand = calloc((size_t)n_cells, sizeof(unsigned long long));
  s->nacc = calloc((size_t)n_cells, sizeof(unsigned long long));
  s->acc = calloc((size_t)n_cells * NMOM, sizeof(double));
  s->aacc = calloc((size_t)n_cells * NMOM, sizeof(double));
  for (int c = 0; c < n_cells; ++c) s->smax[c] = s->smax0;
  init_particles(s);
  index_cells(s);
  return s;
}

/* One DSMC step, in this order: collide within cells (state sorted by cell), with
 * half a sample taken before and half after the collisions when the step is at or
 * past sample_start; move every particle with the body force and the walls; sort
 * into cells again.  Steps are numbered from 1. */
OR_EXPORT int or_step(osim* s, int n) {
  for (int it = 0; it < n; ++it) {
    s->step += 1;
    int sampling = s->step >= s->sample_start;
    if (sampling) sample_all(s, 0.5);
    if (s->collisions && s->nsig > 0.0) collide_all(s);
    if (sampling) {
      sample_all(s, 0.5);
      s->n_samples += 1;
    }
    move_all(s);
    index_cells(s);
  }
  return s->err;
}

OR_EXPORT int or_n_particles(const osim* s) { return s->N; }
OR_EXPORT long long or_step_count(const osim* s) { return s->step; }
OR_EXPORT int or_error(const osim* s) { return s->err; }

/* dt, F, coef, cvhs, vexp, smax0, vinv, lncv as the binary32 values the step uses,
 * and nsig, dt in binary64. */
OR_EXPORT void or_params(const osim* s, float* f6, double* d2) {
  f6[0] = s->dt; f6[1] = s->F; f6[2] = s->coef; f6[3] = s->cvhs; f6[4] = s->vexp;
  f6[5] = s->smax0; f6[6] = s->vinv; f6[7] = s->lncv;
  d2[0] = s->nsig; d2[1] = s->dt_d;
}

OR_EXPORT void or_get_state(const osim* s, float* y, float* vx, float* vy, float* vz) {
  size_t b = (size_t)s->N * 4;
  memcpy(y, s->y, b); memcpy(vx, s->vx, b); memcpy(vy, s->vy, b); memcpy(vz, s->vz, b);
}

OR_EXPORT void or_get_cells(const osim* s, int* offset, float* smax,
                            unsigned long long* ncand, unsigned long long* nacc) {
  int nc = s->n_cells;
  if (offset) memcpy(offset, s->offset, sizeof(int) * ((size_t)nc + 1));
  if (smax) memcpy(smax, s->smax, 4 * (size_t)nc);
  if (ncand) memcpy(ncand, s->ncand, 8 * (size_t)nc);
  if (nacc) memcpy(nacc, s->nacc, 8 * (size_t)nc);
}

OR_EXPORT long long or_get_moments(const osim* s, double* out) {
  memcpy(out, s->acc, sizeof(double) * (size_t)s->n_cells * NMOM);
  return s->n_samples;
}

OR_EXPORT void or_get_abs_moments(const osim* s, double* out) {
  memcpy(out, s->aacc, sizeof(double) * (size_t)s->n_cells * NMOM);
}

OR_EXPORT void or_reset_samples(osim* s) {
  memset(s->acc, 0, sizeof(double) * (size_t)s->n_cells * NMOM);
  memset(s->aacc, 0, sizeof(double) * (size_t)s->n_cells * NMOM);
  memset(s->ncand, 0, 8 * (size_t)s->n_cells);
  memset(s->nacc, 0, 8 * (size_t)s->n_cells);
  s->n_samples = 0;
}

/* ------------------------------------------------------------------------- */
/* Array forms of the scalar routines, for the pins that sweep many inputs. */

OR_EXPORT void or_ln_array(const float* x, float* out, long long n) {
  for (long long i = 0; i < n; ++i) out[i] = or_ln(x[i]);
}

OR_EXPORT void or_exp_array(const float* x, float* out, long long n) {
  for (long long i = 0; i < n; ++i) out[i] = or_exp(x[i]);
}

/* The initial velocities of particles 0..n-1 of a run with this seed (three N(0,1/2)
 * deviates each), without building a run. */
OR_EXPORT int or_init_velocities(uint64_t seed, long long n, float* out3) {
  int ok = 1;
  for (long long p = 0; p < n; ++p) {
    family f = {seed, (uint32_t)p, 0u, 0u, TAG_INIT << 24, 1};
    if (!family_normals(&f, out3 + 3 * p, 3)) ok = 0;
  }
  return ok;
}

/* Re-emission speeds |vy| = sqrt(-ln u) of n bounces (slot p, bounce 0, step 1). */
OR_EXPORT void or_emission_speeds(uint64_t seed, long long n, float* out) {
  for (long long p = 0; p < n; ++p) {
    family f = {seed, (uint32_t)p, 0u, 1u, TAG_MOVE << 24, 1};
    uint32_t w[4];
    family_draw(&f, 0u, w);
    out[p] = sqrtf(-or_ln(or_u01(w[0])));
  }
}
