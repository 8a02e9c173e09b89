// Device building blocks of the docking hot path: counter-based RNG, GA
// operators, pair energy, grid lookup and compensated sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dock_internal.h"

namespace dk {

// Index checks of the bounds-checked build (DOCK_CHECKED): a failed check
// records kCheckBase - site in the call's status word (the first failure
// wins) and returns false; the caller then uses an index known to be in
// bounds, and the persistent loops stop at their next work item. No trap.
// The normal build compiles every check to `true`.
#ifdef DOCK_CHECKED
__device__ __forceinline__ bool check_ok(bool ok, int32_t *word, int site) {
  if (!ok && word != nullptr) atomicCAS(word, 0, kCheckBase - site);
  return ok;
}
#define DK_OK(cond, word, site) ::dk::check_ok((cond), (word), (site))
#define DK_BOUNDS(args) (&(args).bounds)
#else
#define DK_OK(cond, word, site) true
#define DK_BOUNDS(args) nullptr
#endif

// ---- AutoDock4 free-energy constants (the scoring form the paper's muDock
// ---- is "functionally equivalent" to, Section V) ----------------------------
// (double: the FP64 paths use them as they are; FP32 code rounds explicitly)
constexpr double kWVdw = 0.1662, kWHb = 0.1209, kWElec = 0.1406, kWSol = 0.1322;
constexpr double kCoulomb = 332.06363, kQasp = 0.01097, kSigma = 3.6;
constexpr double kDielA = -8.5525, kDielEps0 = 78.4, kDielK = 7.7839, kDielLambda = 0.003627;
constexpr double kDielB = kDielEps0 - kDielA;
// sqrt(W_elec 332.06363) = sqrt(46.688146378) rounded to float: a posed atom
// carries its charge times this, so a pair's Coulomb factor is one product
constexpr float kChargeScale = 6.8328725f;
// Readings of what the paper leaves open.
constexpr float kCutoff2 = 64.0f;   // (8 A)^2 non-bonded cutoff
constexpr float kRmin2 = 0.25f;     // distances floored at 0.5 A
constexpr double kEmax = 1.0e5;     // cap on a pair's raw 12-6 / 12-10 value and on M_t
constexpr float kEout = 1000.0f;    // energy of a ligand atom outside the grid box

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11). Counter (slot, individual, generation,
// ligand id), key (seed, 0). Word 2i / 2i+1 = low / high half of output i.
// ---------------------------------------------------------------------------
struct Words8 {
  uint32_t w[8];
};

// ROLLED: the ten rounds as a loop (the same values, less code where many
// call sites are inlined).
template <bool ROLLED = false>
__device__ __forceinline__ Words8 rng_words(uint64_t seed, uint64_t lig, uint32_t gen,
                                            uint32_t ind, uint32_t slot) {
  uint64_t c0 = slot, c1 = ind, c2 = gen, c3 = lig, k0 = seed, k1 = 0;
#pragma unroll (ROLLED ? 1 : 10)
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ULL, m1 = 0xCA5A826395121157ULL;
    uint64_t hi0 = __umul64hi(m0, c0), lo0 = m0 * c0;
    uint64_t hi1 = __umul64hi(m1, c2), lo1 = m1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  Words8 o;
  o.w[0] = (uint32_t)c0; o.w[1] = (uint32_t)(c0 >> 32);
  o.w[2] = (uint32_t)c1; o.w[3] = (uint32_t)(c1 >> 32);
  o.w[4] = (uint32_t)c2; o.w[5] = (uint32_t)(c2 >> 32);
  o.w[6] = (uint32_t)c3; o.w[7] = (uint32_t)(c3 >> 32);
  return o;
}

// Irwin-Hall normal from the first 12 words of slots (s, s+1):
// (sum of 12 top-24-bit words - 6 * 2^24) * 2^-24, converted round-to-nearest.
template <bool ROLLED = false>
__device__ __forceinline__ float rng_normal(uint64_t seed, uint64_t lig, uint32_t gen,
                                            uint32_t ind, uint32_t s) {
  Words8 a = rng_words<ROLLED>(seed, lig, gen, ind, s);
  Words8 b = rng_words<ROLLED>(seed, lig, gen, ind, s + 1);
  int64_t S = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) S += a.w[i] >> 8;
#pragma unroll
  for (int i = 0; i < 4; ++i) S += b.w[i] >> 8;
  float z = __ll2float_rn(S - 6LL * 16777216LL);
  return __fmul_rn(z, 0x1p-24f);
}

__device__ __forceinline__ float u24(uint32_t w) {
  return __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
}

__device__ __forceinline__ int pick(uint32_t w, int n) {
  return (int)(((uint64_t)w * (uint64_t)n) >> 32);
}

// Order-preserving key of an FP32 score: NaN counts as +inf, -0 as +0.
__device__ __forceinline__ uint32_t score_key(float s) {
  if (s != s) s = __int_as_float(0x7f800000);
  if (s == 0.0f) s = 0.0f;
  uint32_t u = __float_as_uint(s);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ bool better(const float *s, int a, int b) {
  uint32_t ka = score_key(s[a]), kb = score_key(s[b]);
  return ka < kb || (ka == kb && a < b);
}

constexpr float kPiF = 3.14159265358979323846f;
constexpr float kTwoPiF = 6.28318530717958647692f;

__device__ __forceinline__ void quat_normalize(float &w, float &x, float &y, float &z) {
  float n2 = __fmul_rn(w, w);
  n2 = __fadd_rn(n2, __fmul_rn(x, x));
  n2 = __fadd_rn(n2, __fmul_rn(y, y));
  n2 = __fadd_rn(n2, __fmul_rn(z, z));
  float n = __fsqrt_rn(n2);
  if (!(n > 0.0f)) {
    w = 1.0f; x = y = z = 0.0f;
    return;
  }
  w = __fdiv_rn(w, n); x = __fdiv_rn(x, n); y = __fdiv_rn(y, n); z = __fdiv_rn(z, n);
}

// Generation 0 genotype of individual ind (translation uniform in
// [-R/2, R/2)^3 from slot 0, quaternion of 4 normals from slots 1..8,
// torsions uniform in [-pi, pi) from slots 9, 10).
__device__ __forceinline__ void ga_init(float (&g)[DOCK_MAX_GENES], int k, float radius,
                                        uint64_t seed, uint64_t lig, uint32_t ind) {
  Words8 w = rng_words(seed, lig, 0, ind, 0);
  float half = __fmul_rn(0.5f, radius);
#pragma unroll
  for (int m = 0; m < 3; ++m) g[m] = __fadd_rn(__fmul_rn(u24(w.w[m]), radius), -half);
  float qv[4];
#pragma unroll 1
  for (int m = 0; m < 4; ++m) {
    float z = rng_normal(seed, lig, 0, ind, 1 + 2 * m);
#pragma unroll
    for (int mm = 0; mm < 4; ++mm)
      if (mm == m) qv[mm] = z;
  }
  quat_normalize(qv[0], qv[1], qv[2], qv[3]);
  g[3] = qv[0]; g[4] = qv[1]; g[5] = qv[2]; g[6] = qv[3];
  Words8 t0 = rng_words(seed, lig, 0, ind, 9);
  Words8 t1 = t0;
  if (k > 8) t1 = rng_words(seed, lig, 0, ind, 10);
#pragma unroll
  for (int j = 0; j < DOCK_MAX_TORSIONS; ++j) {
    float v = 0.0f;
    if (j < k) {
      uint32_t ww = j < 8 ? t0.w[j] : t1.w[j - 8];
      v = __fadd_rn(__fmul_rn(u24(ww), kTwoPiF), -kPiF);
    }
    g[7 + j] = v;
  }
}

__device__ __forceinline__ int gene_block(int g) { return g < 3 ? g : (g < 7 ? 3 : g - 3); }

// One GA step for individual ind >= 1 of a ligand with k torsions: binary
// tournaments (slot 0 words 0-3), two-point block crossover (words 4-6),
// per-gene mutation decisions (slots 1..3) and Irwin-Hall normal steps
// (slots 4+2g, 5+2g), torsion wrap, quaternion renormalisation.
__device__ __forceinline__ void ga_child(float (&g)[DOCK_MAX_GENES], int k, int P,
                                         const float *prev, const float *score, uint64_t thr_c,
                                         uint64_t thr_m, uint64_t seed, uint64_t lig,
                                         uint32_t gen, uint32_t ind) {
  const int G = 7 + k, B = 4 + k;
  Words8 w = rng_words(seed, lig, gen, ind, 0);
  int a1 = pick(w.w[0], P), a2 = pick(w.w[1], P), b1 = pick(w.w[2], P), b2 = pick(w.w[3], P);
  int pa = better(score, a1, a2) ? a1 : a2;
  int pb = better(score, b1, b2) ? b1 : b2;
  int lo = 0, hi = 0;
  if ((uint64_t)w.w[4] < thr_c) {
    int c1 = pick(w.w[5], B + 1), c2 = pick(w.w[6], B + 1);
    lo = min(c1, c2);
    hi = max(c1, c2);
  }
  const float *A = prev + (int64_t)pa * G, *Bp = prev + (int64_t)pb * G;
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e) {
    float v = 0.0f;
    if (e < G) {
      const int blk = gene_block(e);
      const float *src = (blk >= lo && blk < hi) ? Bp : A;
      v = __ldg(src + e);
    }
    g[e] = v;
  }
  Words8 m0 = rng_words(seed, lig, gen, ind, 1);
  Words8 m1 = m0, m2 = m0;
  if (G > 8) m1 = rng_words(seed, lig, gen, ind, 2);
  if (G > 16) m2 = rng_words(seed, lig, gen, ind, 3);
  uint32_t mask = 0;
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e) {
    uint32_t ww = e < 8 ? m0.w[e] : (e < 16 ? m1.w[e - 8] : m2.w[e - 16]);
    if (e < G && (uint64_t)ww < thr_m) mask |= 1u << e;
  }
  bool qmut = false;
  // mutations are rare: draw each normal in a rolled loop, then apply it
#pragma unroll 1
  while (mask) {
    const int e = __ffs(mask) - 1;
    mask &= mask - 1;
    float z = rng_normal(seed, lig, gen, ind, 4 + 2 * e);
    float sigma = e < 3 ? 1.0f : (e < 7 ? 0.1f : 0.5f);
    float d = __fmul_rn(sigma, z);
    qmut |= (e >= 3 && e < 7);
#pragma unroll
    for (int ee = 0; ee < DOCK_MAX_GENES; ++ee) {
      if (ee == e) {
        float v = __fadd_rn(g[ee], d);
        if (ee >= 7) {
          if (v > kPiF) v = __fadd_rn(v, -kTwoPiF);
          else if (v < -kPiF) v = __fadd_rn(v, kTwoPiF);
        }
        g[ee] = v;
      }
    }
  }
  if (qmut) quat_normalize(g[3], g[4], g[5], g[6]);
}

// The same child computed by the L lanes of a group together: the Philox
// blocks of slot 0 (tournaments, crossover) and slots 1..3 (mutation
// decisions) are spread over the lanes and exchanged by shuffles; every lane
// ends with the full genotype, bit-identical to ga_child.
template <int L>
__device__ __forceinline__ void ga_child_group(float (&g)[DOCK_MAX_GENES], int k, int P,
                                               const float *prev, const float *score,
                                               uint64_t thr_c, uint64_t thr_m, uint64_t seed,
                                               uint64_t lig, uint32_t gen, uint32_t ind, int lane,
                                               unsigned gmask) {
  const int G = 7 + k, B = 4 + k;
  const int nslots = 1 + (G + 7) / 8;  // slot 0 + mutation slots
  // this lane's slots: lane, lane + L, ... (< nslots)
  uint32_t tw[7] = {0, 0, 0, 0, 0, 0, 0};
  uint32_t mask = 0;
  for (int sl = lane; sl < nslots; sl += L) {
    const Words8 w = rng_words(seed, lig, gen, ind, (uint32_t)sl);
    if (sl == 0) {
#pragma unroll
      for (int i = 0; i < 7; ++i) tw[i] = w.w[i];
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int gi = (sl - 1) * 8 + e;
        if (gi < G && (uint64_t)w.w[e] < thr_m) mask |= 1u << gi;
      }
    }
  }
  // slot 0 lives on lane 0 of the group; the mask bits are spread over lanes
#pragma unroll
  for (int i = 0; i < 7; ++i) tw[i] = __shfl_sync(gmask, tw[i], 0, L);
#pragma unroll
  for (int o = 1; o < L; o <<= 1) mask |= __shfl_xor_sync(gmask, mask, o, L);
  const int a1 = pick(tw[0], P), a2 = pick(tw[1], P), b1 = pick(tw[2], P), b2 = pick(tw[3], P);
  const int pa = better(score, a1, a2) ? a1 : a2;
  const int pb = better(score, b1, b2) ? b1 : b2;
  int lo = 0, hi = 0;
  if ((uint64_t)tw[4] < thr_c) {
    const int c1 = pick(tw[5], B + 1), c2 = pick(tw[6], B + 1);
    lo = min(c1, c2);
    hi = max(c1, c2);
  }
  const float *A = prev + (int64_t)pa * G, *Bp = prev + (int64_t)pb * G;
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e) {
    float v = 0.0f;
    if (e < G) {
      const int blk = gene_block(e);
      const float *src = (blk >= lo && blk < hi) ? Bp : A;
      v = __ldg(src + e);
    }
    g[e] = v;
  }
  bool qmut = false;
#pragma unroll 1
  while (mask) {
    const int e = __ffs(mask) - 1;
    mask &= mask - 1;
    float z = rng_normal(seed, lig, gen, ind, 4 + 2 * e);
    float sigma = e < 3 ? 1.0f : (e < 7 ? 0.1f : 0.5f);
    float d = __fmul_rn(sigma, z);
    qmut |= (e >= 3 && e < 7);
#pragma unroll
    for (int ee = 0; ee < DOCK_MAX_GENES; ++ee) {
      if (ee == e) {
        float v = __fadd_rn(g[ee], d);
        if (ee >= 7) {
          if (v > kPiF) v = __fadd_rn(v, -kTwoPiF);
          else if (v < -kPiF) v = __fadd_rn(v, kTwoPiF);
        }
        g[ee] = v;
      }
    }
  }
  if (qmut) quat_normalize(g[3], g[4], g[5], g[6]);
}

// ---------------------------------------------------------------------------
// Compensated sums
// ---------------------------------------------------------------------------
struct Kahan {
  float s = 0.0f, c = 0.0f;  // true sum ~ s - c
  __device__ __forceinline__ void add(float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

// Knuth TwoSum: a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float aa = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// One 128-bit read-only load.
__device__ __forceinline__ float4 ld4(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// ---------------------------------------------------------------------------
// Pair energy (FP32) from a 32-byte pair record
// {c12, c6, c10, cap, qq, ds, bits(i | j << 16), 0} (weights folded in):
//   min(c12 r^-12 - c6 r^-6 - c10 r^-10, cap) + qq / (eps(r) r) + ds exp(-r^2 / 2 sigma^2)
// with eps(r) = A + B / (1 + k exp(-lambda B r)), so 1 / (eps r) = (1 + k e) / ((A (1 + k e) + B) r).
// Zero at r >= 8 A; r floored at 0.5 A. The hardware approximations
// (rsqrt, ex2, rcp, flush-to-zero) see arguments far from the denormal range.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float pair_energy(float r2, const float (&rec)[8]) {
  const float kLb = (float)(-kDielLambda * kDielB * 1.4426950408889634);  // ex2 argument per A
  const float kS = (float)(-1.4426950408889634 / (2.0 * kSigma * kSigma));
  const float dA = (float)kDielA, dB = (float)kDielB, dK = (float)kDielK;
  const float r2c = fmaxf(r2, kRmin2);
  const float ir = rsqrt_ftz(r2c);
  const float ir2 = ir * ir;
  const float r = r2c * ir;
  const float ir4 = ir2 * ir2;
  const float ir6 = ir4 * ir2;
  // c12 r^-12 - c6 r^-6 - c10 r^-10 = r^-6 (c12 r^-6 - (c6 + c10 r^-4))
  const float disp = fminf(ir6 * fmaf(rec[0], ir6, -fmaf(rec[2], ir4, rec[1])), rec[3]);
  const float onek = 1.0f + dK * ex2_ftz(kLb * r);
  const float elec = rec[4] * onek * rcp_ftz((dA * onek + dB) * r);
  const float des = rec[5] * ex2_ftz(kS * r2c);
  const float e = disp + elec + des;
  return r2 < kCutoff2 ? e : 0.0f;
}


// The same pair energy from a 16-byte record {offsets, c12, cb, ds}: cb = c6
// for a 12-6 pair and -c10 for a 12-10 (H-bond) pair, whose sign also picks
// the cap w EMAX; qq = W_elec 332.06363 q_i q_j is the product of the two
// atoms' scaled charges.
__device__ __forceinline__ float pair_energy16(float r2, float c12, float cb, float ds, float qq) {
  const float kLb = (float)(-kDielLambda * kDielB * 1.4426950408889634);  // ex2 argument per A
  const float kS = (float)(-1.4426950408889634 / (2.0 * kSigma * kSigma));
  const float dA = (float)kDielA, dB = (float)kDielB, dK = (float)kDielK;
  const float kCapVdw = (float)((double)kWVdw * kEmax), kCapHb = (float)((double)kWHb * kEmax);
  const float r2c = fmaxf(r2, kRmin2);
  const float ir = rsqrt_ftz(r2c);
  const float ir2 = ir * ir;
  const float r = r2c * ir;
  const float ir4 = ir2 * ir2;
  const float ir6 = ir4 * ir2;
  const bool hb = cb < 0.0f;
  // r^-6 (c12 r^-6 - c6) or r^-6 (c12 r^-6 - c10 r^-4)
  const float disp = fminf(ir6 * fmaf(c12, ir6, -fabsf(cb) * (hb ? ir4 : 1.0f)), hb ? kCapHb : kCapVdw);
  const float onek = 1.0f + dK * ex2_ftz(kLb * r);
  const float elec = qq * onek * rcp_ftz((dA * onek + dB) * r);
  const float des = ds * ex2_ftz(kS * r2c);
  const float e = disp + elec + des;
  return r2 < kCutoff2 ? e : 0.0f;
}

// Grid lookup of M_t + q E + |q| D split in two halves so other work can run
// while the loads are in flight: grid_issue computes the cell and fetches the
// two 32-byte (x, y)-cell records (planes z and z+1) with one 256-bit load
// each, not allocated in L1 (interpolated here in FP32, no texture
// filtering); grid_finish interpolates. A point
// outside the grid box (faces count as inside) gives EOUT.
struct Lookup {
  float c0[8], c1[8];
  float fx, fy, fz, q;
  bool inside;
};

__device__ __forceinline__ Lookup grid_issue(const GridView &G, int t, float q, float x, float y,
                                             float z, int32_t *check_word = nullptr) {
  Lookup L;
  // grid coordinates u = x / h - origin / h (one rounding less than (x - o) / h)
  const float ux = fmaf(x, G.inv_h, G.gx), uy = fmaf(y, G.inv_h, G.gy), uz = fmaf(z, G.inv_h, G.gz);
  const float nm1 = (float)(G.n - 1);
  L.inside = ux >= 0.0f && ux <= nm1 && uy >= 0.0f && uy <= nm1 && uz >= 0.0f && uz <= nm1;
  L.q = q;
  if (L.inside) {
    const int ix = min((int)ux, G.n - 2), iy = min((int)uy, G.n - 2), iz = min((int)uz, G.n - 2);
    L.fx = ux - (float)ix;
    L.fy = uy - (float)iy;
    L.fz = uz - (float)iz;
    const int nc = G.n - 1;
    const int sg = q < 0.0f ? 1 : 0;
    // 32-bit element index (dock_create_pocket bounds the record count)
    int e = ((((2 * t + sg) * G.n + iz) * nc + iy) * nc + ix) * 2;
    if (!DK_OK(e >= 0 && e + G.plane_elems + 1 < G.tex_elems && t < G.n_types, check_word, 9))
      e = 0;
    const int ez = e + G.plane_elems;
    // two 256-bit loads that do not allocate in L1 (the records are read
    // once per atom; L1 keeps the pair records and coordinates instead)
    const float *pz0 = G.xycell + (int64_t)e * 4, *pz1 = G.xycell + (int64_t)ez * 4;
    asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(L.c0[0]), "=f"(L.c0[1]), "=f"(L.c0[2]), "=f"(L.c0[3]), "=f"(L.c0[4]),
                   "=f"(L.c0[5]), "=f"(L.c0[6]), "=f"(L.c0[7]) : "l"(pz0));
    asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(L.c1[0]), "=f"(L.c1[1]), "=f"(L.c1[2]), "=f"(L.c1[3]), "=f"(L.c1[4]),
                   "=f"(L.c1[5]), "=f"(L.c1[6]), "=f"(L.c1[7]) : "l"(pz1));
  }
  return L;
}

__device__ __forceinline__ float grid_finish(const Lookup &L) {
  if (!L.inside) return kEout;
  const float q = L.q, fx = L.fx, fy = L.fy;
  auto plane = [&](const float (&c)[8]) {
    const float v00 = c[0] + q * c[1], v10 = c[2] + q * c[3];
    const float v01 = c[4] + q * c[5], v11 = c[6] + q * c[7];
    const float a = v00 + fx * (v10 - v00), b = v01 + fx * (v11 - v01);
    return a + fy * (b - a);
  };
  const float p0 = plane(L.c0), p1 = plane(L.c1);
  return p0 + L.fz * (p1 - p0);
}

// ---------------------------------------------------------------------------
// Cutoff search in the protein cell list (CellGrid). f(j0, j1) is called for
// each contiguous atom range that can hold an atom within sqrt(rc2) of some
// point of the box [xl, xh] x [yl, yh] x [zl, zh] (a point: lo = hi): the rows
// (cy, cz) from one y-z cell below the box to one above (the y-z cell edge
// equals the 8 A cutoff), a row skipped when its y-z square is sqrt(rc2) or
// farther from the box's y-z rectangle, and in a kept row the x cells that
// meet [xl - e, xh + e], e the half chord of the cutoff sphere at that
// distance. rc2 carries a margin over the cutoff that covers the FP32
// rounding of these bounds; the caller's pair test decides.
// ---------------------------------------------------------------------------
constexpr float kCutoffSearch2 = 64.016f;  // (8 A + 1e-3 A)^2

__device__ __forceinline__ int cell_floor(float u, int d) {
  return (int)floorf(fminf(fmaxf(u, -4.0f), (float)d + 4.0f));  // NaN -> -4
}

template <class F>
__device__ __forceinline__ void cutoff_ranges_box(const CellGrid &C, float xl, float xh, float yl,
                                                  float yh, float zl, float zh, float rc2, F &&f) {
  const int y0 = max(cell_floor((yl - C.loy) * (1.0f / kCellYZ), C.dy) - 1, 0);
  const int y1 = min(cell_floor((yh - C.loy) * (1.0f / kCellYZ), C.dy) + 1, C.dy - 1);
  const int z0 = max(cell_floor((zl - C.loz) * (1.0f / kCellYZ), C.dz) - 1, 0);
  const int z1 = min(cell_floor((zh - C.loz) * (1.0f / kCellYZ), C.dz) + 1, C.dz - 1);
  const float uxl = (xl - C.lox) * (1.0f / kCellX), uxh = (xh - C.lox) * (1.0f / kCellX);
  for (int cz = z0; cz <= z1; ++cz) {
    const float c0 = fmaf((float)cz, kCellYZ, C.loz);
    const float dzv = fmaxf(fmaxf(c0 - zh, zl - (c0 + kCellYZ)), 0.0f);
    for (int cy = y0; cy <= y1; ++cy) {
      const float b0 = fmaf((float)cy, kCellYZ, C.loy);
      const float dyv = fmaxf(fmaxf(b0 - yh, yl - (b0 + kCellYZ)), 0.0f);
      const float d2 = fmaf(dyv, dyv, dzv * dzv);
      if (!(d2 < rc2)) continue;
      const float e = sqrtf(rc2 - d2) * (1.0f / kCellX);
      const int xa = max((int)floorf(fminf(fmaxf(uxl - e, -1.0f), (float)C.dx)), 0);
      const int xb = min((int)floorf(fminf(fmaxf(uxh + e, -1.0f), (float)C.dx)), C.dx - 1);
      if (xa > xb) continue;
      const int row = (cz * C.dy + cy) * C.dx;
      f(__ldg(C.cell_start + row + xa), __ldg(C.cell_start + row + xb + 1));
    }
  }
}

template <class F>
__device__ __forceinline__ void cutoff_ranges(const CellGrid &C, float px, float py, float pz,
                                              float rc2, F &&f) {
  cutoff_ranges_box(C, px, px, py, py, pz, pz, rc2, static_cast<F &&>(f));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace dk
