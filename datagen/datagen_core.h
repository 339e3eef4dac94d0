/*
 * datagen_core.h -- seeded, counter-based synthetic data series generators.
 *
 * This header is the ONE module shared by the CPU oracle side and the GPU side:
 * it produces input bytes only and holds none of the similarity-search method's
 * arithmetic (no normalisation, no PAA, no quantisation, no distances).
 *
 * Every value is a pure function of (seed, series id, point index), so any slice
 * of a collection can be regenerated alone, on the host or on the device, and the
 * two give bit-identical fp32 values:
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 *     as 1, 2, 3", SC'11) supplies 4 x 32 random bits per counter;
 *   - normals come from the Box-Muller transform (Box & Muller, 1958);
 *   - ln, sin and cos are written out here from their series expansions
 *     (ln through the atanh series of (m-1)/(m+1), sin/cos through Taylor series on
 *     a quarter period), using only IEEE-754 single-precision +, -, *, / and sqrt,
 *     each rounded once (no fused multiply-add), so host and device agree bit for bit.
 *
 * The random-walk generator follows the paper's synthetic data recipe (Section IV,
 * "Datasets"): the first point is an N(0,1) draw and every further point adds a new
 * N(0,1) draw to the previous value.
 *
 * Compile the host side with -ffp-contract=off; the device side uses the explicit
 * round-to-nearest intrinsics below, which nvcc never contracts.
 */
#ifndef DATAGEN_CORE_H
#define DATAGEN_CORE_H

#include <stdint.h>

#if defined(__CUDACC__)
#define DG_FN static __host__ __device__ __forceinline__
#else
#define DG_FN static inline
#endif

#if defined(__CUDA_ARCH__)
#define DG_ADD(a, b) __fadd_rn((a), (b))
#define DG_SUB(a, b) __fsub_rn((a), (b))
#define DG_MUL(a, b) __fmul_rn((a), (b))
#define DG_DIV(a, b) __fdiv_rn((a), (b))
#define DG_SQRT(a) __fsqrt_rn((a))
#define DG_F2U(f) __float_as_uint(f)
#define DG_U2F(u) __uint_as_float(u)
#else
#include <math.h>
#include <string.h>
#define DG_ADD(a, b) ((float)((a) + (b)))
#define DG_SUB(a, b) ((float)((a) - (b)))
#define DG_MUL(a, b) ((float)((a) * (b)))
#define DG_DIV(a, b) ((float)((a) / (b)))
#define DG_SQRT(a) sqrtf((a))
static inline uint32_t dg_f2u_host(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static inline float dg_u2f_host(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
#define DG_F2U(f) dg_f2u_host(f)
#define DG_U2F(u) dg_u2f_host(u)
#endif

/* Stream tags: the 4th Philox counter word, so distinct uses of one seed never
 * share random bits. */
enum {
  DG_STREAM_WALK = 0,      /* random-walk steps                           */
  DG_STREAM_NOISE = 1,     /* additive noise on query copies              */
  DG_STREAM_PICK = 2,      /* choice of dataset ids                       */
  DG_STREAM_SHAPE = 3,     /* per-series shape parameters (mixed family)  */
};

typedef struct { uint32_t v[4]; } dg_u32x4;

DG_FN void dg_mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
 * increments 0x9E3779B9 / 0xBB67AE85 (SC'11, Section 5). */
DG_FN dg_u32x4 dg_philox4x32_10(dg_u32x4 ctr, uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint32_t hi0, lo0, hi1, lo1;
    dg_mulhilo(0xD2511F53u, ctr.v[0], &hi0, &lo0);
    dg_mulhilo(0xCD9E8D57u, ctr.v[2], &hi1, &lo1);
    dg_u32x4 n;
    n.v[0] = hi1 ^ ctr.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ ctr.v[3] ^ k1;
    n.v[3] = lo0;
    ctr = n;
  }
  return ctr;
}

/* Four random words for (seed, stream, id, block). */
DG_FN dg_u32x4 dg_bits(uint64_t seed, uint32_t stream, uint64_t id, uint32_t block) {
  dg_u32x4 c;
  c.v[0] = block;
  c.v[1] = (uint32_t)id;
  c.v[2] = (uint32_t)(id >> 32);
  c.v[3] = stream;
  return dg_philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

/* Uniform in (0, 1]: 24 random bits, offset by one ulp so ln() stays finite. */
DG_FN float dg_u01_open0(uint32_t b) {
  return DG_MUL((float)((b >> 8) + 1u), 5.9604644775390625e-08f); /* 2^-24 */
}
/* Uniform in [0, 1). */
DG_FN float dg_u01(uint32_t b) {
  return DG_MUL((float)(b >> 8), 5.9604644775390625e-08f);
}

/* ln(x), x > 0 finite and normal: x = m * 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(r), r = (m-1)/(m+1), |r| <= 0.1716, series to r^11. */
DG_FN float dg_ln(float x) {
  uint32_t bits = DG_F2U(x);
  int e = (int)((bits >> 23) & 0xffu) - 127;
  float m = DG_U2F((bits & 0x007fffffu) | 0x3f800000u);
  if (m > 1.41421356f) { m = DG_MUL(m, 0.5f); e += 1; }
  float r = DG_DIV(DG_SUB(m, 1.0f), DG_ADD(m, 1.0f));
  float r2 = DG_MUL(r, r);
  float p = 0.0909090936f;                          /* 1/11 */
  p = DG_ADD(0.111111112f, DG_MUL(r2, p));          /* 1/9  */
  p = DG_ADD(0.142857149f, DG_MUL(r2, p));          /* 1/7  */
  p = DG_ADD(0.200000003f, DG_MUL(r2, p));          /* 1/5  */
  p = DG_ADD(0.333333343f, DG_MUL(r2, p));          /* 1/3  */
  p = DG_ADD(1.0f, DG_MUL(r2, p));
  float lnm = DG_MUL(2.0f, DG_MUL(r, p));
  return DG_ADD(lnm, DG_MUL((float)e, 0.693147182f)); /* ln 2 */
}

/* sin(x), cos(x) for x in [0, pi/2]: Taylor series to x^13 / x^14 in Horner form.
 * The first omitted terms are below 7e-10 on this interval. */
DG_FN void dg_sincos_q(float x, float* s, float* c) {
  float x2 = DG_MUL(x, x);
  float p = 1.6059043836821613e-10f;                /* +1/13! */
  p = DG_ADD(-2.505210838544172e-08f, DG_MUL(x2, p)); /* -1/11! */
  p = DG_ADD(2.7557319223985893e-06f, DG_MUL(x2, p)); /* +1/9!  */
  p = DG_ADD(-1.984126984126984e-04f, DG_MUL(x2, p)); /* -1/7!  */
  p = DG_ADD(8.333333333333333e-03f, DG_MUL(x2, p));  /* +1/5!  */
  p = DG_ADD(-0.16666666666666666f, DG_MUL(x2, p));   /* -1/3!  */
  p = DG_ADD(1.0f, DG_MUL(x2, p));
  *s = DG_MUL(x, p);
  float q = -1.1470745597729725e-11f;               /* -1/14! */
  q = DG_ADD(2.08767569878681e-09f, DG_MUL(x2, q));   /* +1/12! */
  q = DG_ADD(-2.755731922398589e-07f, DG_MUL(x2, q)); /* -1/10! */
  q = DG_ADD(2.48015873015873e-05f, DG_MUL(x2, q));   /* +1/8!  */
  q = DG_ADD(-1.388888888888889e-03f, DG_MUL(x2, q)); /* -1/6!  */
  q = DG_ADD(4.1666666666666664e-02f, DG_MUL(x2, q)); /* +1/4!  */
  q = DG_ADD(-0.5f, DG_MUL(x2, q));                   /* -1/2!  */
  *c = DG_ADD(1.0f, DG_MUL(x2, q));
}

/* sin(2 pi u), cos(2 pi u) for u in [0, 1): quarter-period reduction is exact
 * (4u and its fraction are exact in fp32), then the quarter-period series. */
DG_FN void dg_sincos_2pi(float u, float* s, float* c) {
  float v = DG_MUL(u, 4.0f);
  int quad = (int)v;
  float f = DG_SUB(v, (float)quad);
  float sq, cq;
  dg_sincos_q(DG_MUL(f, 1.57079632679489662f), &sq, &cq);
  switch (quad & 3) {
    case 0: *s = sq; *c = cq; break;
    case 1: *s = cq; *c = -sq; break;
    case 2: *s = -sq; *c = -cq; break;
    default: *s = -cq; *c = sq; break;
  }
}

/* Two independent N(0,1) draws from one pair of random words (Box-Muller). */
DG_FN void dg_box_muller(uint32_t a, uint32_t b, float* z0, float* z1) {
  float u1 = dg_u01_open0(a);
  float u2 = dg_u01(b);
  float r = DG_SQRT(DG_MUL(-2.0f, dg_ln(u1)));
  float s, c;
  dg_sincos_2pi(u2, &s, &c);
  *z0 = DG_MUL(r, c);
  *z1 = DG_MUL(r, s);
}

/* The four N(0,1) draws number 4*block .. 4*block+3 of (seed, stream, id). */
DG_FN void dg_normal4(uint64_t seed, uint32_t stream, uint64_t id, uint32_t block,
                      float out[4]) {
  dg_u32x4 r = dg_bits(seed, stream, id, block);
  dg_box_muller(r.v[0], r.v[1], &out[0], &out[1]);
  dg_box_muller(r.v[2], r.v[3], &out[2], &out[3]);
}

/* Random walk number `id` of collection `seed`, points [0, len):
 * x_0 = e_0, x_t = x_{t-1} + e_t with e_t ~ N(0,1) (fp32, sequential in t). */
DG_FN void dg_random_walk_one(uint64_t seed, uint64_t id, int len, float* out) {
  float x = 0.0f;
  float e[4];
  for (int t = 0; t < len; ++t) {
    if ((t & 3) == 0) dg_normal4(seed, DG_STREAM_WALK, id, (uint32_t)(t >> 2), e);
    x = (t == 0) ? e[0] : DG_ADD(x, e[t & 3]);
    out[t] = x;
  }
}

/* Laplace(0, b) draw from 32 random bits by inversion: u in (-1/2, 1/2),
 * e = -b sign(u) ln(1 - 2|u|). */
DG_FN float dg_laplace(uint32_t bits, float b) {
  const float u = DG_SUB(dg_u01_open0(bits), 0.5f);  /* (-0.5, 0.5] */
  const float a = u < 0.0f ? -u : u;
  float one_m = DG_SUB(1.0f, DG_MUL(2.0f, a));
  if (one_m < 5.9604644775390625e-08f) one_m = 5.9604644775390625e-08f;
  const float mag = DG_MUL(-b, dg_ln(one_m));
  return u < 0.0f ? -mag : mag;
}

/* Mixed-shape collection: series `id` of collection `seed` is, with probability 1/2
 * each (stream SHAPE), either
 *  - a noisy sinusoid sin(2 pi (f t / len + phi)) + N(0, 0.3), f ~ U[1, 32) cycles,
 *    phi ~ U[0, 1) of a period; or
 *  - a random walk with Laplace(0, 1/sqrt 2) (unit-variance) steps, the steps of one
 *    burst of ceil(len / 20) consecutive points (5% of the series, at a uniform
 *    offset) multiplied by 10. */
DG_FN void dg_mixed_one(uint64_t seed, uint64_t id, int len, float* out) {
  dg_u32x4 sh = dg_bits(seed, DG_STREAM_SHAPE, id, 0);
  float e[4];
  if ((sh.v[0] >> 31) == 0u) {
    const float f = DG_ADD(1.0f, DG_MUL(31.0f, dg_u01(sh.v[1])));
    const float phi = dg_u01(sh.v[2]);
    const float inv_len = DG_DIV(1.0f, (float)len);
    for (int t = 0; t < len; ++t) {
      if ((t & 3) == 0) dg_normal4(seed, DG_STREAM_WALK, id, (uint32_t)(t >> 2), e);
      const float a = DG_ADD(DG_MUL(DG_MUL(f, (float)t), inv_len), phi);
      const float frac = DG_SUB(a, (float)(int)a);
      float sv, cv;
      dg_sincos_2pi(frac, &sv, &cv);
      out[t] = DG_ADD(sv, DG_MUL(0.547722558f, e[t & 3])); /* sqrt(0.3) */
    }
  } else {
    const int burst = (len + 19) / 20;
    const int start = (int)(((uint64_t)sh.v[3] * (uint64_t)(len - burst + 1)) >> 32);
    float x = 0.0f;
    for (int t = 0; t < len; ++t) {
      dg_u32x4 r;
      if ((t & 3) == 0) {
        r = dg_bits(seed, DG_STREAM_WALK, id, (uint32_t)(t >> 2));
        e[0] = dg_laplace(r.v[0], 0.707106769f);
        e[1] = dg_laplace(r.v[1], 0.707106769f);
        e[2] = dg_laplace(r.v[2], 0.707106769f);
        e[3] = dg_laplace(r.v[3], 0.707106769f);
      }
      float step = e[t & 3];
      if (t >= start && t < start + burst) step = DG_MUL(step, 10.0f);
      x = (t == 0) ? step : DG_ADD(x, step);
      out[t] = x;
    }
  }
}

/* Uniform integer in [0, n) for draw number `i` of stream PICK (multiply-shift on
 * 64 random bits; bias below 2^-30 for n < 2^34). */
DG_FN uint64_t dg_pick(uint64_t seed, uint64_t i, uint64_t n) {
  dg_u32x4 r = dg_bits(seed, DG_STREAM_PICK, i, 0);
  uint64_t x = ((uint64_t)r.v[0] << 32) | r.v[1];
  /* high 64 bits of x * n, written with 32-bit limbs for portability */
  uint64_t xl = x & 0xffffffffull, xh = x >> 32;
  uint64_t nl = n & 0xffffffffull, nh = n >> 32;
  uint64_t ll = xl * nl, lh = xl * nh, hl = xh * nl, hh = xh * nh;
  uint64_t mid = (ll >> 32) + (lh & 0xffffffffull) + (hl & 0xffffffffull);
  return hh + (lh >> 32) + (hl >> 32) + (mid >> 32);
}
#endif
