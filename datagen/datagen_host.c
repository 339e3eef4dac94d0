/*
 * datagen_host.c -- host (CPU) side of the seeded input generators.
 * Plain C, OpenMP over series; compiled with -ffp-contract=off so every value is
 * bit-identical to the device side (datagen_device.cu) built from the same header.
 */
#include "datagen_core.h"
#include <stdint.h>

/* Random walks number first_id .. first_id+count-1 of collection `seed`,
 * row-major [count][len]. */
void dg_walks_host(uint64_t seed, int64_t first_id, int64_t count, int32_t len,
                   float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i)
    dg_random_walk_one(seed, (uint64_t)(first_id + i), len, out + i * (int64_t)len);
}

/* Copies of collection members plus N(0, sigma_i^2) noise:
 * out[i][t] = walk(data_seed, ids[i])[t] + sigma[i] * e_{i,t}, with e drawn from
 * stream NOISE of noise_seed keyed by i. */
void dg_noisy_copies_host(uint64_t data_seed, uint64_t noise_seed, const int64_t* ids,
                          const float* sigma, int64_t count, int32_t len, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    float* row = out + i * (int64_t)len;
    dg_random_walk_one(data_seed, (uint64_t)ids[i], len, row);
    float e[4];
    for (int t = 0; t < len; ++t) {
      if ((t & 3) == 0) dg_normal4(noise_seed, DG_STREAM_NOISE, (uint64_t)i, (uint32_t)(t >> 2), e);
      row[t] = DG_ADD(row[t], DG_MUL(sigma[i], e[t & 3]));
    }
  }
}

/* count uniform picks in [0, n) (draws first .. first+count-1 of stream PICK). */
void dg_pick_host(uint64_t seed, int64_t first, int64_t count, int64_t n, int64_t* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = (int64_t)dg_pick(seed, (uint64_t)(first + i), (uint64_t)n);
}

/* Raw Philox4x32-10 block, exposed for known-answer tests. */
void dg_philox_host(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  dg_u32x4 c;
  for (int i = 0; i < 4; ++i) c.v[i] = ctr[i];
  dg_u32x4 r = dg_philox4x32_10(c, key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

/* Elementary functions, exposed so tests can bound their error against libm. */
float dg_ln_host(float x) { return dg_ln(x); }
void dg_sincos_2pi_host(float u, float* s, float* c) { dg_sincos_2pi(u, s, c); }
void dg_normals_host(uint64_t seed, uint32_t stream, uint64_t id, int32_t count, float* out) {
  float e[4];
  for (int t = 0; t < count; ++t) {
    if ((t & 3) == 0) dg_normal4(seed, stream, id, (uint32_t)(t >> 2), e);
    out[t] = e[t & 3];
  }
}

/* Mixed-shape series first_id .. first_id+count-1 of collection `seed`. */
void dg_mixed_host(uint64_t seed, int64_t first_id, int64_t count, int32_t len, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i)
    dg_mixed_one(seed, (uint64_t)(first_id + i), len, out + i * (int64_t)len);
}

/* Members of a mixed collection plus N(0, sigma^2) noise (stream NOISE of noise_seed,
 * keyed by i). */
void dg_mixed_noisy_host(uint64_t data_seed, uint64_t noise_seed, const int64_t* ids, float sigma, int64_t count,
                         int32_t len, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) {
    float* row = out + i * (int64_t)len;
    dg_mixed_one(data_seed, (uint64_t)ids[i], len, row);
    float e[4];
    for (int t = 0; t < len; ++t) {
      if ((t & 3) == 0) dg_normal4(noise_seed, DG_STREAM_NOISE, (uint64_t)i, (uint32_t)(t >> 2), e);
      row[t] = DG_ADD(row[t], DG_MUL(sigma, e[t & 3]));
    }
  }
}
