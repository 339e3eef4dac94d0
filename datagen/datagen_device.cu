/*
 * datagen_device.cu -- device side of the seeded input generators: fills large
 * collections directly in HBM with values bit-identical to datagen_host.c.
 * One thread owns one series (the walk is a sequential sum); a warp stages 32
 * points of its 32 series in shared memory so global stores are whole 128-byte rows.
 */
#include <cuda_runtime.h>
#include "datagen_core.h"

namespace {

constexpr int kWarps = 4;

__global__ void __launch_bounds__(kWarps * 32)
walks_kernel(uint64_t seed, int64_t first_id, int64_t count, int32_t len, float* __restrict__ out) {
  __shared__ float tile[kWarps][32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * 32;
  if (base >= count) return;
  const int64_t my = base + lane;
  float x = 0.0f, e[4];
  for (int t0 = 0; t0 < len; t0 += 32) {
    for (int dt = 0; dt < 32 && t0 + dt < len; ++dt) {
      const int t = t0 + dt;
      if ((t & 3) == 0) dg_normal4(seed, DG_STREAM_WALK, (uint64_t)(first_id + my), (uint32_t)(t >> 2), e);
      x = (t == 0) ? e[0] : DG_ADD(x, e[t & 3]);
      tile[warp][lane][dt] = x;
    }
    __syncwarp();
    const int tcol = t0 + lane;
    for (int r = 0; r < 32; ++r) {
      if (base + r < count && tcol < len) out[(base + r) * (int64_t)len + tcol] = tile[warp][r][lane];
    }
    __syncwarp();
  }
}

__global__ void noisy_kernel(uint64_t data_seed, uint64_t noise_seed, const int64_t* __restrict__ ids,
                             const float* __restrict__ sigma, int64_t count, int32_t len,
                             float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float* row = out + i * (int64_t)len;
  dg_random_walk_one(data_seed, (uint64_t)ids[i], len, row);
  float e[4];
  for (int t = 0; t < len; ++t) {
    if ((t & 3) == 0) dg_normal4(noise_seed, DG_STREAM_NOISE, (uint64_t)i, (uint32_t)(t >> 2), e);
    row[t] = DG_ADD(row[t], DG_MUL(sigma[i], e[t & 3]));
  }
}

// The mixed-shape family: one thread per series, written in place.
__global__ void mixed_kernel(uint64_t seed, int64_t first_id, int64_t count, int32_t len, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  dg_mixed_one(seed, (uint64_t)(first_id + i), len, out + i * (int64_t)len);
}

}  // namespace

extern "C" int dg_mixed_device(uint64_t seed, int64_t first_id, int64_t count, int32_t len, float* out,
                               void* stream) {
  if (count <= 0) return 0;
  if (len <= 0 || out == nullptr) return (int)cudaErrorInvalidValue;
  const int64_t blocks = (count + 127) / 128;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  mixed_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(seed, first_id, count, len, out);
  return (int)cudaGetLastError();
}

extern "C" int dg_walks_device(uint64_t seed, int64_t first_id, int64_t count, int32_t len,
                               float* out, void* stream) {
  if (count <= 0) return 0;
  if (len <= 0 || out == nullptr) return (int)cudaErrorInvalidValue;
  const int64_t warps = (count + 31) / 32;
  const int64_t blocks = (warps + kWarps - 1) / kWarps;
  if (blocks > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
  walks_kernel<<<(unsigned)blocks, kWarps * 32, 0, (cudaStream_t)stream>>>(seed, first_id, count, len, out);
  return (int)cudaGetLastError();
}

/* ids and sigma are device arrays of `count` entries. */
extern "C" int dg_noisy_copies_device(uint64_t data_seed, uint64_t noise_seed, const int64_t* ids,
                                      const float* sigma, int64_t count, int32_t len, float* out,
                                      void* stream) {
  if (count <= 0) return 0;
  if (len <= 0 || out == nullptr || ids == nullptr || sigma == nullptr) return (int)cudaErrorInvalidValue;
  const int64_t blocks = (count + 127) / 128;
  noisy_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(data_seed, noise_seed, ids, sigma, count, len, out);
  return (int)cudaGetLastError();
}
