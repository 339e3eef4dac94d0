// msi_query.cu -- exact k-NN query answering on the GPU (Section III-B, Algorithms 5-9).
//
// The paper's search workers, priority queues and BSF lock become one short chain
// of kernels per query, all on one stream:
//   q_prep          query iSAX summary (Algorithm 5, first step) and the per-segment
//                   squared-gap tables; the approximate-search leaf found by the
//                   query's key, as descending the tree would (Algorithm 5, approxSearch);
//   q_seed          real distances of that leaf's members: the initial BSF;
//   q_seed_select   (k > 1) the k-th smallest of them;
//   q_leaf_filter   lower bound of every leaf against the BSF; survivors become work
//                   items (TraverseRootSubtree, Algorithm 7, flattened over the leaves);
//   q_front         the lowest-bound surviving leaves refined first (the head of the
//                   priority order of ProcessQueue, Algorithm 8);
//   q_filter_blocks bounds of 32-position blocks of the surviving leaves;
//   q_filter_series per-series bounds from the SAX words (Algorithm 9's lower bound),
//                   then, for those that pass, from the fine PAA (64 fp16 segment means
//                   at most) before any row is read;
//   q_refine_rows   real distances of the survivors (CalculateRealDistance,
//                   Algorithm 9); the BSF is an atomicMin on the bits of a
//                   non-negative float, each item re-tested against it (Algorithm 8);
//   q_finalize      the k-th smallest candidate squared distance, FP64 distances of
//                   every candidate within the fp32 error margin of it, and the k
//                   smallest by (FP64 distance, id): the answer.
// Under DTW (Section IV) q_seed, q_front and q_refine_rows have DTW counterparts and
// the FP64 re-check runs in its own kernel. Pruning is conservative: a bound prunes
// only when it exceeds the BSF by more than the fp32 rounding of both sides can
// explain, so the answer is the exact one.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "msi_internal.cuh"

namespace msi {
namespace {

constexpr int kThreads = 256;
// Seed rows a warp takes at once when their fine PAA bounds order them (k = 1).
constexpr int kSeedGroup = 8;

// Programmatic dependent launch (sm_90 and later): the query kernels are launched so
// that one may start while the previous kernel of its stream is finishing (its launch
// latency and set-up overlap that kernel's tail). Each calls pdl_begin() first: the
// wait returns once the previous kernel has completed and its writes are visible (a
// no-op without the launch attribute); the trigger then lets the next kernel launch.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// A candidate: (fp32 squared distance bits << 32) | leaf-order position.
__device__ __forceinline__ unsigned long long pack(float d2, uint32_t pos) {
  return ((unsigned long long)__float_as_uint(d2) << 32) | pos;
}

// Squared Euclidean distance between the z-normalised series `id` and the
// z-normalised query in shared memory; one warp, result in every lane. fp32 with a
// fused multiply-add per point.
__device__ __forceinline__ float warp_sqdist(const IndexView& ix, uint32_t id, float2 ms, const float* qs) {
  const int lane = threadIdx.x & 31;
  const float* row = ix.data + (size_t)id * ix.len;
  float acc = 0.0f;
  if ((ix.len & 3) == 0) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    const float4* q4 = reinterpret_cast<const float4*>(qs);
    const int n4 = ix.len >> 2;
    if (n4 <= 8 * 32) {  // rows of up to 1024 points: every load issued first
      float4 x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = lane + 32 * j;
        x[j] = c < n4 ? __ldg(r4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = lane + 32 * j;
        if (c < n4) {
          float4 z = x[j];
          if (!ix.data_is_z) {
            z.x = znorm_value(z.x, ms.x, ms.y);
            z.y = znorm_value(z.y, ms.x, ms.y);
            z.z = znorm_value(z.z, ms.x, ms.y);
            z.w = znorm_value(z.w, ms.x, ms.y);
          }
          const float4 q = q4[c];
          float d = __fsub_rn(z.x, q.x); acc = __fmaf_rn(d, d, acc);
          d = __fsub_rn(z.y, q.y); acc = __fmaf_rn(d, d, acc);
          d = __fsub_rn(z.z, q.z); acc = __fmaf_rn(d, d, acc);
          d = __fsub_rn(z.w, q.w); acc = __fmaf_rn(d, d, acc);
        }
      }
    } else if (ix.data_is_z) {
      for (int c = lane; c < n4; c += 32) {
        const float4 x = __ldg(r4 + c), q = q4[c];
        float d = __fsub_rn(x.x, q.x); acc = __fmaf_rn(d, d, acc);
        d = __fsub_rn(x.y, q.y); acc = __fmaf_rn(d, d, acc);
        d = __fsub_rn(x.z, q.z); acc = __fmaf_rn(d, d, acc);
        d = __fsub_rn(x.w, q.w); acc = __fmaf_rn(d, d, acc);
      }
    } else {
      for (int c = lane; c < n4; c += 32) {
        const float4 x = __ldg(r4 + c), q = q4[c];
        float d = __fsub_rn(znorm_value(x.x, ms.x, ms.y), q.x); acc = __fmaf_rn(d, d, acc);
        d = __fsub_rn(znorm_value(x.y, ms.x, ms.y), q.y); acc = __fmaf_rn(d, d, acc);
        d = __fsub_rn(znorm_value(x.z, ms.x, ms.y), q.z); acc = __fmaf_rn(d, d, acc);
        d = __fsub_rn(znorm_value(x.w, ms.x, ms.y), q.w); acc = __fmaf_rn(d, d, acc);
      }
    }
  } else {
    for (int t = lane; t < ix.len; t += 32) {
      const float x = __ldg(row + t);
      const float z = ix.data_is_z ? x : znorm_value(x, ms.x, ms.y);
      const float d = __fsub_rn(z, qs[t]);
      acc = __fmaf_rn(d, d, acc);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
  return acc;
}

// Squared iSAX lower bound of one SAX word: s * sum_j T[j][sym_j]. Symbol byte b of
// a 32-bit part becomes its byte offset in the row with one shift and one mask.
template <bool kW16>
__device__ __forceinline__ float word_lb2_t(uint4 wd, const float* Ts, int w, int card, float s) {
  const uint32_t parts[4] = {wd.x, wd.y, wd.z, wd.w};
  const char* tb = reinterpret_cast<const char*>(Ts);
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (kW16 || j < w) {
      const uint32_t p = parts[j >> 2];
      const uint32_t off = (j & 3) == 0 ? (p << 2) & 0x3FCu : (p >> (8 * (j & 3) - 2)) & 0x3FCu;
      acc = __fadd_rn(acc, *reinterpret_cast<const float*>(tb + (size_t)j * card * 4 + off));
    }
  }
  return __fmul_rn(acc, s);
}
// (16 segments, the paper's configuration, takes a path without the per-segment
// test of a run-time segment count)
__device__ __forceinline__ float word_lb2(uint4 wd, const float* Ts, int w, int card, float s) {
  return w == 16 ? word_lb2_t<true>(wd, Ts, w, card, s) : word_lb2_t<false>(wd, Ts, w, card, s);
}

// Squared iSAX lower bound of a leaf from its per-segment symbol envelope: the gap
// between the query's interval [lo_j, up_j] (the PAA value itself for the Euclidean
// distance, the envelope's range for DTW) and the region from the lower edge of the
// smallest symbol to the upper edge of the largest (0 where they meet).
__device__ __forceinline__ float leaf_lb2(const IndexView& ix, int64_t l, const float* up_s, const float* lo_s,
                                          const float* thr_lo_s, const float* thr_up_s) {
  const uint4 lo = ix.env[2 * l], hi = ix.env[2 * l + 1];
  const uint32_t lop[4] = {lo.x, lo.y, lo.z, lo.w}, hip[4] = {hi.x, hi.y, hi.z, hi.w};
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j < ix.w) {
      const int sl = (lop[j >> 2] >> (8 * (j & 3))) & 255, sh = (hip[j >> 2] >> (8 * (j & 3))) & 255;
      const float u = up_s[j], lq = lo_s[j], lower = thr_lo_s[sl], upper = thr_up_s[sh + 1];
      float d = 0.0f;
      if (u < lower) d = __fsub_rn(lower, u);
      else if (lq > upper) d = __fsub_rn(lq, upper);
      acc = __fadd_rn(acc, __fmul_rn(d, d));
    }
  }
  return __fmul_rn(acc, (float)ix.seglen);
}

// k-th smallest (1-based) of `count` 32-bit keys read through get(i), by one block:
// four 8-bit radix passes with a shared histogram.
template <typename Get>
__device__ uint32_t block_select_u32(Get get, uint32_t count, uint32_t k, uint32_t* hist, uint32_t* sel) {
  uint32_t prefix = 0, mask = 0, kk = k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) {
      const uint32_t v = get(i);
      if ((v & mask) == prefix) atomicAdd(&hist[(v >> shift) & 255], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      uint32_t loc[8], tot = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) { loc[b] = hist[lane * 8 + b]; tot += loc[b]; }
      uint32_t incl = tot;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
      }
      const uint32_t excl = incl - tot;
      if (excl < kk && kk <= incl) {
        uint32_t cum = excl;
        for (int b = 0; b < 8; ++b) {
          if (cum + loc[b] >= kk) { sel[0] = (uint32_t)(lane * 8 + b); sel[1] = kk - cum; break; }
          cum += loc[b];
        }
      }
    }
    __syncthreads();
    prefix |= sel[0] << shift;
    mask |= 255u << shift;
    kk = sel[1];
    __syncthreads();
  }
  return prefix;
}

// Block-wide copy of `count` floats from global to shared memory with every load
// issued before the first store (up to 4 float4 per thread in flight), so the copy
// costs one memory round trip instead of one per element.
__device__ __forceinline__ void smem_fill(float* dst, const float* __restrict__ src, int count) {
  const bool vec = ((((uintptr_t)dst) | ((uintptr_t)src)) & 15) == 0;
  const int n4 = vec ? count >> 2 : 0;
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int base = 0; base < n4; base += 4 * blockDim.x) {
    float4 r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = base + j * blockDim.x + threadIdx.x;
      r[j] = i < n4 ? __ldg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = base + j * blockDim.x + threadIdx.x;
      if (i < n4) d4[i] = r[j];
    }
  }
  for (int i = 4 * n4 + threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
}

// Lower bound^2 of series `id` from the fine PAA: sf times the sum over the fine
// segments of the squared gap between the series' mean and the query's interval
// [lo_j, up_j]. The stored mean h is fp16, within e = |h| 2^-11 + 2^-25 of the fp32
// mean (half an fp16 ulp), so each gap is taken e short; every step rounds down.
__device__ __forceinline__ float fine_lb2(const IndexView& ix, const float* fup, const float* flo, uint32_t id) {
  const int chunks = ix.wf >> 3;
  const uint4* src = ix.fine + (size_t)id * chunks;
  float acc = 0.0f;
  for (int c = 0; c < chunks; ++c) {
    const uint4 v = __ldg(src + c);
    const uint32_t parts[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int h2 = 0; h2 < 4; ++h2) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&parts[h2]));
      const float hv[2] = {f.x, f.y};
#pragma unroll
      for (int e2 = 0; e2 < 2; ++e2) {
        const int j = 8 * c + 2 * h2 + e2;
        const float h = hv[e2];
        const float e = __fmaf_ru(fabsf(h), 4.8828125e-4f, 2.98023223876953125e-8f);
        const float g = fmaxf(0.0f, fmaxf(__fsub_rd(__fsub_rd(h, fup[j]), e), __fsub_rd(__fsub_rd(flo[j], h), e)));
        acc = __fmaf_rd(g, g, acc);
      }
    }
  }
  return __fmul_rd(acc, (float)ix.sf);
}

// The same bound for up to 32 series at once (lane i: series id, for the lanes in
// `valid`; the others return 0) by all 32 lanes of the warp together, eight lanes per
// series: in round r of a half, lane 8 g + c reads 16-byte chunk c (segments 8 c ..
// 8 c + 7) of series 16 half + 4 r + g, the half's four loads issued before any
// arithmetic, and the eight partial sums are combined by shuffles. Every step rounds
// down, so the sum stays at or below the exact one in this order too.
__device__ __forceinline__ float warp_fine_lb2_32(const IndexView& ix, const float* fup, const float* flo,
                                                  uint32_t id, unsigned valid) {
  const int lane = threadIdx.x & 31, c = lane & 7, g = lane >> 3;
  const int chunks = ix.wf >> 3;
  float mine = 0.0f;
  if (!valid) return mine;  // the same in every lane
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    if (!((valid >> (16 * half)) & 0xffffu)) continue;  // warp-uniform: no series in this half
    uint4 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int s = 16 * half + 4 * r + g;
      const uint32_t sid = __shfl_sync(kFull, id, s);
      v[r] = ((valid >> s) & 1u) && c < chunks ? __ldg(ix.fine + (size_t)sid * chunks + c) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int base = 16 * half + 4 * r;
      if (!((valid >> base) & 0xfu)) continue;  // warp-uniform: no series in this round
      float acc = 0.0f;
      if (c < chunks) {
        const uint32_t parts[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
        for (int h2 = 0; h2 < 4; ++h2) {
          const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&parts[h2]));
          const float hv[2] = {f.x, f.y};
#pragma unroll
          for (int e2 = 0; e2 < 2; ++e2) {
            const int j = 8 * c + 2 * h2 + e2;
            const float h = hv[e2];
            const float e = __fmaf_ru(fabsf(h), 4.8828125e-4f, 2.98023223876953125e-8f);
            const float gap =
                fmaxf(0.0f, fmaxf(__fsub_rd(__fsub_rd(h, fup[j]), e), __fsub_rd(__fsub_rd(flo[j], h), e)));
            acc = __fmaf_rd(gap, gap, acc);
          }
        }
      }
      acc = __fadd_rd(acc, __shfl_xor_sync(kFull, acc, 1));  // the same sum in all 8 lanes
      acc = __fadd_rd(acc, __shfl_xor_sync(kFull, acc, 2));
      acc = __fadd_rd(acc, __shfl_xor_sync(kFull, acc, 4));
      const float t = __shfl_sync(kFull, acc, 8 * ((lane - base) & 3));
      if (lane >= base && lane < base + 4) mine = t;
    }
  }
  return __fmul_rd(mine, (float)ix.sf);
}

// The same bound computed by a whole warp for one series (lane l takes segments l,
// l + 32, ...); every lane returns lane 0's sum.
__device__ __forceinline__ float warp_fine_lb2(const IndexView& ix, const float* fup, const float* flo, uint32_t id) {
  const int lane = threadIdx.x & 31;
  const __half* src = reinterpret_cast<const __half*>(ix.fine) + (size_t)id * ix.wf;
  float acc = 0.0f;
  for (int j = lane; j < ix.wf; j += 32) {
    const float h = __half2float(src[j]);
    const float e = __fmaf_ru(fabsf(h), 4.8828125e-4f, 2.98023223876953125e-8f);
    const float g = fmaxf(0.0f, fmaxf(__fsub_rd(__fsub_rd(h, fup[j]), e), __fsub_rd(__fsub_rd(flo[j], h), e)));
    acc = __fmaf_rd(g, g, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = __fadd_rd(acc, __shfl_xor_sync(kFull, acc, o));
  return __shfl_sync(kFull, __fmul_rd(acc, (float)ix.sf), 0);
}

// ------------------------------------------------------------------ q_prep
__device__ __forceinline__ void q_prep_body(const IndexView& ix, const float* __restrict__ q, const QueryView& qv, int k) {
  
  if (qv.call) q = qv.call->queries + (size_t)qv.qi * ix.len;
  extern __shared__ float zs[];  // [len]
  __shared__ float thr_up_s[257], thr_lo_s[257];
  __shared__ float paa_s[16];
  __shared__ int sym_s[16];
  __shared__ unsigned long long key_s;
  __shared__ int lo_s, hi_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int v = tid; v <= ix.card; v += blockDim.x) {
    thr_up_s[v] = ix.thr_up[v];
    thr_lo_s[v] = ix.thr_lo[v];
  }
  smem_fill(zs, q, ix.len);  // the raw query, staged with all loads in flight
  __syncthreads();
  if (warp == 0) {
    const Moments m = warp_moments_generic(zs, ix.len);
    __syncwarp();
    for (int t = lane; t < ix.len; t += 32) zs[t] = m.flag != 0 ? 0.0f : znorm_value(zs[t], m.mu, m.rsig);
    __syncwarp();
    int sym = 0;
    if (lane < ix.w) {
      const float p = paa_segment_generic(zs, lane, ix.seglen);
      paa_s[lane] = p;
      sym = sax_symbol(thr_up_s, ix.card, p);
      sym_s[lane] = sym;
    }
    const unsigned long long key = interleave_key(sym, ix.w, ix.bits);
    if (lane == 0) {
      key_s = key;
      qv.st->flag = m.flag;
      if (m.flag < 0) atomicAdd(&qv.counters[ST_BAD_QUERY], 1ull);
    }
  }
  __syncthreads();
  for (int t = tid; t < ix.len; t += blockDim.x) qv.qz[t] = zs[t];
  if (k > 1)
    for (int b = tid; b < 256; b += blockDim.x) qv.khist[b] = 0u;
  // the interval each bound measures gaps to: the PAA value (Euclidean), or for DTW
  // the LB_Keogh envelope reduced per segment (Keogh's PAA envelope: the max of the
  // upper envelope and the min of the lower one over the segment, i.e. the max / min
  // of the query over the segment widened by the warping window)
  __shared__ float iv_up_s[16], iv_lo_s[16];
  if (qv.window >= 0) {
    const int r = qv.window;
    for (int t = tid; t < ix.len; t += blockDim.x) {
      float u = zs[t], l = zs[t];
      const int a = max(0, t - r), b = min(ix.len - 1, t + r);
      for (int x = a; x <= b; ++x) {
        u = fmaxf(u, zs[x]);
        l = fminf(l, zs[x]);
      }
      qv.qenv[t] = u;
      qv.qenv[ix.len + t] = l;
    }
    for (int j = warp; j < ix.w; j += kThreads / 32) {
      const int a = max(0, j * ix.seglen - r), b = min(ix.len - 1, (j + 1) * ix.seglen - 1 + r);
      float u = -INFINITY, l = INFINITY;
      for (int x = a + lane; x <= b; x += 32) {
        u = fmaxf(u, zs[x]);
        l = fminf(l, zs[x]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        u = fmaxf(u, __shfl_xor_sync(kFull, u, o));
        l = fminf(l, __shfl_xor_sync(kFull, l, o));
      }
      if (lane == 0) {
        iv_up_s[j] = u;
        iv_lo_s[j] = l;
      }
    }
  } else if (tid < ix.w) {
    iv_up_s[tid] = paa_s[tid];
    iv_lo_s[tid] = paa_s[tid];
  }
  __syncthreads();
  const int wc = ix.w * ix.card;
  for (int e = tid; e < wc; e += blockDim.x) {
    const int j = e / ix.card, v = e - j * ix.card;
    const float u = iv_up_s[j], l = iv_lo_s[j];
    const float lower = thr_lo_s[v], upper = thr_up_s[v + 1];
    float d = 0.0f;
    if (u < lower) d = __fsub_rn(lower, u);
    else if (l > upper) d = __fsub_rn(l, upper);
    qv.T[e] = __fmul_rn(d, d);
  }
  // coarse table: gap to the union of the regions sharing a kCoarseBits-bit symbol prefix
  {
    const int cb = ix.bits < kCoarseBits ? ix.bits : kCoarseBits, cs = ix.bits - cb;
    for (int e = tid; e < ix.w * kCoarse; e += blockDim.x) {
      const int j = e >> kCoarseBits, c = e & (kCoarse - 1);
      float d = 0.0f;
      if (c < (1 << cb)) {
        const float u = iv_up_s[j], l = iv_lo_s[j];
        const float lower = thr_lo_s[c << cs], upper = thr_up_s[(c + 1) << cs];
        if (u < lower) d = __fsub_rn(lower, u);
        else if (l > upper) d = __fsub_rn(l, upper);
      }
      qv.T5[e] = __fmul_rn(d, d);
    }
  }
  // the same intervals over the fine PAA's segments
  for (int j = tid; j < ix.wf; j += blockDim.x) {
    float u, l;
    if (qv.window >= 0) {
      const int a = max(0, j * ix.sf - qv.window), b = min(ix.len - 1, (j + 1) * ix.sf - 1 + qv.window);
      u = -INFINITY;
      l = INFINITY;
      for (int x = a; x <= b; ++x) {
        u = fmaxf(u, zs[x]);
        l = fminf(l, zs[x]);
      }
    } else {
      float g = 0.0f;
      for (int t = j * ix.sf; t < (j + 1) * ix.sf; ++t) g = __fadd_rn(g, zs[t]);
      u = l = __fdiv_rn(g, (float)ix.sf);
    }
    qv.st->fup[j] = u;
    qv.st->flo[j] = l;
  }
  if (tid < ix.w) {
    qv.st->qpaa[tid] = paa_s[tid];
    qv.st->qup[tid] = iv_up_s[tid];
    qv.st->qlo[tid] = iv_lo_s[tid];
    // a symbol whose region meets the interval (the block filter's clamp needs one):
    // the PAA's own symbol, moved into [symbol of lo, symbol of up] for DTW
    int sym = sym_s[tid];
    if (qv.window >= 0)
      sym = min(max(sym, sax_symbol(thr_up_s, ix.card, iv_lo_s[tid])), sax_symbol(thr_up_s, ix.card, iv_up_s[tid]));
    qv.st->qsym[tid] = sym;
  }
  // approximate search: the last leaf whose first key is <= the query key
  const unsigned long long qkey = key_s;
  if (tid == 0) { lo_s = 0; hi_s = (int)ix.L; }
  __syncthreads();
  while (true) {
    const int lo = lo_s, hi = hi_s;
    if (hi - lo <= 1) break;
    const int step = (hi - lo + blockDim.x - 1) / blockDim.x;
    const int idx = lo + tid * step;
    const bool pred = idx < hi && ix.leaf_key[idx] <= qkey;
    const int cnt = __syncthreads_count(pred);
    if (tid == 0) {
      if (cnt == 0) { hi_s = lo + 1; }  // query key below every probe: keep lo
      else {
        const int nlo = lo + (cnt - 1) * step;
        lo_s = nlo;
        hi_s = min(hi, nlo + step);
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    int64_t l = lo_s;
    if (ix.tree_child) {
      // balanced-split tree: descend from the query's root child by the next bit of
      // each node's split segment (the search above is the fallback when the query's
      // root prefix has no child)
      int32_t node = ix.root_child[qkey >> (64 - ix.root_bits)];
      if (node >= 0) {
        int depth[16];
        for (int j = 0; j < 16; ++j) depth[j] = 1;
        for (int step = 0; step < 16 * 8 + 2 && ix.tree_seg[node] >= 0; ++step) {
          const int j = ix.tree_seg[node];
          const int bit = (sym_s[j] >> (ix.bits - 1 - depth[j])) & 1;
          ++depth[j];
          node = ix.tree_child[2 * node + bit];
        }
        if (ix.tree_seg[node] < 0) l = -1 - ix.tree_child[2 * node];
      }
    }
    int64_t a = ix.leaf_begin[l], b = ix.leaf_begin[l + 1];
    if (b - a < k) {
      b = min(ix.n, max(b, a + (int64_t)k));
      a = min(a, b - (int64_t)k);
    }
    QState* st = qv.st;
    st->qkey = qkey;
    st->seed_a = (uint32_t)a;
    st->seed_b = (uint32_t)b;
    st->thr_bits = 0x7f800000u;
    st->leaf_count = 0;
    st->item_count = 0;
    st->surv_count = 0;
    st->blk_count = 0;
    st->overflow = 0;
    st->nfront = 0;
    st->kbase = 0.0f;
    st->cand_count = (uint32_t)(b - a);
    st->rc_count = 0;
    st->final_bits = 0;
    st->series_refined = 0;
    st->fine_front = 0;
    st->seed_done = (uint32_t)(b - a);
  }
}

__global__ void __launch_bounds__(kThreads)
q_prep(IndexView ix, const float* __restrict__ q, QueryView qv, int k) {
  pdl_begin();
  q_prep_body(ix, q, qv, k);
}

// ------------------------------------------------------------ k-th histogram
// For k > 1 the candidates kept below kbase (the k-th best of the seed and front
// leaves) are counted in 256 equal buckets of [0, kbase). If the buckets up to b hold
// k candidates, at least k computed distances lie below the upper edge of bucket b;
// the bound read off the counts is the upper edge of bucket b + 1, one bucket of room
// for the rounding of the bucket index, so it bounds the k-th computed distance from
// above like any k-th best seen so far.
__device__ __forceinline__ int khist_bucket(float d2, float kbase) {
  return min(255, (int)__fmul_rz(d2, __fdiv_rn(256.0f, kbase)));
}
// One warp: the bound (fp32 bits) from the counts, or 0x7f800000 while fewer than k.
__device__ __forceinline__ unsigned khist_bound(const uint32_t* khist, float kbase, int k) {
  const int lane = threadIdx.x & 31;
  uint32_t v[8], sum = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v[j] = *(volatile const uint32_t*)(khist + 8 * lane + j);
    sum += v[j];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t before = incl - sum;
  int b = 256;
  if (before < (uint32_t)k && incl >= (uint32_t)k) {
    uint32_t run = before;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      run += v[j];
      if (run >= (uint32_t)k) {
        b = 8 * lane + j;
        break;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(kFull, b, o));
  if (b >= 254) return 0x7f800000u;
  return __float_as_uint(__fmul_ru(kbase, (float)(b + 2) * 0.00390625f));
}

// ------------------------------------------------------------------ q_seed
__device__ __forceinline__ void q_seed_body(const IndexView& ix, const QueryView& qv) {
  extern __shared__ __align__(16) float qs[];
  __shared__ float fup_s[kMaxFine], flo_s[kMaxFine];
  const uint32_t a = qv.st->seed_a, b = qv.st->seed_b;
  // the grid covers the largest leaf: a block whose warps start past the seed leaf's
  // rows returns before it loads the query (the same decision in every thread)
  const uint32_t rows_per_block = (kThreads / 32) * ((qv.k == 1 && ix.wf) ? kSeedGroup : 1);
  if ((uint64_t)blockIdx.x * rows_per_block >= b - a) return;
  smem_fill(qs, qv.qz, ix.len);
  for (int j = threadIdx.x; j < ix.wf; j += blockDim.x) {
    fup_s[j] = qv.st->fup[j];
    flo_s[j] = qv.st->flo[j];
  }
  __syncthreads();
  __shared__ unsigned s_min;
  if (threadIdx.x == 0) s_min = 0x7f800000u;
  const uint32_t warps = gridDim.x * (kThreads / 32);
  const int lane = threadIdx.x & 31;
  unsigned best = 0x7f800000u;
  uint32_t n_skip = 0;  // seed rows the fine bound ruled out (counted by every lane)
  auto refine = [&](uint32_t g) {  // row g of the seed: a candidate, and the BSF for k = 1
    const uint32_t pos = a + g;
    const float d2 = warp_sqdist(ix, ix.perm[pos], ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos], qs);
    if (lane == 0) {
      if (g < qv.cand_cap) qv.cand[g] = pack(d2, pos);
      else qv.st->overflow = 1u;
      if (qv.k == 1 && ix.wf) atomicMin(&qv.st->thr_bits, __float_as_uint(d2));  // the screens read it
    }
    best = min(best, __float_as_uint(d2));
  };
  if (qv.k == 1 && ix.wf) {
    // k = 1 with the fine PAA: a warp takes kSeedGroup rows, refines the one with the
    // smallest fine bound (its distance joins the BSF at once), then only the others
    // whose fine bound still passes the BSF; the rest become +inf candidates
    const uint32_t nrow = b - a;
    for (uint32_t g0 = (blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5)) * kSeedGroup; g0 < nrow;
         g0 += warps * kSeedGroup) {
      const uint32_t g = g0 + lane;
      const bool have = lane < kSeedGroup && g < nrow;
      const float flb = warp_fine_lb2_32(ix, fup_s, flo_s, have ? ix.perm[a + g] : 0u, __ballot_sync(kFull, have));
      const float lb = have ? flb : INFINITY;
      float m = lb;
      int mi = lane;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float om = __shfl_xor_sync(kFull, m, o);
        const int oi = __shfl_xor_sync(kFull, mi, o);
        if (om < m || (om == m && oi < mi)) {
          m = om;
          mi = oi;
        }
      }
      if (!(m < INFINITY)) mi = 0;
      refine(g0 + mi);
      const unsigned thr = __shfl_sync(kFull, lane == 0 ? *(volatile unsigned*)&qv.st->thr_bits : 0u, 0);
      const bool rest = have && lane != mi;
      const bool pass = rest && lb <= lb_bound2(thr, qv.eps, qv.tau);
      if (rest && !pass) {
        if (g < qv.cand_cap) qv.cand[g] = pack(INFINITY, a + g);
        else qv.st->overflow = 1u;
      }
      n_skip += __popc(__ballot_sync(kFull, rest && !pass));
      for (unsigned mk = __ballot_sync(kFull, pass); mk; mk &= mk - 1) refine(g0 + __ffs(mk) - 1);
    }
  } else {
    for (uint32_t gw = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); gw < b - a; gw += warps) refine(gw);
  }
  // k = 1: one atomicMin per block, on the block's smallest distance
  __shared__ unsigned s_skip;
  if (threadIdx.x == 0) s_skip = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && best < 0x7f800000u) atomicMin(&s_min, best);
  if ((threadIdx.x & 31) == 0 && n_skip) atomicAdd(&s_skip, n_skip);
  __syncthreads();
  if (threadIdx.x == 0 && qv.k == 1 && s_min < 0x7f800000u) atomicMin(&qv.st->thr_bits, s_min);
  if (threadIdx.x == 0 && s_skip) atomicSub(&qv.st->seed_done, s_skip);
}

__global__ void __launch_bounds__(kThreads)
q_seed(IndexView ix, QueryView qv) {
  pdl_begin();
  q_seed_body(ix, qv);
}

__device__ __forceinline__ void q_seed_select_body(const QueryView& qv, int base) {
  
  __shared__ uint32_t hist[256], sel[2];
  const uint32_t count = min(qv.st->cand_count, qv.cand_cap);
  const unsigned long long* c = qv.cand;
  const uint32_t kth = block_select_u32([&](uint32_t i) { return (uint32_t)(c[i] >> 32); }, count,
                                        (uint32_t)qv.k, hist, sel);
  if (threadIdx.x == 0) qv.st->thr_bits = kth;
  if (!base) return;
  // the candidates so far, counted in 256 buckets of [0, kth): the row refinement adds
  // its own and reads a tighter k-th bound off the counts (see khist_bound)
  const float kb = __uint_as_float(kth);
  if (!(kb > 0.0f && kb < INFINITY)) return;
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) {
    const float d2 = __uint_as_float((uint32_t)(c[i] >> 32));
    if (d2 < kb) atomicAdd(&hist[khist_bucket(d2, kb)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x) qv.khist[b] = hist[b];
  if (threadIdx.x == 0) qv.st->kbase = kb;
}

__global__ void __launch_bounds__(1024)
q_seed_select(QueryView qv, int base) {
  pdl_begin();
  q_seed_select_body(qv, base);
}

// ------------------------------------------------------------------ q_leaf_filter
__device__ __forceinline__ void q_leaf_filter_body(const IndexView& ix, const QueryView& qv) {
  
  __shared__ float thr_up_s[257], thr_lo_s[257], up_s[16], lo_s[16];
  for (int v = threadIdx.x; v <= ix.card; v += blockDim.x) {
    thr_up_s[v] = ix.thr_up[v];
    thr_lo_s[v] = ix.thr_lo[v];
  }
  if (threadIdx.x < ix.w) {
    up_s[threadIdx.x] = qv.st->qup[threadIdx.x];
    lo_s[threadIdx.x] = qv.st->qlo[threadIdx.x];
  }
  __syncthreads();
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  float lb2 = 0.0f;
  if (l < ix.L) {
    const uint32_t b = ix.leaf_begin[l], e = ix.leaf_begin[l + 1];
    const uint32_t sa = qv.st->seed_a, sb = qv.st->seed_b;
    if (!(b >= sa && e <= sb)) {
      lb2 = leaf_lb2(ix, l, up_s, lo_s, thr_lo_s, thr_up_s);
      keep = lb2 <= lb_bound2(qv.st->thr_bits, qv.eps, qv.tau);
    }
  }
  const unsigned m = __ballot_sync(kFull, keep);
  if (m) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&qv.st->leaf_count, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    // work items of at most kItem positions, numbered by a warp prefix sum
    uint32_t b = 0, e = 0, nit = 0;
    if (keep) {
      b = ix.leaf_begin[l];
      e = ix.leaf_begin[l + 1];
      nit = (e - 1) / kItem - b / kItem + 1;  // aligned tiles of kItem positions touched
    }
    uint32_t incl = nit;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t ibase = 0;
    if (lane == 31) ibase = atomicAdd(&qv.st->item_count, incl);
    ibase = __shfl_sync(kFull, ibase, 31) + incl - nit;
    if (keep) {
      const uint32_t slot = base + __popc(m & ((1u << lane) - 1u));
      qv.leaf_list[slot] = (uint32_t)l;
      qv.leaf_lb2[slot] = lb2;
      const uint32_t t0 = b / kItem;
      for (uint32_t j = 0; j < nit; ++j) {
        if (ibase + j < qv.items_cap)
          qv.items[ibase + j] = make_uint4(max(b, (t0 + j) * kItem), min(e, (t0 + j + 1) * kItem), __float_as_uint(lb2),
                                           (uint32_t)l);
        else
          qv.st->overflow = 1u;
      }
    }
  }
  // the block's lowest-bound surviving leaf (ties: lowest leaf), for the early
  // refinement of the most promising leaf
  __shared__ unsigned long long s_min[kThreads / 32];
  unsigned long long mine = keep ? (((unsigned long long)__float_as_uint(lb2) << 32) | (uint32_t)l) : ~0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(kFull, mine, o);
    mine = other < mine ? other : mine;
  }
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = ~0ull;
    for (int w = 0; w < kThreads / 32; ++w) b = s_min[w] < b ? s_min[w] : b;
    qv.blockmin[blockIdx.x] = b;
  }
}

__global__ void __launch_bounds__(kThreads)
q_leaf_filter(IndexView ix, QueryView qv) {
  pdl_begin();
  q_leaf_filter_body(ix, qv);
}

// The m lowest (bound bits << 32 | leaf) keys among the leaf filter's per-block minima
// whose bound passes the BSF as thread 0 reads it (one reading for the whole block,
// so that the block takes one decision): their leaves in s_leaf, their first
// positions in s_beg, the running total of their sizes in s_pre[0..count]. Returns the
// count, the same in every thread.
__device__ int front_leaves(const IndexView& ix, const QueryView& qv, uint32_t nblockmin, int m, uint32_t* s_leaf,
                            uint32_t* s_beg, uint32_t* s_pre) {
  __shared__ int s_count;
  if (threadIdx.x < 32) {  // warp 0 selects (shuffles only); the block waits once
    const int lane = threadIdx.x;
    const unsigned thr = __shfl_sync(kFull, lane == 0 ? *(volatile unsigned*)&qv.st->thr_bits : 0u, 0);
    const float bound2 = lb_bound2(thr, qv.eps, qv.tau);
    if (lane == 0) s_pre[0] = 0;
    unsigned long long last = 0;
    int count = 0;
    for (int round = 0; round < m; ++round) {
      unsigned long long best = ~0ull;
      for (uint32_t i = lane; i < nblockmin; i += 32) {
        const unsigned long long v = qv.blockmin[i];
        if ((round == 0 || v > last) && v < best) best = v;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(kFull, best, o);
        best = other < best ? other : best;
      }
      if (best == ~0ull || __uint_as_float((uint32_t)(best >> 32)) > bound2) break;
      if (lane == 0) {
        const uint32_t l = (uint32_t)best;
        s_leaf[count] = l;
        s_beg[count] = ix.leaf_begin[l];
        s_pre[count + 1] = s_pre[count] + (ix.leaf_begin[l + 1] - ix.leaf_begin[l]);
      }
      last = best;
      ++count;
    }
    if (lane == 0) s_count = count;
  }
  __syncthreads();
  return s_count;
}

// Leaves refined early, by how many neighbours are wanted: k = 1 tightens its BSF
// with every distance, a k-th best needs a wider sample of close series. (For k = 1 a
// block that reads a BSF already tightened by other blocks takes a prefix of the same
// list: the leaves it leaves out are pruned by that BSF.)
__host__ __device__ inline int front_count(int k) { return k == 1 ? 4 : kMaxFront; }

// The lowest-bound surviving leaves (front_count(k) of them), refined before the
// block and series filters so that those run against a tighter BSF (the priority
// order of ProcessQueue, Algorithm 8: the most promising leaves first). Every block
// picks them from the leaf filter's per-block minima (front_leaves); warps take their
// positions in a stride, skipping the seed range. Block 0 records the leaves, which
// the block filter then skips.
__device__ __forceinline__ void q_front_body(const IndexView& ix, const QueryView& qv, uint32_t nblockmin) {
  
  extern __shared__ __align__(16) float qs[];
  __shared__ unsigned s_min;
  __shared__ uint32_t s_leaf[kMaxFront], s_beg[kMaxFront], s_pre[kMaxFront + 1];
  __shared__ float fup_s[kMaxFine], flo_s[kMaxFine];
  smem_fill(qs, qv.qz, ix.len);
  for (int j = threadIdx.x; j < ix.wf; j += blockDim.x) {
    fup_s[j] = qv.st->fup[j];
    flo_s[j] = qv.st->flo[j];
  }
  if (threadIdx.x == 0) s_min = 0x7f800000u;
  const int nf = front_leaves(ix, qv, nblockmin, front_count(qv.k), s_leaf, s_beg, s_pre);
  QState* st = qv.st;
  if (nf == 0) return;  // the same in every thread of the block
  if (blockIdx.x == 0) {
    if (threadIdx.x < nf) st->front_leaf[threadIdx.x] = s_leaf[threadIdx.x];
    if (threadIdx.x == 0) st->nfront = (uint32_t)nf;
  }
  const uint32_t total = s_pre[nf];
  const uint32_t sa = st->seed_a, sb = st->seed_b;
  const unsigned thr = *(volatile unsigned*)&st->thr_bits;
  const float keep2 = keep_bound2(thr, qv.eps);
  const uint32_t warps = gridDim.x * (kThreads / 32);
  const uint32_t gw = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  unsigned bestd = 0x7f800000u;
  uint32_t n_front = 0, n_fine = 0;
  auto position = [&](uint32_t g) {
    int f = 0;
    while (g >= s_pre[f + 1]) ++f;
    return s_beg[f] + (g - s_pre[f]);
  };
  auto refine = [&](uint32_t pos) {
    const uint32_t id = ix.perm[pos];
    const float2 ms = ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos];
    const float d2 = warp_sqdist(ix, id, ms, qs);
    if (lane == 0) {
      ++n_front;
      if (d2 <= keep2) {
        const uint32_t slot = atomicAdd(&st->cand_count, 1u);
        if (slot < qv.cand_cap) qv.cand[slot] = pack(d2, pos);
        else st->overflow = 1u;
      }
    }
    bestd = min(bestd, __float_as_uint(d2));
  };
  const float lbb = lb_bound2(thr, qv.eps, qv.tau);
  if (ix.wf && lbb < INFINITY) {
    // a warp takes 32 rows: each lane bounds one by the fine PAA (against the seed's
    // BSF), and only the rows that pass are read
    for (uint32_t g0 = gw * 32; g0 < total; g0 += warps * 32) {
      const uint32_t g = g0 + lane;
      const uint32_t pos = g < total ? position(g) : 0u;
      const bool screen = g < total && !(pos >= sa && pos < sb);
      const unsigned sm = __ballot_sync(kFull, screen);
      n_fine += __popc(sm);
      // every lane takes part in the warp's bound (it shuffles across all 32 lanes)
      const float flb = warp_fine_lb2_32(ix, fup_s, flo_s, screen ? ix.perm[pos] : 0u, sm);
      const bool want = screen && flb <= lbb;
      for (unsigned m = __ballot_sync(kFull, want); m; m &= m - 1) refine(__shfl_sync(kFull, pos, __ffs(m) - 1));
    }
  } else {
    for (uint32_t g = gw; g < total; g += warps) {
      const uint32_t pos = position(g);
      if (pos >= sa && pos < sb) continue;  // already refined by the seed
      refine(pos);
    }
  }
  __shared__ unsigned s_n, s_nf;
  if (threadIdx.x == 0) s_n = s_nf = 0;
  __syncthreads();
  if (lane == 0) {
    if (bestd < 0x7f800000u) atomicMin(&s_min, bestd);
    if (n_front) atomicAdd(&s_n, n_front);
    if (n_fine) atomicAdd(&s_nf, n_fine);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_n) atomicAdd(&st->series_refined, s_n);  // one global atomic per block
    if (s_nf) atomicAdd(&st->fine_front, s_nf);
    if (qv.k == 1 && s_min < thr) atomicMin(&st->thr_bits, s_min);
  }
}

__global__ void __launch_bounds__(kThreads)
q_front(IndexView ix, QueryView qv, uint32_t nblockmin) {
  pdl_begin();
  q_front_body(ix, qv, nblockmin);
}

// The batched chain's front leaves, picked once per query by one block: the m lowest
// (bound bits << 32 | leaf) keys among the leaf filter's per-block minima whose bound
// passes the BSF as thread 0 reads it (front_leaves' choice, with the whole block
// scanning the minima in each round). Their ids, position ranges and bounds go to the
// query's state, where the front blocks and the block filter read them.
__device__ __forceinline__ void q_front_pick_body(const IndexView& ix, const QueryView& qv, uint32_t nblockmin) {
  __shared__ unsigned long long s_w[kThreads / 32];
  __shared__ unsigned long long s_best;
  __shared__ float s_bound2;
  QState* st = qv.st;
  if (threadIdx.x == 0) s_bound2 = lb_bound2(*(volatile unsigned*)&st->thr_bits, qv.eps, qv.tau);
  const int m = front_count(qv.k);
  const int lane = threadIdx.x & 31;
  unsigned long long last = 0;
  int count = 0;
  for (int round = 0; round < m; ++round) {
    unsigned long long best = ~0ull;
    for (uint32_t i = threadIdx.x; i < nblockmin; i += blockDim.x) {
      const unsigned long long v = qv.blockmin[i];
      if ((round == 0 || v > last) && v < best) best = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(kFull, best, o);
      best = other < best ? other : best;
    }
    if (lane == 0) s_w[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long b = ~0ull;
      for (int w = 0; w < kThreads / 32; ++w) b = s_w[w] < b ? s_w[w] : b;
      s_best = b;
    }
    __syncthreads();
    best = s_best;  // the same in every thread: one decision for the block
    if (best == ~0ull || __uint_as_float((uint32_t)(best >> 32)) > s_bound2) break;
    if (threadIdx.x == 0) {
      const uint32_t l = (uint32_t)best;
      st->front_leaf[count] = l;
      st->front_beg[count] = ix.leaf_begin[l];
      st->front_end[count] = ix.leaf_begin[l + 1];
      st->front_lb[count] = (uint32_t)(best >> 32);
    }
    last = best;
    ++count;
  }
  if (threadIdx.x == 0) st->nfront = (uint32_t)count;
}

// The batched chain's front refinement over the picked leaves (q_front_body's work
// with the pick read from the query's state). A block first drops the leaves whose
// bound the current BSF already prunes (a prefix stays: the bounds ascend), and a
// block whose warps start past the remaining rows returns before loading the query.
__device__ __forceinline__ void q_front_picked_body(const IndexView& ix, const QueryView& qv) {
  extern __shared__ __align__(16) float qs[];
  __shared__ unsigned s_min;
  __shared__ uint32_t s_beg[kMaxFront], s_pre[kMaxFront + 1];
  __shared__ int s_nf;
  __shared__ float fup_s[kMaxFine], flo_s[kMaxFine];
  QState* st = qv.st;
  if (threadIdx.x == 0) {
    const float bound2 = lb_bound2(*(volatile unsigned*)&st->thr_bits, qv.eps, qv.tau);
    const int n = (int)st->nfront;
    int nf = 0;
    s_pre[0] = 0;
    while (nf < n && __uint_as_float(st->front_lb[nf]) <= bound2) {
      s_beg[nf] = st->front_beg[nf];
      s_pre[nf + 1] = s_pre[nf] + (st->front_end[nf] - s_beg[nf]);
      ++nf;
    }
    s_nf = nf;
    s_min = 0x7f800000u;
  }
  __syncthreads();
  const int nf = s_nf;
  const uint32_t total = s_pre[nf];
  const uint32_t warps = gridDim.x * (kThreads / 32);
  const uint32_t w0 = blockIdx.x * (kThreads / 32);
  const bool fine = ix.wf != 0;
  if (nf == 0 || (uint64_t)w0 * (fine ? 32u : 1u) >= total) return;  // the same in every thread
  smem_fill(qs, qv.qz, ix.len);
  for (int j = threadIdx.x; j < ix.wf; j += blockDim.x) {
    fup_s[j] = st->fup[j];
    flo_s[j] = st->flo[j];
  }
  __syncthreads();
  const uint32_t sa = st->seed_a, sb = st->seed_b;
  const unsigned thr = *(volatile unsigned*)&st->thr_bits;
  const float keep2 = keep_bound2(thr, qv.eps);
  const uint32_t gw = w0 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  unsigned bestd = 0x7f800000u;
  uint32_t n_front = 0, n_fine = 0;
  auto position = [&](uint32_t g) {
    int f = 0;
    while (g >= s_pre[f + 1]) ++f;
    return s_beg[f] + (g - s_pre[f]);
  };
  auto refine = [&](uint32_t pos) {
    const uint32_t id = ix.perm[pos];
    const float2 ms = ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos];
    const float d2 = warp_sqdist(ix, id, ms, qs);
    if (lane == 0) {
      ++n_front;
      if (d2 <= keep2) {
        const uint32_t slot = atomicAdd(&st->cand_count, 1u);
        if (slot < qv.cand_cap) qv.cand[slot] = pack(d2, pos);
        else st->overflow = 1u;
      }
    }
    bestd = min(bestd, __float_as_uint(d2));
  };
  const float lbb = lb_bound2(thr, qv.eps, qv.tau);
  if (fine && lbb < INFINITY) {
    for (uint32_t g0 = gw * 32; g0 < total; g0 += warps * 32) {
      const uint32_t g = g0 + lane;
      const uint32_t pos = g < total ? position(g) : 0u;
      const bool screen = g < total && !(pos >= sa && pos < sb);
      const unsigned sm = __ballot_sync(kFull, screen);
      n_fine += __popc(sm);
      // every lane takes part in the warp's bound (it shuffles across all 32 lanes)
      const float flb = warp_fine_lb2_32(ix, fup_s, flo_s, screen ? ix.perm[pos] : 0u, sm);
      const bool want = screen && flb <= lbb;
      for (unsigned m = __ballot_sync(kFull, want); m; m &= m - 1) refine(__shfl_sync(kFull, pos, __ffs(m) - 1));
    }
  } else {
    for (uint32_t g = gw; g < total; g += warps) {
      const uint32_t pos = position(g);
      if (pos >= sa && pos < sb) continue;  // already refined by the seed
      refine(pos);
    }
  }
  __shared__ unsigned s_n, s_nfine;
  if (threadIdx.x == 0) s_n = s_nfine = 0;
  __syncthreads();
  if (lane == 0) {
    if (bestd < 0x7f800000u) atomicMin(&s_min, bestd);
    if (n_front) atomicAdd(&s_n, n_front);
    if (n_fine) atomicAdd(&s_nfine, n_fine);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_n) atomicAdd(&st->series_refined, s_n);
    if (s_nfine) atomicAdd(&st->fine_front, s_nfine);
    if (qv.k == 1 && s_min < thr) atomicMin(&st->thr_bits, s_min);
  }
}

// ------------------------------------------------------------ refinement
// The refinement in three streaming kernels (ProcessQueue and CalculateRealDistance,
// Algorithms 8-9, with the block filter, the per-series filter and the real distances
// decoupled so that each kernel keeps many loads in flight):
//
// q_filter_blocks: a thread per aligned block of 32 positions of a work item (items
//   are the positions of one surviving leaf inside an aligned tile of kItem
//   positions): re-tests the leaf's bound against the current BSF and bounds each
//   of the block's two halves of 16 by its symbol envelope; surviving halves become
//   tasks.
// q_filter_series: a warp per two tasks (16 lanes each) bounds every position by its
//   SAX word (a coarse bound first, then the full one, then the fine PAA's when the
//   index keeps one); survivors {position, bound} go to a per-warp buffer flushed 32
//   at a time to the survivor list. kUnroll task pairs are in flight per warp.
// q_refine_rows: real distances of the survivors whose bound still passes the
//   current BSF, kRows rows per warp at a time. k = 1: the BSF is an atomicMin taken
//   only by a distance below the current BSF. k > 1: the shared candidate histogram
//   (khist_bound), and for k <= 32 each warp's own k best in registers (lane i holds
//   the i-th), published once it has k.
constexpr int kFiltWarps = 8;
constexpr int kUnroll = 4;
constexpr int kBlocksPerItem = kItem / 32;
constexpr int kHalvesPerItem = kItem / 16;  // half-block tasks a work item can yield
constexpr int kRows = 4;
constexpr int kRowWarps = 8;
constexpr int kBlkThreads = 256;

// One thread per (work item, aligned block of 32 positions): re-tests the item's
// leaf bound against the current BSF, bounds each half of the block by its symbol
// envelope (T[j][clamp(query symbol, lo_j, hi_j)] is the gap to the envelope's value
// range), and lists the surviving halves; the list is compacted per warp (one atomic
// per warp).
// Squared iSAX bound of a symbol envelope (per-segment min / max symbols lo, hi):
// T[j][clamp(query symbol, lo_j, hi_j)] is the gap to the envelope's value range.
template <bool kW16>
__device__ __forceinline__ float env_lb2_t(uint4 lo, uint4 hi, const float* Ts, const int* qsym, int w, int card,
                                           float seglen) {
  const uint32_t lop[4] = {lo.x, lo.y, lo.z, lo.w}, hip[4] = {hi.x, hi.y, hi.z, hi.w};
  float acc = 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (kW16 || j < w) {
      const int sl = (lop[j >> 2] >> (8 * (j & 3))) & 255, sh = (hip[j >> 2] >> (8 * (j & 3))) & 255;
      acc = __fadd_rn(acc, Ts[j * card + min(max(qsym[j], sl), sh)]);
    }
  }
  return __fmul_rn(acc, seglen);
}
__device__ __forceinline__ float env_lb2(uint4 lo, uint4 hi, const float* Ts, const int* qsym, int w, int card,
                                         float seglen) {
  return w == 16 ? env_lb2_t<true>(lo, hi, Ts, qsym, w, card, seglen)
                 : env_lb2_t<false>(lo, hi, Ts, qsym, w, card, seglen);
}

__device__ __forceinline__ void q_filter_blocks_body(const IndexView& ix, const QueryView& qv) {
  extern __shared__ __align__(16) float Ts[];  // [w][card]
  __shared__ int qsym_s[16];
  __shared__ uint32_t fl_s[kMaxFront];
  smem_fill(Ts, qv.T, ix.w * ix.card);
  if (threadIdx.x < ix.w) qsym_s[threadIdx.x] = qv.st->qsym[threadIdx.x];
  const uint32_t nfront = qv.st->nfront;
  if (threadIdx.x < nfront) fl_s[threadIdx.x] = qv.st->front_leaf[threadIdx.x];
  const uint32_t ntask = min(qv.st->item_count, qv.items_cap) * kBlocksPerItem;
  const float bound2 = lb_bound2(*(volatile unsigned*)&qv.st->thr_bits, qv.eps, qv.tau);
  const float seglen = (float)ix.seglen;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  __syncthreads();
  for (uint32_t t0 = blockIdx.x * blockDim.x; t0 < ntask; t0 += gridDim.x * blockDim.x) {
    const uint32_t t = t0 + threadIdx.x;
    bool k0 = false, k1 = false;
    uint2 o0 = make_uint2(0, 0), o1 = o0;
    if (t < ntask) {
      const uint4 item = qv.items[t / kBlocksPerItem];
      const uint32_t blk = (item.x / kItem) * kBlocksPerItem + (t % kBlocksPerItem);
      bool front = false;  // a leaf refined early
      for (uint32_t f = 0; f < nfront; ++f) front |= fl_s[f] == item.w;
      if (!front && __uint_as_float(item.z) <= bound2 && blk * 32 < item.y && blk * 32 + 32 > item.x) {
        // the block's positions inside the item, [lo, hi) offsets, and each of its two
        // halves of 16 that holds some of them, bounded by the half's own envelope; a
        // task is a half-block and its [lo, hi) offsets inside the half
        const uint32_t b32 = blk * 32;
        const uint32_t lo_off = max(item.x, b32) - b32, hi_off = min(item.y, b32 + 32) - b32;
        const uint4* he = ix.henv + 4 * (size_t)blk;  // half 2 blk: he[0..1], half 2 blk + 1: he[2..3]
        const bool in0 = lo_off < 16, in1 = hi_off > 16;
        uint4 l0 = make_uint4(0, 0, 0, 0), h0 = l0, l1 = l0, h1 = l0;
        if (in0) {
          l0 = __ldg(he);
          h0 = __ldg(he + 1);
        }
        if (in1) {
          l1 = __ldg(he + 2);
          h1 = __ldg(he + 3);
        }
        k0 = in0 && env_lb2(l0, h0, Ts, qsym_s, ix.w, ix.card, seglen) <= bound2;
        k1 = in1 && env_lb2(l1, h1, Ts, qsym_s, ix.w, ix.card, seglen) <= bound2;
        o0 = make_uint2(2 * blk, lo_off | (min(hi_off, 16u) << 8));
        o1 = make_uint2(2 * blk + 1, (max(lo_off, 16u) - 16) | ((hi_off - 16) << 8));
      }
    }
    // the warp's surviving halves: one atomic for the warp, no block barrier
    const unsigned m0 = __ballot_sync(kFull, k0), m1 = __ballot_sync(kFull, k1);
    if (m0 | m1) {
      const int leader = __ffs(m0 | m1) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&qv.st->blk_count, (uint32_t)(__popc(m0) + __popc(m1)));
      base = __shfl_sync(kFull, base, leader);
      if (k0) {
        const uint32_t slot = base + __popc(m0 & lt);
        if (slot < qv.blks_cap) qv.blks[slot] = o0;
        else qv.st->overflow = 1u;
      }
      if (k1) {
        const uint32_t slot = base + __popc(m0) + __popc(m1 & lt);
        if (slot < qv.blks_cap) qv.blks[slot] = o1;
        else qv.st->overflow = 1u;
      }
    }
  }
}

__global__ void __launch_bounds__(kBlkThreads)
q_filter_blocks(IndexView ix, QueryView qv) {
  pdl_begin();
  q_filter_blocks_body(ix, qv);
}

// One warp per surviving block: bounds every position by its SAX word and buffers
// the survivors {position, bound}, flushed 32 at a time. kUnroll blocks are in flight
// per warp. Each word is first bounded from its kCoarseBits-bit symbol prefixes (T5:
// kCoarse entries per segment, at most two lanes per bank); the words that pass are
// queued per warp and bounded from their full symbols (T) a whole warp at a time.
constexpr int kQueue = 64;

// Coarse bound from the symbols' top kCoarseBits bits. The table entry's byte offset
// inside segment j's row comes straight from the word: symbol byte b of a 32-bit part
// shifted right by 8 b + cshift - 2 and masked to bits 2 .. kCoarseBits + 1 (one shift
// and one mask per segment; cshift >= 2, i.e. symbols of at least kCoarseBits + 2
// bits, else the plain index).
__device__ __forceinline__ float word_lb2_coarse(uint4 wd, const float* T5s, int w, int cshift, float s) {
  const uint32_t parts[4] = {wd.x, wd.y, wd.z, wd.w};
  const char* tb = reinterpret_cast<const char*>(T5s);
  constexpr uint32_t kMask = (uint32_t)(kCoarse - 1) << 2;
  float acc = 0.0f;
  if (cshift >= 2 && w == 16) {  // 16 segments: no per-segment test of the count
    const int sh0 = cshift - 2;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      acc = __fadd_rn(acc, *reinterpret_cast<const float*>(tb + j * kCoarse * 4 +
                                                            ((parts[j >> 2] >> (8 * (j & 3) + sh0)) & kMask)));
  } else if (cshift >= 2) {
    const int sh0 = cshift - 2;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < w)
        acc = __fadd_rn(acc, *reinterpret_cast<const float*>(tb + j * kCoarse * 4 +
                                                              ((parts[j >> 2] >> (8 * (j & 3) + sh0)) & kMask)));
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < w) acc = __fadd_rn(acc, T5s[j * kCoarse + (((parts[j >> 2] >> (8 * (j & 3))) & 255) >> cshift)]);
  }
  return __fmul_rn(acc, s);
}

__device__ __forceinline__ void q_filter_series_body(const IndexView& ix, const QueryView& qv) {
  
  extern __shared__ __align__(16) float Ts[];  // [w][card], then T5 [w][kCoarse]
  float* T5s = Ts + ix.w * ix.card;
  __shared__ uint2 buf_s[kFiltWarps][64];
  __shared__ uint4 qw_s[kFiltWarps][kQueue];
  __shared__ uint32_t qp_s[kFiltWarps][kQueue];
  __shared__ float fup_s[kMaxFine], flo_s[kMaxFine];
  smem_fill(Ts, qv.T, ix.w * ix.card);
  smem_fill(T5s, qv.T5, ix.w * kCoarse);
  for (int j = threadIdx.x; j < ix.wf; j += blockDim.x) {
    fup_s[j] = qv.st->fup[j];
    flo_s[j] = qv.st->flo[j];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint2* buf = buf_s[warp];
  uint4* qw = qw_s[warp];
  uint32_t* qp = qp_s[warp];
  QState* st = qv.st;
  // tasks are half-blocks of 16 positions; a warp takes two at a time (lanes 0-15 the
  // first, 16-31 the second)
  const uint32_t nhalf = min(st->blk_count, qv.blks_cap), ntask = (nhalf + 1) / 2;
  const int hl = lane & 15;
  const uint32_t sa = st->seed_a, sb = st->seed_b;
  const float seglen = (float)ix.seglen;
  const int cshift = ix.bits > kCoarseBits ? ix.bits - kCoarseBits : 0;

  const unsigned lt = (1u << lane) - 1u;
  const uint32_t gw = blockIdx.x * kFiltWarps + warp;
  const uint32_t stride = gridDim.x * kFiltWarps;
  uint32_t nbuf = 0, nq = 0, n_lb = 0, n_fine = 0;
  float bound2 = 0.0f;

  // full bounds of the first 32 queued words (one per lane); survivors to the buffer
  auto drain32 = [&](uint32_t count) {
    const bool have = lane < (int)count;
    const uint32_t p = have ? qp[lane] : 0u;
    float lb2 = have ? word_lb2(qw[lane], Ts, ix.w, ix.card, seglen) : INFINITY;
    bool pass = have && lb2 <= bound2;
    if (pass && ix.wf) {  // the fine PAA's bound, before the series is read
      ++n_fine;
      lb2 = fmaxf(lb2, fine_lb2(ix, fup_s, flo_s, __ldg(ix.perm + p)));
      pass = lb2 <= bound2;
    }
    __syncwarp();
    if (count > 32 && lane < (int)count - 32) {  // move the rest of the queue down
      qw[lane] = qw[32 + lane];
      qp[lane] = qp[32 + lane];
    }
    const unsigned m = __ballot_sync(kFull, pass);
    if (pass) buf[nbuf + __popc(m & lt)] = make_uint2(p, __float_as_uint(lb2));
    nbuf += __popc(m);
    __syncwarp();
    if (nbuf >= 32) {  // flush 32 survivors with one atomic, entry by entry
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&st->surv_count, 32u);
      base = __shfl_sync(kFull, base, 0);
      if (base + lane < qv.surv_cap) qv.surv[base + lane] = buf[lane];
      else st->overflow = 1u;
      __syncwarp();
      if (lane < (int)nbuf - 32) buf[lane] = buf[32 + lane];
      nbuf -= 32;
      __syncwarp();
    }
  };

  for (uint32_t t0 = gw; t0 < ntask; t0 += stride * kUnroll) {
    const unsigned thr = __shfl_sync(kFull, lane == 0 ? *(volatile unsigned*)&st->thr_bits : 0u, 0);
    bound2 = lb_bound2(thr, qv.eps, qv.tau);
    uint2 task[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t r = 2 * (t0 + u * stride) + (lane >> 4);
      task[u] = r < nhalf ? qv.blks[r] : make_uint2(0, 0);  // an empty range when past the end
    }
    uint4 wd[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t p = task[u].x * 16 + hl;
      const bool in = hl >= (int)(task[u].y & 255u) && hl < (int)(task[u].y >> 8);
      wd[u] = in ? __ldg(ix.words + p) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t p = task[u].x * 16 + hl;
      const bool valid = hl >= (int)(task[u].y & 255u) && hl < (int)(task[u].y >> 8) && (p < sa || p >= sb);
      n_lb += valid;
      const bool pass_c = valid && word_lb2_coarse(wd[u], T5s, ix.w, cshift, seglen) <= bound2;
      const unsigned m = __ballot_sync(kFull, pass_c);
      if (pass_c) {
        qw[nq + __popc(m & lt)] = wd[u];
        qp[nq + __popc(m & lt)] = p;
      }
      nq += __popc(m);
      __syncwarp();
      if (nq >= 32) {
        drain32(nq);
        nq -= 32;
      }
    }
  }
  while (nq > 0) {
    const uint32_t c = nq;
    drain32(c);
    nq = c > 32 ? c - 32 : 0;
  }
  // the last partial buffers of the CTA's warps: one atomic for the whole CTA
  __syncwarp();
  __shared__ uint32_t wbase_s[kFiltWarps], cbase_s;
  if (lane == 0) wbase_s[warp] = nbuf;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w2 = 0; w2 < kFiltWarps; ++w2) {
      const uint32_t c = wbase_s[w2];
      wbase_s[w2] = tot;
      tot += c;
    }
    cbase_s = tot ? atomicAdd(&st->surv_count, tot) : 0u;
  }
  __syncthreads();
  if (lane < (int)nbuf) {
    const uint32_t pos = cbase_s + wbase_s[warp] + lane;
    if (pos < qv.surv_cap) qv.surv[pos] = buf[lane];
    else st->overflow = 1u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_lb += __shfl_xor_sync(kFull, n_lb, o);
    n_fine += __shfl_xor_sync(kFull, n_fine, o);
  }
  if (lane == 0 && gw < kMaxRefineWarps) {
    qv.partials[gw] = n_lb;
    qv.partials[2 * kMaxRefineWarps + gw] = gw == 0 ? nhalf : 0u;
    qv.partials[3 * kMaxRefineWarps + gw] = n_fine;
  }
}

__global__ void __launch_bounds__(kFiltWarps * 32)
q_filter_series(IndexView ix, QueryView qv) {
  pdl_begin();
  q_filter_series_body(ix, qv);
}

template <bool KONE>
__device__ __forceinline__ void q_refine_rows_body(const IndexView& ix, const QueryView& qv) {
  
  extern __shared__ __align__(16) float qs[];
  smem_fill(qs, qv.qz, ix.len);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  QState* st = qv.st;
  volatile unsigned int* thr_v = &st->thr_bits;
  // a query whose lists overflowed is run again with room for all n: skip it here
  const uint2* surv = qv.rsurv ? qv.rsurv : qv.surv;
  const uint32_t nsurv = st->overflow ? 0u : (qv.rsurv ? st->ord_count : min(st->surv_count, qv.surv_cap));
  const int k = qv.k;
  const unsigned lt = (1u << lane) - 1u;
  unsigned mine = 0x7f800000u;
  uint32_t n_ref = 0;
  const uint32_t gw = blockIdx.x * kRowWarps + warp;
  const uint32_t step = gridDim.x * kRowWarps * kRows;
  const float kbase = KONE ? 0.0f : st->kbase;  // k > 1: the candidate histogram's range
  uint32_t hist_round = 0;
  // three-stage pipeline over this warp's groups of kRows survivors (lanes < kRows
  // hold one survivor each): the survivor entry of group g + 2 step and the perm /
  // moments of group g + step are in flight while the rows of group g are read
  uint2 sv_a = make_uint2(0, 0), sv_b = make_uint2(0, 0);
  uint32_t id_b = 0;
  float2 ms_b = make_float2(0.f, 0.f);
  const uint32_t g0 = gw * kRows;
  if (lane < kRows && g0 + lane < nsurv) sv_b = surv[g0 + lane];
  if (lane < kRows && g0 + lane < nsurv) {
    id_b = __ldg(ix.perm + sv_b.x);
    if (!ix.data_is_z) ms_b = __ldg(ix.stats + sv_b.x);
  }
  if (lane < kRows && g0 + step + lane < nsurv) sv_a = surv[g0 + step + lane];
  for (uint32_t g = g0; g < nsurv; g += step) {
    const uint2 sv = sv_b;
    const uint32_t myid_cur = id_b;
    const float2 myms_cur = ms_b;
    if (lane < kRows && g + step + lane < nsurv) {
      id_b = __ldg(ix.perm + sv_a.x);
      if (!ix.data_is_z) ms_b = __ldg(ix.stats + sv_a.x);
    }
    sv_b = sv_a;
    if (lane < kRows && g + 2 * step + lane < nsurv) sv_a = surv[g + 2 * step + lane];
    const unsigned thr = __shfl_sync(kFull, lane == 0 ? *thr_v : 0u, 0);
    const float bound2 = lb_bound2(thr, qv.eps, qv.tau);
    const uint32_t myp = sv.x;
    const bool mine_live = lane < kRows && g + lane < nsurv && __uint_as_float(sv.y) <= bound2;
    const uint32_t myid = myid_cur;
    const float2 myms = myms_cur;
    const unsigned rm = __ballot_sync(kFull, mine_live);
    if (!rm) continue;
    uint32_t id[kRows];
    float2 ms[kRows];
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      id[j] = __shfl_sync(kFull, myid, j);
      ms[j].x = __shfl_sync(kFull, myms.x, j);
      ms[j].y = __shfl_sync(kFull, myms.y, j);
    }
    float acc[kRows];
#pragma unroll
    for (int j = 0; j < kRows; ++j) acc[j] = 0.0f;
    if ((ix.len & 3) == 0) {
      const int n4 = ix.len >> 2;
      const float4* q4 = reinterpret_cast<const float4*>(qs);
      for (int c0 = lane; c0 < n4; c0 += 64) {  // two float4 of every row in flight
        float4 x2[2][kRows];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < kRows; ++j)
            x2[h][j] = ((rm >> j) & 1u) && c0 + 32 * h < n4
                           ? __ldg(reinterpret_cast<const float4*>(ix.data + (size_t)id[j] * ix.len) + c0 + 32 * h)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
        const int c = c0 + 32 * h;
        if (c >= n4) break;
        const float4* x = x2[h];
        const float4 q = q4[c];
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
          float4 z = x[j];
          if (!ix.data_is_z) {
            z.x = znorm_value(z.x, ms[j].x, ms[j].y);
            z.y = znorm_value(z.y, ms[j].x, ms[j].y);
            z.z = znorm_value(z.z, ms[j].x, ms[j].y);
            z.w = znorm_value(z.w, ms[j].x, ms[j].y);
          }
          float d = __fsub_rn(z.x, q.x); acc[j] = __fmaf_rn(d, d, acc[j]);
          d = __fsub_rn(z.y, q.y); acc[j] = __fmaf_rn(d, d, acc[j]);
          d = __fsub_rn(z.z, q.z); acc[j] = __fmaf_rn(d, d, acc[j]);
          d = __fsub_rn(z.w, q.w); acc[j] = __fmaf_rn(d, d, acc[j]);
        }
        }
      }
    } else {
      for (int t = lane; t < ix.len; t += 32) {
#pragma unroll
        for (int j = 0; j < kRows; ++j) {
          if ((rm >> j) & 1u) {
            const float x = __ldg(ix.data + (size_t)id[j] * ix.len + t);
            const float z = ix.data_is_z ? x : znorm_value(x, ms[j].x, ms[j].y);
            const float d = __fsub_rn(z, qs[t]);
            acc[j] = __fmaf_rn(d, d, acc[j]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kRows; ++j)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(kFull, acc[j], o);
    n_ref += __popc(rm);
    float d2 = acc[0];
#pragma unroll
    for (int j = 1; j < kRows; ++j)
      if (lane == j) d2 = acc[j];
    const unsigned thr2 = __shfl_sync(kFull, lane == 0 ? *thr_v : 0u, 0);
    const bool keep = mine_live && d2 <= keep_bound2(thr2, qv.eps);
    const unsigned km = __ballot_sync(kFull, keep);
    if (km) {
      const int leader = __ffs(km) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&st->cand_count, (uint32_t)__popc(km));
      base = __shfl_sync(kFull, base, leader);
      const uint32_t slot = base + __popc(km & lt);
      if (keep) {
        if (slot < qv.cand_cap) qv.cand[slot] = pack(d2, myp);
        else st->overflow = 1u;
      }
    }
    if (!KONE && keep && kbase > 0.0f && d2 < kbase) atomicAdd(&qv.khist[khist_bucket(d2, kbase)], 1u);
    if (!KONE && kbase > 0.0f && ((++hist_round & 15) == 0)) {  // every 16 groups: the shared bound
      const unsigned hb = khist_bound(qv.khist, kbase, k);
      if (lane == 0 && hb < thr2) atomicMin(&st->thr_bits, hb);
    }
    if (KONE) {
      if (mine_live && __float_as_uint(d2) < thr2) atomicMin(&st->thr_bits, __float_as_uint(d2));
    } else if (k <= 32) {  // the warp's own k best as well
      const unsigned kth_old = __shfl_sync(kFull, mine, k - 1);
      for (int j = 0; j < kRows; ++j) {
        if (!((rm >> j) & 1u)) continue;
        const unsigned v = __float_as_uint(__shfl_sync(kFull, d2, j));
        if (v >= __shfl_sync(kFull, mine, k - 1)) continue;
        const int pos = __popc(__ballot_sync(kFull, lane < k && mine <= v));
        const unsigned up = __shfl_up_sync(kFull, mine, 1);
        if (lane >= pos && lane < k) mine = lane == pos ? v : up;
      }
      const unsigned kth = __shfl_sync(kFull, mine, k - 1);
      if (lane == 0 && kth < kth_old && kth < thr2) atomicMin(&st->thr_bits, kth);
    }
  }
  if (lane == 0 && gw < kMaxRefineWarps) qv.partials[kMaxRefineWarps + gw] = n_ref;
}

template <bool KONE>
__global__ void __launch_bounds__(kRowWarps * 32)
q_refine_rows(IndexView ix, QueryView qv) {
  pdl_begin();
  q_refine_rows_body<KONE>(ix, qv);
}

// ------------------------------------------------------------------ final pick
// The k-th smallest candidate squared distance T; candidates at or below
// T (1 + eps) are re-checked in FP64 (one block).
__device__ void final_select(const QueryView& qv, uint32_t* hist, uint32_t* sel) {
  const uint32_t count = min(qv.st->cand_count, qv.cand_cap);
  const unsigned long long* c = qv.cand;
  uint32_t kth;
  if (qv.k == 1) {  // the smallest: one block-wide minimum
    if (threadIdx.x == 0) sel[0] = 0xffffffffu;
    __syncthreads();
    uint32_t mn = 0xffffffffu;
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) mn = min(mn, (uint32_t)(c[i] >> 32));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(kFull, mn, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&sel[0], mn);
    __syncthreads();
    kth = sel[0];
  } else {
    kth = block_select_u32([&](uint32_t i) { return (uint32_t)(c[i] >> 32); }, count, (uint32_t)qv.k, hist, sel);
  }
  if (threadIdx.x == 0) qv.st->final_bits = __float_as_uint(__fmul_ru(__uint_as_float(kth), 1.0f + qv.eps));
}

// FP64 re-check of the candidates at or below the k-th candidate distance times
// (1 + eps): one warp per candidate. Lane l adds the FP64 squared differences of the
// points t = l, l + 32, ... in increasing t; the 32 partials are combined by a
// pairwise tree in lane order. No fused operations. The FP64 sum differs from a
// sequential one by a few units in its last place at most (far inside the fp32
// margin), and identical series give identical sums, so exact ties stay ties.
// In rounds of 4 * blockDim candidates, all threads test the candidates against the
// bound and list the passing ones in shared memory (`list`, 4 * blockDim entries);
// then one warp per listed candidate computes its FP64 distance.
__device__ void recheck(const IndexView& ix, const QueryView& qv, uint32_t* list, uint32_t* s_n) {
  const uint32_t count = min(qv.st->cand_count, qv.cand_cap);
  const uint32_t bound = qv.st->final_bits;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = blockDim.x / 32;
  for (uint32_t c0 = 0; c0 < count; c0 += 4 * blockDim.x) {
    if (threadIdx.x == 0) *s_n = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint32_t i = c0 + r * blockDim.x + threadIdx.x;
      if (i < count && (uint32_t)(qv.cand[i] >> 32) <= bound) list[atomicAdd(s_n, 1u)] = i;
    }
    __syncthreads();
    const uint32_t listed = *s_n;
    for (uint32_t li = threadIdx.x >> 5; li < listed; li += warps) {
      const uint32_t pos = (uint32_t)qv.cand[list[li]];
      const uint32_t id = ix.perm[pos];
      const float2 ms = ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos];
      const float* row = ix.data + (size_t)id * ix.len;
      double acc = 0.0;
      for (int t = lane; t < ix.len; t += 32) {
        const float x = row[t];
        const float z = ix.data_is_z ? x : znorm_value(x, ms.x, ms.y);
        const double d = __dsub_rn((double)z, (double)qv.qz[t]);
        acc = __dadd_rn(acc, __dmul_rn(d, d));
      }
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) acc = __dadd_rn(acc, __shfl_xor_sync(kFull, acc, off));
      if (lane == 0) {
        const uint32_t slot = atomicAdd(&qv.st->rc_count, 1u);
        qv.rc_d[slot] = acc;
        qv.rc_id[slot] = id;
      }
    }
    __syncthreads();
  }
}

// (distance bits, id) lexicographic order; non-negative doubles order as their bits.
__device__ __forceinline__ bool key_less(unsigned long long da, uint32_t ia, unsigned long long db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

__device__ void block_bitonic(unsigned long long* sk, uint32_t* si, int n) {
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
        const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
        const bool asc = (lo & size) == 0;
        if (key_less(sk[hi], si[hi], sk[lo], si[lo]) == asc) {
          const unsigned long long tk = sk[lo]; sk[lo] = sk[hi]; sk[hi] = tk;
          const uint32_t ti = si[lo]; si[lo] = si[hi]; si[hi] = ti;
        }
      }
      __syncthreads();
    }
}

constexpr int kSortCap = 2048;  // (distance, id) pairs sorted in shared memory

// The exact answer (one block of 1024 threads): the k-th smallest candidate, the FP64
// re-check of every candidate within the fp32 margin of it, and the k smallest by
// (FP64 distance, id), written to the outputs.
__device__ __forceinline__ void q_finalize_body(const IndexView& ix, const QueryView& qv, int64_t* __restrict__ ids_out, float* __restrict__ dists_out, double* __restrict__ d64_out) {
  
  if (qv.call) {
    const CallDesc c = *qv.call;
    const size_t off = (size_t)qv.qi * qv.k;
    ids_out = c.ids + off;
    dists_out = c.dists ? c.dists + off : nullptr;
    d64_out = c.d64 ? c.d64 + off : nullptr;
  }
  __shared__ unsigned long long sk[kSortCap];
  __shared__ uint32_t si[kSortCap];
  __shared__ uint32_t hist[256], sel[2], s_cnt;
  if (threadIdx.x == 0 && qv.ovf) *qv.ovf = qv.st->overflow;
  if (qv.st->overflow) return;  // the query is run again with room for all n
  if (qv.window < 0) {  // DTW: q_final_pick and q_recheck_dtw did this part
    final_select(qv, hist, sel);
    __syncthreads();
    static_assert(sizeof(sk) >= 4 * 1024 * sizeof(uint32_t), "re-check list must hold 4 * blockDim entries");
    recheck(ix, qv, reinterpret_cast<uint32_t*>(sk), &s_cnt);
    __syncthreads();
  }
  const uint32_t R = qv.st->rc_count;
  const int k = qv.k;
  int nsort;
  if (R <= (uint32_t)kSortCap) {
    nsort = 1;
    while (nsort < (int)R) nsort <<= 1;
    for (int i = threadIdx.x; i < nsort; i += blockDim.x) {
      const bool v = i < (int)R;
      sk[i] = v ? (unsigned long long)__double_as_longlong(qv.rc_d[i]) : ~0ull;
      si[i] = v ? qv.rc_id[i] : ~0u;
    }
    __syncthreads();
  } else {
    // exact k-th (distance, id) key by a 12-digit radix select, then the k keys at
    // or below it
    unsigned long long pre_hi = 0, mask_hi = 0;
    uint32_t pre_lo = 0, mask_lo = 0, kk = (uint32_t)k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int dgt = 0; dgt < 12; ++dgt) {
      for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < R; i += blockDim.x) {
        const unsigned long long dk = (unsigned long long)__double_as_longlong(qv.rc_d[i]);
        const uint32_t id = qv.rc_id[i];
        if ((dk & mask_hi) != pre_hi || (id & mask_lo) != pre_lo) continue;
        const uint32_t b = dgt < 8 ? (uint32_t)(dk >> (8 * (7 - dgt))) & 255u : (id >> (8 * (11 - dgt))) & 255u;
        atomicAdd(&hist[b], 1u);
      }
      __syncthreads();
      if (warp == 0) {
        uint32_t loc[8], tot = 0;
        for (int b = 0; b < 8; ++b) { loc[b] = hist[lane * 8 + b]; tot += loc[b]; }
        uint32_t incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - tot;
        if (excl < kk && kk <= incl) {
          uint32_t cum = excl;
          for (int b = 0; b < 8; ++b) {
            if (cum + loc[b] >= kk) { sel[0] = (uint32_t)(lane * 8 + b); sel[1] = kk - cum; break; }
            cum += loc[b];
          }
        }
      }
      __syncthreads();
      if (dgt < 8) {
        pre_hi |= (unsigned long long)sel[0] << (8 * (7 - dgt));
        mask_hi |= 255ull << (8 * (7 - dgt));
      } else {
        pre_lo |= sel[0] << (8 * (11 - dgt));
        mask_lo |= 255u << (8 * (11 - dgt));
      }
      kk = sel[1];
      __syncthreads();
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < R; i += blockDim.x) {
      const unsigned long long dk = (unsigned long long)__double_as_longlong(qv.rc_d[i]);
      const uint32_t id = qv.rc_id[i];
      if (dk < pre_hi || (dk == pre_hi && id <= pre_lo)) {
        const uint32_t slot = atomicAdd(&s_cnt, 1u);
        if (slot < (uint32_t)kSortCap) { sk[slot] = dk; si[slot] = id; }
      }
    }
    __syncthreads();
    const int got = (int)min(s_cnt, (uint32_t)kSortCap);
    nsort = 1;
    while (nsort < got) nsort <<= 1;
    for (int i = got + threadIdx.x; i < nsort; i += blockDim.x) { sk[i] = ~0ull; si[i] = ~0u; }
    __syncthreads();
  }
  block_bitonic(sk, si, nsort);
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    ids_out[r] = (int64_t)si[r];
    if (dists_out) dists_out[r] = __double2float_rn(__dsqrt_rn(__longlong_as_double((long long)sk[r])));
    if (d64_out) d64_out[r] = __longlong_as_double((long long)sk[r]);
  }
  // sum the refinement's per-warp work counters
  __shared__ unsigned long long s_part[4];
  if (threadIdx.x < 4) s_part[threadIdx.x] = 0;
  __syncthreads();
  {
    unsigned long long a = 0, b = 0, cc = 0, fc = 0;
    for (uint32_t i = threadIdx.x; i < qv.npartials; i += blockDim.x) {
      a += qv.partials[i];
      cc += qv.partials[2 * kMaxRefineWarps + i];
      fc += qv.partials[3 * kMaxRefineWarps + i];
    }
    for (uint32_t i = threadIdx.x; i < qv.npartials_rows; i += blockDim.x) b += qv.partials[kMaxRefineWarps + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
      cc += __shfl_xor_sync(kFull, cc, o);
      fc += __shfl_xor_sync(kFull, fc, o);
    }
    if ((threadIdx.x & 31) == 0) {  // one shared atomic per warp
      atomicAdd(&s_part[0], a);
      atomicAdd(&s_part[1], b);
      atomicAdd(&s_part[2], cc);
      atomicAdd(&s_part[3], fc);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const QState* st = qv.st;
    unsigned long long* c = qv.counters;
    atomicAdd(&c[ST_QUERIES], 1ull);
    atomicAdd(&c[ST_LEAVES_TOTAL], (unsigned long long)ix.L);
    atomicAdd(&c[ST_LEAVES_SURVIVED], (unsigned long long)st->leaf_count);
    atomicAdd(&c[ST_LEAVES_PROCESSED], s_part[2]);
    atomicAdd(&c[ST_SERIES_LB], s_part[0]);
    const unsigned long long seed = st->seed_done;
    atomicAdd(&c[ST_SERIES_REFINED], s_part[1] + seed + st->series_refined);
    atomicAdd(&c[ST_SEED], seed + st->series_refined);
    atomicAdd(&c[ST_CANDIDATES], (unsigned long long)st->cand_count);
    atomicAdd(&c[ST_RECHECKED], (unsigned long long)R);
    atomicAdd(&c[ST_SURVIVORS], (unsigned long long)st->surv_count);
    atomicAdd(&c[ST_FINE], s_part[3]);
    atomicAdd(&c[ST_FINE_FRONT], (unsigned long long)st->fine_front);
  }
}

__global__ void __launch_bounds__(1024)
q_finalize(IndexView ix, QueryView qv, int64_t* __restrict__ ids_out, float* __restrict__ dists_out,
           double* __restrict__ d64_out) {
  pdl_begin();
  q_finalize_body(ix, qv, ids_out, dists_out, d64_out);
}

// ------------------------------------------------------------ batched chain
// A batch of queries runs the same chain with one launch per stage for the whole
// batch: blockIdx.y selects the query (its workspace in a device array of query
// views), blockIdx.x and gridDim.x divide that query's work exactly as in the
// one-query kernels. The batch's queries and outputs come from a call descriptor
// (query qbase + blockIdx.y of the call), so a captured graph serves every call of
// one shape. Queries of a batch share no state: each keeps its own BSF, lists and
// counters, and the answers are those of the same queries run one at a time.
struct BatchArgs {
  const QueryView* __restrict__ qvs;  // [batch] device array: one workspace per query
  int order;                          // 1: the row kernel reads the bound-ordered survivors
  const CallDesc* call;   // queries and outputs of the call
  uint32_t* ovf;          // [batch] per-query overflow flags
  int qbase;              // index of the batch's first query in the call
  int k;
  uint32_t np, npr;       // warps of the series filter and row kernels, per query
};

// The view of query blockIdx.y, read in place (qb_views wrote this call's fields into
// it first), so that a kernel keeps in registers only the fields it uses.
__device__ __forceinline__ const QueryView& batch_view(const BatchArgs& a) { return a.qvs[blockIdx.y]; }

// First stage of every batch: the per-call fields of each query's view.
__global__ void qb_views(QueryView* qvs, BatchArgs a, int count) {
  pdl_begin();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  QueryView& qv = qvs[b];
  qv.k = a.k;
  qv.ovf = a.ovf + b;
  qv.call = a.call;
  qv.qi = a.qbase + b;
  qv.npartials = a.np;
  qv.npartials_rows = a.npr;
  qv.window = -1;
  qv.rsurv = a.order ? qv.surv2 : nullptr;
}

// The priority order of ProcessQueue (Algorithm 8: DeleteMin takes the lowest bound
// first), for the survivors of the series filter: one block per query counts the
// survivors whose bound still passes the current BSF in 256 equal buckets of
// [0, bound), then scatters them bucket by bucket into surv2, so the row kernel's
// warps, which take survivors from the front of the list, refine the lowest bounds
// first and tighten the BSF before the higher ones are read. (Within a bucket the
// order is that of arrival.)
__global__ void __launch_bounds__(1024) qb_order(BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  QState* st = qv.st;
  __shared__ uint32_t hist[256], base[256];
  if (st->overflow) return;  // the query runs again alone
  const uint32_t m = min(st->surv_count, qv.surv_cap);
  const float bound2 = lb_bound2(st->thr_bits, qv.eps, qv.tau);
  // the bucket of a bound: [0, bound2) in 256 equal parts (all in one bucket while the
  // BSF is still unknown)
  const float scale = bound2 < INFINITY && bound2 > 0.0f ? __fdiv_rn(256.0f, bound2) : 0.0f;
  for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const float lb = __uint_as_float(qv.surv[i].y);
    if (lb <= bound2) atomicAdd(&hist[min(255, (int)__fmul_rz(lb, scale))], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the 256 counts by one warp
    const int lane = threadIdx.x;
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = hist[8 * lane + j];
      sum += v[j];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      base[8 * lane + j] = run;
      run += v[j];
    }
    if (lane == 31) st->ord_count = incl;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const uint2 sv = qv.surv[i];
    const float lb = __uint_as_float(sv.y);
    if (lb <= bound2) qv.surv2[atomicAdd(&base[min(255, (int)__fmul_rz(lb, scale))], 1u)] = sv;
  }
}

__global__ void __launch_bounds__(kThreads) qb_prep(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_prep_body(ix, nullptr, qv, a.k);
}
__global__ void __launch_bounds__(kThreads) qb_seed(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_seed_body(ix, qv);
}
__global__ void __launch_bounds__(1024) qb_seed_select(BatchArgs a, int base) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_seed_select_body(qv, base);
}
__global__ void __launch_bounds__(kThreads) qb_leaf_filter(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_leaf_filter_body(ix, qv);
}
// The leaf filter for the whole batch, leaf-major: a thread per leaf loads its
// envelope once, turns it into the 16 region edges, and bounds it against every query
// of the batch from those (the one-query filter's arithmetic, operation for
// operation); each query's survivors, work items and per-block minimum go to its own
// workspace as in q_leaf_filter.
constexpr int kBatchMax = 128;  // queries per leaf-major launch (the batch group cap)
__global__ void __launch_bounds__(kThreads) qb_leaf_filter_lm(IndexView ix, BatchArgs a, int count) {
  pdl_begin();
  __shared__ float thr_up_s[257], thr_lo_s[257];
  __shared__ float paa_s[kBatchMax][16];
  __shared__ float bnd_s[kBatchMax];
  __shared__ uint32_t sa_s[kBatchMax], sb_s[kBatchMax];
  __shared__ unsigned long long bmin_s[kBatchMax];
  for (int v = threadIdx.x; v <= ix.card; v += blockDim.x) {
    thr_up_s[v] = ix.thr_up[v];
    thr_lo_s[v] = ix.thr_lo[v];
  }
  for (int e = threadIdx.x; e < count * 16; e += blockDim.x) {
    const int q = e >> 4, j = e & 15;
    paa_s[q][j] = j < ix.w ? a.qvs[q].st->qpaa[j] : 0.0f;
  }
  for (int q = threadIdx.x; q < count; q += blockDim.x) {
    const QueryView& qv = a.qvs[q];
    bnd_s[q] = lb_bound2(qv.st->thr_bits, qv.eps, qv.tau);
    sa_s[q] = qv.st->seed_a;
    sb_s[q] = qv.st->seed_b;
    bmin_s[q] = ~0ull;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool have = l < ix.L;
  float lower[16], upper[16];
  uint32_t b = 0, e = 0, nit = 0;
  if (have) {
    const uint4 lo = ix.env[2 * l], hi = ix.env[2 * l + 1];
    const uint32_t lop[4] = {lo.x, lo.y, lo.z, lo.w}, hip[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int sl = (lop[j >> 2] >> (8 * (j & 3))) & 255, sh = (hip[j >> 2] >> (8 * (j & 3))) & 255;
      lower[j] = j < ix.w ? thr_lo_s[sl] : -INFINITY;
      upper[j] = j < ix.w ? thr_up_s[sh + 1] : INFINITY;
    }
    b = ix.leaf_begin[l];
    e = ix.leaf_begin[l + 1];
    nit = (e - 1) / kItem - b / kItem + 1;  // aligned tiles of kItem positions touched
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      lower[j] = -INFINITY;
      upper[j] = INFINITY;
    }
  }
  const float seglen = (float)ix.seglen;
  const unsigned lt = (1u << lane) - 1u;
  for (int q = 0; q < count; ++q) {
    bool keep = false;
    float lb2 = 0.0f;
    if (have && !(b >= sa_s[q] && e <= sb_s[q])) {
      // the gap to [lower, upper] without branches: lower <= upper, so at most one
      // difference is positive (a NaN PAA value gives 0, as the compare form does);
      // segments past w have an infinite envelope and add an exact 0
      float acc = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float p = paa_s[q][j];
        const float d = fmaxf(fmaxf(__fsub_rn(lower[j], p), __fsub_rn(p, upper[j])), 0.0f);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
      }
      lb2 = __fmul_rn(acc, seglen);
      keep = lb2 <= bnd_s[q];
    }
    const unsigned m = __ballot_sync(kFull, keep);
    if (!m) continue;
    const QueryView& qv = a.qvs[q];
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&qv.st->leaf_count, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    const uint32_t mynit = keep ? nit : 0u;
    uint32_t incl = mynit;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t ibase = 0;
    if (lane == 31) ibase = atomicAdd(&qv.st->item_count, incl);
    ibase = __shfl_sync(kFull, ibase, 31) + incl - mynit;
    // the warp's lowest (bound, leaf) key: the lowest bound bits, then the lowest leaf
    // among the lanes that hold it (bounds are >= 0, so their bits order as the values)
    const unsigned lbits = __reduce_min_sync(kFull, keep ? __float_as_uint(lb2) : ~0u);
    const unsigned lmin = __reduce_min_sync(kFull, keep && __float_as_uint(lb2) == lbits ? (uint32_t)l : ~0u);
    if (lane == 0) atomicMin(&bmin_s[q], ((unsigned long long)lbits << 32) | lmin);
    if (keep) {
      const uint32_t slot = base + __popc(m & lt);
      qv.leaf_list[slot] = (uint32_t)l;
      qv.leaf_lb2[slot] = lb2;
      const uint32_t t0 = b / kItem;
      for (uint32_t j = 0; j < nit; ++j) {
        if (ibase + j < qv.items_cap)
          qv.items[ibase + j] = make_uint4(max(b, (t0 + j) * kItem), min(e, (t0 + j + 1) * kItem), __float_as_uint(lb2),
                                           (uint32_t)l);
        else
          qv.st->overflow = 1u;
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < count; q += blockDim.x) a.qvs[q].blockmin[blockIdx.x] = bmin_s[q];
}

__global__ void __launch_bounds__(kThreads) qb_front_pick(IndexView ix, BatchArgs a, uint32_t nblockmin) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_front_pick_body(ix, qv, nblockmin);
}
__global__ void __launch_bounds__(kThreads) qb_front(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_front_picked_body(ix, qv);
}
__global__ void __launch_bounds__(kBlkThreads) qb_filter_blocks(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_filter_blocks_body(ix, qv);
}
// (the minimum-blocks hints keep the one-query kernels' occupancy: the query view's
// pointers come from memory here instead of the parameter bank)
__global__ void __launch_bounds__(kFiltWarps * 32, 4) qb_filter_series(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_filter_series_body(ix, qv);
}
template <bool KONE>
__global__ void __launch_bounds__(kRowWarps * 32, 3) qb_refine_rows(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_refine_rows_body<KONE>(ix, qv);
}
__global__ void __launch_bounds__(1024) qb_finalize(IndexView ix, BatchArgs a) {
  pdl_begin();
  const QueryView& qv = batch_view(a);
  q_finalize_body(ix, qv, nullptr, nullptr, nullptr);
}

// ------------------------------------------------------------------ DTW
// Section IV, "MESSI with DTW": the index is unchanged; the bounds measure gaps to
// the query's LB_Keogh envelope (q_prep), and real distances are DTW distances with a
// Sakoe-Chiba band of half-width r: D(i, j) = (q_i - y_j)^2 + min(D(i-1, j-1),
// D(i-1, j), D(i, j-1)) for |i - j| <= r, D(-1, -1) = 0, +inf elsewhere; the
// distance is D(n-1, n-1). The kernels below mirror q_seed, q_front and the row
// refinement with a warp per candidate: the candidate's z values are staged in the
// warp's slice of shared memory, screened by LB_Keogh, then run through the band.
constexpr int kDtwWarps = 4;

// Shared memory of the DTW kernels for series of `len` points: the query, its
// envelope (upper, lower) and per warp a candidate row and a boundary row, in fp32;
// the FP64 re-check holds the query and per warp a row (fp32) and a boundary (FP64).
__host__ __device__ inline size_t dtw_smem(int len) { return sizeof(float) * (size_t)((len + 3) & ~3) * (3 + 2 * kDtwWarps); }
__host__ __device__ inline size_t dtw_check_smem(int len) {
  return sizeof(float) * (size_t)((len + 3) & ~3) * (1 + 3 * kDtwWarps);
}

template <typename V>
__device__ __forceinline__ V dtw_cell(float x, float y, V m);
template <>
__device__ __forceinline__ float dtw_cell<float>(float x, float y, float m) {
  const float d = __fsub_rn(x, y);
  return __fmaf_rn(d, d, m);
}
// FP64: d = x - y, d * d, + m, one rounding each and no fused operation: the same
// bits as a sequential evaluation of the recurrence (a minimum is exact, so the order
// in which cells are visited does not change a cell's value).
template <>
__device__ __forceinline__ double dtw_cell<double>(float x, float y, double m) {
  const double d = __dsub_rn((double)x, (double)y);
  return __dadd_rn(__dmul_rn(d, d), m);
}

// Banded DTW^2 of the query (qs) and a staged candidate (ys), one warp, as a systolic
// wavefront over stripes of 32 query points: lane l owns row i = i0 + l and at step t
// computes the cell (i, jbeg + t - l). The cell above, D(i-1, j), is the value lane
// l - 1 computed one step earlier (a shuffle); the diagonal one, D(i-1, j-1), is the
// value received from lane l - 1 the step before; the left one is the lane's own
// previous value. Lane 0 takes both from `edge`, the last row of the previous stripe,
// which lane 31 writes as it goes (each entry after lane 0 has read it). A stripe
// whose last row has no cell at or below `abandon` ends the computation with +inf:
// every warping path crosses that row and the cells after it add non-negative terms.
// With `cb` (one entry per stripe), a stripe also ends it when its last row's minimum
// plus cb[stripe] exceeds `abandon_cb`: cb holds the LB_Keogh terms of the columns a
// path can only reach in later rows, each of which it visits at least once at a cost
// of at least its term (the cumulative bound of Rakthanmanon et al., KDD 2012).
template <typename V>
__device__ V warp_dtw(const float* qs, const float* ys, V* edge, int n, int r, V abandon,
                      const float* cb = nullptr, float abandon_cb = INFINITY) {
  const int lane = threadIdx.x & 31;
  const V inf = (V)INFINITY;
  for (int j = lane; j < n; j += 32) edge[j] = inf;
  __syncwarp();
  V result = inf;
  for (int i0 = 0; i0 < n; i0 += 32) {
    const int i = i0 + lane;
    const int last = min(n - 1, i0 + 31);
    const int jbeg = max(0, i0 - r), jend = min(n - 1, last + r);
    const int steps = jend - jbeg + 1 + (last - i0);
    const bool row = i < n;
    const float x = row ? qs[i] : 0.0f;
    const int jlo = max(0, i - r), jhi = min(n - 1, i + r);
    const bool writer = lane == 31 && i0 + 32 < n;
    V prev = inf, rowmin = inf;
    // the diagonal predecessor is the value the lane took as "up" one step earlier;
    // lane 0 starts from the edge entry left of jbeg (the origin in the first stripe)
    V upd = lane == 0 ? (jbeg >= 1 ? edge[jbeg - 1] : (i0 == 0 ? (V)0 : inf)) : inf;
    const int jl = row ? jlo : 0x3fffffff;  // an empty band for rows past the end
    const unsigned span = (unsigned)(jhi - jlo);
    const int j0 = jbeg - lane;
    for (int t = 0; t < steps; ++t) {
      const int j = j0 + t;
      const V sh = __shfl_up_sync(kFull, prev, 1);
      const V up = lane == 0 ? (j < n ? edge[j] : inf) : sh;  // j >= 0 for lane 0
      V cur = inf;
      if ((unsigned)(j - jl) <= span) {
        V m = upd < up ? upd : up;
        m = prev < m ? prev : m;
        cur = dtw_cell<V>(x, ys[j], m);
        rowmin = cur < rowmin ? cur : rowmin;
        if (j == n - 1) result = cur;  // kept from the last stripe's row n - 1
      }
      if (writer && (unsigned)j < (unsigned)n) edge[j] = cur;
      prev = cur;
      upd = up;
    }
    __syncwarp();
    if (i0 + 32 < n) {
      const V m31 = __shfl_sync(kFull, rowmin, 31);
      if (m31 > abandon) return inf;
      if (cb && __fadd_rn((float)m31, cb[i0 >> 5]) > abandon_cb) return inf;
    }
  }
  return __shfl_sync(kFull, result, (n - 1) & 31);
}

// The z-normalised values of series `id` into the warp's slice (16-byte aligned).
__device__ __forceinline__ void stage_row(const IndexView& ix, uint32_t id, float2 ms, float* ys) {
  const int lane = threadIdx.x & 31;
  const float* row = ix.data + (size_t)id * ix.len;
  if ((ix.len & 3) == 0) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    float4* y4 = reinterpret_cast<float4*>(ys);
    for (int c = lane; c < (ix.len >> 2); c += 32) {
      float4 v = __ldg(r4 + c);
      if (!ix.data_is_z) {
        v.x = znorm_value(v.x, ms.x, ms.y);
        v.y = znorm_value(v.y, ms.x, ms.y);
        v.z = znorm_value(v.z, ms.x, ms.y);
        v.w = znorm_value(v.w, ms.x, ms.y);
      }
      y4[c] = v;
    }
  } else {
    for (int t = lane; t < ix.len; t += 32) {
      const float v = __ldg(row + t);
      ys[t] = ix.data_is_z ? v : znorm_value(v, ms.x, ms.y);
    }
  }
  __syncwarp();
}

// Real DTW distances of the approximate-search leaf's members (the initial BSF).
// k = 1: each distance abandons above the best so far, which is tightened as the
// members finish; k > 1: every member's full distance (the k-th is picked from them).
__global__ void __launch_bounds__(kDtwWarps * 32)
q_seed_dtw(IndexView ix, QueryView qv) {
  pdl_begin();
  extern __shared__ __align__(16) float sm[];
  const int n4 = (ix.len + 3) & ~3, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* qs = sm;
  float* ys = qs + 3 * n4 + warp * 2 * n4;
  float* edge = ys + n4;
  smem_fill(qs, qv.qz, ix.len);
  __syncthreads();
  QState* st = qv.st;
  volatile unsigned int* thr_v = &st->thr_bits;
  const uint32_t a = st->seed_a, b = st->seed_b;
  for (uint32_t gw = blockIdx.x * kDtwWarps + warp; gw < b - a; gw += gridDim.x * kDtwWarps) {
    const uint32_t pos = a + gw;
    stage_row(ix, ix.perm[pos], ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos], ys);
    const unsigned thr = __shfl_sync(kFull, lane == 0 ? *thr_v : 0u, 0);
    const float ab = qv.k == 1 ? keep_bound2(thr, qv.eps) : INFINITY;
    const float d2 = warp_dtw<float>(qs, ys, edge, ix.len, qv.window, ab);
    if (lane == 0) {
      if (gw < qv.cand_cap) qv.cand[gw] = pack(d2, pos);
      else st->overflow = 1u;
      if (qv.k == 1 && __float_as_uint(d2) < thr) atomicMin(&st->thr_bits, __float_as_uint(d2));
    }
    __syncwarp();
  }
}

// The lowest-bound surviving leaf under DTW (as q_front): refined before the filters,
// its positions excluded from them.
__global__ void __launch_bounds__(kDtwWarps * 32)
q_front_dtw(IndexView ix, QueryView qv, uint32_t nblockmin) {
  pdl_begin();
  extern __shared__ __align__(16) float sm[];
  const int n4 = (ix.len + 3) & ~3, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* qs = sm;
  float* ys = qs + 3 * n4 + warp * 2 * n4;
  float* edge = ys + n4;
  smem_fill(qs, qv.qz, ix.len);
  __shared__ uint32_t s_leaf[kMaxFront], s_beg[kMaxFront], s_pre[kMaxFront + 1];
  __shared__ float fup_s[kMaxFine], flo_s[kMaxFine];
  for (int j = threadIdx.x; j < ix.wf; j += blockDim.x) {
    fup_s[j] = qv.st->fup[j];
    flo_s[j] = qv.st->flo[j];
  }
  const int nf = front_leaves(ix, qv, nblockmin, front_count(qv.k), s_leaf, s_beg, s_pre);
  QState* st = qv.st;
  if (nf == 0) return;  // the same in every thread of the block
  volatile unsigned int* thr_v = &st->thr_bits;
  if (blockIdx.x == 0) {
    if (threadIdx.x < nf) st->front_leaf[threadIdx.x] = s_leaf[threadIdx.x];
    if (threadIdx.x == 0) st->nfront = (uint32_t)nf;
  }
  const uint32_t total = s_pre[nf];
  const uint32_t sa = st->seed_a, sb = st->seed_b;
  __shared__ unsigned s_n, s_nf;
  if (threadIdx.x == 0) s_n = s_nf = 0;
  __syncthreads();
  uint32_t n_front = 0, n_fine = 0;
  for (uint32_t g = blockIdx.x * kDtwWarps + warp; g < total; g += gridDim.x * kDtwWarps) {
    int f = 0;
    while (g >= s_pre[f + 1]) ++f;
    const uint32_t pos = s_beg[f] + (g - s_pre[f]);
    if (pos >= sa && pos < sb) continue;  // already refined by the seed
    if (ix.wf) {  // the fine PAA's bound against the envelope, before the row is read
      const unsigned thr0 = __shfl_sync(kFull, lane == 0 ? *thr_v : 0u, 0);
      ++n_fine;
      if (warp_fine_lb2(ix, fup_s, flo_s, ix.perm[pos]) > lb_bound2(thr0, qv.eps, qv.tau)) continue;
    }
    stage_row(ix, ix.perm[pos], ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos], ys);
    const unsigned thr = __shfl_sync(kFull, lane == 0 ? *thr_v : 0u, 0);
    const float keep2 = keep_bound2(thr, qv.eps);
    const float d2 = warp_dtw<float>(qs, ys, edge, ix.len, qv.window, keep2);
    if (lane == 0) {
      ++n_front;
      if (d2 <= keep2) {
        const uint32_t slot = atomicAdd(&st->cand_count, 1u);
        if (slot < qv.cand_cap) qv.cand[slot] = pack(d2, pos);
        else st->overflow = 1u;
        if (qv.k == 1 && __float_as_uint(d2) < thr) atomicMin(&st->thr_bits, __float_as_uint(d2));
      }
    }
    __syncwarp();
  }
  if (lane == 0 && n_front) atomicAdd(&s_n, n_front);
  if (lane == 0 && n_fine) atomicAdd(&s_nf, n_fine);
  __syncthreads();
  if (threadIdx.x == 0 && s_n) atomicAdd(&st->series_refined, s_n);
  if (threadIdx.x == 0 && s_nf) atomicAdd(&st->fine_front, s_nf);
}

// One warp per survivor of the series filter: re-test its bound against the current
// BSF, stage its row, screen it by LB_Keogh against the envelope and by LB_Keogh with
// the roles exchanged, then its DTW distance (abandoned above the keep bound, with
// the cumulative bounds). The BSF: an atomicMin for k = 1; for k > 1 the shared
// candidate histogram, and for k <= 32 the warp's own k best in registers.
template <bool KONE>
__global__ void __launch_bounds__(kDtwWarps * 32)
q_refine_dtw(IndexView ix, QueryView qv) {
  pdl_begin();
  extern __shared__ __align__(16) float sm[];
  const int n = ix.len, n4 = (n + 3) & ~3, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* qs = sm;
  float* qU = qs + n4;
  float* qL = qU + n4;
  float* ys = qL + n4 + warp * 2 * n4;
  float* edge = ys + n4;
  smem_fill(qs, qv.qz, n);
  smem_fill(qU, qv.qenv, n);
  smem_fill(qL, qv.qenv + n, n);
  __syncthreads();
  QState* st = qv.st;
  volatile unsigned int* thr_v = &st->thr_bits;
  const uint32_t nsurv = st->overflow ? 0u : min(st->surv_count, qv.surv_cap);
  const int k = qv.k;
  unsigned mine = 0x7f800000u;  // lanes < k: this warp's k best, ascending (1 < k <= 32)
  uint32_t n_ref = 0;
  const uint32_t gw = blockIdx.x * kDtwWarps + warp;
  const float kbase = KONE ? 0.0f : st->kbase;
  uint32_t hist_round = 0;
  const int r = qv.window, nstripes = (n + 31) >> 5;
  __shared__ float cb_s[kDtwWarps][MSI_MAX_LEN / 32], ec_s[kDtwWarps][MSI_MAX_LEN / 32];
  float* cb = cb_s[warp];
  float* ecs = ec_s[warp];
  int W = 1;  // envelope table span: the largest power of two <= r + 1
  while (2 * W <= r + 1) W <<= 1;
  for (uint32_t sidx = gw; sidx < nsurv; sidx += gridDim.x * kDtwWarps) {
    const uint2 sv = qv.surv[sidx];
    const unsigned thr = __shfl_sync(kFull, lane == 0 ? *thr_v : 0u, 0);
    if (__uint_as_float(sv.y) > lb_bound2(thr, qv.eps, qv.tau)) continue;
    stage_row(ix, ix.perm[sv.x], ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[sv.x], ys);
    const float keep2 = keep_bound2(thr, qv.eps);
    // LB_Keogh^2 in fp32 (relative error below eps); screened with a factor (1 + eps).
    // The terms go to `edge` (free until the DTW starts) for the cumulative bound.
    const float keep_lb = __fmul_ru(keep2, 1.0f + qv.eps);
    float acc = 0.0f;
    for (int t = lane; t < n; t += 32) {
      const float y = ys[t], u = qU[t], l = qL[t];
      const float d = y > u ? __fsub_rn(y, u) : (y < l ? __fsub_rn(l, y) : 0.0f);
      const float term = __fmul_rn(d, d);
      edge[t] = term;
      acc = __fadd_rn(acc, term);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if (acc > keep_lb) {
      __syncwarp();
      continue;
    }
    // suffix sums of the terms, 32 at a time from the end; then per stripe the sum
    // over the columns beyond its band (j >= 32 (stripe + 1) + r)
    __syncwarp();
    float run = 0.0f;
    for (int c0 = (n - 1) & ~31; c0 >= 0; c0 -= 32) {
      float v = c0 + lane < n ? edge[c0 + lane] : 0.0f;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32) v = __fadd_rn(v, y);
      }
      v = __fadd_rn(v, run);
      if (c0 + lane < n) edge[c0 + lane] = v;
      run = __shfl_sync(kFull, v, 0);
    }
    __syncwarp();
    for (int st_i = lane; st_i < nstripes; st_i += 32) {
      const int j = 32 * (st_i + 1) + r;
      cb[st_i] = j < n ? edge[j] : 0.0f;
      ecs[st_i] = 0.0f;
    }
    __syncwarp();
    // LB_Keogh with the roles exchanged (the candidate's envelope against the query):
    // every row i is visited at least once, at a cost of at least the gap between q_i
    // and the candidate's max / min over |t - i| <= r. The window extremes come from a
    // doubling table (span W) in `edge`, built once for the maxima and once for the
    // minima; the terms are summed per stripe of 32 rows.
    for (int pass = 0; pass < 2; ++pass) {
      for (int t = lane; t < n; t += 32) edge[t] = ys[t];
      __syncwarp();
      for (int h = 1; h < W; h <<= 1) {  // edge[t] = extreme over [t, min(n, t + 2h))
        for (int c0 = 0; c0 < n; c0 += 32) {
          const int t = c0 + lane;
          float v = 0.0f;
          if (t < n) {
            v = edge[t];
            if (t + h < n) v = pass == 0 ? fmaxf(v, edge[t + h]) : fminf(v, edge[t + h]);
          }
          __syncwarp();
          if (t < n) edge[t] = v;
          __syncwarp();
        }
      }
      for (int c0 = 0; c0 < n; c0 += 32) {
        const int t = c0 + lane;
        float term = 0.0f;
        if (t < n) {
          const int a = max(0, t - r), b = min(n - 1, t + r);
          float e = edge[a];
          for (int x = a + W; x + W <= b + 1; x += W) e = pass == 0 ? fmaxf(e, edge[x]) : fminf(e, edge[x]);
          e = pass == 0 ? fmaxf(e, edge[b - W + 1]) : fminf(e, edge[b - W + 1]);
          const float q = qs[t];
          const float d = pass == 0 ? (q > e ? __fsub_rn(q, e) : 0.0f) : (q < e ? __fsub_rn(e, q) : 0.0f);
          term = __fmul_rn(d, d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(kFull, term, o);
        if (lane == 0) ecs[c0 >> 5] += term;
      }
      __syncwarp();
    }
    // total and per-stripe suffix (rows after the stripe) of the exchanged bound
    float ec_total = 0.0f;
    for (int st_i = nstripes - 1; st_i >= 0; --st_i) {  // uniform: every lane keeps the sums
      const float here = ecs[st_i];
      if (lane == 0) cb[st_i] = fmaxf(cb[st_i], ec_total);
      ec_total = __fadd_rn(ec_total, here);
    }
    __syncwarp();
    if (ec_total > keep_lb) continue;
    ++n_ref;
    const float d2 = warp_dtw<float>(qs, ys, edge, n, r, keep2, cb, keep_lb);
    if (lane == 0 && d2 <= keep2) {
      const uint32_t slot = atomicAdd(&st->cand_count, 1u);
      if (slot < qv.cand_cap) qv.cand[slot] = pack(d2, sv.x);
      else st->overflow = 1u;
    }
    const unsigned v = __float_as_uint(d2);
    if (!KONE && kbase > 0.0f) {  // k > 1: the shared candidate histogram (see khist_bound)
      if (lane == 0 && d2 <= keep2 && d2 < kbase) atomicAdd(&qv.khist[khist_bucket(d2, kbase)], 1u);
      if ((++hist_round & 15) == 0) {
        const unsigned hb = khist_bound(qv.khist, kbase, k);
        if (lane == 0 && hb < thr) atomicMin(&st->thr_bits, hb);
      }
    }
    if (KONE) {
      if (lane == 0 && v < thr) atomicMin(&st->thr_bits, v);
    } else if (k <= 32 && v < __shfl_sync(kFull, mine, k - 1)) {
      const int p = __popc(__ballot_sync(kFull, lane < k && mine <= v));
      const unsigned upv = __shfl_up_sync(kFull, mine, 1);
      if (lane >= p && lane < k) mine = lane == p ? v : upv;
      const unsigned kth = __shfl_sync(kFull, mine, k - 1);
      if (lane == 0 && kth < thr) atomicMin(&st->thr_bits, kth);
    }
    __syncwarp();
  }
  if (lane == 0 && gw < kMaxRefineWarps) qv.partials[kMaxRefineWarps + gw] = n_ref;
}

// The k-th smallest candidate and the re-check bound (one block of 1024).
__global__ void __launch_bounds__(1024)
q_final_pick(QueryView qv) {
  pdl_begin();
  __shared__ uint32_t hist[256], sel[2];
  if (qv.st->overflow) return;
  final_select(qv, hist, sel);
}

// FP64 DTW of every candidate at or below the re-check bound: each warp takes 32
// candidates at a time and computes those that pass, one after another.
__global__ void __launch_bounds__(kDtwWarps * 32)
q_recheck_dtw(IndexView ix, QueryView qv) {
  pdl_begin();
  extern __shared__ __align__(16) float sm[];
  const int n4 = (ix.len + 3) & ~3, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* qs = sm;
  float* ys = qs + n4 + warp * 3 * n4;
  double* edge = reinterpret_cast<double*>(ys + n4);  // 16-byte aligned: n4 is a multiple of 4
  if (qv.st->overflow) return;
  smem_fill(qs, qv.qz, ix.len);
  __syncthreads();
  const uint32_t count = min(qv.st->cand_count, qv.cand_cap);
  const uint32_t bound = qv.st->final_bits;
  const uint32_t warps = gridDim.x * kDtwWarps;
  for (uint32_t base = (blockIdx.x * kDtwWarps + warp) * 32; base < count; base += warps * 32) {
    const uint32_t i = base + lane;
    const unsigned long long c = i < count ? qv.cand[i] : ~0ull;
    unsigned m = __ballot_sync(kFull, i < count && (uint32_t)(c >> 32) <= bound);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const uint32_t pos = (uint32_t)__shfl_sync(kFull, c, src);
      const uint32_t id = ix.perm[pos];
      stage_row(ix, id, ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[pos], ys);
      const double d = warp_dtw<double>(qs, ys, edge, ix.len, qv.window, (double)INFINITY);
      if (lane == 0) {
        const uint32_t slot = atomicAdd(&qv.st->rc_count, 1u);
        qv.rc_d[slot] = d;
        qv.rc_id[slot] = id;
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------ lower bounds
__global__ void __launch_bounds__(kThreads)
q_lb_all(IndexView ix, QueryView qv, float* __restrict__ series_lb, float* __restrict__ leaf_lb) {
  __shared__ float thr_up_s[257], thr_lo_s[257], up_s[16], lo_s[16];
  extern __shared__ float Ts[];
  for (int v = threadIdx.x; v <= ix.card; v += blockDim.x) {
    thr_up_s[v] = ix.thr_up[v];
    thr_lo_s[v] = ix.thr_lo[v];
  }
  if (threadIdx.x < ix.w) {
    up_s[threadIdx.x] = qv.st->qup[threadIdx.x];
    lo_s[threadIdx.x] = qv.st->qlo[threadIdx.x];
  }
  smem_fill(Ts, qv.T, ix.w * ix.card);
  __syncthreads();
  // a query with NaN or infinity gets NaN bounds, so that a caller that does not
  // wait for the call (and so gets no error status) cannot mistake them for bounds
  const bool bad = qv.st->flag < 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (series_lb)
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ix.n; p += stride)
      series_lb[ix.perm[p]] = bad ? NAN : __fsqrt_rn(word_lb2(ix.words[p], Ts, ix.w, ix.card, (float)ix.seglen));
  if (leaf_lb)
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < ix.L; l += stride)
      leaf_lb[l] = bad ? NAN : __fsqrt_rn(leaf_lb2(ix, l, up_s, lo_s, thr_lo_s, thr_up_s));
}

// z-normalised collection in collection order, from the index's storage.
__global__ void export_z_kernel(IndexView ix, float* __restrict__ out) {
  for (int64_t p = blockIdx.x; p < ix.n; p += gridDim.x) {
    const uint32_t id = ix.perm[p];
    const float2 ms = ix.data_is_z ? make_float2(0.f, 0.f) : ix.stats[p];
    for (int t = threadIdx.x; t < ix.len; t += blockDim.x) {
      const float x = ix.data[(size_t)id * ix.len + t];
      out[(size_t)id * ix.len + t] = ix.data_is_z ? x : znorm_value(x, ms.x, ms.y);
    }
  }
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

}  // namespace

// One query workspace with room for cand_cap candidates and surv_cap survivors
// (work items, block lists and leaf lists always have room for any query).
int64_t workspace_bytes(const msi_index* ix, uint32_t cand_cap, uint32_t surv_cap, uint32_t items_cap,
                        uint32_t blks_cap);

// Work items any query can need: each leaf touches at most (its size / kItem) + 2
// aligned tiles of kItem positions.
static int64_t full_items(const msi_index* ix) { return ix->n / kItem + 2 * ix->L + 2; }

cudaError_t alloc_workspace(const msi_index* ix, QueryView& qv, uint32_t cand_cap, uint32_t surv_cap,
                            int64_t* bytes, uint32_t items_cap, uint32_t blks_cap) {
  cudaError_t e;
  const size_t items = items_cap ? std::min<size_t>(items_cap, (size_t)full_items(ix)) : (size_t)full_items(ix);
  const size_t blks = blks_cap ? std::min<size_t>(blks_cap, (size_t)kHalvesPerItem * items) : kHalvesPerItem * items;
  if ((e = dalloc(&qv.qz, (size_t)ix->len + 4)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.T, (size_t)ix->w * ix->card)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.T5, (size_t)ix->w * kCoarse)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.st, 1)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.leaf_list, (size_t)ix->L)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.leaf_lb2, (size_t)ix->L)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.items, items)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.blks, blks)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.partials, (size_t)4 * kMaxRefineWarps)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.blockmin, (size_t)(ix->L / kThreads + 2))) != cudaSuccess) return e;
  if ((e = dalloc(&qv.cand, (size_t)cand_cap)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.rc_d, (size_t)cand_cap)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.rc_id, (size_t)cand_cap)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.surv, (size_t)surv_cap)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.qenv, 2 * (size_t)ix->len)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.khist, 256)) != cudaSuccess) return e;
  qv.window = -1;
  qv.cand_cap = cand_cap;
  qv.surv_cap = surv_cap;
  qv.items_cap = (uint32_t)items;
  qv.blks_cap = (uint32_t)blks;
  qv.ovf = nullptr;
  qv.eps = margin_eps();
  qv.tau = margin_tau(ix->len);
  *bytes += workspace_bytes(ix, cand_cap, surv_cap, items_cap, blks_cap);
  return cudaSuccess;
}

// Device bytes of one query workspace (alloc_workspace).
int64_t workspace_bytes(const msi_index* ix, uint32_t cand_cap, uint32_t surv_cap, uint32_t items_cap,
                        uint32_t blks_cap) {
  const int64_t items = items_cap ? std::min<int64_t>(items_cap, full_items(ix)) : full_items(ix);
  const int64_t blks = blks_cap ? std::min<int64_t>(blks_cap, kHalvesPerItem * items) : kHalvesPerItem * items;
  return (int64_t)(3 * ix->len + 4 + 256) * 4 + (int64_t)ix->w * (ix->card + kCoarse) * 4 + (int64_t)ix->L * 8 +
         items * 16 + blks * 8 + 12ll * kMaxRefineWarps + (int64_t)cand_cap * 20 + (int64_t)surv_cap * 8;
}

void free_workspace(QueryView& qv) {
  void* ptrs[] = {qv.qz, qv.T, qv.T5, qv.st, qv.leaf_list, qv.leaf_lb2, qv.items, qv.blks, qv.partials,
                  qv.blockmin, qv.cand, qv.rc_d, qv.rc_id, qv.surv, qv.qenv, qv.khist, qv.surv2};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  qv = QueryView{};
}

// Allocates slot 0 of the query workspace (room for any query) once.
cudaError_t query_setup(msi_index* ix) {
  if (ix->ws_ready) return cudaSuccess;
  QueryView& qv = ix->qv;
  cudaError_t e;
  const uint32_t nn = (uint32_t)ix->n;
  if ((e = alloc_workspace(ix, qv, nn, nn, &ix->device_bytes)) != cudaSuccess) return e;
  if ((e = dalloc(&qv.counters, (size_t)ST_COUNT)) != cudaSuccess) return e;
  if ((e = cudaMemset(qv.counters, 0, sizeof(unsigned long long) * ST_COUNT)) != cudaSuccess) return e;
  if ((e = dalloc(&ix->ws_qraw, (size_t)kQueryChunk * ix->len)) != cudaSuccess) return e;
  if ((e = dalloc(&ix->ws_ids, (size_t)kQueryChunk * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = dalloc(&ix->ws_dists, (size_t)kQueryChunk * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = dalloc(&ix->ws_d64, (size_t)kQueryChunk * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = dalloc(&ix->ws_ovf, (size_t)kQueryChunk)) != cudaSuccess) return e;
  ix->device_bytes += (int64_t)kQueryChunk * (ix->len * 4 + MSI_MAX_K * 20 + 4);
  // DTW kernels: room for the longest series (the attribute is a ceiling only)
  const int dtw_max = (int)dtw_smem(MSI_MAX_LEN), chk_max = (int)dtw_check_smem(MSI_MAX_LEN);
  if ((e = cudaFuncSetAttribute(q_seed_dtw, cudaFuncAttributeMaxDynamicSharedMemorySize, dtw_max)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(q_front_dtw, cudaFuncAttributeMaxDynamicSharedMemorySize, dtw_max)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(q_refine_dtw<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dtw_max)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(q_refine_dtw<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dtw_max)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(q_recheck_dtw, cudaFuncAttributeMaxDynamicSharedMemorySize, chk_max)) != cudaSuccess)
    return e;
  ix->ws_ready = true;
  return cudaSuccess;
}

// Candidate and survivor room of a bounded slot: the seed needs max(leaf capacity, k)
// candidate entries; `requested` (0: the defaults) sets both lists otherwise. The
// default survivor list grows with the collection (a quarter of it): collections
// that prune badly leave millions of survivors per query (60M series of the mixed
// shapes: 0.6M on average at k = 1, and over 4M for 3.5 % of the queries, which
// then reran one by one after their batch).
void slot_capacities(const msi_index* ix, int64_t requested, uint32_t* cand_cap, uint32_t* surv_cap) {
  const int64_t seed_room = std::min<int64_t>(ix->n, (int64_t)ix->cap + MSI_MAX_K);
  *cand_cap = (uint32_t)std::min<int64_t>(
      ix->n, std::max<int64_t>(seed_room, requested ? requested : std::max<int64_t>(1 << 18, seed_room)));
  *surv_cap = (uint32_t)std::min<int64_t>(ix->n, requested ? requested : std::max<int64_t>(1 << 22, ix->n / 4));
}

// Allocates the concurrent query slots (bounded lists), their streams and events.
cudaError_t slots_setup(msi_index* ix) {
  if ((int)ix->slots.size() == ix->nslots) return cudaSuccess;
  cudaError_t e;
  if (!ix->fork_event && (e = cudaEventCreateWithFlags(&ix->fork_event, cudaEventDisableTiming)) != cudaSuccess) return e;
  // the seed needs max(leaf capacity, k) candidate entries
  uint32_t cand_cap, surv_cap;
  slot_capacities(ix, ix->slot_cap, &cand_cap, &surv_cap);
  while ((int)ix->slots.size() < ix->nslots) {
    QueryView qv{};
    if ((e = alloc_workspace(ix, qv, cand_cap, surv_cap, &ix->device_bytes)) != cudaSuccess) {
      free_workspace(qv);
      return e;
    }
    qv.counters = ix->qv.counters;
    cudaStream_t st;
    cudaEvent_t ev;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
      free_workspace(qv);
      return e;
    }
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
      cudaStreamDestroy(st);
      free_workspace(qv);
      return e;
    }
    ix->slots.push_back(qv);
    ix->slot_streams.push_back(st);
    ix->slot_events.push_back(ev);
  }
  return cudaSuccess;
}

// Persistent grid sizes of the filter and refinement kernels (occupancy x SMs),
// computed once per index; query_one divides them among the concurrent queries.
static cudaError_t refine_config(msi_index* ix) {
  if (!ix->grids_ready) {
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device);
    if (e != cudaSuccess) return e;
    const size_t fsmem = sizeof(float) * (size_t)ix->w * ix->card;
    const size_t ssmem = fsmem + sizeof(float) * (size_t)ix->w * kCoarse;
    const size_t rsmem = sizeof(float) * (size_t)((ix->len + 3) & ~3);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_filter_series, kFiltWarps * 32, ssmem)) != cudaSuccess)
      return e;
    ix->grid_series = std::max(1, per_sm) * sms;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qb_filter_series, kFiltWarps * 32, ssmem)) !=
        cudaSuccess)
      return e;
    ix->grid_series_b = std::max(1, per_sm) * sms;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_filter_blocks, kBlkThreads, fsmem)) != cudaSuccess)
      return e;
    ix->grid_blocks = std::max(1, per_sm) * sms;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_refine_rows<true>, kRowWarps * 32, rsmem)) !=
        cudaSuccess)
      return e;
    ix->grid_rows1 = std::max(1, per_sm) * sms;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_refine_rows<false>, kRowWarps * 32, rsmem)) !=
        cudaSuccess)
      return e;
    ix->grid_rowsk = std::max(1, per_sm) * sms;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_refine_dtw<false>, kDtwWarps * 32,
                                                           dtw_smem(ix->len))) != cudaSuccess)
      return e;
    ix->grid_dtw = std::max(1, per_sm) * sms;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, q_recheck_dtw, kDtwWarps * 32,
                                                           dtw_check_smem(ix->len))) != cudaSuccess)
      return e;
    ix->grid_dtw_check = std::max(1, per_sm) * sms;
    ix->grids_ready = true;
  }
  return cudaSuccess;
}

// One query (device pointers), stream-ordered. ev_a / ev_m / ev_b, when given,
// bracket q_filter_series and the row refinement.
// The DTW chain: q_prep (envelope), q_seed_dtw, [q_seed_select], q_leaf_filter,
// q_front_dtw, [q_seed_select], q_filter_blocks, q_filter_series (the Euclidean
// filters run unchanged on the envelope's tables), q_refine_dtw, q_final_pick,
// q_recheck_dtw, q_finalize.
// Launches a query kernel, with programmatic stream serialization when `pdl` (see
// pdl_begin). Used for a query that has the GPU to itself: there it hides each
// kernel's launch latency (one query: 8.1K -> 9.4K queries/s, p50 0.115 -> 0.099 ms
// at 100M x 256). Queries that run concurrently on the query slots launch normally:
// dependents waiting early hold SM resources the other slots' kernels need (8 slots:
// 24.5K -> 21.3K queries/s with it).
template <typename... Params, typename... Args>
static cudaError_t pdl_launch(bool pdl, void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
// A pdl_launch that returns its error from the enclosing function (whose status
// variable is `e`, and whose `pdl` says whether the query runs alone).
#define MSI_LAUNCH(kernel, grid, block, smem, stream, ...)                                          \
  do {                                                                                              \
    if ((e = pdl_launch(pdl, kernel, dim3(grid), dim3(block), smem, stream, __VA_ARGS__)) != cudaSuccess) \
      return e;                                                                                     \
  } while (0)

static cudaError_t query_one_dtw(msi_index* ix, QueryView qv, int share, const float* q_dev, int k, int64_t* ids_dev,
                                 float* dists_dev, double* d64_dev, cudaStream_t s, cudaEvent_t ev_a,
                                 cudaEvent_t ev_m, cudaEvent_t ev_b, int window) {
  cudaError_t e = refine_config(ix);
  if (e != cudaSuccess) return e;
  const bool pdl = share == 1;
  qv.window = std::min(window, ix->len - 1);
  // fp32 DTW sums up to 2 len - 1 cells along a path: relative error below
  // (2 len + 2) 2^-24; the margin covers twice that (both the BSF and the candidate)
  qv.eps = std::max(1.52587890625e-05f, (float)(4 * ix->len + 16) * 5.9604644775390625e-08f);
  const int series_grid = std::max(1, ix->grid_series / share);
  const int blocks_grid = std::max(1, ix->grid_blocks / share);
  const int dtw_grid = std::max(1, ix->grid_dtw / share);
  const int chk_grid = std::max(1, std::min(ix->grid_dtw_check / share, (int)((qv.cand_cap + 127) / 128)));
  qv.npartials = (uint32_t)std::min<int64_t>((int64_t)series_grid * kFiltWarps, kMaxRefineWarps);
  qv.npartials_rows = (uint32_t)std::min<int64_t>((int64_t)dtw_grid * kDtwWarps, kMaxRefineWarps);
  const IndexView v = ix->view();
  const size_t qbytes = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  const size_t dsm = dtw_smem(ix->len), csm = dtw_check_smem(ix->len);
  const size_t fsmem = sizeof(float) * (size_t)ix->w * ix->card;
  MSI_LAUNCH(q_prep, 1, kThreads, qbytes, s, v, q_dev, qv, k);
  const int64_t seed_max = std::max<int64_t>(ix->cap, k);
  MSI_LAUNCH(q_seed_dtw, (unsigned)std::min<int64_t>((seed_max + kDtwWarps - 1) / kDtwWarps, 1024), kDtwWarps * 32, dsm, s, v, qv);
  if (k > 1) MSI_LAUNCH(q_seed_select, 1, 1024, 0, s, qv, 0);
  const uint32_t nlf = (uint32_t)((ix->L + kThreads - 1) / kThreads);
  MSI_LAUNCH(q_leaf_filter, nlf, kThreads, 0, s, v, qv);
  MSI_LAUNCH(q_front_dtw, (unsigned)std::min<int64_t>((ix->cap + kDtwWarps - 1) / kDtwWarps, 512), kDtwWarps * 32, dsm, s, v, qv, nlf);
  if (k > 1) MSI_LAUNCH(q_seed_select, 1, 1024, 0, s, qv, 1);
  MSI_LAUNCH(q_filter_blocks, blocks_grid, kBlkThreads, fsmem, s, v, qv);
  if (ev_a) cudaEventRecord(ev_a, s);
  MSI_LAUNCH(q_filter_series, series_grid, kFiltWarps * 32, fsmem + sizeof(float) * (size_t)ix->w * kCoarse, s, v, qv);
  if (ev_m) cudaEventRecord(ev_m, s);
  if (k == 1) MSI_LAUNCH(q_refine_dtw<true>, dtw_grid, kDtwWarps * 32, dsm, s, v, qv);
  else MSI_LAUNCH(q_refine_dtw<false>, dtw_grid, kDtwWarps * 32, dsm, s, v, qv);
  if (ev_b) cudaEventRecord(ev_b, s);
  MSI_LAUNCH(q_final_pick, 1, 1024, 0, s, qv);
  MSI_LAUNCH(q_recheck_dtw, chk_grid, kDtwWarps * 32, csm, s, v, qv);
  MSI_LAUNCH(q_finalize, 1, 1024, 0, s, v, qv, ids_dev, dists_dev, d64_dev);
  ix->kernel_launches += 10 + (k > 1 ? 2 : 0);
  return cudaGetLastError();
}

cudaError_t grids_setup(msi_index* ix) { return refine_config(ix); }

cudaError_t query_one(msi_index* ix, const QueryView& ws, int share, const float* q_dev, int k, int64_t* ids_dev,
                      float* dists_dev, double* d64_dev, uint32_t* ovf, cudaStream_t s, cudaEvent_t ev_a,
                      cudaEvent_t ev_m, cudaEvent_t ev_b, int window, const CallDesc* call, int qi) {
  share = std::max(1, share);
  if (window >= 0) {
    QueryView qv = ws;
    qv.k = k;
    qv.ovf = ovf;
    return query_one_dtw(ix, qv, share, q_dev, k, ids_dev, dists_dev, d64_dev, s, ev_a, ev_m, ev_b, window);
  }
  cudaError_t e = refine_config(ix);
  if (e != cudaSuccess) return e;
  const bool pdl = share == 1;
  QueryView qv = ws;
  qv.k = k;
  qv.ovf = ovf;
  qv.window = -1;
  qv.call = call;
  qv.qi = qi;
  const int series_grid = std::max(1, ix->grid_series / share);
  const int rows_grid = std::max(1, (k == 1 ? ix->grid_rows1 : ix->grid_rowsk) / share);
  const int blocks_grid = std::max(1, ix->grid_blocks / share);
  const size_t fsmem = sizeof(float) * (size_t)ix->w * ix->card;
  qv.npartials = (uint32_t)std::min<int64_t>((int64_t)series_grid * kFiltWarps, kMaxRefineWarps);
  qv.npartials_rows = (uint32_t)std::min<int64_t>((int64_t)rows_grid * kRowWarps, kMaxRefineWarps);
  const IndexView v = ix->view();
  const size_t qbytes = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  MSI_LAUNCH(q_prep, 1, kThreads, qbytes, s, v, q_dev, qv, k);
  const int64_t seed_max = std::max<int64_t>(ix->cap, k);
  // a warp per seed row; k = 1 with the fine PAA: a warp per kSeedGroup rows
  const int64_t seed_per_block = (k == 1 && ix->wf) ? 8 * kSeedGroup : 8;
  MSI_LAUNCH(q_seed, (unsigned)std::min<int64_t>((seed_max + seed_per_block - 1) / seed_per_block, 1024), kThreads,
             qbytes, s, v, qv);
  if (k > 1) MSI_LAUNCH(q_seed_select, 1, 1024, 0, s, qv, 0);
  const uint32_t nlf = (uint32_t)((ix->L + kThreads - 1) / kThreads);
  MSI_LAUNCH(q_leaf_filter, nlf, kThreads, 0, s, v, qv);
  MSI_LAUNCH(q_front, (unsigned)std::min<int64_t>((ix->cap + 7) / 8, 256), kThreads, qbytes, s, v, qv, nlf);
  if (k > 1) MSI_LAUNCH(q_seed_select, 1, 1024, 0, s, qv, 1);  // the k-th best over seed and front
  MSI_LAUNCH(q_filter_blocks, blocks_grid, kBlkThreads, fsmem, s, v, qv);
  if (ev_a) cudaEventRecord(ev_a, s);
  MSI_LAUNCH(q_filter_series, series_grid, kFiltWarps * 32, fsmem + sizeof(float) * (size_t)ix->w * kCoarse, s, v, qv);
  if (ev_m) cudaEventRecord(ev_m, s);
  const size_t rsmem = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  if (k == 1) MSI_LAUNCH(q_refine_rows<true>, rows_grid, kRowWarps * 32, rsmem, s, v, qv);
  else MSI_LAUNCH(q_refine_rows<false>, rows_grid, kRowWarps * 32, rsmem, s, v, qv);
  if (ev_b) cudaEventRecord(ev_b, s);
  MSI_LAUNCH(q_finalize, 1, 1024, 0, s, v, qv, ids_dev, dists_dev, d64_dev);
  // q_prep, q_seed, q_leaf_filter, q_front, q_filter_blocks, q_filter_series,
  // q_refine_rows, q_finalize, and q_seed_select twice for k > 1.
  ix->kernel_launches += 8 + (k > 1 ? 2 : 0);
  return cudaGetLastError();
}

// Batch workspaces: the candidate list as a query slot's, survivor lists of n / 8
// entries (at least 2^20, at most 2^24), room for any query's work items, and block
// tasks for n / 16 positions (at least 2^21): a query that needs more overflows and is
// run again alone with room for all n. (Smaller lists made k = 100 queries overflow:
// 783 of 4096 at 100M x 256 with 2^18 items and n / 16 survivors.) A slot capacity
// given at build time bounds these lists as it bounds a slot's.
static void batch_capacities(const msi_index* ix, uint32_t* cand_cap, uint32_t* surv_cap, uint32_t* items_cap,
                             uint32_t* blks_cap) {
  uint32_t sc;
  slot_capacities(ix, ix->slot_cap, cand_cap, &sc);
  if (ix->slot_cap) {
    *surv_cap = sc;
    *items_cap = (uint32_t)std::max(256, ix->slot_cap / 4);
    *blks_cap = 0;  // 16 per item
    return;
  }
  *surv_cap = (uint32_t)std::min<int64_t>(ix->n, std::min<int64_t>(1 << 24, std::max<int64_t>(1 << 20, ix->n / 8)));
  *items_cap = 0;  // room for any query
  *blks_cap = (uint32_t)std::min<int64_t>(kHalvesPerItem * full_items(ix), std::max<int64_t>(1 << 22, ix->n / 8));
}

cudaError_t batch_setup(msi_index* ix) {
  cudaError_t e;
  if ((e = refine_config(ix)) != cudaSuccess) return e;
  if (ix->batch_dense && !ix->tc_ready && (e = tc_setup(ix)) != cudaSuccess) return e;
  const int G = std::max(1, ix->batch_group);
  if ((int)ix->bws.size() < G) {
    uint32_t cc, sc, ic, bc;
    batch_capacities(ix, &cc, &sc, &ic, &bc);
    while ((int)ix->bws.size() < G) {
      QueryView qv{};
      if ((e = alloc_workspace(ix, qv, cc, sc, &ix->device_bytes, ic, bc)) != cudaSuccess) {
        free_workspace(qv);
        return e;
      }
      qv.counters = ix->qv.counters;
      ix->bws.push_back(qv);
      ix->bws_dirty = true;
    }
  }
  // the bound-ordered copy of the survivors, only while ordering is on
  if (ix->batch_order) {
    uint32_t cc, sc, ic, bc;
    batch_capacities(ix, &cc, &sc, &ic, &bc);
    for (auto& qv : ix->bws)
      if (!qv.surv2) {
        if ((e = dalloc(&qv.surv2, (size_t)sc)) != cudaSuccess) return e;
        ix->device_bytes += (int64_t)sc * 8;
        ix->bws_dirty = true;
      }
  }
  if (ix->bws_dev_cap < (int)ix->bws.size()) {
    if (ix->bws_dev) cudaFree(ix->bws_dev);
    ix->bws_dev = nullptr;
    ix->bws_dev_cap = 0;
    if ((e = cudaMalloc(&ix->bws_dev, sizeof(QueryView) * ix->bws.size())) != cudaSuccess) return e;
    ix->bws_dev_cap = (int)ix->bws.size();
    ix->bws_dirty = true;
  }
  // the device views must name the workspaces that exist now (every view is rewritten
  // whenever one was allocated or freed)
  if (ix->bws_dirty) {
    if ((e = cudaMemcpy(ix->bws_dev, ix->bws.data(), sizeof(QueryView) * ix->bws.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return e;
    ix->bws_dirty = false;
  }
  return cudaSuccess;
}

// Frees the batch workspaces beyond the first `keep` (no batch may be in flight).
void batch_release(msi_index* ix, int keep) {
  uint32_t cc, sc, ic, bc;
  batch_capacities(ix, &cc, &sc, &ic, &bc);
  while ((int)ix->bws.size() > keep) {
    ix->device_bytes -= workspace_bytes(ix, cc, sc, ic, bc) + (ix->bws.back().surv2 ? (int64_t)sc * 8 : 0);
    free_workspace(ix->bws.back());
    ix->bws.pop_back();
    ix->bws_dirty = true;
  }
}

cudaError_t query_batch(msi_index* ix, int count, int k, const CallDesc* call, int qbase, uint32_t* ovf,
                        cudaStream_t s, cudaEvent_t ev_a, cudaEvent_t ev_m, cudaEvent_t ev_b) {
  cudaError_t e;
  if (count < 1 || count > (int)ix->bws.size() || count > 65535) return cudaErrorInvalidValue;
  if (ix->bws_dirty) return cudaErrorNotReady;  // batch_setup has not written the views
  if ((e = refine_config(ix)) != cudaSuccess) return e;  // grid sizes, once per index
  if (ix->batch_order && !ix->batch_dense)  // batch_setup allocates the ordered copies
    for (int i = 0; i < count; ++i)
      if (!ix->bws[i].surv2) return cudaErrorNotReady;
  const bool pdl = ix->batch_pdl;
  const int share = std::max(1, ix->batch_share);
  const int series_grid = std::max(1, ix->grid_series_b / share);
  const int rows_grid = std::max(1, (k == 1 ? ix->grid_rows1 : ix->grid_rowsk) / share);
  const int blocks_grid = std::max(1, ix->grid_blocks / share);
  BatchArgs a;
  a.qvs = ix->bws_dev;
  a.order = ix->batch_order && !ix->batch_dense ? 1 : 0;
  a.call = call;
  a.ovf = ovf;
  a.qbase = qbase;
  a.k = k;
  a.np = (uint32_t)std::min<int64_t>((int64_t)series_grid * kFiltWarps, kMaxRefineWarps);
  a.npr = (uint32_t)std::min<int64_t>((int64_t)rows_grid * kRowWarps, kMaxRefineWarps);
  const IndexView v = ix->view();
  const unsigned B = (unsigned)count;
  const size_t qbytes = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  const size_t fsmem = sizeof(float) * (size_t)ix->w * ix->card;
  if (ix->batch_dense) {
    // the tensor-core filter in place of the leaf, block and series filters: the seed
    // leaf gives each query its first k-th best, one pass over the collection per
    // tc_queries_per_pass queries bounds every (series, query) pair, the row kernel
    // computes the survivors' distances
    if (!ix->tc_ready) return cudaErrorNotReady;  // batch_setup prepares it
    a.np = 0;  // no series filter: its per-warp counters are not read
    MSI_LAUNCH(qb_views, (B + 127) / 128, 128, 0, s, ix->bws_dev, a, count);
    MSI_LAUNCH(qb_prep, dim3(1, B), kThreads, qbytes, s, v, a);
    const int64_t seed_max = std::max<int64_t>(ix->cap, k);
    const int64_t seed_per_block = (k == 1 && ix->wf) ? 8 * kSeedGroup : 8;
    MSI_LAUNCH(qb_seed, dim3((unsigned)std::min<int64_t>((seed_max + seed_per_block - 1) / seed_per_block, 1024), B),
               kThreads, qbytes, s, v, a);
    if (k > 1) MSI_LAUNCH(qb_seed_select, dim3(1, B), 1024, 0, s, a, 1);
    const int per = tc_queries_per_pass(ix->len);
    int passes = 0;
    if (ev_a) cudaEventRecord(ev_a, s);
    for (int p0 = 0; p0 < count; p0 += per, ++passes)
      if ((e = tc_filter(ix, ix->bws_dev, p0, std::min(per, count - p0), s)) != cudaSuccess) return e;
    if (ev_m) cudaEventRecord(ev_m, s);
    const size_t rsmem = sizeof(float) * (size_t)((ix->len + 3) & ~3);
    if (k == 1) MSI_LAUNCH(qb_refine_rows<true>, dim3(rows_grid, B), kRowWarps * 32, rsmem, s, v, a);
    else MSI_LAUNCH(qb_refine_rows<false>, dim3(rows_grid, B), kRowWarps * 32, rsmem, s, v, a);
    if (ev_b) cudaEventRecord(ev_b, s);
    MSI_LAUNCH(qb_finalize, dim3(1, B), 1024, 0, s, v, a);
    ix->kernel_launches += 6 + passes + (k > 1 ? 1 : 0);
    return cudaGetLastError();
  }
  MSI_LAUNCH(qb_views, (B + 127) / 128, 128, 0, s, ix->bws_dev, a, count);
  MSI_LAUNCH(qb_prep, dim3(1, B), kThreads, qbytes, s, v, a);
  const int64_t seed_max = std::max<int64_t>(ix->cap, k);
  const int64_t seed_per_block = (k == 1 && ix->wf) ? 8 * kSeedGroup : 8;
  MSI_LAUNCH(qb_seed, dim3((unsigned)std::min<int64_t>((seed_max + seed_per_block - 1) / seed_per_block, 1024), B),
             kThreads, qbytes, s, v, a);
  if (k > 1) MSI_LAUNCH(qb_seed_select, dim3(1, B), 1024, 0, s, a, 0);
  const uint32_t nlf = (uint32_t)((ix->L + kThreads - 1) / kThreads);
  if (count <= kBatchMax) MSI_LAUNCH(qb_leaf_filter_lm, nlf, kThreads, 0, s, v, a, count);
  else MSI_LAUNCH(qb_leaf_filter, dim3(nlf, B), kThreads, 0, s, v, a);
  MSI_LAUNCH(qb_front_pick, dim3(1, B), kThreads, 0, s, v, a, nlf);
  MSI_LAUNCH(qb_front, dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>((ix->cap + 7) / 8, 256) / share), B),
             kThreads, qbytes, s, v, a);
  if (k > 1) MSI_LAUNCH(qb_seed_select, dim3(1, B), 1024, 0, s, a, 1);
  MSI_LAUNCH(qb_filter_blocks, dim3(blocks_grid, B), kBlkThreads, fsmem, s, v, a);
  if (ev_a) cudaEventRecord(ev_a, s);
  MSI_LAUNCH(qb_filter_series, dim3(series_grid, B), kFiltWarps * 32, fsmem + sizeof(float) * (size_t)ix->w * kCoarse, s,
             v, a);
  if (ix->batch_order) MSI_LAUNCH(qb_order, dim3(1, B), 1024, 0, s, a);
  if (ev_m) cudaEventRecord(ev_m, s);
  const size_t rsmem = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  if (k == 1) MSI_LAUNCH(qb_refine_rows<true>, dim3(rows_grid, B), kRowWarps * 32, rsmem, s, v, a);
  else MSI_LAUNCH(qb_refine_rows<false>, dim3(rows_grid, B), kRowWarps * 32, rsmem, s, v, a);
  if (ev_b) cudaEventRecord(ev_b, s);
  MSI_LAUNCH(qb_finalize, dim3(1, B), 1024, 0, s, v, a);
  ix->kernel_launches += 10 + (k > 1 ? 2 : 0) + (ix->batch_order ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t export_z(msi_index* ix, float* z_dev, cudaStream_t s) {
  export_z_kernel<<<4096, 128, 0, s>>>(ix->view(), z_dev);
  return cudaGetLastError();
}

// The lower-bound pipeline on caller-provided query scratch (qz, T, T5, st,
// counters inside `qv`); used by the entry point that allocates nothing.
cudaError_t lower_bounds_on(const msi_index* ix, const QueryView& qv_in, const float* q_dev, float* series_lb_dev,
                            float* leaf_lb_dev, cudaStream_t s) {
  QueryView qv = qv_in;
  qv.k = 1;
  qv.window = -1;  // Euclidean bounds
  const IndexView v = ix->view();
  const size_t qbytes = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  q_prep<<<1, kThreads, qbytes, s>>>(v, q_dev, qv, 1);
  q_lb_all<<<1024, kThreads, sizeof(float) * (size_t)ix->w * ix->card, s>>>(v, qv, series_lb_dev, leaf_lb_dev);
  return cudaGetLastError();
}

cudaError_t lower_bounds(msi_index* ix, const float* q_dev, float* series_lb_dev, float* leaf_lb_dev,
                         cudaStream_t s) {
  QueryView qv = ix->qv;
  qv.k = 1;
  const IndexView v = ix->view();
  const size_t qbytes = sizeof(float) * (size_t)((ix->len + 3) & ~3);
  q_prep<<<1, kThreads, qbytes, s>>>(v, q_dev, qv, 1);
  q_lb_all<<<1024, kThreads, sizeof(float) * (size_t)ix->w * ix->card, s>>>(v, qv, series_lb_dev, leaf_lb_dev);
  return cudaGetLastError();
}

}  // namespace msi
