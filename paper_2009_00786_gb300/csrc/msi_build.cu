// msi_build.cu -- index construction on the GPU (Section III-A, Algorithms 1-4).
//
// The paper's CPU pipeline (index workers computing iSAX summaries into per-root-
// subtree buffers, then building subtrees with node splits) becomes four data-
// parallel phases:
//   1. summarise: one warp per series computes the canonical z-normalisation, the
//      PAA, the SAX word and an interleaved 64-bit key (ConvertToiSAX, Algorithm 3);
//   2. sort: stable LSD radix sort of (key, id), which groups series exactly as the
//      iSAX tree does (the first `segments` key bits are the root subtree);
//   3. split: a capacity-bounded binary split of key ranges, one bit per level, the
//      flat equivalent of SplitNode (Algorithm 4), leaves as contiguous ranges;
//   4. envelopes: per-leaf minimum / maximum symbol of every segment.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "msi_internal.cuh"

namespace msi {
namespace {

#define MSI_TRY(x)                      \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

// ------------------------------------------------------------------ summarise
constexpr int kSumWarps = 8;

// A series' SAX word and moments side by side: one 32-byte sector, so that the
// gathers into leaf order fetch one sector per series instead of two.
struct __align__(32) SumRec {
  uint4 word;
  float2 stats;  // (mu, 1/sigma)
  float2 pad;
};

struct SumOut {
  SumRec* rec;                  // [n] collection order: word and moments
  unsigned long long* keys;     // [n]
  uint32_t* ids;                // [n] iota
  float* z_out;                 // [n][len] or nullptr (borrowed data)
  unsigned long long* first_bad;  // min id of a non-finite series
  uint4* fine;                  // [n][wf / 8] collection order: fine PAA (fp16), or nullptr
  int wf, sf;                   // its segments and their length
};

// Writes the warp's fine PAA (fp16, staged in shared memory) as wf / 8 uint4 values.
__device__ __forceinline__ void emit_fine(const __half* fs, int64_t i, const SumOut& o) {
  const int lane = threadIdx.x & 31, chunks = o.wf / 8;
  __syncwarp();
  if (lane < chunks) o.fine[i * chunks + lane] = reinterpret_cast<const uint4*>(fs)[lane];
}

// Writes the word (symbols in a per-warp byte buffer) and the key.
__device__ __forceinline__ void emit_word(uint8_t* sw, int sym_lane, int w, int bits, int64_t i,
                                          const SumOut& o) {
  const int lane = threadIdx.x & 31;
  const unsigned long long key = interleave_key(sym_lane, w, bits);
  if (lane == 0) {
    const uint4 word = *reinterpret_cast<const uint4*>(sw);
    o.rec[i].word = word;
    o.keys[i] = key;
    o.ids[i] = (uint32_t)i;
  }
}

// Fast path: len = 128 * NC, segment length s = 4 * G with G a power of two <= 32
// (every segment inside one 128-point chunk). Each lane holds its points in
// registers as NC float4 values, so the series is read once with coalesced 512-byte
// warp loads; sums follow the canonical order exactly.
template <int NC>
__global__ void __launch_bounds__(kSumWarps * 32)
summarise_fast(const float* __restrict__ src, int64_t n, int w, int card, int bits, int G,
               const float* __restrict__ thr_up_g, SumOut o) {
  __shared__ float thr_s[257];
  __shared__ __align__(16) uint8_t sw_s[kSumWarps][16];
  __shared__ __align__(16) __half fs_s[kSumWarps][kMaxFine];
  __shared__ float paa_s[kSumWarps][16];
  for (int v = threadIdx.x; v <= card; v += blockDim.x) thr_s[v] = thr_up_g[v];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int len = NC * 128;
  const int s = 4 * G;
  const int segs_per_chunk = 128 / s;
  // len, s and sf are powers of two here: their exact reciprocals
  const float inv_len = 1.0f / (float)len, inv_s = 1.0f / (float)s;
  const float inv_sf = o.sf ? 1.0f / (float)o.sf : 0.0f;
  uint8_t* sw = sw_s[warp];
  __half* fs = fs_s[warp];
  const int sf = o.sf;  // fine segment length: 1, 2, or 4 Gf (Gf lanes per segment)
  for (int64_t i = (int64_t)blockIdx.x * kSumWarps + warp; i < n; i += (int64_t)gridDim.x * kSumWarps) {
    const float4* row = reinterpret_cast<const float4*>(src + i * len);
    float4 v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = __ldcs(row + c * 32 + lane);
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      acc = __fadd_rn(acc, v[c].x);
      acc = __fadd_rn(acc, v[c].y);
      acc = __fadd_rn(acc, v[c].z);
      acc = __fadd_rn(acc, v[c].w);
    }
    const float mu = div_pow2(tree32(acc), inv_len);
    float acc2 = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float d = __fsub_rn(v[c].x, mu);
      acc2 = __fmaf_rn(d, d, acc2);
      d = __fsub_rn(v[c].y, mu);
      acc2 = __fmaf_rn(d, d, acc2);
      d = __fsub_rn(v[c].z, mu);
      acc2 = __fmaf_rn(d, d, acc2);
      d = __fsub_rn(v[c].w, mu);
      acc2 = __fmaf_rn(d, d, acc2);
    }
    const Moments m = finish_moments(mu, tree32(acc2), len, inv_len);
    if (m.flag < 0 && lane == 0) atomicMin(o.first_bad, (unsigned long long)i);
    const bool cst = m.flag != 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float4 z;
      z.x = cst ? 0.0f : znorm_value(v[c].x, m.mu, m.rsig);
      z.y = cst ? 0.0f : znorm_value(v[c].y, m.mu, m.rsig);
      z.z = cst ? 0.0f : znorm_value(v[c].z, m.mu, m.rsig);
      z.w = cst ? 0.0f : znorm_value(v[c].w, m.mu, m.rsig);
      if (o.z_out) __stcs(reinterpret_cast<float4*>(o.z_out + i * len) + c * 32 + lane, z);
      if (o.fine) {  // this lane's points are 4 (32 c + lane) .. + 3
        const int t0 = 4 * (32 * c + lane);
        if (sf == 1) {
          fs[t0] = __float2half_rn(z.x);
          fs[t0 + 1] = __float2half_rn(z.y);
          fs[t0 + 2] = __float2half_rn(z.z);
          fs[t0 + 3] = __float2half_rn(z.w);
        } else if (sf == 2) {
          fs[t0 / 2] = __float2half_rn(__fmul_rn(__fadd_rn(z.x, z.y), 0.5f));
          fs[t0 / 2 + 1] = __float2half_rn(__fmul_rn(__fadd_rn(z.z, z.w), 0.5f));
        } else {
          float gf = __fadd_rn(__fadd_rn(__fadd_rn(z.x, z.y), z.z), z.w);
          for (int off = 1; off < sf / 4; off <<= 1) gf = __fadd_rn(gf, __shfl_xor_sync(kFull, gf, off));
          if ((lane & (sf / 4 - 1)) == 0) fs[t0 / sf] = __float2half_rn(div_pow2(gf, inv_sf));
        }
      }
      float g = __fadd_rn(__fadd_rn(__fadd_rn(z.x, z.y), z.z), z.w);
      for (int off = 1; off < G; off <<= 1) g = __fadd_rn(g, __shfl_xor_sync(kFull, g, off));
      if ((lane & (G - 1)) == 0) {
        const int j = c * segs_per_chunk + lane / G;
        if (j < 16) paa_s[warp][j] = div_pow2(g, inv_s);
      }
    }
    // one symbol search for all segments: lane j takes segment j
    __syncwarp();
    const int sym = lane < w ? sax_symbol(thr_s, card, paa_s[warp][lane]) : 0;
    if (lane < 16) sw[lane] = (uint8_t)sym;
    __syncwarp();
    if (lane == 0) o.rec[i].stats = make_float2(m.mu, m.rsig);
    emit_word(sw, sym, w, bits, i, o);
    if (o.fine) emit_fine(fs, i, o);
    __syncwarp();
  }
}

// ------------------------------------------------ summarise, two series per warp
// The same canonical arithmetic with each half-warp on its own series: half-lane h
// holds the points of canonical lanes h and h + 16 (parts A and B), so every point
// is summed into the partial of its canonical lane exactly as above; the 16 lane
// partials of each part are combined by the same pairwise tree (xor offsets 1..8
// stay inside a half) and the last step of the 32-lane tree adds the two parts. The
// shuffles, divisions and the key's ballots serve two series at once, and every lane
// keeps twice the loads in flight.
//
// SAX symbol by a cell table: the value axis [-4, 4) in 1024 cells of 1/128; cell_lo[c]
// is the number of thresholds at or below the left edge of cell c - 1 (one cell of room
// for the rounding of the cell index), a lower bound of the symbol of any value whose
// computed cell is c; exact comparisons with the next thresholds (at most a few) then
// give the symbol: the number of thresholds at or below the value.
constexpr int kSymCells = 1024;
__device__ __forceinline__ int sax_symbol_cells(const float* thr_up_s, const uint8_t* cell_lo, int card, float p) {
  const float x = fminf(fmaxf(floorf(__fmul_rn(__fadd_rn(p, 4.0f), 128.0f)), 0.0f), (float)(kSymCells - 1));
  int sym = cell_lo[(int)x];
  while (sym < card - 1 && thr_up_s[sym + 1] <= p) ++sym;
  return sym;
}

// The interleaved key of the half-warp's word (lanes h < w of the half hold sym_h).
__device__ __forceinline__ unsigned long long interleave_key_half(int sym, int w, int bits, int hl, int half) {
  unsigned long long key = 0;
  int used = 0;
  for (int p = bits - 1; p >= 0 && used < 64; --p) {
    const unsigned m = __ballot_sync(kFull, hl < w && ((sym >> p) & 1));
    const unsigned mh = (m >> (16 * half)) & 0xffffu;
    const unsigned rev = __brev(mh) >> (32 - w);  // segment 0 in the top bit of w
    const int take = (64 - used) < w ? (64 - used) : w;
    key = (key << take) | (unsigned long long)(rev >> (w - take));
    used += take;
  }
  return used < 64 ? key << (64 - used) : key;
}

// Pairwise tree over xor offsets 1 .. width / 2 inside a half-warp.
__device__ __forceinline__ float tree_half(float v, int width) {
  for (int off = 1; off < width && off < 16; off <<= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

// NC <= 4 (len <= 512) and G <= 16 (segments of at most 64 points).
// Pairs of rows per warp in summarise_pair's shared-memory ring: the pair being
// summarised and the next one in flight (a third stage measured no faster).
template <int NC>
constexpr int kPairStages = 2;
template <int NC>
constexpr size_t pair_ring_bytes() {
  return (size_t)kSumWarps * kPairStages<NC> * 2 * NC * 32 * sizeof(float4);
}

__host__ __device__ constexpr int ilog2c(int v) { return v > 1 ? 1 + ilog2c(v >> 1) : 0; }

// kG, kSF, kW, kBits: the segment's float4 groups, the fine PAA's points per segment,
// the segments and the symbol bits fixed at compile time (0, or -1 for kSF: read from
// the arguments), so that the trees unroll and the shape's branches fold away; the
// arithmetic and its order are the same either way.
template <int NC, int kG = 0, int kSF = -1, int kW = 0, int kBits = 0>
__global__ void __launch_bounds__(kSumWarps * 32)
summarise_pair(const float* __restrict__ src, int64_t n, int w_rt, int card, int bits_rt, int G_rt,
               const float* __restrict__ thr_up_g, const uint8_t* __restrict__ cell_lo_g, SumOut o) {
  const int G = kG ? kG : G_rt, w = kW ? kW : w_rt, bits = kBits ? kBits : bits_rt;
  // per warp a ring of kPairStages<NC> pairs of rows in shared memory, filled by
  // 16-byte asynchronous copies kPairStages - 1 pairs ahead; every lane copies and
  // later reads only its own float4s, so the ring needs no synchronisation between lanes
  constexpr int S = kPairStages<NC>;
  extern __shared__ __align__(16) float4 ring_s[];  // [kSumWarps][S][2 halves][NC * 32]
  __shared__ float thr_s[257];
  __shared__ uint8_t cell_s[kSymCells];
  __shared__ __align__(16) uint8_t sw_s[kSumWarps][2][16];
  __shared__ __align__(16) __half fs_s[kSumWarps][2][kMaxFine];
  __shared__ float paa_s[kSumWarps][2][16];
  for (int v = threadIdx.x; v <= card; v += blockDim.x) thr_s[v] = thr_up_g[v];
  for (int c = threadIdx.x; c < kSymCells; c += blockDim.x) cell_s[c] = cell_lo_g[c];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int half = lane >> 4, hl = lane & 15;
  const int len = NC * 128;
  const int s = 4 * G;
  const int segs_per_chunk = 128 / s;
  const int sf = kSF >= 0 ? kSF : o.sf;
  // len, s and sf are powers of two here: their exact reciprocals, and shifts for the
  // per-chunk index divisions by G and sf
  const float inv_len = 1.0f / (float)len, inv_s = 1.0f / (float)s;
  const float inv_sf = sf ? 1.0f / (float)sf : 0.0f;
  const int lg_g = kG ? ilog2c(kG) : __ffs(G) - 1;
  const int lg_sf = kSF >= 0 ? ilog2c(kSF > 0 ? kSF : 1) : (sf ? __ffs(sf) - 1 : 0);
  uint8_t* sw = sw_s[warp][half];
  __half* fs = fs_s[warp][half];
  float* paa = paa_s[warp][half];
  float4* ring = ring_s + (size_t)warp * S * 2 * NC * 32 + half * NC * 32;  // stage st at + st * 2 NC 32
  const int64_t first = 2 * ((int64_t)blockIdx.x * kSumWarps + warp), stride = 2 * (int64_t)gridDim.x * kSumWarps;
  // this lane's float4s of the pair starting at p0 (the half past the end re-reads p0)
  // into stage st; one commit group per pair, empty past the end
  auto issue = [&](int64_t p0, int st) {
    if (p0 < n) {
      const int64_t i = p0 + half < n ? p0 + half : p0;
      const float4* row = reinterpret_cast<const float4*>(src + i * len);
      float4* dst = ring + st * 2 * NC * 32;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        cp_async16(dst + c * 32 + hl, row + c * 32 + hl);
        cp_async16(dst + c * 32 + hl + 16, row + c * 32 + hl + 16);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int st = 0; st < S - 1; ++st) issue(first + st * stride, st);
  int stage = 0;
  for (int64_t i0 = first; i0 < n; i0 += stride) {
    issue(i0 + (S - 1) * stride, stage == 0 ? S - 1 : stage - 1);  // the slot this lane read last
    cp_async_wait<S - 1>();  // pair i0 has landed (this lane's copies)
    const int64_t i = i0 + half;
    const bool valid = i < n;
    // part A: canonical lane hl, part B: canonical lane hl + 16 (float4 index 32 c + lane)
    float4 va[NC], vb[NC];
    const float4* cur = ring + stage * 2 * NC * 32;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      va[c] = cur[c * 32 + hl];
      vb[c] = cur[c * 32 + hl + 16];
    }
    stage = stage == S - 1 ? 0 : stage + 1;
    float sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      sa = __fadd_rn(sa, va[c].x); sb = __fadd_rn(sb, vb[c].x);
      sa = __fadd_rn(sa, va[c].y); sb = __fadd_rn(sb, vb[c].y);
      sa = __fadd_rn(sa, va[c].z); sb = __fadd_rn(sb, vb[c].z);
      sa = __fadd_rn(sa, va[c].w); sb = __fadd_rn(sb, vb[c].w);
    }
    const float mu = div_pow2(__fadd_rn(tree_half(sa, 16), tree_half(sb, 16)), inv_len);
    float qa = 0.0f, qb = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float d = __fsub_rn(va[c].x, mu); qa = __fmaf_rn(d, d, qa);
      d = __fsub_rn(vb[c].x, mu); qb = __fmaf_rn(d, d, qb);
      d = __fsub_rn(va[c].y, mu); qa = __fmaf_rn(d, d, qa);
      d = __fsub_rn(vb[c].y, mu); qb = __fmaf_rn(d, d, qb);
      d = __fsub_rn(va[c].z, mu); qa = __fmaf_rn(d, d, qa);
      d = __fsub_rn(vb[c].z, mu); qb = __fmaf_rn(d, d, qb);
      d = __fsub_rn(va[c].w, mu); qa = __fmaf_rn(d, d, qa);
      d = __fsub_rn(vb[c].w, mu); qb = __fmaf_rn(d, d, qb);
    }
    const Moments m = finish_moments(mu, __fadd_rn(tree_half(qa, 16), tree_half(qb, 16)), len, inv_len);
    if (valid && m.flag < 0 && hl == 0) atomicMin(o.first_bad, (unsigned long long)i);
    const bool cst = m.flag != 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        const float4 x = part ? vb[c] : va[c];
        const int L = hl + 16 * part;  // canonical lane
        float4 z;
        z.x = cst ? 0.0f : znorm_value(x.x, m.mu, m.rsig);
        z.y = cst ? 0.0f : znorm_value(x.y, m.mu, m.rsig);
        z.z = cst ? 0.0f : znorm_value(x.z, m.mu, m.rsig);
        z.w = cst ? 0.0f : znorm_value(x.w, m.mu, m.rsig);
        if (o.z_out && valid) __stcs(reinterpret_cast<float4*>(o.z_out + i * len) + c * 32 + L, z);
        if (o.fine) {  // this canonical lane's points are 4 (32 c + L) .. + 3
          const int t0 = 4 * (32 * c + L);
          if (sf == 1) {
            fs[t0] = __float2half_rn(z.x);
            fs[t0 + 1] = __float2half_rn(z.y);
            fs[t0 + 2] = __float2half_rn(z.z);
            fs[t0 + 3] = __float2half_rn(z.w);
          } else if (sf == 2) {
            fs[t0 / 2] = __float2half_rn(__fmul_rn(__fadd_rn(z.x, z.y), 0.5f));
            fs[t0 / 2 + 1] = __float2half_rn(__fmul_rn(__fadd_rn(z.z, z.w), 0.5f));
          } else {
            float gf = __fadd_rn(__fadd_rn(__fadd_rn(z.x, z.y), z.z), z.w);
            gf = tree_half(gf, sf / 4);  // sf / 4 <= 16 consecutive canonical lanes, one part
            if ((L & (sf / 4 - 1)) == 0) fs[t0 >> lg_sf] = __float2half_rn(div_pow2(gf, inv_sf));
          }
        }
        // PAA: groups of 4 points, G consecutive canonical lanes per segment (G <= 16,
        // so a segment lies in one part), combined by the pairwise tree
        float g = __fadd_rn(__fadd_rn(__fadd_rn(z.x, z.y), z.z), z.w);
        g = tree_half(g, G);
        if ((L & (G - 1)) == 0) {
          const int j = c * segs_per_chunk + (L >> lg_g);
          if (j < 16) paa[j] = div_pow2(g, inv_s);
        }
      }
    }
    __syncwarp();
    int sym = 0;
    if (hl < w) sym = sax_symbol_cells(thr_s, cell_s, card, paa[hl]);
    if (hl < 16) sw[hl] = (uint8_t)sym;
    __syncwarp();
    const unsigned long long key = interleave_key_half(sym, w, bits, hl, half);
    if (valid && hl == 0) {
      o.rec[i].stats = make_float2(m.mu, m.rsig);
      o.rec[i].word = *reinterpret_cast<const uint4*>(sw);
      o.keys[i] = key;
      o.ids[i] = (uint32_t)i;
    }
    if (o.fine) {
      __syncwarp();
      const int chunks = o.wf / 8;
      if (valid && hl < chunks) o.fine[i * chunks + hl] = reinterpret_cast<const uint4*>(fs)[hl];
    }
    __syncwarp();
  }
  cp_async_wait<0>();  // the ring's last (empty) groups, before the block ends
}

// Generic path: any length up to MSI_MAX_LEN and any segment length. The warp
// stages the z values in shared memory and lanes j < w reduce their segment in the
// canonical order.
constexpr int kGenWarps = 4;
__global__ void __launch_bounds__(kGenWarps * 32)
summarise_generic(const float* __restrict__ src, int64_t n, int len, int w, int card, int bits,
                  const float* __restrict__ thr_up_g, SumOut o) {
  extern __shared__ float zs_all[];  // [kGenWarps][len]
  __shared__ float thr_s[257];
  __shared__ __align__(16) uint8_t sw_s[kGenWarps][16];
  __shared__ __align__(16) __half fs_s[kGenWarps][kMaxFine];
  for (int v = threadIdx.x; v <= card; v += blockDim.x) thr_s[v] = thr_up_g[v];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* zs = zs_all + warp * len;
  uint8_t* sw = sw_s[warp];
  const int s = len / w;
  for (int64_t i = (int64_t)blockIdx.x * kGenWarps + warp; i < n; i += (int64_t)gridDim.x * kGenWarps) {
    const float* x = src + i * len;
    const Moments m = warp_moments_generic(x, len);
    if (m.flag < 0 && lane == 0) atomicMin(o.first_bad, (unsigned long long)i);
    const bool cst = m.flag != 0;
    for (int t = lane; t < len; t += 32) {
      const float z = cst ? 0.0f : znorm_value(x[t], m.mu, m.rsig);
      zs[t] = z;
    }
    __syncwarp();
    if (o.z_out)
      for (int t = lane; t < len; t += 32) o.z_out[i * len + t] = zs[t];
    int sym = 0;
    if (lane < w) sym = sax_symbol(thr_s, card, paa_segment_generic(zs, lane, s));
    if (lane < 16) sw[lane] = lane < w ? (uint8_t)sym : 0;
    __syncwarp();
    if (lane == 0) o.rec[i].stats = make_float2(m.mu, m.rsig);
    emit_word(sw, sym, w, bits, i, o);
    if (o.fine) {
      for (int j = lane; j < o.wf; j += 32) {
        float g = 0.0f;
        for (int t = j * o.sf; t < (j + 1) * o.sf; ++t) g = __fadd_rn(g, zs[t]);
        fs_s[warp][j] = __float2half_rn(__fdiv_rn(g, (float)o.sf));
      }
      emit_fine(fs_s[warp], i, o);
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ radix sort
// Stable LSD radix sort of (u64 key, u32 value), 8-bit digits. Per pass: a tile
// histogram (upsweep), an exclusive scan of the digit-major histogram, and a stable
// scatter through a tile sorted in shared memory.
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;

__global__ void __launch_bounds__(kRsThreads)
rs_upsweep(const unsigned long long* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
           int64_t tiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll 4
  for (int r = 0; r < kRsRounds; ++r) {
    const int64_t idx = base + r * kRsThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// The stable scatter: each round of 256 keys is ranked inside the tile with warp
// match and per-digit warp prefixes; every key goes to its rank among the tile's keys
// of equal digit in shared memory, and the tile is then written out in that order, so
// keys of one digit leave as one contiguous run instead of one scattered store each.
// The tile's count of digit d is the difference of consecutive scanned offsets
// (digit-major). A thread loads its 16 keys and values of the tile before the first
// round, so the rounds wait on no global load.
constexpr size_t kRsSmem = (size_t)kRsTile * (sizeof(unsigned long long) + sizeof(uint32_t));
__global__ void __launch_bounds__(kRsThreads)
rs_scatter_local(const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
                 unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
                 const uint32_t* __restrict__ offs, int64_t tiles) {
  constexpr int kW = kRsThreads / 32;
  extern __shared__ __align__(16) unsigned char rs_smem[];
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(rs_smem);
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + kRsTile);
  __shared__ uint32_t run[256], lstart[256], gstart[256];
  __shared__ uint32_t wc[kW][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  const int count = (int)((n - base) < (int64_t)kRsTile ? (n - base) : (int64_t)kRsTile);
  const unsigned lt = (1u << lane) - 1u;
  {  // this tile's digit counts, their exclusive scan (tile-local starts), global starts
    const int64_t idx = (int64_t)threadIdx.x * tiles + blockIdx.x;
    const uint32_t g0 = offs[idx];
    const uint32_t g1 = (idx + 1 < 256 * tiles) ? offs[idx + 1] : (uint32_t)n;
    gstart[threadIdx.x] = g0;
    const uint32_t c = g1 - g0;
    // block exclusive scan of the 256 counts (one per thread)
    uint32_t x = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wc[0][warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint32_t t = lane < kW ? wc[0][lane] : 0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, t, off);
        if (lane >= off) t += y;
      }
      if (lane < kW) wc[1][lane] = t;
    }
    __syncthreads();
    const uint32_t st = (warp ? wc[1][warp - 1] : 0u) + x - c;
    lstart[threadIdx.x] = st;
    run[threadIdx.x] = st;
    __syncthreads();
  }
  unsigned long long kr[kRsRounds];
  uint32_t vr[kRsRounds];
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const int li = r * kRsThreads + threadIdx.x;
    kr[r] = li < count ? kin[base + li] : 0ull;
    vr[r] = li < count ? vin[base + li] : 0u;
  }
  // keep the loads here, all in flight together (the compiler would otherwise move
  // each one down to its round)
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) asm volatile("" : "+l"(kr[r]), "+r"(vr[r]));
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
    for (int q = 0; q < kW; ++q) wc[q][threadIdx.x] = 0;
    __syncthreads();
    const int li = r * kRsThreads + threadIdx.x;
    const bool valid = li < count;
    const unsigned long long key = kr[r];
    const uint32_t val = vr[r];
    const int d = valid ? (int)((key >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(kFull, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[threadIdx.x];
#pragma unroll
      for (int q = 0; q < kW; ++q) {
        const uint32_t c = wc[q][threadIdx.x];
        wc[q][threadIdx.x] = acc;
        acc += c;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wc[warp][d] + (uint32_t)rank;  // tile-local sorted position
      sk[pos] = key;
      sv[pos] = val;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < count; i += kRsThreads) {
    const unsigned long long key = sk[i];
    const int d = (int)((key >> shift) & 255);
    const uint32_t dst = gstart[d] + ((uint32_t)i - lstart[d]);
    kout[dst] = key;
    vout[dst] = sv[i];
  }
}

// ------------------------------------------------------------------ scan (u32)
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < kScanThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, t, off);
      if (lane >= off) t += y;
    }
    if (lane < kScanThreads / 32) ws[lane] = t;
  }
  __syncthreads();
  const uint32_t warp_off = warp ? ws[warp - 1] : 0;
  *total = ws[kScanThreads / 32 - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads)
scan_tile_sums(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_sums_inplace(uint32_t* __restrict__ sums, int64_t m) {
  uint32_t carry = 0;
  for (int64_t base = 0; base < m; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const uint32_t v = i < m ? sums[i] : 0;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, &total);
    if (i < m) sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kScanThreads)
scan_tiles(const uint32_t* __restrict__ in, int64_t n, const uint32_t* __restrict__ sums,
           uint32_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// Exclusive scan of n u32 values (in may equal out). `sums` holds ceil(n / tile).
cudaError_t exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums, cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 0) return cudaSuccess;
  scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  scan_sums_inplace<<<1, kScanThreads, 0, s>>>(sums, tiles);
  scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ leaf split
struct Node {
  uint32_t begin, end;
};

// One level of the binary split. A node at depth d (its keys share their first d
// bits) becomes a leaf once d >= root_bits and it holds at most `cap` series;
// otherwise it splits on key bit d into the members with that bit 0 and 1
// (SplitNode, Algorithm 4: one more bit of one segment). Nodes whose keys are
// identical in all 64 bits are cut into consecutive pieces of `cap`.
// `out` holds node_cap entries; a level that would exceed it sets *overflow and
// drops the node (the host then fails the build).
__global__ void split_level(const unsigned long long* __restrict__ keys, const Node* __restrict__ in,
                            const uint32_t* __restrict__ in_count, Node* __restrict__ out,
                            uint32_t* __restrict__ out_count, uint8_t* __restrict__ leaf_flag, int depth,
                            int root_bits, int total_bits, uint32_t cap, uint32_t node_cap,
                            uint32_t* __restrict__ overflow) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *in_count) return;
  const Node nd = in[i];
  const uint32_t size = nd.end - nd.begin;
  if (depth >= root_bits && size <= cap) {
    leaf_flag[nd.begin] = 1;
    return;
  }
  if (depth >= total_bits) {
    for (uint32_t p = nd.begin; p < nd.end; p += cap) leaf_flag[p] = 1;
    return;
  }
  const int bit = 63 - depth;
  uint32_t lo = nd.begin, hi = nd.end;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if ((keys[mid] >> bit) & 1ull) hi = mid; else lo = mid + 1;
  }
  if (lo > nd.begin) {
    const uint32_t slot = atomicAdd(out_count, 1u);
    if (slot < node_cap) out[slot] = Node{nd.begin, lo}; else *overflow = 1u;
  }
  if (lo < nd.end) {
    const uint32_t slot = atomicAdd(out_count, 1u);
    if (slot < node_cap) out[slot] = Node{lo, nd.end}; else *overflow = 1u;
  }
}

// ------------------------------------------------------- balanced split
// MSI_BUILD_BALANCED_SPLIT: below the root fan-out a node above capacity splits on
// the segment whose next symbol bit divides its members most evenly (SplitNode,
// Section II-B), segments with bits left only. Each node is one CTA: it counts the
// next bit of every segment over its members, picks the segment, and partitions its
// range stably on that bit (ids and words move together). Node depths are 4 bits per
// segment. A node whose members agree on the chosen bit passes to the next level
// whole; one with no bit left in any segment is cut into pieces of `cap`.
struct BNode {
  uint32_t begin, end, id, pad;
  unsigned long long depth;  // bits used per segment, 4 bits each
};

__device__ __forceinline__ int bnode_depth(unsigned long long d, int j) { return (int)((d >> (4 * j)) & 15ull); }

__device__ __forceinline__ uint32_t word_symbol(uint4 wd, int j) {
  const uint32_t part = j < 4 ? wd.x : (j < 8 ? wd.y : (j < 12 ? wd.z : wd.w));
  return (part >> (8 * (j & 3))) & 255u;
}

// root children as balanced-split nodes: ids 0..R-1, one bit per segment; the root
// table maps each key prefix to its child
__global__ void bal_roots(const Node* __restrict__ nodes, const uint32_t* __restrict__ count,
                          const unsigned long long* __restrict__ keys, int w, int root_bits,
                          BNode* __restrict__ out, int32_t* __restrict__ root_child) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *count) return;
  const Node nd = nodes[i];
  unsigned long long depth = 0;
  for (int j = 0; j < w; ++j) depth |= 1ull << (4 * j);
  out[i] = BNode{nd.begin, nd.end, i, 0u, depth};
  root_child[keys[nd.begin] >> (64 - root_bits)] = (int32_t)i;
}

__global__ void gather_words(const uint32_t* __restrict__ ids, int64_t n, const SumRec* __restrict__ rec,
                             uint4* __restrict__ words_out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) words_out[p] = rec[ids[p]].word;
}

__global__ void __launch_bounds__(kScanThreads)
bal_split(const BNode* __restrict__ in, uint32_t* __restrict__ ids, uint4* __restrict__ words,
          uint32_t* __restrict__ ids_tmp, uint4* __restrict__ words_tmp, BNode* __restrict__ out,
          uint32_t* __restrict__ out_count, uint32_t out_cap, uint8_t* __restrict__ leaf_flag,
          int32_t* __restrict__ tree_child, int8_t* __restrict__ tree_seg, uint32_t* __restrict__ tree_count,
          uint32_t tree_cap, int w, int bits, uint32_t cap, uint32_t* __restrict__ overflow) {
  const BNode nd = in[blockIdx.x];
  const uint32_t size = nd.end - nd.begin;
  bool open = false;  // some segment has a bit left
  for (int j = 0; j < w; ++j) open |= bnode_depth(nd.depth, j) < bits;
  if (size <= cap || !open) {
    for (uint32_t p = nd.begin + threadIdx.x * cap; p < nd.end; p += blockDim.x * cap) leaf_flag[p] = 1;
    if (threadIdx.x == 0) {
      tree_child[2 * nd.id] = tree_child[2 * nd.id + 1] = -1 - (int32_t)nd.begin;  // leaf index later
      tree_seg[nd.id] = -1;
    }
    return;
  }
  __shared__ uint32_t ones[16];
  __shared__ int s_j;
  if (threadIdx.x < 16) ones[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (uint32_t p0 = nd.begin; p0 < nd.end; p0 += blockDim.x) {
    const uint32_t p = p0 + threadIdx.x;
    const uint4 wd = p < nd.end ? words[p] : make_uint4(0, 0, 0, 0);
    for (int j = 0; j < w; ++j) {
      const int b = bnode_depth(nd.depth, j);
      const bool bit = p < nd.end && b < bits && ((word_symbol(wd, j) >> (bits - 1 - b)) & 1u);
      const unsigned m = __ballot_sync(kFull, bit);
      if (lane == 0 && m) atomicAdd(&ones[j], (uint32_t)__popc(m));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = -1;
    long long best_gap = 0;
    for (int j = 0; j < w; ++j) {
      if (bnode_depth(nd.depth, j) >= bits) continue;
      long long gap = 2ll * ones[j] - (long long)size;
      gap = gap < 0 ? -gap : gap;
      if (best < 0 || gap < best_gap) {
        best = j;
        best_gap = gap;
      }
    }
    s_j = best;
  }
  __syncthreads();
  const int j = s_j;
  const int b = bnode_depth(nd.depth, j);
  const uint32_t n1 = ones[j], n0 = size - n1;
  uint32_t base0 = 0, base1 = 0;
  for (uint32_t p0 = nd.begin; p0 < nd.end; p0 += blockDim.x) {
    const uint32_t p = p0 + threadIdx.x;
    const bool in = p < nd.end;
    const uint4 wd = in ? words[p] : make_uint4(0, 0, 0, 0);
    const uint32_t id = in ? ids[p] : 0u;
    const uint32_t bit = in ? (word_symbol(wd, j) >> (bits - 1 - b)) & 1u : 0u;
    uint32_t tot1;
    const uint32_t ex1 = block_exclusive_scan(bit, &tot1);
    if (in) {
      const uint32_t dst = bit ? nd.begin + n0 + base1 + ex1 : nd.begin + base0 + (threadIdx.x - ex1);
      ids_tmp[dst] = id;
      words_tmp[dst] = wd;
    }
    base1 += tot1;
    base0 += min((uint32_t)blockDim.x, nd.end - p0) - tot1;
  }
  __syncthreads();
  for (uint32_t p = nd.begin + threadIdx.x; p < nd.end; p += blockDim.x) {
    ids[p] = ids_tmp[p];
    words[p] = words_tmp[p];
  }
  if (threadIdx.x == 0) {
    const unsigned long long d2 = nd.depth + (1ull << (4 * j));
    int32_t c[2] = {-1, -1};
    const uint32_t lo[2] = {nd.begin, nd.begin + n0}, hi[2] = {nd.begin + n0, nd.end};
    for (int h = 0; h < 2; ++h) {
      if (lo[h] == hi[h]) continue;
      const uint32_t id = atomicAdd(tree_count, 1u);
      const uint32_t slot = atomicAdd(out_count, 1u);
      if (id >= tree_cap || slot >= out_cap) {
        *overflow = 1u;
        continue;
      }
      c[h] = (int32_t)id;
      out[slot] = BNode{lo[h], hi[h], id, 0u, d2};
    }
    // a side without members points to the other, so routing always reaches a leaf
    tree_child[2 * nd.id] = c[0] >= 0 ? c[0] : c[1];
    tree_child[2 * nd.id + 1] = c[1] >= 0 ? c[1] : c[0];
    tree_seg[nd.id] = (int8_t)j;
  }
}

// leaf entries of the tree: first position -> leaf index
__global__ void bal_leaf_ids(int32_t* __restrict__ tree_child, const int8_t* __restrict__ tree_seg,
                             const uint32_t* __restrict__ count, const uint32_t* __restrict__ rank) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *count || tree_seg[i] >= 0) return;
  const uint32_t begin = (uint32_t)(-1 - tree_child[2 * i]);
  tree_child[2 * i] = tree_child[2 * i + 1] = -1 - (int32_t)rank[begin];
}

__global__ void flags_to_u32(const uint8_t* __restrict__ f, int64_t n, uint32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = f[i];
}

__global__ void write_leaf_begin(const uint8_t* __restrict__ f, const uint32_t* __restrict__ rank, int64_t n,
                                 uint32_t* __restrict__ leaf_begin) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && f[i]) leaf_begin[rank[i]] = (uint32_t)i;
}

// ------------------------------------------------------------------ envelopes
__global__ void envelopes(const uint4* __restrict__ words, const uint32_t* __restrict__ leaf_begin, int64_t L,
                          const unsigned long long* __restrict__ keys_sorted, uint4* __restrict__ env,
                          uint64_t* __restrict__ leaf_key) {
  const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (l >= L) return;
  const uint32_t b = leaf_begin[l], e = leaf_begin[l + 1];
  uint4 lo = make_uint4(~0u, ~0u, ~0u, ~0u), hi = make_uint4(0, 0, 0, 0);
  for (uint32_t p = b + lane; p < e; p += 32) {
    const uint4 w = words[p];
    lo.x = __vminu4(lo.x, w.x); lo.y = __vminu4(lo.y, w.y); lo.z = __vminu4(lo.z, w.z); lo.w = __vminu4(lo.w, w.w);
    hi.x = __vmaxu4(hi.x, w.x); hi.y = __vmaxu4(hi.y, w.y); hi.z = __vmaxu4(hi.z, w.z); hi.w = __vmaxu4(hi.w, w.w);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo.x = __vminu4(lo.x, __shfl_xor_sync(kFull, lo.x, off));
    lo.y = __vminu4(lo.y, __shfl_xor_sync(kFull, lo.y, off));
    lo.z = __vminu4(lo.z, __shfl_xor_sync(kFull, lo.z, off));
    lo.w = __vminu4(lo.w, __shfl_xor_sync(kFull, lo.w, off));
    hi.x = __vmaxu4(hi.x, __shfl_xor_sync(kFull, hi.x, off));
    hi.y = __vmaxu4(hi.y, __shfl_xor_sync(kFull, hi.y, off));
    hi.z = __vmaxu4(hi.z, __shfl_xor_sync(kFull, hi.z, off));
    hi.w = __vmaxu4(hi.w, __shfl_xor_sync(kFull, hi.w, off));
  }
  if (lane == 0) {
    env[2 * l] = lo;
    env[2 * l + 1] = hi;
    leaf_key[l] = keys_sorted[b];
  }
}

// Envelope of every aligned block of 32 leaf-order positions and of each of its two
// halves of 16 (one warp per block: the first four shuffle levels close the halves,
// the fifth the block).
__global__ void block_envelopes(const uint4* __restrict__ words, int64_t n, uint4* __restrict__ benv,
                                uint4* __restrict__ henv) {
  const int64_t blk = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (blk * 32 >= n) return;
  const int64_t p = blk * 32 + lane;
  uint4 lo = make_uint4(~0u, ~0u, ~0u, ~0u), hi = make_uint4(0, 0, 0, 0);
  if (p < n) lo = hi = words[p];
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    if (off == 16 && (lane & 15) == 0 && blk * 32 + lane < n) {  // a half with at least one position
      const int64_t hb = 2 * blk + (lane >> 4);
      henv[2 * hb] = lo;
      henv[2 * hb + 1] = hi;
    }
    lo.x = __vminu4(lo.x, __shfl_xor_sync(kFull, lo.x, off));
    lo.y = __vminu4(lo.y, __shfl_xor_sync(kFull, lo.y, off));
    lo.z = __vminu4(lo.z, __shfl_xor_sync(kFull, lo.z, off));
    lo.w = __vminu4(lo.w, __shfl_xor_sync(kFull, lo.w, off));
    hi.x = __vmaxu4(hi.x, __shfl_xor_sync(kFull, hi.x, off));
    hi.y = __vmaxu4(hi.y, __shfl_xor_sync(kFull, hi.y, off));
    hi.z = __vmaxu4(hi.z, __shfl_xor_sync(kFull, hi.z, off));
    hi.w = __vmaxu4(hi.w, __shfl_xor_sync(kFull, hi.w, off));
  }
  if (lane == 0) {
    benv[2 * blk] = lo;
    benv[2 * blk + 1] = hi;
  }
}

__global__ void gather_leaf_order(const uint32_t* __restrict__ perm, int64_t n, const SumRec* __restrict__ rec,
                                  uint4* __restrict__ words_out, float2* __restrict__ stats_out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t id = perm[p];
  words_out[p] = rec[id].word;
  stats_out[p] = rec[id].stats;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

// The build's temporaries: carved from one device allocation reserved up front (one
// cudaMalloc and one cudaFree instead of one per array), with a fallback to separate
// allocations should the reservation run short.
struct Freer {
  std::vector<void*> ptrs;
  char* base = nullptr;
  size_t cap = 0, used = 0;
  ~Freer() {
    for (void* p : ptrs) cudaFree(p);
    if (base) cudaFree(base);
  }
  cudaError_t reserve(size_t bytes) {
    cudaError_t e = cudaMalloc((void**)&base, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      base = nullptr;
      return cudaSuccess;  // the separate allocations below still work (or fail alone)
    }
    cap = bytes;
    return cudaSuccess;
  }
  template <typename T>
  cudaError_t get(T** p, size_t count) {
    const size_t bytes = (sizeof(T) * (count ? count : 1) + 255) & ~size_t(255);
    if (base && used + bytes <= cap) {
      *p = reinterpret_cast<T*>(base + used);
      used += bytes;
      return cudaSuccess;
    }
    cudaError_t e = dalloc(p, count);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t block_envelopes_of(msi_index* ix, cudaStream_t s) {
  const int64_t nblk = (ix->n + 31) / 32;
  block_envelopes<<<grid_for(nblk * 32, 256), 256, 0, s>>>(ix->words, ix->n, ix->benv, ix->henv);
  return cudaGetLastError();
}

// Builds every device structure of `ix` (shape fields, thresholds and data pointers
// already set). `src_dev` holds the raw collection on the device; with `in_place`
// it is ix->data_owned and is overwritten by its z-normalised values.
cudaError_t build_index(msi_index* ix, const float* src_dev, bool in_place, cudaStream_t s,
                        int64_t* first_bad, const char** stage) {
  (void)in_place;
  const int64_t n = ix->n;
  const int len = ix->len, w = ix->w;
  Freer tmp;
  SumOut o;
  unsigned long long* keys_alt;
  uint32_t* ids_alt;
  *stage = "allocating build scratch";
  {  // words, keys and ids twice, moments, flags, ranks, radix histograms, the nodes of
     // a level (and the balanced split's sort buffers); 64 MB of room for the rest
    const int64_t tiles_b = (n + kRsTile - 1) / kRsTile;
    const bool bal = (ix->flags & MSI_BUILD_BALANCED_SPLIT) != 0;
    const size_t want = (size_t)n * (32 + 4 + 8 + 8 + 4 + 1 + 4 + (bal ? 36 : 0)) + (size_t)tiles_b * 1024 +
                        (size_t)16 * std::min<int64_t>(n, (1ll << std::min(w * ix->bits, 20)) + 2 * (n / ix->cap) + 2) +
                        ((size_t)64 << 20);
    MSI_TRY(tmp.reserve(want));
  }
  MSI_TRY(tmp.get(&o.rec, n));
  MSI_TRY(tmp.get(&o.keys, n));
  MSI_TRY(tmp.get(&o.ids, n));
  MSI_TRY(tmp.get(&keys_alt, n));
  MSI_TRY(tmp.get(&ids_alt, n));
  MSI_TRY(tmp.get(&o.first_bad, 1));
  o.z_out = ix->data_owned;  // nullptr when borrowed
  o.fine = nullptr;
  o.wf = (ix->flags & MSI_BUILD_NO_FINE_BOUND) ? 0 : fine_segments(len, w);
  o.sf = o.wf ? len / o.wf : 0;
  if (o.wf) {  // written by the summarise kernel straight into the index (collection order)
    MSI_TRY(dalloc(&ix->fine, (size_t)n * (o.wf / 8)));
    o.fine = ix->fine;
  }
  MSI_TRY(cudaMemsetAsync(o.first_bad, 0xff, sizeof(unsigned long long), s));

  // 1. summarise
  *stage = "summarise";
  int dev_sms = 0;
  MSI_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ix->device));
  const int s_len = ix->seglen;
  const int G = s_len / 4;
  const bool fast = (len % 128 == 0) && (len / 128) <= 16 && (s_len % 4 == 0) && G >= 1 && G <= 32 &&
                    (G & (G - 1)) == 0 && ((len / 128) & (len / 128 - 1)) == 0;
  const bool pair = fast && len / 128 <= 4 && G <= 16 && (o.sf == 0 || o.sf <= 64);
  if (pair) {
    // the symbol cell table: thresholds t_1..t_{card-1} at or below the left edge of
    // the previous cell (-4 + (c - 1) / 128), counted on the host from the same table
    // (ascending, so a binary search); it lives in the index, so the upload needs no wait
    static_assert(sizeof(ix->h_sym_cells) == kSymCells, "cell table size");
    ix->h_sym_cells[0] = 0;
    for (int c = 1; c < kSymCells; ++c) {
      const double edge = -4.0 + (double)(c - 1) / 128.0;
      int lo = 1, hi = ix->card;  // first v in [1, card) with t_v > edge, or card
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if ((double)ix->h_thr_up[mid] <= edge) lo = mid + 1;
        else hi = mid;
      }
      ix->h_sym_cells[c] = (uint8_t)(lo - 1);
    }
    uint8_t* cell_d;
    MSI_TRY(tmp.get(&cell_d, kSymCells));
    MSI_TRY(cudaMemcpyAsync(cell_d, ix->h_sym_cells, kSymCells, cudaMemcpyHostToDevice, s));
    const int64_t pairs = (n + 1) / 2;
    const int64_t blocks = std::min<int64_t>((pairs + kSumWarps - 1) / kSumWarps, (int64_t)dev_sms * 64);
    // the row rings pass the 48 KB default from 256 points on: raise the limit per width
    MSI_TRY(cudaFuncSetAttribute(summarise_pair<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_ring_bytes<1>()));
    MSI_TRY(cudaFuncSetAttribute(summarise_pair<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_ring_bytes<2>()));
    MSI_TRY(cudaFuncSetAttribute(summarise_pair<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_ring_bytes<4>()));
    MSI_TRY(cudaFuncSetAttribute(summarise_pair<2, 4, 4, 16, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_ring_bytes<2>()));
    // 256 points, 16 segments of 16, 64 fine segments of 4, 8-bit symbols: its own
    // compiled shape; every other shape reads these from the arguments
    const bool shape_256_16 = len == 256 && G == 4 && o.sf == 4 && w == 16 && ix->bits == 8;
    if (shape_256_16)
      summarise_pair<2, 4, 4, 16, 8><<<(unsigned)blocks, kSumWarps * 32, pair_ring_bytes<2>(), s>>>(
          src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, cell_d, o);
    else switch (len / 128) {
      case 1: summarise_pair<1><<<(unsigned)blocks, kSumWarps * 32, pair_ring_bytes<1>(), s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, cell_d, o); break;
      case 2: summarise_pair<2><<<(unsigned)blocks, kSumWarps * 32, pair_ring_bytes<2>(), s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, cell_d, o); break;
      default: summarise_pair<4><<<(unsigned)blocks, kSumWarps * 32, pair_ring_bytes<4>(), s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, cell_d, o); break;
    }
  } else if (fast) {
    const int64_t blocks = std::min<int64_t>((n + kSumWarps - 1) / kSumWarps, (int64_t)dev_sms * 64);
    switch (len / 128) {
      case 1: summarise_fast<1><<<(unsigned)blocks, kSumWarps * 32, 0, s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, o); break;
      case 2: summarise_fast<2><<<(unsigned)blocks, kSumWarps * 32, 0, s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, o); break;
      case 4: summarise_fast<4><<<(unsigned)blocks, kSumWarps * 32, 0, s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, o); break;
      case 8: summarise_fast<8><<<(unsigned)blocks, kSumWarps * 32, 0, s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, o); break;
      default: summarise_fast<16><<<(unsigned)blocks, kSumWarps * 32, 0, s>>>(src_dev, n, w, ix->card, ix->bits, G, ix->thr_up, o); break;
    }
  } else {
    const size_t smem = sizeof(float) * (size_t)len * kGenWarps;
    if (smem > 48 * 1024)
      MSI_TRY(cudaFuncSetAttribute(summarise_generic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t blocks = std::min<int64_t>((n + kGenWarps - 1) / kGenWarps, (int64_t)dev_sms * 32);
    summarise_generic<<<(unsigned)blocks, kGenWarps * 32, smem, s>>>(src_dev, n, len, w, ix->card, ix->bits,
                                                                     ix->thr_up, o);
  }
  MSI_TRY(cudaGetLastError());
  unsigned long long bad = 0;
  MSI_TRY(cudaMemcpyAsync(&bad, o.first_bad, sizeof bad, cudaMemcpyDeviceToHost, s));
  MSI_TRY(cudaStreamSynchronize(s));
  if (bad != ~0ull) {
    *first_bad = (int64_t)bad;
    return cudaSuccess;
  }
  *first_bad = -1;

  // 2. sort (key, id), stable, 8 passes of 8 bits
  *stage = "sort";
  const int64_t tiles = (n + kRsTile - 1) / kRsTile;
  uint32_t *hist, *sums;
  MSI_TRY(tmp.get(&hist, (size_t)tiles * 256));
  MSI_TRY(tmp.get(&sums, (size_t)((tiles * 256 + kScanTile - 1) / kScanTile + 1)));
  unsigned long long *ka = o.keys, *kb = keys_alt;
  uint32_t *va = o.ids, *vb = ids_alt;
  MSI_TRY(cudaFuncSetAttribute(rs_scatter_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRsSmem));
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 8 * pass;
    rs_upsweep<<<(unsigned)tiles, kRsThreads, 0, s>>>(ka, n, shift, hist, tiles);
    MSI_TRY(exclusive_scan(hist, hist, tiles * 256, sums, s));
    rs_scatter_local<<<(unsigned)tiles, kRsThreads, kRsSmem, s>>>(ka, va, kb, vb, n, shift, hist, tiles);
    MSI_TRY(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  // after 8 passes the sorted keys / ids are back in (ka, va) == (o.keys, o.ids)

  // 3. leaf split
  *stage = "leaf split";
  const int total_bits = std::min(64, w * ix->bits);
  const int root_bits = std::min(w, total_bits);
  // Nodes of one depth are disjoint non-empty ranges. Below depth root_bits there
  // are at most 2^depth of them; from there on only nodes above capacity split, at
  // most n / cap of them, two children each.
  const int64_t node_cap = std::min<int64_t>(n, (1ll << root_bits) + 2 * (n / ix->cap) + 2);
  Node *na, *nb;
  uint32_t* counts;  // [2] in, out; [2] overflow
  uint8_t* flags;
  MSI_TRY(tmp.get(&na, node_cap));
  MSI_TRY(tmp.get(&nb, node_cap));
  MSI_TRY(tmp.get(&counts, 3));
  MSI_TRY(tmp.get(&flags, n + 1));
  MSI_TRY(cudaMemsetAsync(flags, 0, (size_t)n + 1, s));
  MSI_TRY(cudaMemsetAsync(counts + 2, 0, sizeof(uint32_t), s));
  const Node root{0u, (uint32_t)n};
  const uint32_t one = 1;
  MSI_TRY(cudaMemcpyAsync(na, &root, sizeof root, cudaMemcpyHostToDevice, s));
  MSI_TRY(cudaMemcpyAsync(counts, &one, sizeof one, cudaMemcpyHostToDevice, s));
  const bool balanced = (ix->flags & MSI_BUILD_BALANCED_SPLIT) != 0;
  // round-robin: every level to the last key bit; balanced: the root fan-out only
  const int last_depth = balanced ? root_bits - 1 : total_bits;
  for (int depth = 0; depth <= last_depth; ++depth) {
    MSI_TRY(cudaMemsetAsync(counts + 1, 0, sizeof(uint32_t), s));
    split_level<<<grid_for(node_cap, 256), 256, 0, s>>>(ka, na, counts, nb, counts + 1, flags, depth, root_bits,
                                                       total_bits, (uint32_t)ix->cap, (uint32_t)node_cap,
                                                       counts + 2);
    MSI_TRY(cudaGetLastError());
    MSI_TRY(cudaMemcpyAsync(counts, counts + 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    std::swap(na, nb);
  }
  uint32_t* tree_count = nullptr;
  if (balanced) {
    *stage = "balanced split";
    uint32_t R = 0;
    MSI_TRY(cudaMemcpyAsync(&R, counts, sizeof R, cudaMemcpyDeviceToHost, s));
    MSI_TRY(cudaStreamSynchronize(s));
    // each level adds at most two nodes per node above capacity (at most n / cap of
    // them); a chain of levels is at most w * bits long
    const int64_t per_level = 2 * (n / ix->cap + 1);
    const int64_t level_cap = std::max<int64_t>(R, per_level);
    const int64_t tree_cap = std::min<int64_t>(0x7ffffff0ll, (int64_t)R + per_level * (w * ix->bits + 1));
    ix->root_bits = root_bits;
    MSI_TRY(dalloc(&ix->root_child, (size_t)1 << root_bits));
    MSI_TRY(dalloc(&ix->tree_child, 2 * (size_t)tree_cap));
    MSI_TRY(dalloc(&ix->tree_seg, (size_t)tree_cap));
    MSI_TRY(cudaMemsetAsync(ix->root_child, 0xff, sizeof(int32_t) << root_bits, s));
    BNode *ba, *bb;
    uint4 *wsort, *wtmp;
    uint32_t* itmp;
    MSI_TRY(tmp.get(&ba, level_cap));
    MSI_TRY(tmp.get(&bb, level_cap));
    MSI_TRY(tmp.get(&wsort, n));
    MSI_TRY(tmp.get(&wtmp, n));
    MSI_TRY(tmp.get(&itmp, n));
    MSI_TRY(tmp.get(&tree_count, 1));
    MSI_TRY(cudaMemcpyAsync(tree_count, counts, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    bal_roots<<<grid_for(R, 256), 256, 0, s>>>(na, counts, ka, w, root_bits, ba, ix->root_child);
    gather_words<<<grid_for(n, 256), 256, 0, s>>>(va, n, o.rec, wsort);
    MSI_TRY(cudaGetLastError());
    uint32_t live = R;
    for (int level = 0; live > 0; ++level) {
      if (level > w * ix->bits + 1) {  // every level uses one more bit of some segment
        *stage = "balanced split: too many levels";
        return cudaErrorUnknown;
      }
      MSI_TRY(cudaMemsetAsync(counts + 1, 0, sizeof(uint32_t), s));
      bal_split<<<live, kScanThreads, 0, s>>>(ba, va, wsort, itmp, wtmp, bb, counts + 1, (uint32_t)level_cap, flags,
                                              ix->tree_child, ix->tree_seg, tree_count, (uint32_t)tree_cap, w,
                                              ix->bits, (uint32_t)ix->cap, counts + 2);
      MSI_TRY(cudaGetLastError());
      MSI_TRY(cudaMemcpyAsync(&live, counts + 1, sizeof live, cudaMemcpyDeviceToHost, s));
      MSI_TRY(cudaStreamSynchronize(s));
      std::swap(ba, bb);
    }
    uint32_t tn = 0;
    MSI_TRY(cudaMemcpyAsync(&tn, tree_count, sizeof tn, cudaMemcpyDeviceToHost, s));
    MSI_TRY(cudaStreamSynchronize(s));
    ix->tree_nodes = std::min<int64_t>(tn, tree_cap);
  }
  // leaf begins: exclusive scan of the flags gives each leaf's rank
  uint32_t* rank;
  uint32_t* sums2;
  MSI_TRY(tmp.get(&rank, n + 1));
  MSI_TRY(tmp.get(&sums2, (size_t)((n + 1 + kScanTile - 1) / kScanTile + 1)));
  flags_to_u32<<<grid_for(n + 1, 256), 256, 0, s>>>(flags, n + 1, rank);
  MSI_TRY(exclusive_scan(rank, rank, n + 1, sums2, s));
  if (balanced) {
    bal_leaf_ids<<<grid_for(ix->tree_nodes, 256), 256, 0, s>>>(ix->tree_child, ix->tree_seg, tree_count, rank);
    MSI_TRY(cudaGetLastError());
    ix->device_bytes += (int64_t)(sizeof(int32_t) << ix->root_bits) + 9 * ix->tree_nodes;
  }
  uint32_t L32 = 0, node_overflow = 0;
  MSI_TRY(cudaMemcpyAsync(&L32, rank + n, sizeof L32, cudaMemcpyDeviceToHost, s));
  MSI_TRY(cudaMemcpyAsync(&node_overflow, counts + 2, sizeof node_overflow, cudaMemcpyDeviceToHost, s));
  MSI_TRY(cudaStreamSynchronize(s));
  ix->L = L32;
  if (node_overflow || ix->L < 1) {
    *stage = "leaf split: node list overflow";
    return cudaErrorUnknown;
  }

  // 4. final structures
  *stage = "allocating index";
  MSI_TRY(dalloc(&ix->words, n));
  MSI_TRY(dalloc(&ix->perm, n));
  MSI_TRY(dalloc(&ix->stats, n));
  MSI_TRY(dalloc(&ix->leaf_begin, ix->L + 1));
  MSI_TRY(dalloc(&ix->env, 2 * ix->L));
  MSI_TRY(dalloc(&ix->leaf_key, ix->L));
  const int64_t nblk = (n + 31) / 32, nhb = (n + 15) / 16;
  MSI_TRY(dalloc(&ix->benv, 2 * nblk));
  MSI_TRY(dalloc(&ix->henv, 2 * nhb));
  ix->device_bytes += (int64_t)n * (16 + 4 + 8) + (ix->L + 1) * 4 + ix->L * (32 + 8) + nblk * 32 + nhb * 32;
  *stage = "envelopes";
  write_leaf_begin<<<grid_for(n, 256), 256, 0, s>>>(flags, rank, n, ix->leaf_begin);
  const uint32_t nn = (uint32_t)n;
  MSI_TRY(cudaMemcpyAsync(ix->leaf_begin + ix->L, &nn, sizeof nn, cudaMemcpyHostToDevice, s));
  MSI_TRY(cudaMemcpyAsync(ix->perm, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  gather_leaf_order<<<grid_for(n, 256), 256, 0, s>>>(ix->perm, n, o.rec, ix->words, ix->stats);
  if (o.wf) {
    ix->wf = o.wf;
    ix->sf = o.sf;
    ix->device_bytes += (int64_t)n * 2 * o.wf;
  }
  envelopes<<<grid_for(ix->L * 32, 256), 256, 0, s>>>(ix->words, ix->leaf_begin, ix->L, ka, ix->env, ix->leaf_key);
  block_envelopes<<<grid_for(nblk * 32, 256), 256, 0, s>>>(ix->words, n, ix->benv, ix->henv);
  MSI_TRY(cudaGetLastError());
  MSI_TRY(cudaStreamSynchronize(s));
  return cudaSuccess;
}

}  // namespace msi
