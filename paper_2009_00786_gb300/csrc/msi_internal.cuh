// msi_internal.cuh -- index layout and device helpers shared by the library's
// translation units (msi_api.cu, msi_build.cu, msi_query.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "../../include/msi.h"

namespace msi {

constexpr int kWarp = 32;
constexpr int kItem = 256;  // leaf positions per refinement work item
constexpr int kMaxRefineWarps = 1 << 16;
constexpr int kMaxFront = 8;  // leaves refined before the filters, at most
// Concurrent queries divide the persistent grids of their kernels by at most this (the
// default of an index's grid share; msi_autotune may choose another): the queries then
// oversubscribe the GPU and the hardware interleaves their blocks, where dividing by
// the number of queries would leave SMs idle whenever the queries' phases do not line
// up (100M x 256: 16 queries at 1/3 of the grid each 31.6K q/s, 8 queries at 1/8 each
// 24.0K).
constexpr int kSlotGridShare = 3;
constexpr int kDefaultQuerySlots = 16;
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ index
// Device-side view of an index, passed to kernels by value.
struct IndexView {
  const float* data;        // [n][len] collection: z-normalised (owned) or raw (borrowed)
  int data_is_z;            // 1: data holds z values; 0: z = (x - mu) * rsig on the fly
  const float2* stats;      // [n] leaf order: (mu, 1/sigma), 1/sigma = 0 for constant series
  const uint4* words;       // [n] leaf order: iSAX word, one byte per segment, zero padded
  const uint32_t* perm;     // [n] leaf order -> collection id
  const uint32_t* leaf_begin; // [L+1]
  const uint4* env;         // [L][2]: per-segment min symbols, max symbols
  const uint4* benv;        // [ceil(n/32)][2]: the same over aligned blocks of 32 leaf positions
                            //   (kept in the index file; the block filter reads henv)
  const uint4* henv;        // [ceil(n/16)][2]: the same over aligned half-blocks of 16 positions
  const uint64_t* leaf_key; // [L]: interleaved key of each leaf's first member
  const float* thr_up;      // [card+1]: region upper edges: thr_up[v] = smallest float >= beta_v,
                            //   thr_up[0] = -inf, thr_up[card] = +inf (also the SAX thresholds)
  const float* thr_lo;      // [card+1]: conservative lower edges: largest float <= beta_v
  // balanced-split tree (MSI_BUILD_BALANCED_SPLIT; null otherwise): the node of each
  // root prefix (-1: none), each node's children (a leaf: both -1 - leaf index) and
  // split segment (-1 for a leaf)
  const int32_t* root_child;
  const int32_t* tree_child;
  const int8_t* tree_seg;
  // [n][wf / 8] collection order (indexed by id = perm[position]): the series' means
  // over wf equal segments of sf points (the fine PAA), fp16 rounded to nearest; null
  // when wf = 0. Kept in collection order: its reads are random anyway (only series
  // whose iSAX bound passed are bounded by it), and the build then writes it once.
  const uint4* fine;
  int64_t n;
  int64_t L;
  int len, w, card, bits, seglen, root_bits;
  int wf, sf;
};

constexpr int kMaxFine = 64;
// The coarse bound of the series filter reads each symbol's first kCoarseBits bits:
// a table of kCoarse entries per segment (6 bits: two-way bank conflicts at most, and
// at 100M x 256 the batched series filter ran 1.27 ms per 100 queries against 1.42 ms
// with 5 bits).
constexpr int kCoarseBits = 6;
constexpr int kCoarse = 1 << kCoarseBits;
// Segments of the fine PAA: the largest of 64, 32, 16, 8 that divides len into
// segments of a power-of-two length and exceeds the iSAX word's w; 0 when none does.
__host__ __device__ inline int fine_segments(int len, int w) {
  for (int wf = kMaxFine; wf >= 8; wf >>= 1) {
    const int sf = len / wf;
    if (len % wf == 0 && (sf & (sf - 1)) == 0 && wf > w) return wf;
  }
  return 0;
}

// Per-query device state (one instance per in-flight query).
struct QState {
  float qpaa[16];
  float qup[16], qlo[16];       // per-segment interval the bounds measure gaps to: the PAA
                                // value (Euclidean) or the envelope's [min, max] (DTW)
  float fup[kMaxFine], flo[kMaxFine];  // the same over the fine PAA's segments
  int32_t qsym[16];             // a symbol inside that interval, per segment
  unsigned long long qkey;
  uint32_t seed_a, seed_b;      // leaf-order positions refined by the approximate search
  unsigned int thr_bits;        // fp32 bits of the current k-th best squared distance
  unsigned int leaf_count;      // leaves that passed the leaf filter
  unsigned int item_count;      // refinement work items (<= kItem positions of one leaf)
  unsigned int surv_count;      // series whose bound passed the series filter
  unsigned int blk_count;       // half-blocks (16 positions) whose envelope bound passed
  unsigned int overflow;        // a candidate or survivor list ran out of room
  float kbase;                  // k > 1: the k-th best after the seed and front leaves; the
                                // range [0, kbase) of the candidate histogram (0: none yet)
  uint32_t nfront;              // leaves refined early (the lowest-bound survivors)
  uint32_t front_leaf[8];       // their ids; the filters skip them
  uint32_t front_beg[8], front_end[8];  // batched chain: their position ranges
  unsigned int front_lb[8];     // batched chain: their bounds (fp32 bits, ascending)
  unsigned int cand_count;      // candidates appended
  unsigned int rc_count;        // FP64 re-checks appended
  unsigned int final_bits;      // k-th smallest candidate squared distance (fp32 bits)
  unsigned int series_refined;
  unsigned int fine_front;      // front-leaf rows bounded by the fine PAA
  unsigned int seed_done;       // seed rows whose distance was computed
  int32_t flag;                 // 1 constant query, -1 non-finite query
  unsigned int ord_count;       // survivors in bound order (surv2), when ordered
};

// Device-wide work counters (u64), in msi_query_stats field order.
enum StatSlot {
  ST_QUERIES = 0, ST_LEAVES_TOTAL, ST_LEAVES_SURVIVED, ST_LEAVES_PROCESSED, ST_SERIES_LB,
  ST_SERIES_REFINED, ST_SEED, ST_CANDIDATES, ST_RECHECKED, ST_BAD_QUERY, ST_SURVIVORS, ST_FINE, ST_FINE_FRONT,
  ST_TC_PAIRS, ST_COUNT
};

// Base pointers of one batched call. A query launched from a cached CUDA graph finds
// its input and outputs here (query qi of the call) instead of in kernel arguments, so
// one graph serves every call of the same shape.
struct CallDesc {
  const float* queries;  // [nq][len]
  int64_t* ids;          // [nq][k]
  float* dists;          // [nq][k], or nullptr
  double* d64;           // [nq][k], or nullptr
};

struct QueryView {
  float* qz;                    // [len]
  float* T;                     // [w][card] squared per-segment gap, query PAA to each symbol
  float* T5;                    // [w][kCoarse] the same to each kCoarseBits-bit symbol prefix (coarse regions)
  QState* st;
  uint32_t* leaf_list;          // [L]
  float* leaf_lb2;              // [L]
  uint4* items;                 // [n / kItem + 2L]: {first pos, end pos, leaf bound^2 bits, leaf}
  uint2* surv;                  // [n]: {leaf-order position, bound^2 bits} of filter survivors
  uint2* surv2;                 // [surv_cap]: the same in ascending bound buckets (batch workspaces)
  const uint2* rsurv;           // the list the row kernel reads: surv2 when ordered, else null (surv)
  uint2* blks;                  // [16 (n / kItem + 2L)]: {half-block index, lo | hi << 8} of surviving halves
  unsigned long long* blockmin; // [L / 256 + 2]: per leaf-filter block, min (bound^2 bits << 32 | leaf)
  unsigned long long* cand;     // [n]: (fp32 d^2 bits << 32) | id
  double* rc_d;                 // [n]
  uint32_t* rc_id;              // [n]
  unsigned long long* counters; // [ST_COUNT]
  uint32_t* partials;           // [4][kMaxRefineWarps]: per-warp work counters of the refinement
  uint32_t npartials;           // warps of the series filter launch
  uint32_t npartials_rows;      // warps of the row (or DTW) refinement launch
  uint32_t cand_cap;            // entries of cand / rc_d / rc_id
  uint32_t surv_cap;            // entries of surv
  uint32_t items_cap;           // entries of items (a query that needs more overflows)
  uint32_t blks_cap;            // entries of blks (likewise)
  uint32_t* ovf;                // per-query overflow flag written by q_finalize (or nullptr)
  float* qenv;                  // [2][len]: LB_Keogh envelope of the query, upper then lower (DTW)
  uint32_t* khist;              // [256]: k > 1, kept candidates per bucket of [0, kbase)
  int window = -1;              // DTW: Sakoe-Chiba half-width; -1: Euclidean distance
  const CallDesc* call = nullptr; // graph replay: the call's pointers (query qi of it)
  int qi = 0;
  int k;
  float eps;                    // relative margin on squared distances
  float tau;                    // absolute margin on lower bounds (distance units)
};

// ----------------------------------------------------- canonical fp32 arithmetic
// The z-normalisation and PAA are computed in one fixed order (the CPU oracle
// follows the same order) because the SAX symbols are integers decided by them:
//   lane of point t = (t / 4) mod 32; each lane sums its points in increasing t;
//   the 32 lane partials are combined by a pairwise tree in lane order;
//   mu = S1 / n; V likewise over fma(d, d, .) with d = x_t - mu;
//   sigma = sqrt(V / n); constant if sigma < 1e-30 or sigma <= 1e-6 |mu| (z = 0);
//   z_t = (x_t - mu) * (1 / sigma); every step a single IEEE rounding.
__device__ __forceinline__ float tree32(float v) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) v = __fadd_rn(v, __shfl_xor_sync(kFull, v, off));
  return v;
}

struct Moments {
  float mu;
  float rsig;  // 1/sigma, 0 for a constant series
  int flag;    // 0 normal, 1 constant, -1 non-finite
};

// x / d for a power of two d: the product with its exact reciprocal, the same
// correctly rounded value as the division at a fraction of its instructions (both are
// the exact quotient rounded once).
__device__ __forceinline__ float div_pow2(float x, float inv_d) { return __fmul_rn(x, inv_d); }

// mu = S1 / n already rounded; v = the combined sum of squared deviations. inv_len
// > 0: len is a power of two and inv_len its exact reciprocal (v / n by div_pow2).
__device__ __forceinline__ Moments finish_moments(float mu, float v, int len, float inv_len = 0.0f) {
  Moments m;
  const float n = (float)len;
  m.mu = mu;
  const float sigma = __fsqrt_rn(inv_len > 0.0f ? div_pow2(v, inv_len) : __fdiv_rn(v, n));
  if (!isfinite(m.mu) || !isfinite(sigma)) {
    m.flag = -1;
    m.rsig = 0.0f;
  } else if (sigma < 1e-30f || sigma <= __fmul_rn(1e-6f, fabsf(m.mu))) {
    m.flag = 1;
    m.rsig = 0.0f;
  } else {
    m.flag = 0;
    m.rsig = __fdiv_rn(1.0f, sigma);
  }
  return m;
}

// Canonical moments of one series in global or shared memory, any length (one warp).
__device__ __forceinline__ Moments warp_moments_generic(const float* x, int len) {
  const int lane = threadIdx.x & 31;
  float acc = 0.0f;
  for (int c = 0; c * 128 < len; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = c * 128 + 4 * lane + i;
      if (t < len) acc = __fadd_rn(acc, x[t]);
    }
  const float mu = __fdiv_rn(tree32(acc), (float)len);
  float acc2 = 0.0f;
  for (int c = 0; c * 128 < len; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = c * 128 + 4 * lane + i;
      if (t < len) {
        const float d = __fsub_rn(x[t], mu);
        acc2 = __fmaf_rn(d, d, acc2);
      }
    }
  return finish_moments(mu, tree32(acc2), len);
}

__device__ __forceinline__ float znorm_value(float x, float mu, float rsig) {
  return __fmul_rn(__fsub_rn(x, mu), rsig);
}

// Canonical PAA of segment j from z values in memory: groups of 4 consecutive points
// summed in order, groups combined by a pairwise tree in group order when the
// segment length is 4 * 2^m; a sequential sum otherwise; then divided by s.
__device__ __forceinline__ float paa_segment_generic(const float* z, int j, int s) {
  const float* seg = z + j * s;
  float sum;
  const int g = s >> 2;
  if ((s & 3) == 0 && (g & (g - 1)) == 0) {
    // pairwise tree over the group sums, as a binary-counter stack
    float stack[16];
    int level[16];
    int top = 0;
    for (int i = 0; i < g; ++i) {
      float v = __fadd_rn(__fadd_rn(__fadd_rn(seg[4 * i], seg[4 * i + 1]), seg[4 * i + 2]), seg[4 * i + 3]);
      int lv = 0;
      while (top > 0 && level[top - 1] == lv) {
        v = __fadd_rn(stack[top - 1], v);
        --top;
        ++lv;
      }
      stack[top] = v;
      level[top] = lv;
      ++top;
    }
    sum = stack[0];
  } else {
    sum = seg[0];
    for (int t = 1; t < s; ++t) sum = __fadd_rn(sum, seg[t]);
  }
  return __fdiv_rn(sum, (float)s);
}

// SAX symbol: number of thresholds t_1..t_{card-1} at or below p (thr_up[1..card-1]).
__device__ __forceinline__ int sax_symbol(const float* thr_up_s, int card, float p) {
  int lo = 1, hi = card;  // answer sym = (first index v in [1, card) with thr_up[v] > p) - 1
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (thr_up_s[mid] <= p) lo = mid + 1; else hi = mid;
  }
  return lo - 1;
}

// Interleaved key of a word from one symbol per lane (lanes j < w hold sym_j): bit
// planes from the most significant, each plane listing segment 0 first; the first
// 64 bits, left aligned.
__device__ __forceinline__ unsigned long long interleave_key(int sym, int w, int bits) {
  const int lane = threadIdx.x & 31;
  unsigned long long key = 0;
  int used = 0;
  for (int p = bits - 1; p >= 0 && used < 64; --p) {
    const unsigned m = __ballot_sync(kFull, lane < w && ((sym >> p) & 1));
    const unsigned rev = __brev(m) >> (32 - w);  // segment 0 in the top bit of w
    const int take = (64 - used) < w ? (64 - used) : w;
    key = (key << take) | (unsigned long long)(rev >> (w - take));
    used += take;
  }
  return used < 64 ? key << (64 - used) : key;
}

// ------------------------------------------------------- async copies, mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for the phase of parity `parity` of barrier b, at most about `limit_ns`
// nanoseconds; false when it gave up.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* b, uint32_t parity, uint64_t limit_ns) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 63) == 63) {
      const uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > limit_ns) return false;
    }
  }
}
// One bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16),
// completing on barrier b's transaction count.
// 16-byte asynchronous copy into shared memory (global -> L2 -> shared, no L1), its
// commit group, and the wait until at most N of this thread's newest groups are pending.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}

// ------------------------------------------------------------------ margins
// The two margins of the exactness argument for series of `len` points: eps relative
// on squared distances (2^-16), tau absolute on lower bounds (1e-3 at len 256, growing
// with the square root of the length as the fp32 PAA rounding of a bound does).
inline float margin_eps() { return 1.52587890625e-05f; }
inline float margin_tau(int len) { return 1e-3f * fmaxf(1.0f, sqrtf((float)len / 256.0f)); }

// Lower-bound pruning threshold for a k-th best squared distance `thr`:
// (sqrt(thr) (1 + eps) + tau)^2, rounded up; +inf while thr is unknown.
__device__ __forceinline__ float lb_bound2(unsigned thr_bits, float eps, float tau) {
  const float thr = __uint_as_float(thr_bits);
  if (!(thr < INFINITY)) return INFINITY;
  const float b = __fadd_ru(__fmul_ru(__fsqrt_ru(thr), 1.0f + eps), tau);
  return __fmul_ru(b, b);
}
// Squared distances at or below thr (1 + eps) are kept as candidates.
__device__ __forceinline__ float keep_bound2(unsigned thr_bits, float eps) {
  const float thr = __uint_as_float(thr_bits);
  if (!(thr < INFINITY)) return INFINITY;
  return __fmul_ru(thr, 1.0f + eps);
}

}  // namespace msi

// -------------------------------------------------------------- host index
struct msi_index {
  int device = 0;
  int64_t n = 0;
  int32_t len = 0, w = 0, card = 0, bits = 0, seglen = 0, cap = 0;
  uint32_t flags = 0;
  bool data_is_z = false;
  float* data_owned = nullptr;
  const float* data = nullptr;
  uint4* words = nullptr;
  uint32_t* perm = nullptr;
  float2* stats = nullptr;
  int64_t L = 0;
  uint32_t* leaf_begin = nullptr;
  uint4* env = nullptr;
  uint4* benv = nullptr;
  uint4* henv = nullptr;  // half-block envelopes: computed from the words (build and load)
  uint64_t* leaf_key = nullptr;
  float* thr_up = nullptr;
  float* thr_lo = nullptr;
  int32_t* root_child = nullptr;  // balanced-split tree (see IndexView)
  int32_t* tree_child = nullptr;
  int8_t* tree_seg = nullptr;
  int64_t tree_nodes = 0;
  uint4* fine = nullptr;  // fine PAA (see IndexView); wf = 0: not kept
  int wf = 0, sf = 0;
  int root_bits = 0;
  float h_thr_up[257];
  float h_thr_lo[257];
  uint8_t h_sym_cells[1024];  // the build's symbol cell table (host copy, read by an async upload)
  int64_t device_bytes = 0;
  cudaStream_t own_stream = nullptr;
  // query workspace (allocated on first use): slot 0 has room for any query; the
  // slots used to run several queries at once have bounded candidate / survivor
  // lists, and a query that overflows them is run again on slot 0
  bool ws_ready = false;
  msi::QueryView qv{};
  std::vector<msi::QueryView> slots;
  // batched chain: one workspace per query of a batch (bounded lists), and their
  // views in device memory for the batch kernels
  std::vector<msi::QueryView> bws;
  msi::QueryView* bws_dev = nullptr;
  int bws_dev_cap = 0;
  bool bws_dirty = false;    // bws changed since bws_dev was written
  bool batch_chain = true;   // batched calls run the batched chain (false: the query slots)
  int batch_group = 128;     // most queries per batched launch
  int batch_share = 4;       // the batched kernels give each query 1/batch_share of a grid
  bool batch_pdl = true;     // stages of a batch overlap their launch with the previous tail
  bool batch_dense = false;  // batched chain: the tensor-core filter instead of the iSAX filters
  bool batch_order = false;  // batched chain: survivors refined in ascending bound order
  // tensor-core filter (msi_tc.cu), set up on first use: collection id -> leaf
  // position, collection-order moments, an abort flag, the collection's TMA map
  bool tc_ready = false;
  uint32_t* iperm = nullptr;
  float2* cstats = nullptr;
  int* tc_err = nullptr;
  void* tc_map = nullptr;
  int tc_grid = 0;
  int64_t tc_aborts = 0;
  std::vector<cudaStream_t> slot_streams;
  std::vector<cudaEvent_t> slot_events;
  cudaEvent_t fork_event = nullptr;
  uint32_t* ws_ovf = nullptr;   // [kQueryChunk]
  // batched calls replay one CUDA graph per (queries, k); the call's pointers go to
  // call_dev (from pinned call_host) before each replay
  struct BatchGraph {
    int64_t nq;
    int32_t k;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<BatchGraph> graphs;
  msi::CallDesc* call_dev = nullptr;
  msi::CallDesc* call_host = nullptr;
  bool use_graphs = true;
  int nslots = msi::kDefaultQuerySlots;
  int grid_share = msi::kSlotGridShare;  // batched calls: grids divided by min(nslots, this)
  int slot_cap = 0;
  int64_t overflow_reruns = 0;
  float* ws_qraw = nullptr;     // staging for host queries [kQueryChunk][len]
  int64_t* ws_ids = nullptr;    // staging for host outputs [kQueryChunk][MSI_MAX_K]
  float* ws_dists = nullptr;
  double* ws_d64 = nullptr;
  bool grids_ready = false;  // persistent grid sizes of every refinement mode
  int grid_series = 0, grid_blocks = 0, grid_rows1 = 0, grid_rowsk = 0;
  int grid_series_b = 0;  // the batched chain's series filter (its own register budget)
  int grid_dtw = 0, grid_dtw_check = 0;  // DTW refinement and FP64 re-check
  bool timing = false;
  std::vector<cudaEvent_t> events;  // refinement timing: three per query (start, after filter, end)
  double refine_ms = 0.0;
  double filter_ms = 0.0;
  int64_t refine_launches = 0;
  std::atomic<int64_t> kernel_launches{0};  // query_one runs on caller and server threads

  msi::IndexView view() const {
    msi::IndexView v;
    v.data = data;
    v.data_is_z = data_is_z ? 1 : 0;
    v.stats = stats;
    v.words = words;
    v.perm = perm;
    v.leaf_begin = leaf_begin;
    v.env = env;
    v.benv = benv;
    v.henv = henv;
    v.leaf_key = leaf_key;
    v.thr_up = thr_up;
    v.thr_lo = thr_lo;
    v.root_child = root_child;
    v.tree_child = tree_child;
    v.tree_seg = tree_seg;
    v.root_bits = root_bits;
    v.fine = fine;
    v.wf = wf;
    v.sf = sf;
    v.n = n;
    v.L = L;
    v.len = len;
    v.w = w;
    v.card = card;
    v.bits = bits;
    v.seglen = seglen;
    return v;
  }
};

namespace msi {
constexpr int kQueryChunk = 1024;

// Build pipeline (msi_build.cu). All device pointers; stream-ordered.
cudaError_t build_index(msi_index* ix, const float* src_dev, bool in_place, cudaStream_t s,
                        int64_t* first_bad, const char** stage);
// Block and half-block envelopes of the leaf-order words (ix->words, ix->benv,
// ix->henv allocated); enqueued on s.
cudaError_t block_envelopes_of(msi_index* ix, cudaStream_t s);

// Query pipeline (msi_query.cu).
cudaError_t query_setup(msi_index* ix);
cudaError_t slots_setup(msi_index* ix);
// items_cap: work items (and 16x that many half-block tasks) a query may list; 0: room
// for any query. A query that needs more is flagged as overflowed and run again.
// blks_cap: half-block tasks (0: 16 per work item).
cudaError_t alloc_workspace(const msi_index* ix, QueryView& qv, uint32_t cand_cap, uint32_t surv_cap,
                            int64_t* bytes, uint32_t items_cap = 0, uint32_t blks_cap = 0);
void slot_capacities(const msi_index* ix, int64_t requested, uint32_t* cand_cap, uint32_t* surv_cap);
int64_t workspace_bytes(const msi_index* ix, uint32_t cand_cap, uint32_t surv_cap, uint32_t items_cap = 0,
                        uint32_t blks_cap = 0);
void free_workspace(QueryView& qv);
// window < 0: Euclidean distance; window >= 0: DTW with that Sakoe-Chiba half-width.
// call != nullptr: q_dev / ids_dev / dists_dev / d64_dev are ignored and query qi of
// the call descriptor is searched instead (Euclidean only).
cudaError_t query_one(msi_index* ix, const QueryView& ws, int share, const float* q_dev, int k, int64_t* ids_dev,
                      float* dists_dev, double* d64_dev, uint32_t* ovf, cudaStream_t s, cudaEvent_t ev_a,
                      cudaEvent_t ev_m, cudaEvent_t ev_b, int window = -1, const CallDesc* call = nullptr,
                      int qi = 0);
// Persistent grid sizes of the query kernels, computed once per index.
cudaError_t grids_setup(msi_index* ix);
// Batched chain (msi_query.cu): workspaces for ix->batch_group queries; then one launch
// per stage for `count` queries of the call descriptor, queries qbase .. qbase+count-1
// (count <= batch_group), each flagging in ovf[i] whether its bounded lists overflowed.
cudaError_t batch_setup(msi_index* ix);
void batch_release(msi_index* ix, int keep);
// Tensor-core filter (msi_tc.cu): queries per pass for series of `len` points (0: not
// available), one-time set-up, release, and one pass over the collection for queries
// q0 .. q0+nq-1 of a batch (nq <= the pass size).
int tc_queries_per_pass(int len);
cudaError_t tc_setup(msi_index* ix);
void tc_free(msi_index* ix);
cudaError_t tc_filter(msi_index* ix, const QueryView* qvs_dev, int q0, int nq, cudaStream_t s);
// ev_a / ev_m / ev_b, when given, bracket the series filter and the row kernel.
cudaError_t query_batch(msi_index* ix, int count, int k, const CallDesc* call, int qbase, uint32_t* ovf,
                        cudaStream_t s, cudaEvent_t ev_a, cudaEvent_t ev_m, cudaEvent_t ev_b);
cudaError_t export_z(msi_index* ix, float* z_dev, cudaStream_t s);
cudaError_t lower_bounds(msi_index* ix, const float* q_dev, float* series_lb_dev, float* leaf_lb_dev,
                         cudaStream_t s);
// Sets the calling thread's msi_last_error() text (msi_api.cu).
void set_last_error(const char* what);
// Frees an index and all its device memory (msi_api.cu).
void destroy_index(msi_index* ix);
// Region edge tables of a cardinality: up[v] = smallest float >= beta_v, lo[v] =
// largest float <= beta_v, v = 0..card (msi_api.cu).
void breakpoint_edges(int card, float* up, float* lo);
cudaError_t lower_bounds_on(const msi_index* ix, const QueryView& qv, const float* q_dev, float* series_lb_dev,
                            float* leaf_lb_dev, cudaStream_t s);
}  // namespace msi
