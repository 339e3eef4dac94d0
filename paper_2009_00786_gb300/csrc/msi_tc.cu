// msi_tc.cu -- the dense filter of a batched search on the tensor cores (sm_103a).
//
// The paper prunes with iSAX lower bounds and reads a series only when its bound
// passes (Section III-B, Algorithms 7-9). On collections where those bounds prune
// little, a batch of queries is served better by one streaming pass over the whole
// collection that bounds every (series, query) pair from the dot products of the
// contraction D = |z|^2 + |q|^2 - 2 z.q, computed for a tile of 128 series against up
// to 128 queries per tensor-core instruction sequence. The tensor cores compute only
// a filter: x.q is taken in TF32 with fp32 accumulation, and a certified bound on its
// error turns the estimate into a lower bound of D; pairs whose lower bound passes the
// query's threshold become survivors whose distances are computed in fp32 by the row
// kernel and re-checked in FP64 at the k-th boundary, as every other candidate is.
//
// Kernel shape (one CTA per SM, persistent over 128-series tiles):
//   warp 0      TMA producer: each tile's rows, one 128-byte-wide k-block of 32 points
//               per stage, straight from the fp32 collection (raw or z-normalised)
//               into shared memory in the 128-byte-swizzled K-major layout;
//   warp 1      TMEM allocation and the MMA issuer (one thread): per tile, len / 8
//               tcgen05.mma.kind::tf32 instructions (M = 128 series, N = the queries,
//               K = 8) into one of two TMEM accumulators;
//   warps 2-17  epilogue: each thread owns one series (TMEM lane) and a quarter of the
//               queries (columns), reads those dot products with tcgen05.ld, forms the
//               bounds and appends survivors; four warps per scheduler hide the
//               latency of each warp's dependent arithmetic.
// The queries (z-normalised, fp32, zero padded) stay in shared memory for the whole
// kernel in the same swizzled layout. Every wait is bounded: a wait that runs out
// (about a second) raises the CTA's abort flag, every role leaves its loop, copies
// and MMAs in flight are waited for (again bounded) and TMEM is freed; the host then
// runs the affected queries again on the pruned path.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "msi_internal.cuh"

namespace msi {
namespace {

constexpr int kEpiWarps = 16;       // 4 per TMEM lane quarter, each a quarter of the columns
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTcThreads = 64 + kEpiThreads;  // producer, MMA, epilogue
constexpr int kTileRows = 128;      // UMMA M
constexpr int kStages = 5;          // k-blocks of the row tile in flight
constexpr int kKb = 32;             // points per k-block (128 bytes of fp32)
constexpr int kStageBytes = kTileRows * 128;
constexpr uint64_t kWaitNs = 1000000000ull;  // one second

// Waits for the phase of parity `parity` of barrier b to complete; false when the
// CTA's abort flag is (or becomes) set, or after about a second (which sets it).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 63) == 63) {
      if (*abort_flag) return false;
      const uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitNs) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled
// layout: rows of 128 bytes, 8-row atoms 1024 bytes apart (the stride dimension
// offset); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: D fp32, A and B TF32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileRows >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Barrier 1 over the epilogue threads, returning whether any of them passed
// `pred` (so that all four warps take the same decision).
__device__ __forceinline__ bool epilogue_any(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(kEpiThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 4 / 8 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
  const QueryView* __restrict__ qvs;  // the batch's query views
  int q0, nq;                         // queries q0 .. q0 + nq - 1 of the batch (nq <= N)
  const uint32_t* __restrict__ iperm; // [n] collection id -> leaf-order position
  const float2* __restrict__ cstats;  // [n] collection order (mu, 1/sigma)
  int64_t ntiles;
  int kblocks;                        // ceil(len / 32)
  int* err;                           // set when a CTA gave up on a wait
  unsigned long long* pairs;          // (series, query) pairs bounded (a device counter)
};

// Certified lower bound of D = |z|^2 + |q|^2 - 2 z.q from the TF32 dot product p~ of
// the stored row x (raw: z = (x - mu) rsig; or z itself, then mu = 0, rsig = 1) and
// the fp32 query q (|q|^2 = qq, sum q = S, |q| <= qn):
//   z.q = rsig (x.q - mu S);  |x| <= sqrt(len (mu^2 + sigma^2)) (population moments);
//   |p~ - x.q| <= 2^-8 |x| |q| covers both operands rounded (or truncated) to TF32's
//   10 fraction bits (2 * 2^-10 relative, plus its square) and the fp32 accumulation
//   of len terms (len 2^-22 relative at most), with a factor of two to spare;
//   |z|^2 is len for a non-constant series (0 for a constant one) within len 2^-14.
// The bound's own fp32 evaluation (a few round-to-nearest operations on values of at
// most 4 len) is covered by the absolute term len 2^-14 + 1e-3 and the 2^-19 terms.
// Rearranged per pair: lb = (|z|^2 - c0) + qq + a mu S - a x.q - b |q| - c |S|, with
// a = 2 rsig, b = 2 rsig (2^-8 + 2^-19) |x|, c = 2 rsig 2^-19 |mu|, c0 = len 2^-14 + 1e-3:
// four fused multiply-adds against per-query constants {S, |S|, |q|, bound - qq}.
constexpr float kTf32Rel = 0.00390625f + 1.9073486e-6f;  // 2^-8 + 2^-19
constexpr float kFp32Rel = 1.9073486e-6f;                  // 2^-19

template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
q_tc_filter(const __grid_constant__ CUtensorMap tmap, IndexView ix, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the operand tiles (the swizzle atoms)
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int kb_count = a.kblocks;
  unsigned char* Qs = smem;                                   // [kblocks][N rows x 128 B]
  unsigned char* As = Qs + (size_t)kb_count * N * 128;        // [kStages][128 rows x 128 B]
  __shared__ __align__(8) uint64_t full_bar[kStages], empty_bar[kStages], tfull_bar[2], tempty_bar[2], done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;
  __shared__ float qq_s[N], S_s[N], qn_s[N];
  __shared__ float4 qc_s[N];  // per query: S, |S|, |q|, this tile's bound - |q|^2
  __shared__ uint32_t sa_s[N], sb_s[N];
  __shared__ QState* st_s[N];
  __shared__ uint2* surv_s[N];
  __shared__ uint32_t cap_s[N];
  __shared__ float eps_s, tau_s;
  __shared__ int k_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  volatile int* abort_flag = &abort_s;

  // ---- queries into shared memory (swizzled K-major), their norms and sums
  if (tid == 0) abort_s = 0;
  for (int j = warp; j < N; j += kTcThreads / 32) {
    const bool have = j < a.nq;
    const QueryView* qv = have ? &a.qvs[a.q0 + j] : nullptr;
    const float* qz = have ? qv->qz : nullptr;
    double sq = 0.0, sm = 0.0;
    for (int t = lane; t < kb_count * kKb; t += 32) {
      const float v = (have && t < ix.len) ? qz[t] : 0.0f;
      sq += (double)v * (double)v;
      sm += (double)v;
      const int kb = t / kKb, c = (t % kKb) * 4;
      const int chunk = c >> 4, r8 = j & 7;
      unsigned char* dst = Qs + (size_t)kb * N * 128 + (size_t)(j >> 3) * 1024 + r8 * 128 + ((chunk ^ r8) << 4) + (c & 15);
      *reinterpret_cast<float*>(dst) = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sq += __shfl_xor_sync(kFull, sq, o);
      sm += __shfl_xor_sync(kFull, sm, o);
    }
    if (lane == 0) {
      qq_s[j] = (float)sq;
      S_s[j] = (float)sm;
      qn_s[j] = __fsqrt_ru(__fmul_ru((float)sq, 1.0f + 1e-6f));
      if (have) {
        QState* st = qv->st;
        st_s[j] = st;
        surv_s[j] = qv->surv;
        cap_s[j] = qv->surv_cap;
        sa_s[j] = st->seed_a;
        sb_s[j] = st->seed_b;
        if (j == 0) {
          eps_s = qv->eps;
          tau_s = qv->tau;
          k_s = qv->k;
        }
      } else {
        st_s[j] = nullptr;
        surv_s[j] = nullptr;
        cap_s[j] = 0;
        sa_s[j] = sb_s[j] = 0;
      }
    }
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], kEpiThreads);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the queries, for the tensor cores
  constexpr uint32_t kCols = 2 * N < 32 ? 32 : 2 * N;           // two accumulators of N columns
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = tf32_idesc(N);

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0, inflight = 0;
      for (int64_t t = blockIdx.x; t < a.ntiles && !*abort_flag; t += gridDim.x) {
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (!mbar_wait(&empty_bar[s], ph ^ 1, abort_flag)) break;
          mbar_expect_tx(&full_bar[s], kStageBytes);
          tma_load_2d(As + (size_t)s * kStageBytes, &tmap, kb * kKb, (int)(t * kTileRows), &full_bar[s]);
          inflight = it + 1;
        }
      }
      // on abort: wait (bounded) for the copies issued and not consumed, so that
      // none writes shared memory after the CTA has left
      if (*abort_flag) {
        const uint64_t t0 = global_ns();
        for (uint32_t j = inflight > kStages ? inflight - kStages : 0; j < inflight; ++j)
          while (!mbar_try(&full_bar[j % kStages], (j / kStages) & 1) && global_ns() - t0 < kWaitNs) {
          }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, local = 0;
      bool issued = false;
      for (int64_t t = blockIdx.x; t < a.ntiles && !*abort_flag; t += gridDim.x, ++local) {
        const uint32_t acc = local & 1, aph = (local >> 1) & 1;
        if (!mbar_wait(&tempty_bar[acc], aph ^ 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t d = tmem + acc * N;
        bool ok = true;
        for (int kb = 0; kb < kb_count; ++kb, ++it) {
          const int s = it % kStages;
          if (!mbar_wait(&full_bar[s], (it / kStages) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(As + (size_t)s * kStageBytes);
          const uint32_t b_base = smem_u32(Qs + (size_t)kb * N * 128);
#pragma unroll
          for (int kk = 0; kk < kKb / 8; ++kk)
            mma_tf32(d, sw128_desc(a_base + kk * 32), sw128_desc(b_base + kk * 32), idesc, (kb | kk) ? 1u : 0u);
          mma_commit(&empty_bar[s]);  // the stage is free once these MMAs have read it
          issued = true;
        }
        if (!ok) break;
        mma_commit(&tfull_bar[acc]);
      }
      // every MMA issued has completed before TMEM is freed
      if (issued) {
        mma_commit(&done_bar);
        const uint64_t t0 = global_ns();
        while (!mbar_try(&done_bar, 0) && global_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else {
    // ---------------------------------------------------------- epilogue
    const int g = warp & 3;            // TMEM lanes 32 g .. 32 g + 31 (the warp's quarter)
    constexpr int CW = N / 4;          // columns (queries) per epilogue warp
    const int col0 = ((warp - 2) >> 2) * CW;
    const int er = tid - 64;           // 0 .. kEpiThreads - 1: epilogue thread index
    const int row = g * 32 + lane;
    const float len = (float)ix.len;
    const float eps = eps_s, tau = tau_s;
    const int k = k_s;
    const float c0 = __fmaf_ru(len, 6.1035156e-5f, 1e-3f);
    const int my_q = max(0, min(a.nq, col0 + CW) - col0);  // real queries among this thread's columns
    unsigned long long pairs = 0;
    uint32_t local = 0;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++local) {
      // this tile's pruning bounds, from each query's current k-th best (the barrier
      // first: every thread is done with the previous tile's)
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory");
      if (er < N) {
        QState* st = st_s[er];
        const float lbb = st ? lb_bound2(*(volatile unsigned*)&st->thr_bits, eps, tau) : -INFINITY;
        qc_s[er] = make_float4(S_s[er], fabsf(S_s[er]), qn_s[er], lbb - qq_s[er]);
      }
      const uint32_t acc = local & 1, aph = (local >> 1) & 1;
      const bool ready = mbar_wait(&tfull_bar[acc], aph, abort_flag);
      // one decision for all epilogue warps (and the bounds above become visible)
      if (epilogue_any(!ready)) break;
      tc_fence_after();
      const int64_t id = t * kTileRows + row;
      const bool valid = id < ix.n;
      // the row's terms (a row past the end never passes)
      float am = 0.f, a2 = 0.f, b = 0.f, c = 0.f, base = INFINITY;
      uint32_t pos = 0;
      if (valid) {
        const float2 ms = __ldg(&a.cstats[id]);
        pos = __ldg(&a.iperm[id]);
        base = -c0;  // |z|^2 - c0, |z|^2 = 0 for a constant series (z = 0)
        if (ms.y > 0.0f) {
          const float mu = ix.data_is_z ? 0.0f : ms.x, rsig = ix.data_is_z ? 1.0f : ms.y;
          const float sig = ix.data_is_z ? 1.0f : __frcp_ru(ms.y);
          const float xn = __fmul_ru(__fsqrt_ru(__fmul_ru(len, __fmaf_ru(mu, mu, __fmul_ru(sig, sig)))), 1.0001f);
          a2 = 2.0f * rsig;
          am = a2 * mu;
          b = __fmul_ru(__fmul_ru(a2, kTf32Rel), xn);
          c = __fmul_ru(__fmul_ru(a2, kFp32Rel), fabsf(mu));
          base = len - c0;
        }
        pairs += (unsigned long long)my_q;
      }
      float v[CW];
      const uint32_t taddr = tmem + ((uint32_t)(g * 32) << 16) + acc * N + col0;
      if constexpr (CW == 32) tmem_ld32(taddr, v);
      else if constexpr (CW == 16) tmem_ld16(taddr, v);
      else if constexpr (CW == 8) tmem_ld8(taddr, v);
      else tmem_ld4(taddr, v);
      // the pairs whose bound passes, as a bit mask (no branch per pair); slots past
      // nq carry a bound of -inf and never pass
      uint32_t keep = 0;
#pragma unroll
      for (int i = 0; i < CW; ++i) {
        const float4 q = qc_s[col0 + i];  // S, |S|, |q|, bound - qq
        float tt = __fmaf_rn(am, q.x, base);
        tt = __fmaf_rn(-c, q.y, tt);
        tt = __fmaf_rn(-b, q.z, tt);
        tt = __fmaf_rn(-a2, v[i], tt);  // lb - qq
        keep |= (tt <= q.w ? 1u : 0u) << i;
        v[i] = tt;
      }
      tc_fence_before();
      mbar_arrive(&tempty_bar[acc]);  // the accumulator is free: the values are in registers
      // the rare survivors (one warp-wide test; the loop indexes v statically)
      if (__any_sync(kFull, keep != 0)) {
#pragma unroll
        for (int i = 0; i < CW; ++i) {
          const int j = col0 + i;
          if (!((keep >> i) & 1u) || (pos >= sa_s[j] && pos < sb_s[j])) continue;  // seed rows: candidates already
          const float lbq = v[i] + qq_s[j];
          const float lb = fmaxf(0.0f, lbq);
          QState* st = st_s[j];
          const uint32_t slot = atomicAdd(&st->surv_count, 1u);
          if (slot < cap_s[j]) surv_s[j][slot] = make_uint2(pos, __float_as_uint(lb));
          else st->overflow = 1u;
          if (k == 1) {  // the pair's upper bound, lb + 2 (margin), bounds the 1-NN distance
            const float4 q = qc_s[j];
            const float m = __fmaf_ru(b, q.z, __fmaf_ru(c, q.y, c0));
            const float ub = __fmul_ru(__fadd_ru(lbq, __fmul_ru(2.0f, m)), 1.0f + 2.4e-7f);
            atomicMin(&st->thr_bits, __float_as_uint(fmaxf(ub, 0.0f)));
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(kFull, pairs, o);
    if (lane == 0 && pairs) atomicAdd(a.pairs, pairs);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
  if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
}

// id -> leaf position and collection-order moments, for the dense filter
__global__ void tc_inverse(IndexView ix, uint32_t* __restrict__ iperm, float2* __restrict__ cstats) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < ix.n; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t id = ix.perm[p];
    iperm[id] = (uint32_t)p;
    cstats[id] = ix.stats[p];
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <int N>
size_t tc_smem(int kblocks) {
  return 1024 + (size_t)kblocks * N * 128 + (size_t)kStages * kStageBytes;
}

template <int N>
cudaError_t launch_tc(const CUtensorMap& map, const IndexView& v, const TcArgs& a, int grid, cudaStream_t s) {
  q_tc_filter<N><<<grid, kTcThreads, tc_smem<N>(a.kblocks), s>>>(map, v, a);
  return cudaGetLastError();
}

template <int N>
cudaError_t tc_attr(int kblocks) {
  return cudaFuncSetAttribute(q_tc_filter<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<N>(kblocks));
}

}  // namespace

// Queries per pass of the dense filter for series of `len` points: the largest of
// 128, 64, 32, 16 whose fp32 queries fit 128 KB of shared memory; 0 when the filter
// cannot run (len not a multiple of 4, the row pitch TMA needs, or too long).
int tc_queries_per_pass(int len) {
  if (len % 4 != 0) return 0;
  const int kb = (len + kKb - 1) / kKb;
  for (int n = 128; n >= 16; n >>= 1)
    if ((size_t)kb * n * 128 <= (size_t)128 * 1024) return n;
  return 0;
}

cudaError_t tc_setup(msi_index* ix) {
  if (ix->tc_ready) return cudaSuccess;
  cudaError_t e;
  if (!encode_fn() || tc_queries_per_pass(ix->len) == 0 || ix->n > 0x7fffff00LL) return cudaErrorNotSupported;
  if ((e = cudaMalloc(&ix->iperm, sizeof(uint32_t) * (size_t)ix->n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ix->cstats, sizeof(float2) * (size_t)ix->n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ix->tc_err, sizeof(int))) != cudaSuccess) return e;
  ix->device_bytes += (int64_t)ix->n * 12;
  tc_inverse<<<2048, 256, 0, ix->own_stream>>>(ix->view(), ix->iperm, ix->cstats);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ix->tc_err, 0, sizeof(int), ix->own_stream)) != cudaSuccess) return e;
  // the collection as a 2-D fp32 tensor [n][len]: boxes of 32 points x 128 series,
  // 128-byte swizzle, zero fill beyond either edge
  CUtensorMap* map = new CUtensorMap;
  const cuuint64_t dims[2] = {(cuuint64_t)ix->len, (cuuint64_t)ix->n};
  const cuuint64_t strides[1] = {(cuuint64_t)ix->len * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKb, (cuuint32_t)kTileRows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ix->data), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    delete map;
    return cudaErrorInvalidValue;
  }
  ix->tc_map = map;
  if ((e = cudaStreamSynchronize(ix->own_stream)) != cudaSuccess) return e;
  // the shared memory of every accumulator width a pass of this length can use
  const int kb = (ix->len + kKb - 1) / kKb, per = tc_queries_per_pass(ix->len);
  if ((e = tc_attr<16>(kb)) != cudaSuccess || (per >= 32 && (e = tc_attr<32>(kb)) != cudaSuccess) ||
      (per >= 64 && (e = tc_attr<64>(kb)) != cudaSuccess) || (per >= 128 && (e = tc_attr<128>(kb)) != cudaSuccess))
    return e;
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix->device)) != cudaSuccess) return e;
  ix->tc_grid = sms;
  ix->tc_ready = true;
  return cudaSuccess;
}

void tc_free(msi_index* ix) {
  if (ix->iperm) cudaFree(ix->iperm);
  if (ix->cstats) cudaFree(ix->cstats);
  if (ix->tc_err) cudaFree(ix->tc_err);
  delete static_cast<CUtensorMap*>(ix->tc_map);
  ix->iperm = nullptr;
  ix->cstats = nullptr;
  ix->tc_err = nullptr;
  ix->tc_map = nullptr;
  ix->tc_ready = false;
}

cudaError_t tc_filter(msi_index* ix, const QueryView* qvs_dev, int q0, int nq, cudaStream_t s) {
  const int per = tc_queries_per_pass(ix->len);
  if (!ix->tc_ready || per == 0 || nq < 1 || nq > per) return cudaErrorInvalidValue;
  TcArgs a;
  a.qvs = qvs_dev;
  a.q0 = q0;
  a.nq = nq;
  a.iperm = ix->iperm;
  a.cstats = ix->cstats;
  a.ntiles = (ix->n + kTileRows - 1) / kTileRows;
  a.kblocks = (ix->len + kKb - 1) / kKb;
  a.err = ix->tc_err;
  a.pairs = ix->qv.counters + ST_TC_PAIRS;
  const IndexView v = ix->view();
  const CUtensorMap& map = *static_cast<const CUtensorMap*>(ix->tc_map);
  const int grid = (int)std::min<int64_t>(ix->tc_grid, a.ntiles);
  // the narrowest accumulator that holds the pass's queries
  if (nq <= 16) return launch_tc<16>(map, v, a, grid, s);
  if (nq <= 32) return launch_tc<32>(map, v, a, grid, s);
  if (nq <= 64) return launch_tc<64>(map, v, a, grid, s);
  return launch_tc<128>(map, v, a, grid, s);
}

}  // namespace msi
