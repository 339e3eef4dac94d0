// msi_api.cu -- the C ABI of include/msi.h: argument checks, device memory,
// streams, the breakpoint tables, and the order in which the build and query
// kernels run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "msi_internal.cuh"

namespace {

thread_local std::string g_err;

msi_status fail(msi_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
msi_status fail(msi_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

msi_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error for the next call
  if (e == cudaErrorMemoryAllocation) return fail(MSI_ENOMEM, "%s: out of device memory", what);
  return fail(MSI_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Is `p` device memory of `device`? Host memory (pinned or pageable) answers false.
bool is_device_ptr(const void* p, int device, bool* other_device) {
  *other_device = false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    if (a.device != device) *other_device = true;
    return true;
  }
  return false;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------- breakpoints
// beta = Phi^{-1}(p) by Newton's method on Phi(x) - p, with Phi(x) = erfc(-x/sqrt 2)/2
// and Phi'(x) = exp(-x^2/2)/sqrt(2 pi), started from the logistic approximation
// x0 = (sqrt 3 / pi) ln(p / (1 - p)).
double normal_quantile(double p) {
  const double kPi = 3.14159265358979323846;
  double x = std::sqrt(3.0) / kPi * std::log(p / (1.0 - p));
  for (int it = 0; it < 100; ++it) {
    const double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
    const double d = std::exp(-0.5 * x * x) / std::sqrt(2.0 * kPi);
    const double step = f / d;
    x -= step;
    if (std::fabs(step) <= 1e-17 * std::fmax(1.0, std::fabs(x))) break;
  }
  return x;
}

// Region edges for cardinality c: up[v] = smallest float >= beta_v (the SAX decision
// thresholds), lo[v] = largest float <= beta_v; v = 0 and v = c are -inf / +inf.
void region_edges(int c, float* up, float* lo) {
  up[0] = lo[0] = -INFINITY;
  up[c] = lo[c] = INFINITY;
  for (int v = 1; v < c; ++v) {
    const double b = (2 * v == c) ? 0.0 : normal_quantile((double)v / (double)c);
    float f = (float)b;
    while ((double)f < b) f = std::nextafter(f, INFINITY);
    while ((double)std::nextafter(f, -INFINITY) >= b) f = std::nextafter(f, -INFINITY);
    up[v] = f;
    float g = (float)b;
    while ((double)g > b) g = std::nextafter(g, -INFINITY);
    while ((double)std::nextafter(g, INFINITY) <= b) g = std::nextafter(g, INFINITY);
    lo[v] = g;
  }
}

void free_index(msi_index* ix) {
  if (!ix) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != ix->device) cudaSetDevice(ix->device);
  void* ptrs[] = {ix->data_owned, ix->words,     ix->perm,         ix->stats,   ix->leaf_begin, ix->env,
                  ix->benv,       ix->leaf_key,  ix->thr_up,       ix->thr_lo,  ix->qv.counters, ix->ws_qraw,
                  ix->ws_ids,     ix->ws_dists,  ix->ws_ovf,       ix->ws_d64,  ix->root_child,  ix->tree_child,
                  ix->tree_seg,   ix->fine,      ix->henv};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  msi::free_workspace(ix->qv);
  for (auto& qv : ix->slots) msi::free_workspace(qv);
  for (auto& qv : ix->bws) msi::free_workspace(qv);
  msi::tc_free(ix);
  if (ix->bws_dev) cudaFree(ix->bws_dev);
  for (cudaStream_t st : ix->slot_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : ix->slot_events) cudaEventDestroy(ev);
  if (ix->fork_event) cudaEventDestroy(ix->fork_event);
  for (auto& g : ix->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (ix->call_dev) cudaFree(ix->call_dev);
  if (ix->call_host) cudaFreeHost(ix->call_host);
  for (cudaEvent_t ev : ix->events)
    if (ev) cudaEventDestroy(ev);
  if (ix->own_stream) cudaStreamDestroy(ix->own_stream);
  if (cur >= 0 && cur != ix->device) cudaSetDevice(cur);
  delete ix;
}

}  // namespace

namespace msi {
void set_last_error(const char* what) { g_err = what; }
void destroy_index(msi_index* ix) { free_index(ix); }
void breakpoint_edges(int card, float* up, float* lo) { region_edges(card, up, lo); }
}  // namespace msi

extern "C" {

int32_t msi_abi_version(void) { return MSI_ABI_VERSION; }

const char* msi_status_str(msi_status s) {
  switch (s) {
    case MSI_OK: return "MSI_OK";
    case MSI_EINVAL: return "MSI_EINVAL";
    case MSI_ENOMEM: return "MSI_ENOMEM";
    case MSI_ECUDA: return "MSI_ECUDA";
    case MSI_ETIMEOUT: return "MSI_ETIMEOUT";
    case MSI_EINTERNAL: return "MSI_EINTERNAL";
  }
  return "MSI_UNKNOWN";
}

const char* msi_last_error(void) { return g_err.c_str(); }

msi_status msi_build(const float* series, int64_t n, int32_t len, int32_t segments, int32_t cardinality,
                     const msi_build_opts* opts, msi_index** out) {
  g_err.clear();
  if (!out) return fail(MSI_EINVAL, "out is NULL");
  *out = nullptr;
  if (!series) return fail(MSI_EINVAL, "series is NULL");
  if (n < 1 || n > 0xfffffffeLL) return fail(MSI_EINVAL, "n = %lld outside [1, 2^32-2]", (long long)n);
  if (len < 1 || len > MSI_MAX_LEN) return fail(MSI_EINVAL, "len = %d outside [1, %d]", len, MSI_MAX_LEN);
  if (segments < 1 || segments > MSI_MAX_SEGMENTS)
    return fail(MSI_EINVAL, "segments = %d outside [1, %d]", segments, MSI_MAX_SEGMENTS);
  if (len % segments != 0) return fail(MSI_EINVAL, "len = %d is not a multiple of segments = %d", len, segments);
  if (cardinality < 2 || cardinality > MSI_MAX_CARDINALITY || (cardinality & (cardinality - 1)))
    return fail(MSI_EINVAL, "cardinality = %d is not a power of two in [2, 256]", cardinality);
  const int32_t cap = (opts && opts->leaf_capacity) ? opts->leaf_capacity : MSI_DEFAULT_LEAF_CAPACITY;
  if (cap < 1 || cap > (1 << 24)) return fail(MSI_EINVAL, "leaf_capacity = %d outside [1, 2^24]", cap);
  const uint32_t flags = opts ? opts->flags : 0u;
  if (flags & ~(MSI_BUILD_BORROW | MSI_BUILD_BALANCED_SPLIT | MSI_BUILD_NO_FINE_BOUND)) return fail(MSI_EINVAL, "unknown build flags 0x%x", flags);
  const int32_t slots = (opts && opts->query_slots) ? opts->query_slots : msi::kDefaultQuerySlots;
  if (slots < 1 || slots > 64) return fail(MSI_EINVAL, "query_slots = %d outside [1, 64]", slots);
  const int32_t slot_cap = opts ? opts->slot_capacity : 0;
  if (slot_cap < 0) return fail(MSI_EINVAL, "slot_capacity = %d is negative", slot_cap);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
  bool other = false;
  const bool on_dev = is_device_ptr(series, dev, &other);
  if (other) return fail(MSI_EINVAL, "series lives on another device than the current one (%d)", dev);
  if ((flags & MSI_BUILD_BORROW) && !on_dev) return fail(MSI_EINVAL, "MSI_BUILD_BORROW needs device memory");
  // kernels read rows with 16-byte vector loads
  const bool aligned = ((uintptr_t)series & 15u) == 0;
  if ((flags & MSI_BUILD_BORROW) && !aligned)
    return fail(MSI_EINVAL, "a borrowed collection must start on a 16-byte boundary");

  msi_index* ix = new msi_index();
  ix->device = dev;
  ix->n = n;
  ix->len = len;
  ix->w = segments;
  ix->card = cardinality;
  ix->bits = 0;
  while ((1 << ix->bits) < cardinality) ++ix->bits;
  ix->seglen = len / segments;
  ix->cap = cap;
  ix->flags = flags;
  ix->nslots = slots;
  ix->slot_cap = slot_cap;
  region_edges(cardinality, ix->h_thr_up, ix->h_thr_lo);

  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  if ((e = cudaStreamCreateWithFlags(&ix->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    free_index(ix);
    return cuda_fail(e, "creating the index stream");
  }
  if (!s) s = ix->own_stream;
  const size_t tb = sizeof(float) * (size_t)(cardinality + 1);
  if ((e = cudaMalloc(&ix->thr_up, tb)) != cudaSuccess || (e = cudaMalloc(&ix->thr_lo, tb)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ix->thr_up, ix->h_thr_up, tb, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ix->thr_lo, ix->h_thr_lo, tb, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    free_index(ix);
    return cuda_fail(e, "uploading breakpoint tables");
  }
  const size_t data_bytes = sizeof(float) * (size_t)n * len;
  const float* src = series;
  bool in_place = false;
  if (flags & MSI_BUILD_BORROW) {
    ix->data = series;
    ix->data_is_z = false;
  } else {
    if ((e = cudaMalloc(&ix->data_owned, data_bytes)) != cudaSuccess) {
      free_index(ix);
      return cuda_fail(e, "allocating the collection copy");
    }
    ix->device_bytes += (int64_t)data_bytes;
    ix->data = ix->data_owned;
    ix->data_is_z = true;
    if (!on_dev || !aligned) {
      if ((e = cudaMemcpyAsync(ix->data_owned, series, data_bytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               s)) != cudaSuccess) {
        free_index(ix);
        return cuda_fail(e, "copying the collection to the device");
      }
      src = ix->data_owned;
      in_place = true;
    }
  }
  int64_t first_bad = -1;
  const char* stage = "build";
  e = msi::build_index(ix, src, in_place, s, &first_bad, &stage);
  if (e != cudaSuccess) {
    free_index(ix);
    return cuda_fail(e, stage);
  }
  if (first_bad >= 0) {
    free_index(ix);
    return fail(MSI_EINVAL, "series %lld holds NaN or infinity (or its moments overflow)", (long long)first_bad);
  }
  *out = ix;
  return MSI_OK;
}

msi_status msi_knn(msi_index* ix, const float* queries, int64_t nq, int32_t k, int64_t* ids, float* dists,
                   void* stream) {
  return msi_knn_ex(ix, queries, nq, k, ids, dists, nullptr, stream);
}

// window < 0: Euclidean k-NN (msi_knn_ex); window >= 0: DTW k-NN (msi_knn_dtw).
// Enqueues `cnt` Euclidean queries on the concurrent query slots (query i on slot
// i mod nslots) between a fork from and a join back into stream s. With `call`, the
// kernels take the queries and outputs from that descriptor (graph capture); else
// from the pointers given.
// With the batched chain (ix->batch_chain) the queries run in groups of at most
// batch_group queries, one launch per stage per group, and `call` must be given.
static cudaError_t enqueue_batch(msi_index* ix, cudaStream_t s, int64_t cnt, int32_t k, const float* qd,
                                 int64_t* id_base, float* d_base, double* d64_base, const msi::CallDesc* call) {
  cudaError_t e;
  if (ix->batch_chain) {
    if (!call) return cudaErrorInvalidValue;
    const int64_t G = std::max(1, ix->batch_group);
    for (int64_t g0 = 0; g0 < cnt; g0 += G)
      if ((e = msi::query_batch(ix, (int)std::min<int64_t>(G, cnt - g0), k, call, (int)g0, ix->ws_ovf + g0, s,
                                nullptr, nullptr, nullptr)) != cudaSuccess)
        return e;
    return cudaSuccess;
  }
  if ((e = cudaEventRecord(ix->fork_event, s)) != cudaSuccess) return e;
  for (int sl = 0; sl < ix->nslots; ++sl)
    if ((e = cudaStreamWaitEvent(ix->slot_streams[sl], ix->fork_event, 0)) != cudaSuccess) return e;
  const int share = std::min(ix->nslots, ix->grid_share);
  for (int64_t i = 0; i < cnt; ++i) {
    const int sl = (int)(i % ix->nslots);
    if (call)
      e = msi::query_one(ix, ix->slots[sl], share, nullptr, k, nullptr, nullptr, nullptr, ix->ws_ovf + i,
                         ix->slot_streams[sl], nullptr, nullptr, nullptr, -1, call, (int)i);
    else
      e = msi::query_one(ix, ix->slots[sl], share, qd + i * ix->len, k, id_base + i * k,
                         d_base ? d_base + i * k : nullptr, d64_base ? d64_base + i * k : nullptr, ix->ws_ovf + i,
                         ix->slot_streams[sl], nullptr, nullptr, nullptr, -1);
    if (e != cudaSuccess) return e;
  }
  for (int sl = 0; sl < ix->nslots; ++sl)
    if ((e = cudaEventRecord(ix->slot_events[sl], ix->slot_streams[sl])) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, ix->slot_events[sl], 0)) != cudaSuccess)
      return e;
  return cudaSuccess;
}

constexpr int kMaxBatchGraphs = 8;  // query shapes remembered per index

// Records enqueue_batch for `cnt` queries as a CUDA graph whose queries and outputs
// come from ix->call_dev; *launches = the kernels it holds.
static cudaError_t capture_batch(msi_index* ix, cudaStream_t s, int64_t cnt, int32_t k, cudaGraphExec_t* exec,
                                 int64_t* launches) {
  cudaError_t e;
  if (!ix->call_dev && (e = cudaMalloc(&ix->call_dev, sizeof(msi::CallDesc))) != cudaSuccess) return e;
  if (!ix->call_host && (e = cudaMallocHost(&ix->call_host, sizeof(msi::CallDesc))) != cudaSuccess) return e;
  if ((e = msi::grids_setup(ix)) != cudaSuccess) return e;
  if (ix->batch_chain && (e = msi::batch_setup(ix)) != cudaSuccess) return e;
  const int64_t before = ix->kernel_launches.load();
  if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
  const cudaError_t le = enqueue_batch(ix, s, cnt, k, nullptr, nullptr, nullptr, nullptr, ix->call_dev);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(s, &graph);
  *launches = ix->kernel_launches.load() - before;
  ix->kernel_launches -= *launches;  // counted when the graph runs
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return le != cudaSuccess ? le : e;
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e;
}

static msi_status knn_impl(msi_index* ix, const float* queries, int64_t nq, int32_t k, int32_t window, int64_t* ids,
                           float* dists, double* sqdists64, void* stream) {
  g_err.clear();
  if (!ix) return fail(MSI_EINVAL, "index is NULL");
  if (nq < 0) return fail(MSI_EINVAL, "nq = %lld is negative", (long long)nq);
  if (k < 1 || k > MSI_MAX_K || (int64_t)k > ix->n)
    return fail(MSI_EINVAL, "k = %d outside [1, min(n = %lld, %d)]", k, (long long)ix->n, MSI_MAX_K);
  if (nq == 0) return MSI_OK;
  if (!queries || !ids) return fail(MSI_EINVAL, "queries or ids is NULL");
  DeviceGuard guard(ix->device);
  bool o1 = false, o2 = false, o3 = false, o4 = false;
  const bool q_dev = is_device_ptr(queries, ix->device, &o1);
  const bool ids_dev = is_device_ptr(ids, ix->device, &o2);
  const bool d_dev = dists ? is_device_ptr(dists, ix->device, &o3) : true;
  const bool d64_dev = sqdists64 ? is_device_ptr(sqdists64, ix->device, &o4) : true;
  if (o1 || o2 || o3 || o4) return fail(MSI_EINVAL, "an argument lives on another device than the index");
  cudaError_t e = msi::query_setup(ix);
  if (e != cudaSuccess) return cuda_fail(e, "allocating the query workspace");
  cudaStream_t s = stream ? (cudaStream_t)stream : ix->own_stream;
  unsigned long long* bad_flag = ix->qv.counters + msi::ST_BAD_QUERY;
  if ((e = cudaMemsetAsync(bad_flag, 0, sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(e, "msi_knn");
  const int64_t chunk = msi::kQueryChunk;
  if (ix->timing && ix->events.size() < (size_t)(3 * chunk)) {
    while (ix->events.size() < (size_t)(3 * chunk)) {
      cudaEvent_t a;
      if ((e = cudaEventCreate(&a)) != cudaSuccess) return cuda_fail(e, "creating timing events");
      ix->events.push_back(a);
    }
  }
  const bool host_out = !ids_dev || !d_dev || !d64_dev;
  // several queries run concurrently on the query slots
  // (DTW queries use the full workspace: their survivor lists outgrow a slot's)
  // timing: the batched chain records its events around each group's series filter
  // and row kernel (launched directly, not from a graph); the slot form times queries
  // one at a time instead
  const bool batched = nq > 1 && (ix->batch_chain || (ix->nslots > 1 && !ix->timing)) && window < 0;
  int64_t timed = 0;  // entries of ix->events used by this chunk (three each)
  if (batched && !ix->batch_chain && (e = msi::slots_setup(ix)) != cudaSuccess)
    return cuda_fail(e, "allocating query slots");
  if (batched && ix->batch_chain) {
    if ((e = msi::batch_setup(ix)) != cudaSuccess) return cuda_fail(e, "allocating the batch workspaces");
    if (!ix->call_dev && (e = cudaMalloc(&ix->call_dev, sizeof(msi::CallDesc))) != cudaSuccess)
      return cuda_fail(e, "allocating the call descriptor");
    if (!ix->call_host && (e = cudaMallocHost(&ix->call_host, sizeof(msi::CallDesc))) != cudaSuccess)
      return cuda_fail(e, "allocating the call descriptor");
  }
  for (int64_t c0 = 0; c0 < nq; c0 += chunk) {
    const int64_t cnt = std::min<int64_t>(chunk, nq - c0);
    const float* qd = queries + c0 * ix->len;
    if (!q_dev) {
      if ((e = cudaMemcpyAsync(ix->ws_qraw, qd, sizeof(float) * cnt * ix->len, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(e, "copying queries to the device");
      qd = ix->ws_qraw;
    }
    int64_t* id_base = ids_dev ? ids + c0 * k : ix->ws_ids;
    float* d_base = dists ? (d_dev ? dists + c0 * k : ix->ws_dists) : nullptr;
    double* d64_base = sqdists64 ? (d64_dev ? sqdists64 + c0 * k : ix->ws_d64) : nullptr;
    timed = 0;
    if (batched && ix->timing) {  // the batched chain, group by group, with events
      *ix->call_host = msi::CallDesc{qd, id_base, d_base, d64_base};
      if ((e = cudaMemcpyAsync(ix->call_dev, ix->call_host, sizeof(msi::CallDesc), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        return cuda_fail(e, "copying the call descriptor");
      const int64_t G = std::max(1, ix->batch_group);
      for (int64_t g0 = 0; g0 < cnt; g0 += G, ++timed)
        if ((e = msi::query_batch(ix, (int)std::min<int64_t>(G, cnt - g0), k, ix->call_dev, (int)g0, ix->ws_ovf + g0,
                                  s, ix->events[3 * timed], ix->events[3 * timed + 1], ix->events[3 * timed + 2])) !=
            cudaSuccess)
          return cuda_fail(e, "launching the batched query kernels");
    } else if (batched) {
      // A (queries, k) shape seen before runs as one CUDA graph, replayed with this
      // call's pointers; a new shape launches its kernels directly (and is remembered).
      msi_index::BatchGraph* g = nullptr;
      for (auto& h : ix->graphs)
        if (h.nq == cnt && h.k == k) g = &h;
      if (ix->use_graphs && !g) {
        if (ix->graphs.size() >= (size_t)kMaxBatchGraphs) {  // forget the oldest shape
          if (ix->graphs.front().exec) cudaGraphExecDestroy(ix->graphs.front().exec);
          ix->graphs.erase(ix->graphs.begin());
        }
        ix->graphs.push_back({cnt, k, nullptr, 0});
      } else if (ix->use_graphs && !g->exec &&
                 (e = capture_batch(ix, s, cnt, k, &g->exec, &g->launches)) != cudaSuccess) {
        return cuda_fail(e, "capturing the batched query graph");
      }
      if (g && g->exec) {
        *ix->call_host = msi::CallDesc{qd, id_base, d_base, d64_base};
        if ((e = cudaMemcpyAsync(ix->call_dev, ix->call_host, sizeof(msi::CallDesc), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaGraphLaunch(g->exec, s)) != cudaSuccess)
          return cuda_fail(e, "launching the batched query graph");
        ix->kernel_launches += g->launches;
      } else if (ix->batch_chain) {
        *ix->call_host = msi::CallDesc{qd, id_base, d_base, d64_base};
        if ((e = cudaMemcpyAsync(ix->call_dev, ix->call_host, sizeof(msi::CallDesc), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = enqueue_batch(ix, s, cnt, k, nullptr, nullptr, nullptr, nullptr, ix->call_dev)) != cudaSuccess)
          return cuda_fail(e, "launching the batched query kernels");
      } else if ((e = enqueue_batch(ix, s, cnt, k, qd, id_base, d_base, d64_base, nullptr)) != cudaSuccess) {
        return cuda_fail(e, "launching the query kernels");
      }
    }
    for (int64_t i = 0; !batched && i < cnt; ++i) {
      cudaEvent_t ea = nullptr, em = nullptr, eb = nullptr;
      if (ix->timing) {
        ea = ix->events[3 * i];
        em = ix->events[3 * i + 1];
        eb = ix->events[3 * i + 2];
        timed = i + 1;
      }
      e = msi::query_one(ix, ix->qv, 1, qd + i * ix->len, k, id_base + i * k, d_base ? d_base + i * k : nullptr,
                         d64_base ? d64_base + i * k : nullptr, nullptr, s, ea, em, eb, window);
      if (e != cudaSuccess) return cuda_fail(e, "launching the query kernels");
    }
    if (batched) {
      // run any query that overflowed a slot's bounded lists again on slot 0
      std::vector<uint32_t> ovf(cnt);
      int tc_abort = 0;
      if ((e = cudaMemcpyAsync(ovf.data(), ix->ws_ovf, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost, s)) !=
              cudaSuccess ||
          (ix->tc_ready && (e = cudaMemcpyAsync(&tc_abort, ix->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
                               cudaSuccess) ||
          (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "query execution");
      if (tc_abort) {  // a tensor-core filter gave up on a wait: every query of the chunk again
        for (auto& o : ovf) o = 1u;
        ++ix->tc_aborts;
        if ((e = cudaMemsetAsync(ix->tc_err, 0, sizeof(int), s)) != cudaSuccess) return cuda_fail(e, "query execution");
      }
      for (int64_t i = 0; i < cnt; ++i) {
        if (!ovf[i]) continue;
        e = msi::query_one(ix, ix->qv, 1, qd + i * ix->len, k, id_base + i * k, d_base ? d_base + i * k : nullptr,
                           d64_base ? d64_base + i * k : nullptr, nullptr, s, nullptr, nullptr, nullptr, window);
        if (e != cudaSuccess) return cuda_fail(e, "launching the query kernels");
        ++ix->overflow_reruns;
      }
    }
    if (!ids_dev &&
        (e = cudaMemcpyAsync(ids + c0 * k, ix->ws_ids, sizeof(int64_t) * cnt * k, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
      return cuda_fail(e, "copying ids to the host");
    if (dists && !d_dev &&
        (e = cudaMemcpyAsync(dists + c0 * k, ix->ws_dists, sizeof(float) * cnt * k, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
      return cuda_fail(e, "copying distances to the host");
    if (sqdists64 && !d64_dev &&
        (e = cudaMemcpyAsync(sqdists64 + c0 * k, ix->ws_d64, sizeof(double) * cnt * k, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
      return cuda_fail(e, "copying distances to the host");
    if (host_out || ix->timing || c0 + chunk < nq) {
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "query execution");
    }
    if (ix->timing) {
      for (int64_t i = 0; i < timed; ++i) {
        float ms = 0.f;
        float fms = 0.f;
        if (cudaEventElapsedTime(&ms, ix->events[3 * i], ix->events[3 * i + 2]) == cudaSuccess &&
            cudaEventElapsedTime(&fms, ix->events[3 * i], ix->events[3 * i + 1]) == cudaSuccess) {
          ix->refine_ms += ms;
          ix->filter_ms += fms;
          ++ix->refine_launches;
        }
      }
    }
  }
  if (!stream || host_out) {
    unsigned long long bad = 0;
    if ((e = cudaMemcpyAsync(&bad, bad_flag, sizeof bad, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_fail(e, "query execution");
    if (bad) return fail(MSI_EINVAL, "%llu queries hold NaN or infinity", bad);
  }
  return MSI_OK;
}

msi_status msi_knn_ex(msi_index* ix, const float* queries, int64_t nq, int32_t k, int64_t* ids, float* dists,
                      double* sqdists64, void* stream) {
  return knn_impl(ix, queries, nq, k, -1, ids, dists, sqdists64, stream);
}

namespace {
void forget_graphs(msi_index* ix) {
  for (auto& g : ix->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  ix->graphs.clear();
}
}  // namespace

namespace {
struct Sched {
  bool chain;
  int slots, share, group, bshare;
  bool dense;
};
Sched get_sched(const msi_index* ix) {
  return Sched{ix->batch_chain, ix->nslots, ix->grid_share, ix->batch_group, ix->batch_share, ix->batch_dense};
}
void put_sched(msi_index* ix, const Sched& c) {
  ix->batch_chain = c.chain;
  ix->nslots = c.slots;
  ix->grid_share = c.share;
  ix->batch_group = c.group;
  ix->batch_share = c.bshare;
  ix->batch_dense = c.chain && c.dense;
}
// Releases the slot and batch workspaces the index's schedule does not use (no call
// may be in flight).
void release_unused(msi_index* ix) {
  uint32_t cand_cap = 0, surv_cap = 0;
  msi::slot_capacities(ix, ix->slot_cap, &cand_cap, &surv_cap);
  const int keep = ix->batch_chain ? 0 : ix->nslots;
  while ((int)ix->slots.size() > keep) {
    msi::free_workspace(ix->slots.back());
    ix->device_bytes -= msi::workspace_bytes(ix, cand_cap, surv_cap);
    cudaStreamDestroy(ix->slot_streams.back());
    cudaEventDestroy(ix->slot_events.back());
    ix->slots.pop_back();
    ix->slot_streams.pop_back();
    ix->slot_events.pop_back();
  }
  msi::batch_release(ix, ix->batch_chain ? ix->batch_group : 0);
}
}  // namespace

msi_status msi_schedule_set(msi_index* ix, const msi_schedule* sc) {
  g_err.clear();
  if (!ix || !sc) return fail(MSI_EINVAL, "index or schedule is NULL");
  if (sc->query_slots < 1 || sc->query_slots > 64 || sc->grid_share < 1 || sc->grid_share > 64 ||
      sc->batch_group < 1 || sc->batch_group > 1024 || sc->batch_share < 1 || sc->batch_share > 64)
    return fail(MSI_EINVAL, "schedule outside query_slots 1..64, grid_share 1..64, batch_group 1..1024, "
                            "batch_share 1..64");
  DeviceGuard guard(ix->device);
  cudaError_t e = cudaStreamSynchronize(ix->own_stream);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "msi_schedule_set");
  forget_graphs(ix);  // graphs hold the previous schedule's launches
  if (sc->batch_dense && msi::tc_queries_per_pass(ix->len) == 0)
    return fail(MSI_EINVAL, "the tensor-core filter needs len a multiple of 4 and at most 2048");
  put_sched(ix, Sched{sc->batch_chain != 0, sc->query_slots, sc->grid_share, sc->batch_group, sc->batch_share,
                      sc->batch_dense != 0});
  ix->batch_pdl = sc->batch_overlap != 0;
  ix->batch_order = sc->batch_order != 0;
  release_unused(ix);
  return MSI_OK;
}

msi_status msi_schedule_get(const msi_index* ix, msi_schedule* sc) {
  g_err.clear();
  if (!ix || !sc) return fail(MSI_EINVAL, "index or schedule is NULL");
  sc->batch_chain = ix->batch_chain ? 1 : 0;
  sc->query_slots = ix->nslots;
  sc->grid_share = ix->grid_share;
  sc->batch_group = ix->batch_group;
  sc->batch_share = ix->batch_share;
  sc->batch_overlap = ix->batch_pdl ? 1 : 0;
  sc->batch_dense = ix->batch_dense ? 1 : 0;
  sc->batch_order = ix->batch_order ? 1 : 0;
  return MSI_OK;
}

msi_status msi_autotune(msi_index* ix, const float* queries, int64_t nq, int32_t k, int32_t reps,
                        msi_tune_result* out, void* stream) {
  g_err.clear();
  if (!ix || !queries) return fail(MSI_EINVAL, "index or queries is NULL");
  if (nq < 2) return fail(MSI_EINVAL, "nq = %lld: a schedule needs at least 2 queries", (long long)nq);
  if (k < 1 || k > MSI_MAX_K || (int64_t)k > ix->n)
    return fail(MSI_EINVAL, "k = %d outside [1, min(n = %lld, %d)]", k, (long long)ix->n, MSI_MAX_K);
  if (reps < 0) return fail(MSI_EINVAL, "reps = %d is negative", reps);
  if (reps == 0) reps = 3;
  DeviceGuard guard(ix->device);
  cudaStream_t s = stream ? (cudaStream_t)stream : ix->own_stream;
  const Sched keep = get_sched(ix);
  const bool keep_timing = ix->timing;
  ix->timing = false;
  int64_t* ids = nullptr;
  float* dists = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  msi_status st = MSI_OK;
  double best = -1.0, def_rate = 0.0;
  Sched best_s = keep;
  int count = 0;
  // the candidates: the index's own schedule first, then the batched chain, then slots
  std::vector<Sched> cands{keep};
  auto add = [&](const Sched& c) {
    for (const Sched& o : cands)
      if (o.chain == c.chain && o.dense == c.dense &&
          (c.chain ? (o.group == c.group && o.bshare == c.bshare) : (o.slots == c.slots && o.share == c.share)))
        return;
    cands.push_back(c);
  };
  for (int g : {32, 64, 128})
    for (int bs : {1, 2, 4, 8}) add(Sched{true, keep.slots, keep.share, (int)std::min<int64_t>(g, nq), bs, false});
  // the tensor-core filter: one pass over the collection per pass of queries, so the
  // largest group it takes in one pass
  const int per = msi::tc_queries_per_pass(ix->len);
  if (per > 0)
    for (int bs : {1, 4}) add(Sched{true, keep.slots, keep.share, (int)std::min<int64_t>(per, nq), bs, true});
  for (int sl : {4, 8, 12, 16, 24, 32})
    for (int sh : {1, 2, 3, 4, 6})
      if (sh <= sl) add(Sched{false, sl, sh, keep.group, keep.bshare, false});
  if ((e = cudaMalloc(&ids, sizeof(int64_t) * (size_t)nq * k)) != cudaSuccess ||
      (e = cudaMalloc(&dists, sizeof(float) * (size_t)nq * k)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = cuda_fail(e, "autotune buffers");
  } else {
    bool batch_released = false;
    for (const Sched& c : cands) {
      if (st != MSI_OK) break;
      forget_graphs(ix);  // graphs hold the previous schedule's streams and grids
      if (!c.chain && !batch_released) {  // the slot candidates do not hold batch workspaces too
        msi::batch_release(ix, 0);
        batch_released = true;
      }
      put_sched(ix, c);
      for (int w = 0; w < 3 && st == MSI_OK; ++w) st = knn_impl(ix, queries, nq, k, -1, ids, dists, nullptr, s);
      if (st != MSI_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == MSI_OK; ++r) st = knn_impl(ix, queries, nq, k, -1, ids, dists, nullptr, s);
      if (st != MSI_OK) break;
      float ms = 0.f;
      if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        st = cuda_fail(e, "autotune timing");
        break;
      }
      const double rate = ms > 0.f ? (double)nq * reps / (ms * 1e-3) : 0.0;
      if (count == 0) def_rate = rate;
      ++count;
      if (rate > best) {
        best = rate;
        best_s = c;
      }
    }
  }
  if (ids) cudaFree(ids);
  if (dists) cudaFree(dists);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  forget_graphs(ix);
  ix->timing = keep_timing;
  put_sched(ix, st == MSI_OK ? best_s : keep);
  cudaStreamSynchronize(s);
  release_unused(ix);
  if (st != MSI_OK) return st;
  if (out) {
    out->query_slots = best_s.slots;
    out->grid_share = best_s.share;
    out->queries_per_s = best;
    out->candidates = count;
    out->default_queries_per_s = def_rate;
    out->batch_chain = best_s.chain ? 1 : 0;
    out->batch_group = best_s.group;
    out->batch_share = best_s.bshare;
    out->batch_dense = best_s.dense ? 1 : 0;
  }
  return MSI_OK;
}

msi_status msi_knn_dtw(msi_index* ix, const float* queries, int64_t nq, int32_t k, int32_t window, int64_t* ids,
                       float* dists, double* sqdists64, void* stream) {
  g_err.clear();
  if (window < 0) return fail(MSI_EINVAL, "window = %d is negative", window);
  return knn_impl(ix, queries, nq, k, window, ids, dists, sqdists64, stream);
}

void msi_free(msi_index* ix) { free_index(ix); }

msi_status msi_index_info_get(const msi_index* ix, msi_index_info* info) {
  g_err.clear();
  if (!ix || !info) return fail(MSI_EINVAL, "index or info is NULL");
  info->n = ix->n;
  info->len = ix->len;
  info->segments = ix->w;
  info->cardinality = ix->card;
  info->leaf_capacity = ix->cap;
  info->leaves = ix->L;
  info->device_bytes = ix->device_bytes;
  info->flags = ix->flags;
  info->device = ix->device;
  info->fine_segments = ix->wf;
  return MSI_OK;
}

msi_status msi_index_export(const msi_index* cix, const msi_export* ex) {
  g_err.clear();
  if (!cix || !ex) return fail(MSI_EINVAL, "index or export is NULL");
  msi_index* ix = const_cast<msi_index*>(cix);
  DeviceGuard guard(ix->device);
  cudaError_t e;
  const int64_t n = ix->n, L = ix->L;
  std::vector<uint32_t> perm;
  if (ex->words || ex->perm) {
    perm.resize(n);
    if ((e = cudaMemcpy(perm.data(), ix->perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "export");
    if (ex->perm) std::memcpy(ex->perm, perm.data(), sizeof(uint32_t) * n);
  }
  if (ex->words) {
    std::vector<uint4> wl(n);
    if ((e = cudaMemcpy(wl.data(), ix->words, sizeof(uint4) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "export");
    for (int64_t p = 0; p < n; ++p)
      std::memcpy(ex->words + (int64_t)perm[p] * ix->w, &wl[p], (size_t)ix->w);
  }
  if (ex->leaf_begin &&
      (e = cudaMemcpy(ex->leaf_begin, ix->leaf_begin, sizeof(uint32_t) * (L + 1), cudaMemcpyDeviceToHost)) !=
          cudaSuccess)
    return cuda_fail(e, "export");
  if (ex->env_lo || ex->env_hi) {
    std::vector<uint4> env(2 * L);
    if ((e = cudaMemcpy(env.data(), ix->env, sizeof(uint4) * 2 * L, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "export");
    for (int64_t l = 0; l < L; ++l) {
      if (ex->env_lo) std::memcpy(ex->env_lo + l * ix->w, &env[2 * l], (size_t)ix->w);
      if (ex->env_hi) std::memcpy(ex->env_hi + l * ix->w, &env[2 * l + 1], (size_t)ix->w);
    }
  }
  if (ex->thresholds) std::memcpy(ex->thresholds, ix->h_thr_up + 1, sizeof(float) * (ix->card - 1));
  if (ex->fine && ix->fine &&  // kept in collection order
      (e = cudaMemcpy(ex->fine, ix->fine, sizeof(uint16_t) * (size_t)n * ix->wf, cudaMemcpyDeviceToHost)) !=
          cudaSuccess)
    return cuda_fail(e, "export");
  if (ex->znorm) {
    const size_t bytes = sizeof(float) * (size_t)n * ix->len;
    if (ix->data_is_z) {
      if ((e = cudaMemcpy(ex->znorm, ix->data, bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "export");
    } else {
      float* tmp = nullptr;
      if ((e = cudaMalloc(&tmp, bytes)) != cudaSuccess) return cuda_fail(e, "export");
      e = msi::export_z(ix, tmp, ix->own_stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ix->own_stream);
      if (e == cudaSuccess) e = cudaMemcpy(ex->znorm, tmp, bytes, cudaMemcpyDeviceToHost);
      cudaFree(tmp);
      if (e != cudaSuccess) return cuda_fail(e, "export");
    }
  }
  return MSI_OK;
}

msi_status msi_lower_bounds(msi_index* ix, const float* query, float* series_lb, float* leaf_lb, void* stream) {
  g_err.clear();
  if (!ix || !query) return fail(MSI_EINVAL, "index or query is NULL");
  DeviceGuard guard(ix->device);
  cudaError_t e = msi::query_setup(ix);
  if (e != cudaSuccess) return cuda_fail(e, "allocating the query workspace");
  cudaStream_t s = stream ? (cudaStream_t)stream : ix->own_stream;
  bool other = false;
  const float* qd = query;
  if (!is_device_ptr(query, ix->device, &other)) {
    if ((e = cudaMemcpyAsync(ix->ws_qraw, query, sizeof(float) * ix->len, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return cuda_fail(e, "copying the query");
    qd = ix->ws_qraw;
  } else if (other) {
    return fail(MSI_EINVAL, "query lives on another device");
  }
  float *sl = nullptr, *ll = nullptr;
  if (series_lb && (e = cudaMalloc(&sl, sizeof(float) * ix->n)) != cudaSuccess) return cuda_fail(e, "lower bounds");
  if (leaf_lb && (e = cudaMalloc(&ll, sizeof(float) * ix->L)) != cudaSuccess) {
    cudaFree(sl);
    return cuda_fail(e, "lower bounds");
  }
  e = msi::lower_bounds(ix, qd, sl, ll, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && sl) e = cudaMemcpy(series_lb, sl, sizeof(float) * ix->n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ll) e = cudaMemcpy(leaf_lb, ll, sizeof(float) * ix->L, cudaMemcpyDeviceToHost);
  cudaFree(sl);
  cudaFree(ll);
  if (e != cudaSuccess) return cuda_fail(e, "lower bounds");
  return MSI_OK;
}

msi_status msi_query_stats_get(msi_index* ix, msi_query_stats* st, int32_t reset) {
  g_err.clear();
  if (!ix || !st) return fail(MSI_EINVAL, "index or stats is NULL");
  std::memset(st, 0, sizeof *st);
  if (!ix->ws_ready) return MSI_OK;
  DeviceGuard guard(ix->device);
  unsigned long long c[msi::ST_COUNT];
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(c, ix->qv.counters, sizeof(unsigned long long) * msi::ST_COUNT, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "reading counters");
  st->queries = (int64_t)c[msi::ST_QUERIES];
  st->leaves_total = (int64_t)c[msi::ST_LEAVES_TOTAL];
  st->leaves_survived = (int64_t)c[msi::ST_LEAVES_SURVIVED];
  st->blocks_examined = (int64_t)c[msi::ST_LEAVES_PROCESSED];
  st->series_lower_bounded = (int64_t)c[msi::ST_SERIES_LB];
  st->series_refined = (int64_t)c[msi::ST_SERIES_REFINED];
  st->seed_series = (int64_t)c[msi::ST_SEED];
  st->candidates = (int64_t)c[msi::ST_CANDIDATES];
  st->rechecked = (int64_t)c[msi::ST_RECHECKED];
  st->refine_launches = ix->refine_launches;
  st->refine_ms = ix->refine_ms;
  st->filter_ms = ix->filter_ms;
  st->kernel_launches = ix->kernel_launches.load();
  st->survivors = (int64_t)c[msi::ST_SURVIVORS];
  st->fine_bounded = (int64_t)c[msi::ST_FINE];
  st->front_fine_bounded = (int64_t)c[msi::ST_FINE_FRONT];
  st->overflow_reruns = ix->overflow_reruns;
  st->tc_pairs = (int64_t)c[msi::ST_TC_PAIRS];
  if (reset) {
    if ((e = cudaMemset(ix->qv.counters, 0, sizeof(unsigned long long) * msi::ST_COUNT)) != cudaSuccess)
      return cuda_fail(e, "resetting counters");
    ix->refine_ms = 0.0;
    ix->filter_ms = 0.0;
    ix->refine_launches = 0;
    ix->kernel_launches = 0;
    ix->overflow_reruns = 0;
  }
  return MSI_OK;
}

msi_status msi_set_timing(msi_index* ix, int32_t enable) {
  g_err.clear();
  if (!ix) return fail(MSI_EINVAL, "index is NULL");
  ix->timing = enable != 0;
  return MSI_OK;
}

}  // extern "C"
