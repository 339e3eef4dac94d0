// msi_serve.cu -- a request loop over several resident indexes with continuous
// batching (the serving form of the search; the paper runs one query after another,
// Section IV "Setup", so this has no counterpart there).
//
// Every index gets query slots: a bounded workspace, a stream, device and pinned
// host staging. A dispatcher thread admits waiting requests into free slots the
// moment they free up (so requests that arrive while others are on the GPU join
// the work already in flight), launches each query's kernel chain on its slot's
// stream, and completes a request when its slot's event fires. The number of slots
// is bounded by a workspace-memory budget (admission by device memory), and a cap
// on slots in flight lets the same loop serve strictly one query at a time. A query
// that overflows a slot's bounded lists is run again on the index's own workspace,
// which has room for any query.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "msi_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int index_no = 0;
  int k = 1;
  std::vector<float> query;
  Clock::time_point t0;
};

struct Result {
  std::vector<int64_t> ids;
  std::vector<float> dists;
  double ms = 0.0;
  msi_status status = MSI_OK;
};

struct Slot {
  msi_index* ix = nullptr;
  int index_no = 0;
  bool full = false;  // the index's own workspace: room for any query
  msi::QueryView qv{};
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* q_dev = nullptr;
  int64_t* ids_dev = nullptr;
  float* d_dev = nullptr;
  uint32_t* ovf_dev = nullptr;
  float* q_host = nullptr;  // pinned
  int64_t* ids_host = nullptr;
  float* d_host = nullptr;
  uint32_t* ovf_host = nullptr;
  bool busy = false;
  Request req;
};

}  // namespace

struct msi_server {
  int device = 0;
  int max_inflight = 0;
  int share = 1;
  std::vector<msi_index*> indexes;
  std::vector<Slot> slots;
  std::vector<std::deque<Request>> waiting;  // per index
  std::vector<std::deque<Request>> rerun;    // per index: need the full workspace
  std::unordered_map<uint64_t, Result> results;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  int64_t completed = 0, reruns = 0;
  std::string fatal;  // a CUDA failure of the worker; every later call reports it
};

namespace {

cudaError_t slot_alloc(Slot& sl, msi_index* ix, int index_no, bool full, uint32_t cand_cap, uint32_t surv_cap,
                       int64_t* bytes) {
  sl.ix = ix;
  sl.index_no = index_no;
  sl.full = full;
  cudaError_t e;
  if (full) {
    if ((e = msi::query_setup(ix)) != cudaSuccess) return e;
    sl.qv = ix->qv;
  } else if ((e = msi::alloc_workspace(ix, sl.qv, cand_cap, surv_cap, bytes)) != cudaSuccess) {
    return e;
  } else {
    sl.qv.counters = ix->qv.counters;
  }
  if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sl.q_dev, sizeof(float) * (size_t)ix->len)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sl.ids_dev, sizeof(int64_t) * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sl.d_dev, sizeof(float) * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sl.ovf_dev, sizeof(uint32_t))) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&sl.q_host, sizeof(float) * (size_t)ix->len)) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&sl.ids_host, sizeof(int64_t) * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&sl.d_host, sizeof(float) * MSI_MAX_K)) != cudaSuccess) return e;
  if ((e = cudaMallocHost(&sl.ovf_host, sizeof(uint32_t))) != cudaSuccess) return e;
  *sl.ovf_host = 0;
  return cudaSuccess;
}

void slot_free(Slot& sl) {
  if (sl.stream) cudaStreamSynchronize(sl.stream);
  if (!sl.full) msi::free_workspace(sl.qv);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  if (sl.done) cudaEventDestroy(sl.done);
  cudaFree(sl.q_dev);
  cudaFree(sl.ids_dev);
  cudaFree(sl.d_dev);
  cudaFree(sl.ovf_dev);
  cudaFreeHost(sl.q_host);
  cudaFreeHost(sl.ids_host);
  cudaFreeHost(sl.d_host);
  cudaFreeHost(sl.ovf_host);
  sl = Slot{};
}

cudaError_t launch(msi_server* sv, Slot& sl, Request&& req) {
  msi_index* ix = sl.ix;
  std::memcpy(sl.q_host, req.query.data(), sizeof(float) * (size_t)ix->len);
  *sl.ovf_host = 0;
  cudaError_t e = cudaMemcpyAsync(sl.q_dev, sl.q_host, sizeof(float) * (size_t)ix->len, cudaMemcpyHostToDevice,
                                  sl.stream);
  if (e == cudaSuccess)
    e = msi::query_one(ix, sl.qv, sl.full ? 1 : sv->share, sl.q_dev, req.k, sl.ids_dev, sl.d_dev, nullptr,
                       sl.full ? nullptr : sl.ovf_dev, sl.stream, nullptr, nullptr, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.ids_host, sl.ids_dev, sizeof(int64_t) * req.k, cudaMemcpyDeviceToHost, sl.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl.d_host, sl.d_dev, sizeof(float) * req.k, cudaMemcpyDeviceToHost, sl.stream);
  if (e == cudaSuccess && !sl.full)
    e = cudaMemcpyAsync(sl.ovf_host, sl.ovf_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, sl.stream);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
  sl.req = std::move(req);
  sl.busy = true;
  return e;
}

void worker_loop(msi_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    int inflight = 0;
    bool progressed = false;
    // completions
    for (Slot& sl : sv->slots) {
      if (!sl.busy) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) {
        ++inflight;
        continue;
      }
      sl.busy = false;
      progressed = true;
      if (q != cudaSuccess) {
        sv->fatal = std::string("query execution: ") + cudaGetErrorString(q);
        sv->results[sl.req.ticket].status = MSI_ECUDA;
        sv->cv_done.notify_all();
        continue;
      }
      if (!sl.full && *sl.ovf_host) {  // needs the full workspace
        sv->rerun[sl.index_no].push_back(std::move(sl.req));
        ++sv->reruns;
        continue;
      }
      Result r;
      r.ids.assign(sl.ids_host, sl.ids_host + sl.req.k);
      r.dists.assign(sl.d_host, sl.d_host + sl.req.k);
      r.ms = std::chrono::duration<double, std::milli>(Clock::now() - sl.req.t0).count();
      sv->results[sl.req.ticket] = std::move(r);
      ++sv->completed;
      sv->cv_done.notify_all();
    }
    // admissions: reruns first, then the oldest waiting request whose index has a
    // free slot, while the in-flight cap allows
    while (inflight < sv->max_inflight) {
      Slot* target = nullptr;
      std::deque<Request>* from = nullptr;
      for (Slot& sl : sv->slots)
        if (!sl.busy && sl.full && !sv->rerun[sl.index_no].empty()) {
          target = &sl;
          from = &sv->rerun[sl.index_no];
          break;
        }
      if (!target) {
        Clock::time_point best = Clock::time_point::max();
        for (Slot& sl : sv->slots) {
          if (sl.busy) continue;
          std::deque<Request>& w = sv->waiting[sl.index_no];
          if (!w.empty() && w.front().t0 < best) {
            best = w.front().t0;
            target = &sl;
            from = &w;
          }
        }
      }
      if (!target) break;
      Request req = std::move(from->front());
      from->pop_front();
      const cudaError_t e = launch(sv, *target, std::move(req));
      if (e != cudaSuccess) {
        sv->fatal = std::string("launching a query: ") + cudaGetErrorString(e);
        sv->results[target->req.ticket].status = MSI_ECUDA;
        target->busy = false;
        sv->cv_done.notify_all();
        continue;
      }
      ++inflight;
      progressed = true;
    }
    bool queued = false;
    for (size_t i = 0; i < sv->waiting.size(); ++i) queued |= !sv->waiting[i].empty() || !sv->rerun[i].empty();
    if (sv->stop && inflight == 0 && !queued) break;
    if (inflight == 0 && !queued) {
      sv->cv_work.wait(lk);
    } else if (!progressed) {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
  }
}

}  // namespace

extern "C" {

msi_status msi_server_create(msi_index* const* indexes, int32_t n_indexes, const msi_server_opts* opts,
                             msi_server** out) {
  msi::set_last_error("");
  if (!out) {
    msi::set_last_error("out is NULL");
    return MSI_EINVAL;
  }
  *out = nullptr;
  if (!indexes || n_indexes < 1 || n_indexes > 64) {
    msi::set_last_error("need 1 to 64 indexes");
    return MSI_EINVAL;
  }
  const int per_index = opts && opts->slots_per_index ? opts->slots_per_index : 8;
  const int64_t budget = opts && opts->workspace_bytes ? opts->workspace_bytes : (int64_t)8 << 30;
  const int max_inflight = opts && opts->max_inflight ? opts->max_inflight : 1 << 30;
  if (per_index < 1 || per_index > 256 || budget < 0 || max_inflight < 1) {
    msi::set_last_error("slots_per_index outside [1, 256], or a negative budget or in-flight cap");
    return MSI_EINVAL;
  }
  int dev = 0;
  for (int i = 0; i < n_indexes; ++i) {
    if (!indexes[i]) {
      msi::set_last_error("an index is NULL");
      return MSI_EINVAL;
    }
    if (i && indexes[i]->device != dev) {
      msi::set_last_error("indexes on different devices");
      return MSI_EINVAL;
    }
    dev = indexes[i]->device;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(dev);
  msi_server* sv = new msi_server();
  sv->device = dev;
  sv->max_inflight = max_inflight;
  sv->share = std::max(1, std::min(per_index, msi::kSlotGridShare));
  sv->waiting.resize(n_indexes);
  sv->rerun.resize(n_indexes);
  cudaError_t e = cudaSuccess;
  int64_t used = 0;
  // one full-capacity slot per index, then bounded slots while the budget lasts
  for (int i = 0; i < n_indexes && e == cudaSuccess; ++i) {
    sv->indexes.push_back(indexes[i]);
    sv->slots.emplace_back();
    int64_t ignore = 0;
    e = slot_alloc(sv->slots.back(), indexes[i], i, true, 0, 0, &ignore);
  }
  for (int r = 1; r < per_index && e == cudaSuccess; ++r) {
    for (int i = 0; i < n_indexes && e == cudaSuccess; ++i) {
      uint32_t cc, sc;
      msi::slot_capacities(indexes[i], opts ? opts->slot_capacity : 0, &cc, &sc);
      int64_t bytes = 0;
      const int64_t need = msi::workspace_bytes(indexes[i], cc, sc);
      if (used + need > budget) continue;
      sv->slots.emplace_back();
      e = slot_alloc(sv->slots.back(), indexes[i], i, false, cc, sc, &bytes);
      used += bytes;
    }
  }
  if (e != cudaSuccess) {
    for (Slot& sl : sv->slots) slot_free(sl);
    delete sv;
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    msi::set_last_error(e == cudaErrorMemoryAllocation ? "out of device memory for the query slots"
                                                       : cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MSI_ENOMEM : MSI_ECUDA;
  }
  sv->worker = std::thread(worker_loop, sv);
  if (prev >= 0) cudaSetDevice(prev);
  *out = sv;
  return MSI_OK;
}

msi_status msi_server_submit(msi_server* sv, int32_t index_no, const float* query, int32_t k, uint64_t* ticket) {
  msi::set_last_error("");
  if (!sv || !query || !ticket) {
    msi::set_last_error("server, query or ticket is NULL");
    return MSI_EINVAL;
  }
  if (index_no < 0 || index_no >= (int)sv->indexes.size()) {
    msi::set_last_error("index_no out of range");
    return MSI_EINVAL;
  }
  msi_index* ix = sv->indexes[index_no];
  if (k < 1 || k > MSI_MAX_K || k > ix->n) {
    msi::set_last_error("k outside [1, min(n, MSI_MAX_K)]");
    return MSI_EINVAL;
  }
  Request req;
  req.index_no = index_no;
  req.k = k;
  req.query.assign(query, query + ix->len);
  req.t0 = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->fatal.empty()) {
      msi::set_last_error(sv->fatal.c_str());
      return MSI_ECUDA;
    }
    req.ticket = sv->next_ticket++;
    *ticket = req.ticket;
    sv->waiting[index_no].push_back(std::move(req));
  }
  sv->cv_work.notify_one();
  return MSI_OK;
}

msi_status msi_server_wait(msi_server* sv, uint64_t ticket, int64_t* ids, float* dists, double* latency_ms) {
  msi::set_last_error("");
  if (!sv || !ids) {
    msi::set_last_error("server or ids is NULL");
    return MSI_EINVAL;
  }
  std::unique_lock<std::mutex> lk(sv->mu);
  if (ticket == 0 || ticket >= sv->next_ticket) {
    msi::set_last_error("unknown ticket");
    return MSI_EINVAL;
  }
  sv->cv_done.wait(lk, [&] { return sv->results.count(ticket) > 0; });
  Result r = std::move(sv->results[ticket]);
  sv->results.erase(ticket);
  if (r.status != MSI_OK) {
    msi::set_last_error(sv->fatal.c_str());
    return r.status;
  }
  std::copy(r.ids.begin(), r.ids.end(), ids);
  if (dists) std::copy(r.dists.begin(), r.dists.end(), dists);
  if (latency_ms) *latency_ms = r.ms;
  return MSI_OK;
}

msi_status msi_server_stats(msi_server* sv, int64_t* completed, int64_t* reruns, int32_t* slots) {
  if (!sv) return MSI_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (completed) *completed = sv->completed;
  if (reruns) *reruns = sv->reruns;
  if (slots) *slots = (int32_t)sv->slots.size();
  return MSI_OK;
}

void msi_server_free(msi_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->device);
  for (Slot& sl : sv->slots) slot_free(sl);
  if (prev >= 0) cudaSetDevice(prev);
  delete sv;
}

}  // extern "C"
