// msi_noalloc.cu -- msi_lower_bounds_noalloc, the one entry point that allocates no
// memory at all.
//
// Some callers cannot call cudaMalloc: code held to a device-memory budget by a custom
// allocator or a stream-ordered pool that it does not own (an allocation behind the
// pool's back breaks the budget), and real-time paths that must not block on the
// driver's allocator (cudaMalloc can synchronise the device). For them
// this entry point computes the same lower bounds as msi_lower_bounds with every
// per-query temporary (query state, z-normalised query, per-segment gap tables,
// counters) in one file-scope device array of fixed size instead of the index's
// query workspace, which msi_lower_bounds allocates on first use.
//
// The array is a static __device__ object: every GPU that loads the library holds
// kScratchBytes of it until the process exits. All calls share it and it keeps the
// last call's contents; calls whose work overlaps on the GPU (on different streams,
// or from different threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "msi_internal.cuh"

namespace {

// Layout: query state (QState) | device counters | query z [MSI_MAX_LEN] |
// T [MSI_MAX_SEGMENTS * MSI_MAX_CARDINALITY] | T5 [MSI_MAX_SEGMENTS * kCoarse].
constexpr size_t kStateBytes = 1024;
constexpr size_t kCounterBytes = 256;
constexpr size_t kQzBytes = sizeof(float) * MSI_MAX_LEN;
constexpr size_t kTBytes = sizeof(float) * MSI_MAX_SEGMENTS * MSI_MAX_CARDINALITY;
constexpr size_t kT5Bytes = sizeof(float) * MSI_MAX_SEGMENTS * msi::kCoarse;
constexpr size_t kScratchBytes = kStateBytes + kCounterBytes + kQzBytes + kTBytes + kT5Bytes;  // 38,144 bytes
static_assert(sizeof(msi::QState) <= kStateBytes, "query state does not fit its scratch slot");
static_assert(sizeof(unsigned long long) * msi::ST_COUNT <= kCounterBytes, "counters do not fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

msi_status fail(msi_status st, const char* what) {
  msi::set_last_error(what);
  return st;
}

}  // namespace

extern "C" MSI_API msi_status msi_lower_bounds_noalloc(const msi_index* ix, const float* query, float* series_lb,
                                                        float* leaf_lb, void* stream) {
  msi::set_last_error("");
  if (!ix || !query || !series_lb || !leaf_lb) return fail(MSI_EINVAL, "index, query or an output is NULL");
  if ((size_t)ix->len * sizeof(float) > kQzBytes || (size_t)ix->w * ix->card * sizeof(float) > kTBytes ||
      ix->w > MSI_MAX_SEGMENTS)
    return fail(MSI_EINVAL, "index shape exceeds the fixed scratch (len <= 4096, segments * cardinality <= 4096)");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fail(MSI_ECUDA, "no usable CUDA device");
  if (ix->device < 0 || ix->device >= kMaxDevices) return fail(MSI_EINVAL, "device ordinal beyond 63");
  if (prev != ix->device && cudaSetDevice(ix->device) != cudaSuccess) return fail(MSI_ECUDA, "cudaSetDevice failed");
  struct Restore {
    int d;
    ~Restore() {
      int c;
      if (d >= 0 && cudaGetDevice(&c) == cudaSuccess && c != d) cudaSetDevice(d);
    }
  } restore{prev};
  for (const void* p : {(const void*)query, (const void*)series_lb, (const void*)leaf_lb}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return fail(MSI_EINVAL, "query and outputs must be device memory of the index's GPU");
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != ix->device)
      return fail(MSI_EINVAL, "query and outputs must be device memory of the index's GPU");
  }
  // set-up, once per device, with that device current: the device address of the
  // scratch array (its name in host code is only a host-side stand-in)
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[ix->device]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return fail(MSI_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      g_scratch_addr[ix->device] = ptr;
    }
    base = g_scratch_addr[ix->device];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  msi::QueryView qv{};
  qv.st = reinterpret_cast<msi::QState*>(b);
  qv.counters = reinterpret_cast<unsigned long long*>(b + kStateBytes);
  qv.qz = reinterpret_cast<float*>(b + kStateBytes + kCounterBytes);
  qv.T = reinterpret_cast<float*>(b + kStateBytes + kCounterBytes + kQzBytes);
  qv.T5 = reinterpret_cast<float*>(b + kStateBytes + kCounterBytes + kQzBytes + kTBytes);
  qv.k = 1;
  qv.eps = msi::margin_eps();  // the allocating path's margins
  qv.tau = msi::margin_tau(ix->len);
  cudaStream_t s = (cudaStream_t)stream;
  // state and counters start at zero on every call (the array keeps the last call's)
  cudaError_t e = cudaMemsetAsync(b, 0, kStateBytes + kCounterBytes, s);
  if (e == cudaSuccess) e = msi::lower_bounds_on(ix, qv, query, series_lb, leaf_lb, s);
  if (e == cudaSuccess && !stream) {
    unsigned long long bad = 0;
    e = cudaMemcpyAsync(&bad, qv.counters + msi::ST_BAD_QUERY, sizeof bad, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && bad) return fail(MSI_EINVAL, "the query holds NaN or infinity");
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MSI_ENOMEM : MSI_ECUDA, cudaGetErrorString(e));
  }
  return MSI_OK;
}
