// msi_merge.cu -- msi_merge_topk: the exchange step of a search over a collection split
// across GPUs. Every series is summarised and searched on its own (Section III), so a
// collection split into contiguous ranges is searched range by range; the answer over
// the whole collection is the k smallest of the ranges' answers in (FP64 squared
// distance, id) order, the order each range's answer already has.
//
// One block per query. Every part's list is sorted, so a candidate's position in the
// merged order is its position in its own list plus, for every other part, the number
// of that part's entries before it (a binary search); ids are distinct across parts,
// so positions are distinct and each candidate below k writes itself. No sort, no
// shared buffer, and the result is the same whatever the launch shape.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "msi_internal.cuh"

namespace {

// (d, id) strictly before (d2, id2)? Non-negative doubles order as their bit patterns.
__device__ __forceinline__ bool before(unsigned long long d, int64_t id, unsigned long long d2, int64_t id2) {
  return d < d2 || (d == d2 && id < id2);
}

// Entries of sorted list (ld, li)[0..m) that come before (d, id).
__device__ __forceinline__ int count_before(const double* ld, const int64_t* li, int m, unsigned long long d,
                                            int64_t id) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (before((unsigned long long)__double_as_longlong(ld[mid]), li[mid], d, id)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(256)
merge_topk_kernel(const int64_t* __restrict__ ids, const double* __restrict__ d64, int parts, int64_t nq, int kin,
                  int k, int64_t* __restrict__ out_ids, float* __restrict__ out_d, double* __restrict__ out_d64) {
  const int64_t q = blockIdx.x;
  const int total = parts * kin;
  for (int c = threadIdx.x; c < total; c += blockDim.x) {
    const int p = c / kin, j = c - p * kin;
    const size_t base = ((size_t)p * nq + q) * kin;
    const double dv = d64[base + j];
    const int64_t idv = ids[base + j];
    const unsigned long long db = (unsigned long long)__double_as_longlong(dv);
    int rank = j;
    for (int o = 0; o < parts && rank < k; ++o) {
      if (o == p) continue;
      const size_t ob = ((size_t)o * nq + q) * kin;
      rank += count_before(d64 + ob, ids + ob, kin, db, idv);
    }
    if (rank < k) {
      const size_t r = (size_t)q * k + rank;
      out_ids[r] = idv;
      if (out_d64) out_d64[r] = dv;
      if (out_d) out_d[r] = __double2float_rn(__dsqrt_rn(dv));
    }
  }
}

thread_local char g_err_buf[256];

msi_status fail(msi_status s, const char* what) {
  std::snprintf(g_err_buf, sizeof g_err_buf, "%s", what);
  msi::set_last_error(g_err_buf);
  return s;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" MSI_API msi_status msi_merge_topk(const int64_t* ids, const double* sqdists64, int32_t parts, int64_t nq,
                                             int32_t k_in, int32_t k, int64_t* out_ids, float* out_dists,
                                             double* out_sqdists64, void* stream) {
  msi::set_last_error("");
  if (!ids || !sqdists64 || !out_ids) return fail(MSI_EINVAL, "ids, distances or out_ids is NULL");
  if (parts < 1 || nq < 0 || k_in < 1 || k < 1 || (int64_t)k > (int64_t)parts * k_in || k > MSI_MAX_K ||
      k_in > MSI_MAX_K || (int64_t)parts * k_in > (1 << 20) || nq > 0x7fffffffLL)
    return fail(MSI_EINVAL, "need parts >= 1, nq >= 0, 1 <= k_in <= 1024, 1 <= k <= min(parts * k_in, 1024)");
  if (nq == 0) return MSI_OK;
  const size_t in_n = (size_t)parts * nq * k_in, out_n = (size_t)nq * k;
  const bool dev_in = on_device(ids) && on_device(sqdists64);
  const bool dev_out = on_device(out_ids) && (!out_dists || on_device(out_dists)) &&
                       (!out_sqdists64 || on_device(out_sqdists64));
  cudaStream_t s = (cudaStream_t)stream;
  // host arrays are staged through one device buffer (inputs, then outputs)
  void* stage = nullptr;
  size_t stage_bytes = 0;
  if (!dev_in) stage_bytes += in_n * (sizeof(int64_t) + sizeof(double));
  if (!dev_out) stage_bytes += out_n * (sizeof(int64_t) + sizeof(float) + sizeof(double));
  cudaError_t e = cudaSuccess;
  if (stage_bytes && (e = cudaMalloc(&stage, stage_bytes)) != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? MSI_ENOMEM : MSI_ECUDA, "staging buffer");
  }
  char* sp = static_cast<char*>(stage);
  const int64_t* ids_d = ids;
  const double* d_d = sqdists64;
  if (!dev_in) {
    int64_t* a = reinterpret_cast<int64_t*>(sp);
    double* b = reinterpret_cast<double*>(sp + in_n * sizeof(int64_t));
    sp += in_n * (sizeof(int64_t) + sizeof(double));
    e = cudaMemcpyAsync(a, ids, in_n * sizeof(int64_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b, sqdists64, in_n * sizeof(double), cudaMemcpyDefault, s);
    ids_d = a;
    d_d = b;
  }
  int64_t* oi = out_ids;
  float* od = out_dists;
  double* o64 = out_sqdists64;
  if (!dev_out) {  // ids, then FP64 distances, then fp32 distances: each stays aligned
    oi = reinterpret_cast<int64_t*>(sp);
    o64 = reinterpret_cast<double*>(sp + out_n * sizeof(int64_t));
    od = reinterpret_cast<float*>(sp + out_n * (sizeof(int64_t) + sizeof(double)));
  }
  if (e == cudaSuccess) {
    merge_topk_kernel<<<(unsigned)nq, 256, 0, s>>>(ids_d, d_d, parts, nq, k_in, k, oi, od, o64);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev_out) {
    e = cudaMemcpyAsync(out_ids, oi, out_n * sizeof(int64_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess && out_dists) e = cudaMemcpyAsync(out_dists, od, out_n * sizeof(float), cudaMemcpyDefault, s);
    if (e == cudaSuccess && out_sqdists64)
      e = cudaMemcpyAsync(out_sqdists64, o64, out_n * sizeof(double), cudaMemcpyDefault, s);
  }
  if (e == cudaSuccess && (!stream || stage)) e = cudaStreamSynchronize(s);
  if (stage) cudaFree(stage);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(MSI_ECUDA, cudaGetErrorString(e));
  }
  return MSI_OK;
}
