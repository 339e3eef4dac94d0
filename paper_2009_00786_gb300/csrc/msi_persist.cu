// msi_persist.cu -- saving an index to a file and loading it back.
//
// The paper builds its index in memory for every run (Section III-A); a saved index
// lets a collection be searched again without the summarisation, sort and split
// passes. The file holds a fixed header (parameters, array sizes and an FNV-1a
// checksum of the index arrays) followed by the arrays in a fixed order: SAX words,
// leaf order, per-series moments, leaf boundaries, leaf envelopes, block envelopes,
// leaf keys, the balanced-split tree when there is one, the fine PAA when there is one
// and, for an index that owns its collection, the z-normalised collection.
// A borrowed collection is not written; loading such an index takes the collection
// again. Everything is little-endian, as both hosts that run this library are.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "msi_internal.cuh"

namespace {

constexpr char kMagic[8] = {'M', 'S', 'I', 'I', 'N', 'D', 'E', 'X'};
constexpr uint32_t kVersion = 3;  // 3: the fine PAA in collection order
constexpr size_t kStage = size_t(64) << 20;  // pinned staging buffer

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n;
  int32_t len, w, card, bits, seglen, cap;
  uint32_t flags;
  int32_t data_is_z;
  int64_t L;
  int64_t nblk;
  uint64_t index_checksum;  // FNV-1a over every array but the collection
  int64_t tree_nodes;       // balanced-split tree (0 without one)
  int64_t root_bits;
  uint64_t reserved[2];
};

// One array of the file: device pointer and byte count.
struct Section {
  void* dev;
  size_t bytes;
};

std::vector<Section> sections(msi_index* ix, int64_t nblk, bool with_data) {
  std::vector<Section> v = {
      {ix->words, sizeof(uint4) * (size_t)ix->n},
      {ix->perm, sizeof(uint32_t) * (size_t)ix->n},
      {ix->stats, sizeof(float2) * (size_t)ix->n},
      {ix->leaf_begin, sizeof(uint32_t) * (size_t)(ix->L + 1)},
      {ix->env, sizeof(uint4) * 2 * (size_t)ix->L},
      {ix->benv, sizeof(uint4) * 2 * (size_t)nblk},
      {ix->leaf_key, sizeof(uint64_t) * (size_t)ix->L},
  };
  if (ix->tree_child) {  // balanced-split tree
    v.push_back({ix->root_child, sizeof(int32_t) << ix->root_bits});
    v.push_back({ix->tree_child, 2 * sizeof(int32_t) * (size_t)ix->tree_nodes});
    v.push_back({ix->tree_seg, sizeof(int8_t) * (size_t)ix->tree_nodes});
  }
  if (ix->fine) v.push_back({ix->fine, sizeof(uint16_t) * (size_t)ix->n * ix->wf});
  if (with_data) v.push_back({ix->data_owned, sizeof(float) * (size_t)ix->n * ix->len});
  return v;
}

uint64_t fnv1a(uint64_t h, const unsigned char* p, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

msi_status fail(msi_status st, const std::string& what) {
  msi::set_last_error(what.c_str());
  return st;
}

msi_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? MSI_ENOMEM : MSI_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

}  // namespace

extern "C" {

msi_status msi_index_save(msi_index* ix, const char* path) {
  msi::set_last_error("");
  if (!ix || !path) return fail(MSI_EINVAL, "index or path is NULL");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ix->device) cudaSetDevice(ix->device);
  const int64_t nblk = (ix->n + 31) / 32;
  const bool with_data = ix->data_owned != nullptr;
  std::vector<Section> secs = sections(ix, nblk, with_data);
  Pinned stage;
  cudaError_t e = cudaMallocHost(&stage.p, kStage);
  msi_status st = MSI_OK;
  File out;
  FileHeader h{};
  if (e != cudaSuccess) {
    st = cuda_fail(e, "allocating the staging buffer");
    goto done;
  }
  // the index arrays are finished once the index's streams are idle
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    st = cuda_fail(e, "waiting for the index");
    goto done;
  }
  out.f = fopen(path, "wb");
  if (!out.f) {
    st = fail(MSI_EINTERNAL, std::string("cannot create ") + path);
    goto done;
  }
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(FileHeader);
  h.n = ix->n;
  h.len = ix->len;
  h.w = ix->w;
  h.card = ix->card;
  h.bits = ix->bits;
  h.seglen = ix->seglen;
  h.cap = ix->cap;
  h.flags = ix->flags;
  h.data_is_z = ix->data_is_z ? 1 : 0;
  h.L = ix->L;
  h.nblk = nblk;
  h.tree_nodes = ix->tree_child ? ix->tree_nodes : 0;
  h.root_bits = ix->tree_child ? ix->root_bits : 0;
  // the header goes first with a zero checksum and is rewritten at the end
  if (fwrite(&h, sizeof h, 1, out.f) != 1) {
    st = fail(MSI_EINTERNAL, "writing the header");
    goto done;
  }
  {
    uint64_t sum = 1469598103934665603ull;
    for (size_t si = 0; si < secs.size(); ++si) {
      const bool data = with_data && si + 1 == secs.size();
      for (size_t off = 0; off < secs[si].bytes; off += kStage) {
        const size_t b = std::min(kStage, secs[si].bytes - off);
        if ((e = cudaMemcpy(stage.p, (char*)secs[si].dev + off, b, cudaMemcpyDeviceToHost)) != cudaSuccess) {
          st = cuda_fail(e, "reading the index from the device");
          goto done;
        }
        if (!data) sum = fnv1a(sum, (const unsigned char*)stage.p, b);
        if (fwrite(stage.p, 1, b, out.f) != b) {
          st = fail(MSI_EINTERNAL, "writing the index arrays");
          goto done;
        }
      }
    }
    h.index_checksum = sum;
    if (fseek(out.f, 0, SEEK_SET) != 0 || fwrite(&h, sizeof h, 1, out.f) != 1 || fflush(out.f) != 0) {
      st = fail(MSI_EINTERNAL, "finishing the header");
      goto done;
    }
  }
done:
  if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
  return st;
}

msi_status msi_index_load(const char* path, const float* series, const msi_build_opts* opts, msi_index** out) {
  msi::set_last_error("");
  if (!path || !out) return fail(MSI_EINVAL, "path or out is NULL");
  *out = nullptr;
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return fail(MSI_EINVAL, std::string("cannot open ") + path);
  FileHeader h{};
  if (fread(&h, sizeof h, 1, in.f) != 1 || std::memcmp(h.magic, kMagic, 8) != 0)
    return fail(MSI_EINVAL, "not an index file");
  if (h.version != kVersion || h.header_bytes != sizeof(FileHeader))
    return fail(MSI_EINVAL, "unsupported index file version");
  const bool shape_ok = h.n >= 1 && h.n <= 0xfffffffeLL && h.len >= 1 && h.len <= MSI_MAX_LEN && h.w >= 1 &&
                        h.w <= MSI_MAX_SEGMENTS && h.len % h.w == 0 && h.seglen == h.len / h.w && h.card >= 2 &&
                        h.card <= MSI_MAX_CARDINALITY && (h.card & (h.card - 1)) == 0 && (1 << h.bits) == h.card &&
                        h.cap >= 1 && h.L >= 1 && h.L <= h.n && h.nblk == (h.n + 31) / 32 &&
                        (h.flags & ~(MSI_BUILD_BORROW | MSI_BUILD_BALANCED_SPLIT | MSI_BUILD_NO_FINE_BOUND)) == 0 &&
                        h.data_is_z == ((h.flags & MSI_BUILD_BORROW) ? 0 : 1);
  const bool tree = (h.flags & MSI_BUILD_BALANCED_SPLIT) != 0;
  const bool tree_ok = tree ? (h.root_bits == h.w && h.tree_nodes >= 1 && h.tree_nodes <= 2 * h.n + (1ll << h.w))
                            : (h.root_bits == 0 && h.tree_nodes == 0);
  if (!shape_ok || !tree_ok) return fail(MSI_EINVAL, "inconsistent index file header");
  const bool borrow = (h.flags & MSI_BUILD_BORROW) != 0;
  // the fine PAA's shape follows from the parameters, as in the build
  const int wf = (h.flags & MSI_BUILD_NO_FINE_BOUND) ? 0 : msi::fine_segments(h.len, h.w);
  if (borrow && !series) return fail(MSI_EINVAL, "the index borrows its collection: pass the same collection");
  if (!borrow && series) return fail(MSI_EINVAL, "the index holds its collection: series must be NULL");
  // the file size must match the header before anything is allocated
  {
    const size_t idx_bytes = (sizeof(uint4) + sizeof(uint32_t) + sizeof(float2)) * (size_t)h.n +
                             sizeof(uint32_t) * (size_t)(h.L + 1) + sizeof(uint4) * 2 * (size_t)h.L +
                             sizeof(uint4) * 2 * (size_t)h.nblk + sizeof(uint64_t) * (size_t)h.L;
    const size_t tree_bytes = tree ? (sizeof(int32_t) << h.root_bits) + 9 * (size_t)h.tree_nodes : 0;
    const size_t fine_bytes = sizeof(uint16_t) * (size_t)h.n * wf;
    const size_t want = sizeof(FileHeader) + idx_bytes + tree_bytes + fine_bytes +
                        (borrow ? 0 : sizeof(float) * (size_t)h.n * h.len);
    if (fseek(in.f, 0, SEEK_END) != 0) return fail(MSI_EINTERNAL, "seeking the index file");
    const long long got = ftell(in.f);
    if (got < 0 || (size_t)got != want) return fail(MSI_EINVAL, "truncated or oversized index file");
    if (fseek(in.f, sizeof(FileHeader), SEEK_SET) != 0) return fail(MSI_EINTERNAL, "seeking the index file");
  }
  const int32_t slots = (opts && opts->query_slots) ? opts->query_slots : msi::kDefaultQuerySlots;
  if (slots < 1 || slots > 64) return fail(MSI_EINVAL, "query_slots outside [1, 64]");
  const int32_t slot_cap = opts ? opts->slot_capacity : 0;
  if (slot_cap < 0) return fail(MSI_EINVAL, "slot_capacity is negative");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "no usable CUDA device");
  if (borrow) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, series) != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev) {
      cudaGetLastError();
      return fail(MSI_EINVAL, "a borrowed collection must be device memory on the current device");
    }
    if (((uintptr_t)series & 15u) != 0) return fail(MSI_EINVAL, "a borrowed collection must start on a 16-byte boundary");
  }
  msi_index* ix = new msi_index();
  ix->device = dev;
  ix->n = h.n;
  ix->len = h.len;
  ix->w = h.w;
  ix->card = h.card;
  ix->bits = h.bits;
  ix->seglen = h.seglen;
  ix->cap = h.cap;
  ix->flags = h.flags;
  ix->nslots = slots;
  ix->slot_cap = slot_cap;
  ix->L = h.L;
  ix->data_is_z = !borrow;
  ix->tree_nodes = h.tree_nodes;
  ix->root_bits = (int)h.root_bits;
  msi::breakpoint_edges(h.card, ix->h_thr_up, ix->h_thr_lo);
  Pinned stage;
  msi_status st = MSI_OK;
  std::vector<Section> secs;
  uint64_t sum = 1469598103934665603ull;
  const size_t tb = sizeof(float) * (size_t)(h.card + 1);
  if ((e = cudaStreamCreateWithFlags(&ix->own_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaMalloc(&ix->thr_up, tb)) != cudaSuccess || (e = cudaMalloc(&ix->thr_lo, tb)) != cudaSuccess ||
      (e = cudaMemcpy(ix->thr_up, ix->h_thr_up, tb, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ix->thr_lo, ix->h_thr_lo, tb, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&ix->words, sizeof(uint4) * (size_t)h.n)) != cudaSuccess ||
      (e = cudaMalloc(&ix->perm, sizeof(uint32_t) * (size_t)h.n)) != cudaSuccess ||
      (e = cudaMalloc(&ix->stats, sizeof(float2) * (size_t)h.n)) != cudaSuccess ||
      (e = cudaMalloc(&ix->leaf_begin, sizeof(uint32_t) * (size_t)(h.L + 1))) != cudaSuccess ||
      (e = cudaMalloc(&ix->env, sizeof(uint4) * 2 * (size_t)h.L)) != cudaSuccess ||
      (e = cudaMalloc(&ix->benv, sizeof(uint4) * 2 * (size_t)h.nblk)) != cudaSuccess ||
      (e = cudaMalloc(&ix->henv, sizeof(uint4) * 2 * (size_t)((h.n + 15) / 16))) != cudaSuccess ||
      (e = cudaMalloc(&ix->leaf_key, sizeof(uint64_t) * (size_t)h.L)) != cudaSuccess ||
      (tree && (e = cudaMalloc(&ix->root_child, sizeof(int32_t) << h.root_bits)) != cudaSuccess) ||
      (tree && (e = cudaMalloc(&ix->tree_child, 2 * sizeof(int32_t) * (size_t)h.tree_nodes)) != cudaSuccess) ||
      (tree && (e = cudaMalloc(&ix->tree_seg, (size_t)h.tree_nodes)) != cudaSuccess) ||
      (wf && (e = cudaMalloc(&ix->fine, sizeof(uint16_t) * (size_t)h.n * wf)) != cudaSuccess) ||
      (!borrow && (e = cudaMalloc(&ix->data_owned, sizeof(float) * (size_t)h.n * h.len)) != cudaSuccess) ||
      (e = cudaMallocHost(&stage.p, kStage)) != cudaSuccess) {
    st = cuda_fail(e, "allocating the index");
    goto fail_out;
  }
  ix->data = borrow ? series : ix->data_owned;
  ix->wf = wf;
  ix->sf = wf ? h.len / wf : 0;
  ix->device_bytes = (int64_t)2 * wf * h.n + (int64_t)(sizeof(uint4) + sizeof(uint32_t) + sizeof(float2)) * h.n +
                     (int64_t)(4 + 32 + 8) * h.L + 32 * h.nblk + 32 * ((h.n + 15) / 16) +
                     (borrow ? 0 : 4 * h.n * h.len);
  secs = sections(ix, h.nblk, !borrow);
  for (size_t si = 0; si < secs.size(); ++si) {
    const bool data = !borrow && si + 1 == secs.size();
    for (size_t off = 0; off < secs[si].bytes; off += kStage) {
      const size_t b = std::min(kStage, secs[si].bytes - off);
      if (fread(stage.p, 1, b, in.f) != b) {
        st = fail(MSI_EINVAL, "reading the index arrays");
        goto fail_out;
      }
      if (!data) sum = fnv1a(sum, (const unsigned char*)stage.p, b);
      if ((e = cudaMemcpy((char*)secs[si].dev + off, stage.p, b, cudaMemcpyHostToDevice)) != cudaSuccess) {
        st = cuda_fail(e, "copying the index to the device");
        goto fail_out;
      }
    }
  }
  if (sum != h.index_checksum) {
    st = fail(MSI_EINVAL, "index file checksum mismatch");
    goto fail_out;
  }
  // the half-block envelopes are not stored: computed from the loaded words
  if ((e = msi::block_envelopes_of(ix, ix->own_stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(ix->own_stream)) != cudaSuccess) {
    st = cuda_fail(e, "computing the block envelopes");
    goto fail_out;
  }
  *out = ix;
  return MSI_OK;
fail_out:
  msi::destroy_index(ix);
  return st;
}

}  // extern "C"
