/*
 * msi.h -- exact k-nearest-neighbour similarity search over an in-memory collection
 * of z-normalised data series summarised by iSAX, on one NVIDIA GB300 GPU (sm_103a).
 *
 * Method: MESSI (Peng, Fatourou, Palpanas, "MESSI: In-Memory Data Series Indexing").
 * The calls follow the paper's problem statement (Section II-A, "Similarity Search"):
 * given a collection of series of one length n and a query of that length, return
 * the series at the smallest Euclidean distance; here generalised to the k smallest.
 *
 * Conventions shared by every call:
 *  - Every call returns an msi_status; on failure msi_last_error() gives a detail
 *    string for the calling thread. No exception crosses this boundary.
 *  - Array arguments are plain pointers. Unless a call says otherwise a pointer may
 *    address host memory or device memory of the index's GPU; the library detects
 *    which (cudaPointerGetAttributes) and copies what it needs. The caller keeps
 *    ownership of everything it passes.
 *  - Layouts are row-major and densely packed: a collection is float[n][len].
 *  - `stream` arguments are cudaStream_t values passed as void*. NULL means the
 *    library's own stream, and the call returns only after its work is complete.
 *    With a non-NULL stream, work is ordered on that stream; outputs in host memory
 *    are complete when the call returns, outputs in device memory once the stream
 *    reaches the call's work.
 *  - Calls on one index must not overlap in time (they share the index's query
 *    workspace); distinct indexes are independent.
 */
#ifndef MSI_H
#define MSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point is exported from the shared library. */
#if defined(__GNUC__)
#define MSI_API __attribute__((visibility("default")))
#else
#define MSI_API
#endif

#define MSI_ABI_VERSION 3
#define MSI_MAX_SEGMENTS 16          /* one SAX word fits 16 bytes                    */
#define MSI_MAX_CARDINALITY 256      /* 8-bit symbols (Section II-B)                  */
#define MSI_MAX_LEN 4096             /* longest series                                */
#define MSI_MAX_K 1024               /* most neighbours per query                     */
#define MSI_DEFAULT_LEAF_CAPACITY 2000 /* leaf capacity used in Section IV            */

typedef enum msi_status {
  MSI_OK = 0,
  MSI_EINVAL = 1,     /* an argument is out of range, NULL, or the input holds NaN/inf */
  MSI_ENOMEM = 2,     /* device memory for the index or its workspace is short         */
  MSI_ECUDA = 3,      /* a CUDA runtime call failed (no device, launch failure, ...)   */
  MSI_ETIMEOUT = 4,   /* reserved: a bounded device-side wait ran out                  */
  MSI_EINTERNAL = 5   /* an internal consistency check failed                          */
} msi_status;

typedef struct msi_index msi_index; /* opaque; owns all the device memory it uses */

/* Build flags. */
#define MSI_BUILD_BORROW 0x1u /* index a DEVICE collection in place, without a copy: the
                                 caller keeps the buffer alive and unchanged until
                                 msi_free; distances z-normalise its values on the fly */
#define MSI_BUILD_BALANCED_SPLIT 0x2u /* split each node that exceeds the leaf capacity on the
                                 segment whose next symbol bit divides its members most
                                 evenly (Section II-B), and route the approximate search
                                 down that tree; default: one bit per level, segments in
                                 turn (both give exact answers)                        */
#define MSI_BUILD_NO_FINE_BOUND 0x4u /* keep no fine PAA. By default the index also stores
                                 each series' means over wf equal segments (wf = the
                                 largest of 64, 32, 16, 8 above `segments` that splits
                                 len into power-of-two lengths; none if no such wf) as
                                 fp16, 2 wf bytes per series, and the search bounds every
                                 series that passes the iSAX bound by them before it
                                 reads the series (a PAA lower bound, Section II-B, over
                                 finer segments; answers are the same either way)      */

typedef struct msi_build_opts {
  int32_t leaf_capacity; /* most series per leaf; 0 selects MSI_DEFAULT_LEAF_CAPACITY */
  uint32_t flags;        /* MSI_BUILD_* bits                                          */
  void* stream;          /* cudaStream_t or NULL                                       */
  int32_t query_slots;   /* Euclidean queries msi_knn runs at once; 0 selects 16, 1 runs*/
                         /* them one after another                                     */
  int32_t slot_capacity; /* candidates / survivors a concurrent slot holds; 0 selects  */
                         /* max(2^18, leaf_capacity + MSI_MAX_K) and max(2^22, n / 4); */
                         /* at most n each; a query                                   */
                         /* that needs more is run again with room for all n          */
} msi_build_opts;

/*
 * msi_build -- summarise a collection and build its index (Section III-A, Algorithms
 * 1-4: CreateIndex, IndexWorker, CalculateiSAXSummaries, TreeConstruction).
 *
 * Each series is z-normalised (Section II-A: mean 0, standard deviation 1, population
 * moments; a constant series becomes all zeros), cut into `segments` equal segments
 * whose means form its PAA (Section II-B), and each mean is quantised to one of
 * `cardinality` symbols against N(0,1) equiprobable breakpoints, giving the series'
 * iSAX word. Series are grouped into leaves of at most leaf_capacity members by the
 * bits of their words taken one bit of every segment at a time, most significant
 * first, splitting a group in two on the next bit while it is over capacity; the
 * first `segments` bits always split (the root fan-out of Section II-B). Each leaf
 * keeps the per-segment minimum and maximum symbol of its members.
 *
 *   series       float[n][len], host or device. Copied unless MSI_BUILD_BORROW.
 *   n            number of series, 1 .. 2^32-2.
 *   len          points per series, 1 .. MSI_MAX_LEN, a multiple of `segments`.
 *   segments     1 .. MSI_MAX_SEGMENTS.
 *   cardinality  a power of two in [2, 256].
 *   opts         NULL for the defaults.
 *   out          receives the index; set to NULL on failure (no partial index).
 * Errors: MSI_EINVAL (arguments; a series holding NaN or infinity), MSI_ENOMEM,
 * MSI_ECUDA.
 */
MSI_API msi_status msi_build(const float* series, int64_t n, int32_t len, int32_t segments,
                     int32_t cardinality, const msi_build_opts* opts, msi_index** out);

/*
 * msi_knn -- exact k-NN search, one query after another (Section III-B, Algorithms 5-9:
 * ExactSearch, SearchWorker, TraverseRootSubtree, ProcessQueue, CalculateRealDistance).
 *
 * Every query is z-normalised like the collection. The answer is exactly the k
 * series at the smallest Euclidean distance between z-normalised values, ordered by
 * distance and then by lower id (ties go to the lower id). The distance itself is
 * the square root of the FP64 sum of squared differences, rounded to float.
 *
 *   index    an index from msi_build.
 *   queries  float[nq][len], host or device.
 *   nq       number of queries, >= 0 (0 is a no-op).
 *   k        neighbours per query, 1 .. min(n, MSI_MAX_K).
 *   ids      int64[nq][k]: ids (row positions in the collection), host or device.
 *   dists    float[nq][k]: Euclidean distances, host or device; may be NULL.
 *   stream   see the conventions above.
 * With nq > 1 the queries run concurrently on the index's query slots
 * (msi_build_opts.query_slots), each slot on its own stream joined back to `stream`;
 * the call then waits for its work before returning, whatever the output memory.
 * Errors: MSI_EINVAL, MSI_ENOMEM (query workspace), MSI_ECUDA.
 */
MSI_API msi_status msi_knn(msi_index* index, const float* queries, int64_t nq, int32_t k, int64_t* ids,
                   float* dists, void* stream);

/*
 * msi_knn_ex -- msi_knn that also returns, per neighbour, the FP64 squared distance
 * the exact pick ordered by (the paper's answer is the BSF distance, Algorithm 5;
 * this is its squared FP64 value before rounding). Answers computed over disjoint
 * parts of a collection merge exactly by (sqdists64, id).
 *   sqdists64  double[nq][k], host or device; may be NULL (then this is msi_knn).
 * Other arguments and errors as msi_knn.
 */
MSI_API msi_status msi_knn_ex(msi_index* index, const float* queries, int64_t nq, int32_t k, int64_t* ids,
                              float* dists, double* sqdists64, void* stream);

/*
 * Exact k-NN under Dynamic Time Warping (Section IV, "MESSI with DTW"): the same
 * index, searched with the LB_Keogh envelope of each query (the per-segment maximum
 * of its upper envelope and minimum of its lower one give the iSAX lower bounds),
 * and DTW as the real distance, with a Sakoe-Chiba warping window of half-width
 * `window` points (the paper uses 10% of the length: window = len / 10):
 *   DTW^2(q, y) = D(len-1, len-1),  D(i, j) = (q_i - y_j)^2 + min(D(i-1, j-1),
 *   D(i-1, j), D(i, j-1)) for |i - j| <= window, D(-1, -1) = 0, +inf elsewhere,
 * on the z-normalised query and series. The answer is the k smallest by (FP64
 * DTW^2, id), like msi_knn_ex's; dists = sqrt(DTW^2) rounded to fp32 and
 * sqdists64 = the FP64 DTW^2 (either may be NULL).
 *   window  >= 0; values >= len mean an unconstrained warping (len - 1).
 * Other arguments, layouts and errors as msi_knn_ex; MSI_EINVAL for a negative
 * window.
 */
MSI_API msi_status msi_knn_dtw(msi_index* index, const float* queries, int64_t nq, int32_t k, int32_t window,
                               int64_t* ids, float* dists, double* sqdists64, void* stream);

/*
 * Writes the index to a file (no counterpart in the paper, which builds its index in
 * memory for every run, Section III-A): its parameters, its arrays (SAX words, leaf
 * order, per-series moments, leaves, envelopes, block envelopes, keys) with a
 * checksum, and for an index that owns its collection the z-normalised collection. A
 * borrowed collection (MSI_BUILD_BORROW) is not written.
 *   path  file name, created or truncated.
 * Waits for the device. Errors: MSI_EINVAL (NULL argument), MSI_ECUDA (device read),
 * MSI_EINTERNAL (file I/O; msi_last_error names the step).
 */
MSI_API msi_status msi_index_save(msi_index* index, const char* path);

/*
 * Reads an index written by msi_index_save onto the current device.
 *   series  for an index saved from a borrowed collection: the same collection, device
 *           memory on the current device, 16-byte aligned, kept alive by the caller;
 *           NULL for an index that holds its collection.
 *   opts    query_slots and slot_capacity as in msi_build (leaf capacity and flags
 *           come from the file); may be NULL.
 *   out     receives the index (free with msi_free).
 * The file is checked (magic, version, parameters, exact size, checksum of the index
 * arrays) before and while it is read. Errors: MSI_EINVAL (not an index file, a
 * truncated or inconsistent one, a series pointer missing or not expected),
 * MSI_ENOMEM / MSI_ECUDA; nothing is returned on error.
 */
MSI_API msi_status msi_index_load(const char* path, const float* series, const msi_build_opts* opts,
                                  msi_index** out);

/* Releases the index and all its device memory. NULL is a no-op. */
MSI_API void msi_free(msi_index* index);

/* Static name of a status code. */
MSI_API const char* msi_status_str(msi_status status);

/* Detail of the calling thread's last failure ("" if none). Valid until the thread's
 * next msi_* call. */
MSI_API const char* msi_last_error(void);

/* ABI version of the loaded library (MSI_ABI_VERSION). */
MSI_API int32_t msi_abi_version(void);

typedef struct msi_index_info {
  int64_t n;              /* series                                   */
  int32_t len;            /* points per series                        */
  int32_t segments;       /* PAA segments (word length in symbols)    */
  int32_t cardinality;    /* symbols per segment                      */
  int32_t leaf_capacity;  /* most series per leaf                     */
  int64_t leaves;         /* leaves built                             */
  int64_t device_bytes;   /* device memory the index holds            */
  uint32_t flags;         /* MSI_BUILD_* flags it was built with      */
  int32_t device;         /* CUDA device ordinal                      */
  int32_t fine_segments;  /* segments of the fine PAA (0: none kept)  */
} msi_index_info;

/* Shape and size of an index. `info` is a host pointer. */
MSI_API msi_status msi_index_info_get(const msi_index* index, msi_index_info* info);

/*
 * msi_index_export -- copy the index's summaries to HOST memory, for inspection and
 * tests. Every pointer may be NULL to skip that array.
 *   words       uint8[n][segments]: the iSAX word of each series, in collection order.
 *   perm        uint32[n]: collection id of the series at each leaf-order position.
 *   leaf_begin  uint32[leaves+1]: first leaf-order position of each leaf, then n.
 *   env_lo/hi   uint8[leaves][segments]: per-leaf minimum / maximum symbol.
 *   thresholds  float[cardinality-1]: the fp32 quantisation thresholds in use (the
 *               smallest float at or above each N(0,1) breakpoint).
 *   znorm       float[n][len]: z-normalised collection (collection order).
 *   fine        uint16[n][fine_segments]: the fine PAA, fp16 bit patterns, collection
 *               order (ignored when the index keeps none).
 */
typedef struct msi_export {
  uint8_t* words;
  uint32_t* perm;
  uint32_t* leaf_begin;
  uint8_t* env_lo;
  uint8_t* env_hi;
  float* thresholds;
  float* znorm;
  uint16_t* fine;
} msi_export;
MSI_API msi_status msi_index_export(const msi_index* index, const msi_export* out);

/*
 * msi_lower_bounds -- the iSAX lower bound (mindist between the query's PAA and an
 * iSAX region, Section II-B; used by Algorithms 7 and 9) of one query against every
 * series and every leaf, as the search computes it (fp32). HOST outputs.
 *   query     float[len], host or device (raw; z-normalised here).
 *   series_lb float[n] in collection order, or NULL.
 *   leaf_lb   float[leaves], or NULL.
 * A query holding NaN or infinity gets NaN bounds.
 */
MSI_API msi_status msi_lower_bounds(msi_index* index, const float* query, float* series_lb, float* leaf_lb,
                            void* stream);

/* Work counters of the msi_knn calls since the last reset (all queries summed). */
typedef struct msi_query_stats {
  int64_t queries;
  int64_t leaves_total;          /* leaves examined by the leaf filter              */
  int64_t leaves_survived;       /* leaves whose bound did not exceed the threshold */
  int64_t blocks_examined;       /* half-blocks of 16 leaf positions whose envelope  */
                                 /* bound passed                                    */
  int64_t series_lower_bounded;  /* per-series lower bounds computed                */
  int64_t series_refined;        /* real distances computed (seed leaf included)    */
  int64_t seed_series;           /* real distances of the approximate-search seed   */
  int64_t candidates;            /* (distance, id) pairs kept for the final pick    */
  int64_t rechecked;             /* FP64 re-computations at the k-th boundary       */
  int64_t refine_launches;       /* refinements timed (one per query)               */
  double refine_ms;              /* summed device time of q_filter_series and the   */
                                 /* row (or DTW) refinement (timing enabled only)   */
  double filter_ms;              /* the q_filter_series part of refine_ms           */
  int64_t kernel_launches;       /* kernels the query path launched (all queries)   */
  int64_t survivors;             /* series that passed the series filter (the SAX-  */
                                 /* word bound, then the fine PAA bound when the    */
                                 /* index keeps one; re-tested before refinement)   */
  int64_t fine_bounded;          /* series the series filter bounded by the fine PAA */
  int64_t front_fine_bounded;    /* front-leaf rows bounded by the fine PAA         */
  int64_t overflow_reruns;       /* batched queries whose bounded slot lists ran out */
  int64_t tc_pairs;              /* (series, query) pairs bounded by the tensor-core */
                                 /* filter                                          */
                                 /* of room and that ran again on the full workspace */
} msi_query_stats;

/* Reads the counters (host pointer), optionally resetting them. Reading synchronises
 * with the index's last call. */
MSI_API msi_status msi_query_stats_get(msi_index* index, msi_query_stats* stats, int32_t reset);

/* Enables (1) or disables (0) CUDA-event timing of the refinement kernels (events
 * recorded on the query stream around them; the call then waits for its work). */
MSI_API msi_status msi_set_timing(msi_index* index, int32_t enable);

/*
 * The schedule of batched msi_knn calls (nq > 1, Euclidean). The paper runs one
 * query after another (Section IV, "Setup"); here a call's queries run together in
 * one of two forms, with the same answers:
 *  - the batched chain (batch_chain = 1, the default): one kernel launch per stage of
 *    the search for a group of up to batch_group queries, each query with its own
 *    workspace and 1/batch_share of each persistent grid;
 *  - query slots (batch_chain = 0): each query runs its own chain of launches on one
 *    of query_slots streams, its grids divided by min(query_slots, grid_share).
 * msi_schedule_set changes it (MSI_EINVAL outside: query_slots 1..64, grid_share
 * 1..64, batch_group 1..1024, batch_share 1..64); msi_schedule_get reads it.
 */
typedef struct msi_schedule {
  int32_t batch_chain;
  int32_t query_slots;
  int32_t grid_share;
  int32_t batch_group;
  int32_t batch_share;
  int32_t batch_overlap;  /* chain form: 1 launches each stage early (programmatic
                             dependent launch) so it starts as the previous ends */
  int32_t batch_dense;    /* chain form: 1 replaces the leaf, block and series filters
                             by the tensor-core filter (one streaming pass over the
                             collection per pass of queries; len a multiple of 4,
                             at most 2048) */
  int32_t batch_order;    /* chain form: 1 refines the series filter's survivors in
                             ascending lower-bound order (a bucket sort per query) */
} msi_schedule;
MSI_API msi_status msi_schedule_set(msi_index* index, const msi_schedule* schedule);
MSI_API msi_status msi_schedule_get(const msi_index* index, msi_schedule* schedule);

/*
 * msi_autotune -- choose the batched-query schedule of an index by measurement.
 * This call times msi_knn on `queries` (nq >= 2 of them, host or device, as msi_knn)
 * with k neighbours for every candidate schedule: the batched chain with groups of
 * {32, 64, 128} queries (at most nq) and batch shares {1, 2, 4, 8}; the same with the
 * tensor-core filter (groups of one filter pass, shares {1, 4}) where len allows it;
 * query slots {4, 8, 12, 16, 24, 32} with grid shares {1, 2, 3, 4, 6} up to the slot
 * count.
 * Each candidate runs `reps` timed calls (0 selects 3) after three untimed ones, with
 * CUDA events on `stream` (NULL: the index's stream). The fastest schedule
 * (queries/s) stays with the index; answers are the same under every schedule. `out`
 * (host, may be NULL) receives the choice. Workspaces the choice does not use are
 * released.
 * Errors: MSI_EINVAL for a NULL index or queries, nq < 2 or k outside msi_knn's
 * range; MSI_ENOMEM / MSI_ECUDA as msi_knn. On error the index keeps its schedule.
 */
typedef struct msi_tune_result {
  int32_t query_slots;   /* the schedule chosen (slots form)                     */
  int32_t grid_share;
  double queries_per_s;  /* its measured rate                                    */
  int32_t candidates;    /* schedules measured                                   */
  double default_queries_per_s;  /* the rate of the index's schedule before tuning */
  int32_t batch_chain;   /* the form chosen, and its group and share (chain form) */
  int32_t batch_group;
  int32_t batch_share;
  int32_t batch_dense;   /* the tensor-core filter chosen                        */
} msi_tune_result;
MSI_API msi_status msi_autotune(msi_index* index, const float* queries, int64_t nq, int32_t k, int32_t reps,
                                msi_tune_result* out, void* stream);

/*
 * Serving: a request loop over several resident indexes with continuous batching.
 * The paper answers one query after another (Section IV, "Setup"); this has no
 * counterpart there. Each index gets query slots (a bounded workspace, a stream and
 * staging buffers); a dispatcher thread admits waiting requests into free slots as
 * soon as slots free up, so requests arriving while others run join the work in
 * flight. Answers are exactly those of msi_knn. Indexes attached to a server must
 * not be used by other calls until the server is freed.
 */
typedef struct msi_server msi_server;

typedef struct msi_server_opts {
  int32_t slots_per_index;  /* query slots per index, the first with room for any query; */
                            /* 0 selects 8; each divides the grids by at most 3       */
  int64_t workspace_bytes;  /* device bytes the bounded slots may use (admission by     */
                            /* memory: slots beyond it are not created); 0 selects 8 GiB */
  int32_t max_inflight;     /* most queries on the GPU at once; 0: no cap, 1: one at a time */
  int32_t slot_capacity;    /* candidate / survivor room of a bounded slot (0: default)  */
} msi_server_opts;

/* Starts a server over n_indexes indexes (host array of handles); opts may be NULL.
 * Errors: MSI_EINVAL, MSI_ENOMEM (slots), MSI_ECUDA. */
MSI_API msi_status msi_server_create(msi_index* const* indexes, int32_t n_indexes, const msi_server_opts* opts,
                                     msi_server** out);

/* Queues one query (HOST memory, float[len] of index `index_no`) for its k nearest
 * neighbours (1 .. min(n, MSI_MAX_K)); *ticket names it for msi_server_wait. */
MSI_API msi_status msi_server_submit(msi_server* server, int32_t index_no, const float* query, int32_t k,
                                     uint64_t* ticket);

/* Waits for a ticket's answer: ids int64[k] and dists float[k] (HOST memory; dists
 * may be NULL) and the time from submission to completion in ms (may be NULL). */
MSI_API msi_status msi_server_wait(msi_server* server, uint64_t ticket, int64_t* ids, float* dists,
                                   double* latency_ms);

/* Requests completed, queries rerun on a full workspace, and slots in use. */
MSI_API msi_status msi_server_stats(msi_server* server, int64_t* completed, int64_t* reruns, int32_t* slots);

/* Finishes the queued requests, stops the loop and releases the slots. */
MSI_API void msi_server_free(msi_server* server);

/*
 * msi_merge_topk -- the one exchange of a search over a collection split across GPUs
 * by contiguous ranges of series. Every series is summarised and searched on its own
 * (Section III), so each range is indexed and searched alone; the answer over the
 * whole collection is the k smallest of the ranges' answers in (FP64 squared
 * distance, collection id) order, which is the order msi_knn_ex returns.
 *   ids        int64[parts][nq][k_in]: each part's answer (collection ids, distinct
 *              across parts), each row sorted by (sqdists64, id) as msi_knn_ex gives it.
 *   sqdists64  double[parts][nq][k_in]: the FP64 squared distances of those ids.
 *   out_ids    int64[nq][k]; out_dists float[nq][k] = sqrt rounded to fp32 (may be NULL);
 *              out_sqdists64 double[nq][k] (may be NULL). Ascending (distance, id).
 * Arrays may be host or device memory (host arrays are staged through a temporary
 * device buffer). Stream as for every call (NULL: the call waits).
 * Errors: MSI_EINVAL (NULL pointers; parts < 1; k_in or k outside [1, 1024]; k above
 * parts * k_in), MSI_ENOMEM, MSI_ECUDA.
 */
MSI_API msi_status msi_merge_topk(const int64_t* ids, const double* sqdists64, int32_t parts, int64_t nq,
                                  int32_t k_in, int32_t k, int64_t* out_ids, float* out_dists,
                                  double* out_sqdists64, void* stream);

/*
 * msi_lower_bounds_noalloc -- msi_lower_bounds for callers that cannot allocate
 * device memory. The paper has no counterpart: it exists for code that must not
 * call cudaMalloc, such as code held to a device-memory budget by an allocator or
 * pool it does not own (an allocation behind its back breaks the budget), and
 * latency-critical paths that must not wait on the driver's allocator (cudaMalloc
 * can synchronise the device).
 *
 * It computes the same lower bounds, with the same kernels, and calls no cudaMalloc,
 * cudaFree or allocating library routine: the per-query temporaries (query state,
 * z-normalised query, per-segment gap tables, counters; 38,144 bytes) live in one
 * fixed file-scope device array that every GPU loading the library holds until the
 * process exits. Every call shares that array and finds the previous call's contents
 * in it (it clears what must start at zero); calls whose work overlaps on the GPU
 * race on it, so the caller serialises them. The first call on a device looks up the
 * array's device address (once per device); make that first call before any stream
 * capture begins.
 *
 *   index      an index from msi_build (its query workspace is not used).
 *   query      float[len] in DEVICE memory of the index's GPU (raw; z-normalised here).
 *   series_lb  float[n] in DEVICE memory: bound per series, collection order.
 *   leaf_lb    float[leaves] in DEVICE memory: bound per leaf.
 *   stream     cudaStream_t or NULL (NULL: the legacy default stream, and the call
 *              waits for its work and reports a non-finite query). A non-finite
 *              query gets NaN in every output, so a caller that passes a stream
 *              and does not wait still cannot take it for a bound.
 * Errors: MSI_EINVAL (NULL or host pointers; an index whose len exceeds 4096 or whose
 * segments * cardinality exceeds 4096 does not fit the fixed scratch; a non-finite
 * query), MSI_ECUDA.
 */
MSI_API msi_status msi_lower_bounds_noalloc(const msi_index* index, const float* query, float* series_lb,
                                            float* leaf_lb, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MSI_H */
