/*
 * kann.h -- C ABI of the B300 (sm_103a) batched HNSW search library.
 *
 * The library runs the query-time path of the composable ANN method of
 * kANNolo (Delfino et al., 2025): k-NN search -- for a query, find the k
 * dataset vectors closest to it (problem statement, Sec. 1) -- over an HNSW graph (Sec. 2,
 * citing Malkov & Yashunin) whose items are dense vectors (L2 or inner
 * product), Product-Quantization codes (Sec. 2, citing Jegou et al.) or
 * sparse term/weight vectors (Sec. 3, Table 1).
 *
 * Conventions shared by every call:
 *   - Every call returns an int status (KANN_OK = 0 or a KANN_E* code);
 *     kann_status_str() names it.  Nothing is launched when a call fails
 *     argument validation.
 *   - Distances are "smaller is better": L2 = sum (q - x)^2 (squared, no
 *     root), IP = -sum q * x.  Results are ordered by the total order on
 *     (distance, id): distance first (NaN counts as +inf), then id.
 *   - Pointers named d_* are DEVICE pointers owned by the caller.  The index
 *     borrows them: the caller keeps them alive and unchanged until
 *     kann_index_destroy().  The index owns only a small host-side record.
 *   - Pointers named h_* are HOST pointers, read or written before the call
 *     returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Search and exact-k-NN calls are asynchronous on it; the only
 *     host synchronisation is inside kann_index_upload's validation.
 *   - Integer ids are int32 (n < 2^31).  Missing results are id -1 with
 *     distance +inf.
 */
#ifndef KANN_H
#define KANN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------*/
#define KANN_OK 0
#define KANN_EINVAL 1   /* bad argument (null pointer, size, k/ef range, alignment) */
#define KANN_ENOMEM 2   /* a host allocation or the shared-memory budget failed */
#define KANN_ECUDA 3    /* a CUDA runtime call failed; see kann_last_cuda_error() */
#define KANN_EFORMAT 4  /* graph/vector description is inconsistent (ids out of range, degree caps) */
#define KANN_ETIMEOUT 5 /* a bounded device wait ran out */

/* ---- per-query status bits (optional d_status output of kann_search_ex) -*/
#define KANN_QSTAT_HOPCAP 1u    /* layer-0 expansions hit opts.max_hops; result is the W reached */
#define KANN_QSTAT_FORGOT 2u    /* the visited table forgot ids (cleared, or an id found no free slot;
                                   results unaffected, the forgotten ids were evaluated again) */
#define KANN_QSTAT_BAD_ID 4u    /* an adjacency entry >= n was met and skipped */
#define KANN_QSTAT_QUERY_TRUNCATED 8u /* sparse query with more than 512 terms: the terms after the first
                                         512 (in term order) were dropped */

/* ---- enums --------------------------------------------------------------*/
#define KANN_L2 0
#define KANN_IP 1

#define KANN_F32 0   /* IEEE binary32 */
#define KANN_F16 1   /* IEEE binary16, round-to-nearest-even from FP32 */
#define KANN_BF16 2  /* bfloat16, round-to-nearest-even from FP32 */
#define KANN_E4M3 3  /* OCP FP8 E4M3 with a per-vector FP32 scale s: x = s * code */

#define KANN_PQ_LUT_F32 0       /* kann_search_opts.pq_lut */
#define KANN_PQ_LUT_F16 1
#define KANN_PQ_LUT_U8 2

#define KANN_VISITED_AUTO 0     /* kann_search_opts.visited_format */
#define KANN_VISITED_COMPACT 1
#define KANN_VISITED_WIDE 2

/* Search limits of this build. */
#define KANN_MAX_EF 1024    /* ef_eff = max(ef, k) must not exceed this */
#define KANN_MAX_M0 64      /* layer-0 degree cap (M0 = 2M, so M <= 32) */
#define KANN_MAX_DIM 4096   /* dense dimension */
#define KANN_MAX_EXPAND 4   /* kann_search_opts.expand */

/* ---- index descriptions -------------------------------------------------*/

/* The HNSW graph (Malkov & Yashunin), serialised with fixed-width rows.
 *   d_level      [n] int8      level of each node (0 = layer 0 only)
 *   d_l0         [n][M0] int32 layer-0 neighbours, -1 padded
 *   d_upper_slot [n] int32     row of the node in d_upper, -1 if level 0
 *   d_upper      [n_upper][max_level][M] int32, layer l at index l - 1,
 *                -1 padded (may be NULL when max_level == 0)
 * entry is the entry point (a node of level max_level). */
typedef struct {
  int64_t n;
  int32_t M;
  int32_t M0;
  int32_t max_level;
  int32_t entry;
  int64_t n_upper;
  const int8_t* d_level;
  const int32_t* d_l0;
  const int32_t* d_upper_slot;
  const int32_t* d_upper;
} kann_graph_desc;

/* Dense vectors [n][d] in `dtype`, rows `row_stride_bytes` apart (a multiple
 * of 16, >= d * element size; d * element size must itself be a multiple of
 * 16).  d_scale [n] FP32 is required for KANN_E4M3 and ignored otherwise. */
typedef struct {
  int32_t dtype;
  int32_t d;
  int32_t metric;
  int32_t reserved;
  const void* d_data;
  const float* d_scale;
  int64_t row_stride_bytes;
} kann_vectors_desc;

/* Product quantization (Jegou et al.): m subspaces of dsub dims, ksub = 256
 * centroids each; d_codes [n][m] uint8, d_codebooks [m][256][dsub] FP32.
 * The ADC distance is sum_j LUT[j][code_j] with the per-query table LUT built
 * on the device for `metric`. */
typedef struct {
  int32_t m;
  int32_t ksub;
  int32_t dsub;
  int32_t metric;
  const uint8_t* d_codes;
  const float* d_codebooks;
} kann_pq_desc;

/* Sparse vectors in CSR: d_indptr [n+1] int64, d_terms [nnz] uint16 sorted
 * and unique within a row, d_weights [nnz] FP32; term ids < vocab.
 * Measure: IP (distance = -sum over shared terms of w_q * w_x). */
typedef struct {
  const int64_t* d_indptr;
  const uint16_t* d_terms;
  const float* d_weights;
  int32_t vocab;
  int32_t reserved;
} kann_sparse_desc;

typedef struct kann_index kann_index_t;

/* Build a device-resident index from caller-owned device arrays (Sec. 2:
 * the dataset holds the items and their encoding, the index decides which
 * items a query is compared with).  Exactly one traversal source
 * must be given: `v` (dense), `pq`, or `sp`.  `rerank` (nullable) is a dense
 * KANN_F32 (exact) or KANN_BF16 copy of the same items with the same d and
 * metric, used to re-rank the traversal's best candidates.  The graph's metadata and
 * degree caps are validated on the host; with `validate_ids` != 0 the
 * adjacency arrays are also scanned on the device for ids outside [0, n)
 * (one synchronising call).  On success *out owns a host record only.
 * Errors: KANN_EINVAL (nulls, sizes, alignment), KANN_EFORMAT (metadata or
 * ids inconsistent), KANN_ECUDA, KANN_ENOMEM. */
int kann_index_upload(kann_index_t** out, const kann_graph_desc* g, const kann_vectors_desc* v,
                      const kann_pq_desc* pq, const kann_sparse_desc* sp, const kann_vectors_desc* rerank,
                      int validate_ids);

/* Release the host record.  Borrowed device arrays are untouched. */
int kann_index_destroy(kann_index_t* idx);

/* Optional search settings (zero-initialise, then set what is needed). */
typedef struct {
  int32_t rerank;          /* 0: no re-rank; R > 0: re-rank the best min(R, |W|) traversal
                              candidates from the index's rerank copy (FP32 arithmetic);
                              -1: R = ef_eff.  R must be >= k. */
  int32_t max_hops;        /* cap on layer-0 expansions per query; 0 = 1,000,000 */
  int32_t hash_bits;       /* log2 of the slots of the per-query visited table (5..16);
                              0 = automatic (4,096 compact slots; wide: >= 8 efmax, 1,024..8,192) */
  int32_t warps_per_block; /* dense and sparse: queries per CTA (one warp each); 0 = automatic.
                              A PQ search always runs one query per CTA of 8 warps that
                              share the query's lookup table */
  int32_t lanes_per_row;   /* lanes sharing one row gather (power of two <= 32); 0 = automatic */
  int32_t lean;            /* dense rows of 2 chunks per lane: 1 = half the row batches in
                              flight for a 64-register budget (more warps per SM), -1 = off,
                              0 = automatic (off) */
  int32_t pq_lut;          /* PQ index only: the per-query table's format.
                              KANN_PQ_LUT_F32 (0): FP32 entries.
                              KANN_PQ_LUT_F16 (1): FP16 (entries scaled by the power of two
                              that brings the largest |entry| to at most 2^15, rounded to
                              nearest; each row's FP32 sum scaled back): half the shared memory.
                              KANN_PQ_LUT_U8 (2): uint8 values v = rint(clamp((entry - min_j) /
                              scale, 0, 255)), min_j the minimum of subspace j, scale = (largest
                              max_j - min_j) / 255, entries in FP32: a quarter of the shared
                              memory (four queries per SM at m = 192).  Rows are ordered by the
                              exact integer sum of their values; the distance reported (without
                              re-rank) is sum_j min_j + scale * sum (two FP32 roundings). */
  uint32_t* d_status;      /* [n] per-query KANN_QSTAT_* bits, nullable */
  int32_t* d_counters;     /* [n][4] per-query counters, nullable: layer-0 distance
                              evaluations, layer-0 expansions, upper-layer distance
                              evaluations, upper-layer hops */
  int32_t* d_work_counter; /* non-null: persistent work-stealing launch (one CTA set per SM,
                              each warp takes the next query from this device counter,
                              which the call zeroes on `stream` first); null: one warp per
                              query in a plain grid */
  const int32_t* d_n;      /* persistent mode only, nullable: device int holding the number
                              of queries to run (clamped to n), read by the kernel -- lets a
                              captured CUDA graph serve batches of varying size */
  int32_t visited_format;  /* visited table: 0 = automatic (compact when the index allows),
                              1 = compact: 16-bit slots in buckets of 8, an id stored as an
                              invertible multiply of its bits split into bucket and slot value
                              (needs n <= 2^(hash_bits + 12); KANN_EINVAL otherwise),
                              2 = wide: 32-bit id slots.  Both may forget ids (a forgotten id
                              is evaluated again), neither reports an unvisited id as visited,
                              so results do not depend on this choice */
  int32_t expand;          /* dense indices: layer-0 entries expanded per step.  0 or 1 = the
                              HNSW search step (one expansion, the parity form); 2..KANN_MAX_EXPAND
                              = a batched variant that marks that many best unexpanded entries
                              expanded at once, evaluates all their unvisited neighbours in one
                              batch and keeps the ef best -- a different search (it may expand an
                              entry the one-at-a-time step would evict first), with more rows in
                              flight per dependent step; its results are defined by that rule,
                              not by the one-expansion search.  PQ and sparse indices: KANN_EINVAL
                              unless 0 or 1.  max_hops counts expansions */
  int32_t team;            /* dense and sparse indices: warps sharing one query.  0 or 1 = one
                              warp per query (warps_per_block of them per CTA); 2 or 4 = one
                              query per CTA of that many warps: warp 0 runs the search and at
                              every distance and re-rank batch each warp evaluates one slice
                              of the candidates, every row by one lane group as in the one-warp
                              search, so results are identical bit for bit (more warps per SM
                              when each query's shared memory limits them; warps_per_block is
                              then ignored).  PQ indices always run teams of 8 warps and take
                              0 only; with expand > 1: KANN_EINVAL unless 0 or 1 */
} kann_search_opts;

/* HNSW K-NN-SEARCH (Malkov & Yashunin Alg. 5) for n dense FP32 queries
 * d_queries [n][d]: greedy descent from the entry point through layers
 * max_level..1, then the ef-bounded beam on layer 0 (ef_eff = max(ef, k)),
 * one expansion per step in (distance, id) order, then the k best.
 * Outputs d_ids [n][k] int32 and d_dists [n][k] FP32.  For a PQ index the
 * queries are the raw FP32 vectors (d = m * dsub) and the per-query ADC
 * table is built on the device.  n == 0 is a no-op.
 * Errors: KANN_EINVAL (k < 1, ef_eff > KANN_MAX_EF, sparse index, nulls). */
int kann_search(const kann_index_t* idx, const float* d_queries, int n, int k, int ef, int32_t* d_ids,
                float* d_dists, void* stream);

/* kann_search with options (re-rank, status, counters, tuning). */
int kann_search_ex(const kann_index_t* idx, const float* d_queries, int n, int k, int ef, int32_t* d_ids,
                   float* d_dists, const kann_search_opts* opts, void* stream);

/* Mixed batch: query i uses k = d_k[i] and ef = d_ef[i] (both device int32
 * arrays; 1 <= k <= kmax, ef_eff <= efmax).  Outputs are [n][kmax]; entries
 * past query i's k are id -1 / +inf.  Same search as kann_search_ex. */
int kann_search_batch(const kann_index_t* idx, const float* d_queries, int n, const int32_t* d_k,
                      const int32_t* d_ef, int kmax, int efmax, int32_t* d_ids, float* d_dists,
                      const kann_search_opts* opts, void* stream);

/* Device bytes a batch of n queries (k <= kmax, ef <= efmax) needs besides
 * the index, for admission by device memory: the caller's query rows (n * d
 * FP32; for a sparse index only the CSR offsets, (n + 1) * 8 -- term and
 * weight bytes come on top), per-query k and ef words (8 n), the outputs
 * (n * kmax * 8), per-query status words (4 n) and the persistent launch's
 * two counters (8).  The search itself allocates no device memory: beam,
 * candidates and visited table live in shared memory.  Returns 0 when no
 * search with these settings can run (null index, n < 0, kmax < 1,
 * max(efmax, kmax) > KANN_MAX_EF, or a per-warp shared-memory need above the
 * device's limit). */
size_t kann_search_workspace_bytes(const kann_index_t* idx, int n, int kmax, int efmax);

/* kann_search_workspace_bytes for a search with options `opts` (nullable =
 * defaults): the same byte count, and 0 exactly when kann_search_batch with
 * these n, kmax, efmax and options would be refused (argument checks and the
 * shared-memory plan are the search's own -- for example a PQ table in FP16
 * fits where the FP32 table does not, and a PQ search that needs it gives up
 * visited-table bits to fit).  The pointer options (d_status, d_counters,
 * d_work_counter, d_n) are ignored. */
size_t kann_search_workspace_bytes_ex(const kann_index_t* idx, int n, int kmax, int efmax,
                                      const kann_search_opts* opts);

/* Sparse-query search over a sparse index: queries in CSR (d_q_indptr [n+1]
 * int64, d_q_terms uint16 sorted unique per row, d_q_weights FP32). */
int kann_search_sparse(const kann_index_t* idx, const int64_t* d_q_indptr, const uint16_t* d_q_terms,
                       const float* d_q_weights, int n, int k, int ef, int32_t* d_ids, float* d_dists,
                       const kann_search_opts* opts, void* stream);

/* Exact k-NN by brute force (the ground truth recall is measured against):
 * d_queries [nq][d] and d_base [nb][d], both in `dtype` (KANN_F32 or
 * KANN_BF16 / KANN_F16 for the tensor-core path), row-major, contiguous.
 * Scores for L2 are ||x||^2 - 2 q.x (+ ||q||^2) accumulated in FP32; the k best
 * per query are returned sorted by (distance, id) in d_ids / d_dists.
 * d_ws is caller-owned device scratch of at least
 * kann_exact_knn_workspace_bytes(...) bytes.  d_queries, d_base and d_ws
 * must be 16-byte aligned, d_ids and d_dists 4-byte aligned, and d a
 * multiple of 4.  Errors: KANN_EINVAL (sizes, nulls, alignment; nothing is
 * launched). */
int kann_exact_knn(const void* d_queries, const void* d_base, int nq, int64_t nb, int d, int metric, int dtype,
                   int k, int32_t* d_ids, float* d_dists, void* d_ws, size_t ws_bytes, void* stream);

size_t kann_exact_knn_workspace_bytes(int nq, int64_t nb, int d, int k, int dtype);

/* Exact k-NN for sparse inner product (ground truth of the sparse measure):
 * base CSR (d_indptr [nb+1], d_terms, d_weights) and query CSR (d_q_indptr
 * [nq+1], d_q_terms, d_q_weights), term ids < vocab (vocab * 4 bytes plus
 * 16 KB must fit one CTA's shared memory: vocab <= ~50k).  Distance = -IP in
 * FP32; d_ids / d_dists [nq][k] sorted by (distance, id); k <= 128.  Cost is
 * one full pass over the base per query: meant for sampled ground truth. */
int kann_exact_knn_sparse(const int64_t* d_indptr, const uint16_t* d_terms, const float* d_weights, int64_t nb,
                          const int64_t* d_q_indptr, const uint16_t* d_q_terms, const float* d_q_weights, int nq,
                          int vocab, int k, int32_t* d_ids, float* d_dists, void* stream);

/* kann_exact_knn_noalloc: the same exact k-NN, for callers that cannot
 * allocate device memory -- for example code running inside a host
 * application whose device memory is owned by another allocator (a
 * framework's caching allocator, an inference server that reserves the
 * whole GPU up front), or latency-critical paths where cudaMalloc is not
 * allowed because it can synchronise the device.  It calls no cudaMalloc,
 * cudaFree or other allocating routine: its scratch is one static device
 * array of KANN_NOALLOC_SCRATCH_BYTES per GPU, held by every GPU that loads
 * this library until the process exits.  The caller still passes inputs and
 * outputs as for kann_exact_knn.
 *   - The first call on a device looks up that array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.  The address is kept for the life of the process: after
 *     cudaDeviceReset (or any other teardown of the device's primary context)
 *     the kept address is stale, so do not call this function again in that
 *     process.
 *   - Arguments and their alignment are checked as for kann_exact_knn.
 *   - Returns KANN_EINVAL when the request needs more scratch than the array
 *     holds, i.e. kann_exact_knn_workspace_bytes(nq, nb, d, k, dtype) >
 *     KANN_NOALLOC_SCRATCH_BYTES (split the queries into smaller batches).
 *   - Every call shares the array, which keeps the previous call's contents
 *     (nothing in it needs to start at zero).  Calls that overlap on the GPU
 *     (concurrent streams, or several host threads) race on it: serialise
 *     them.
 * The paper has no counterpart to this call. */
#define KANN_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int kann_exact_knn_noalloc(const void* d_queries, const void* d_base, int nq, int64_t nb, int d, int metric,
                           int dtype, int k, int32_t* d_ids, float* d_dists, void* stream);

/* Convert FP32 rows d_x [n][d] to a storage format on the device:
 * KANN_F16 / KANN_BF16 (round to nearest even) into d_out [n][d] 16-bit, or
 * KANN_E4M3 with per-row scale s = max|x| / 448 (FP32 division) and codes
 * RNE_satfinite(x / s) into d_out [n][d] uint8 and d_scale [n] (an all-zero
 * row gets s = 0 and zero codes).  Asynchronous on `stream`. */
int kann_quantize(const float* d_x, int64_t n, int d, int dtype, void* d_out, float* d_scale, void* stream);

/* ---- PQ codebooks (device) -------------------------------------------------
 * Product Quantization (Sec. 2, citing Jegou et al.) as index preparation:
 * kann_pq_train trains 256 centroids per subspace (m subspaces of
 * dsub = d / m <= 16 dims) on FP32 rows d_x [n][d] (n >= 256): k-means++
 * seeding (centroid c drawn with the counter-based SplitMix64 uniform keyed by
 * (seed ^ (j + 1) * 0xD1B54A32D192ED03, c), the first row whose running sum of
 * squared distances to the nearest centroid so far reaches u * the total),
 * then `iters` Lloyd iterations (nearest centroid, strictly smaller wins;
 * means; an empty centroid moves to the farthest row), all in FP64 -- the
 * steps of the oracle's reading, equal to it bit for bit on integer data.
 * Writes d_codebooks [m][256][dsub] (FP32, rounded from FP64); d_ws is
 * caller scratch of kann_pq_train_workspace_bytes(n, d, m).  kann_pq_encode
 * writes d_codes [n][m]: nearest centroid per subspace under L2 in FP32, ties
 * to the lowest index.  Both are asynchronous on `stream`. */
size_t kann_pq_train_workspace_bytes(int64_t n, int d, int m);
int kann_pq_train(const float* d_x, int64_t n, int d, int m, int iters, uint64_t seed, float* d_codebooks, void* d_ws,
                  size_t ws_bytes, void* stream);
int kann_pq_encode(const float* d_x, int64_t n, int d, int m, const float* d_codebooks, uint8_t* d_codes,
                   void* stream);

/* ---- graph construction (host, multi-threaded) ---------------------------
 * The indexing pipeline of the paper (Sec. 2, Fig. 1) ends in an HNSW graph;
 * search treats it as a fixed input.  These host calls build one in the
 * serialised layout above from FP32 dense rows h_x [n][d] or a CSR sparse set.
 *
 * kann_hnsw_levels: the level of every node, level = floor(-ln U / ln M)
 * with U in (0, 1] from a counter-based SplitMix64 draw keyed by (seed, id);
 * writes h_level [n] and returns max_level and n_upper for sizing.
 *
 * kann_hnsw_build_dense / _sparse: insert ids 0..n-1 with `nthreads` threads
 * (0 = all cores), Malkov & Yashunin's neighbour-selection heuristic, degree
 * caps M (upper layers) and 2M (layer 0).  Output arrays are caller-owned
 * host buffers sized by kann_hnsw_levels: h_l0 [n][2M], h_upper_slot [n],
 * h_upper [n_upper][max_level][M]; *h_entry receives the entry point. */
int kann_hnsw_levels(int64_t n, int M, uint64_t seed, int8_t* h_level, int32_t* h_max_level, int64_t* h_n_upper);

int kann_hnsw_build_dense(const float* h_x, int64_t n, int d, int metric, int M, int ef_construction, uint64_t seed,
                          int nthreads, const int8_t* h_level, int32_t* h_l0, int32_t* h_upper_slot,
                          int32_t* h_upper, int32_t* h_entry);

int kann_hnsw_build_sparse(const int64_t* h_indptr, const uint16_t* h_terms, const float* h_weights, int64_t n,
                           int M, int ef_construction, uint64_t seed, int nthreads, const int8_t* h_level,
                           int32_t* h_l0, int32_t* h_upper_slot, int32_t* h_upper, int32_t* h_entry);

/* ---- graph construction (layer 0 on the device) ---------------------------
 * The same HNSW (Malkov & Yashunin Alg. 1 with the Alg. 4 heuristic, caps M
 * and 2M, levels from kann_hnsw_levels) with the layer-0 insertions on the
 * GPU.  The nodes of level >= 1 (about n / M) are inserted first, on the host
 * with `nthreads` threads (all their layers); the level-0 nodes follow in id
 * order, in batches of at most 1/32 of the nodes already inserted (and
 * at most `batch`, 0 = 65,536): each batch node's efConstruction best
 * candidates come from the library's search on the graph so far, it keeps up
 * to M of them by the heuristic, and each kept neighbour appends the node to
 * its list or, past 2M, shrinks its list with the same heuristic.  Nodes of
 * one batch do not link to each other, and a node takes at most 16 reverse
 * links per batch (the others keep their forward edge only).  Distances are
 * FP32.  d_x [n][d] FP32 device rows (16-byte aligned, d a multiple of 4);
 * h_level [n] host levels; outputs are caller-owned device arrays sized as
 * for kann_hnsw_build_dense: d_l0 [n][2M], d_upper_slot [n], d_upper
 * [n_upper][max_level][M] (may be NULL when max_level == 0); *h_entry
 * receives the entry point.  d_ws is device scratch of
 * kann_hnsw_build_device_workspace_bytes(n, d, M, ef_construction, batch)
 * bytes.  Synchronises `stream` (the host part needs the upper nodes' rows).
 * Errors: KANN_EINVAL, KANN_ECUDA. */
size_t kann_hnsw_build_device_workspace_bytes(int64_t n, int d, int M, int ef_construction, int batch);
int kann_hnsw_build_device(const float* d_x, int64_t n, int d, int metric, int M, int ef_construction, uint64_t seed,
                           int batch, int nthreads, const int8_t* h_level, int32_t* d_l0, int32_t* d_upper_slot,
                           int32_t* d_upper, int32_t* h_entry, void* d_ws, size_t ws_bytes, void* stream);

/* The same build over sparse vectors (the sparse IP measure, Sec. 3 Table 1):
 * device CSR d_indptr [n+1] int64, d_terms uint16 (sorted, unique per row,
 * < vocab), d_weights FP32 with nnz = d_indptr[n] entries; distance -IP in
 * FP32 (a merge-join of the two term lists).  The batch nodes are searched
 * with kann_search_sparse (a node's first 512 terms).  d_ws holds
 * kann_hnsw_build_device_sparse_workspace_bytes(n, nnz, M, ef_construction,
 * batch) bytes (the batch queries are gathered there as a CSR). */
size_t kann_hnsw_build_device_sparse_workspace_bytes(int64_t n, int64_t nnz, int M, int ef_construction, int batch);
int kann_hnsw_build_device_sparse(const int64_t* d_indptr, const uint16_t* d_terms, const float* d_weights,
                                  int64_t n, int vocab, int M, int ef_construction, uint64_t seed, int batch,
                                  int nthreads, const int8_t* h_level, int32_t* d_l0, int32_t* d_upper_slot,
                                  int32_t* d_upper, int32_t* h_entry, void* d_ws, size_t ws_bytes, void* stream);

/* ---- diagnostics --------------------------------------------------------*/
const char* kann_status_str(int status);
/* The cudaError_t of the most recent failed CUDA call in this thread. */
int kann_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KANN_H */
