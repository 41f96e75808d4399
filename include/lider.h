/*
 * lider.h -- C ABI of LIDER batched query search on one B300 (sm_103a).
 *
 * LIDER (arXiv 2205.00970) indexes dense embeddings with a clustering-based
 * two-layer architecture (Sec. 3.2): k-means clusters, and inside each cluster
 * a core model made of ESK-LSH hashkey arrays (Sec. 4), key re-scaling
 * (Sec. 5.1) and one simplified two-stage RMI per array (Sec. 5.2).  A query
 * is routed to its nearest clusters, hashed, located in every sorted array,
 * expanded bi-directionally, and its candidates are scored by exact inner
 * product; the per-cluster top-k lists are merged (Sec. 3.3.2, Sec. 6.2).
 *
 * Conventions for every entry point:
 *   - return LIDER_OK (0) on success, a negative LIDER_E* code otherwise; the
 *     message of the last failure on the calling thread is lider_last_error();
 *   - no C++ exception crosses this boundary;
 *   - pointers documented "device" must be CUDA device (or managed) memory on
 *     the current device; "host" pointers are ordinary host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is enqueued on it and, unless stated otherwise, the
 *     call returns before that work completes;
 *   - matrices are row-major FP32 with rows of d contiguous floats;
 *   - there is no CPU fallback: without a usable CUDA device every call that
 *     needs one fails with LIDER_ECUDA.
 */
#ifndef LIDER_H_
#define LIDER_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LIDER_OK        0
#define LIDER_EINVAL   -1   /* an argument is out of range or inconsistent   */
#define LIDER_ENOMEM   -2   /* a device allocation failed                     */
#define LIDER_ECUDA    -3   /* a CUDA runtime call or kernel launch failed    */
#define LIDER_ELIMIT   -4   /* a size exceeds a documented implementation cap */
#define LIDER_ETIMEDOUT -5  /* lider_server_wait: the request is still running */

#define LIDER_HASH_PSTABLE    0  /* h = floor((a.x + b) / W), Sec. 4.1 (p-stable)    */
#define LIDER_HASH_HYPERPLANE 1  /* h = [a.x >= 0], Sec. 4.1 (random hyperplane, one
                                    bit per hash; b and W are not used)          */

/* How a query picks its c clusters (Sec. 3.2 and Sec. 3.3.2). */
#define LIDER_ROUTE_EXACT 0   /* exact scan: the c best scores q.mu - |mu|^2/2 over
                                 all centroids                                     */
#define LIDER_ROUTE_CORE  1   /* Layer-1 centroids retriever: a core model (the same
                                 ESK-LSH projections, sorted arrays and RMIs) over
                                 the centroids; the query is located and expanded
                                 by r0 * c positions in each array and the c best of
                                 the centroids found, by the same score, are probed */

/* How candidates are scored.  SIMT, TENSOR and F16 return the same results
 * bit for bit: the exact FP32 top-k of each query's candidate union (the two
 * tensor modes select by an approximate score plus a guard band of twice its
 * proven error bound, then re-score that list exactly on the CUDA cores). */
#define LIDER_SCORE_TENSOR 0   /* tcgen05 tensor cores, 3 TF32 products per FP32 product */
#define LIDER_SCORE_SIMT   1   /* FP32 FMA on the CUDA cores                             */
#define LIDER_SCORE_BF16   2   /* served form: BF16 corpus copy scored on the tensor
                                  cores (FP32 accumulation), then an FP32 re-rank of a
                                  shortlist of rerank * k candidates per query (not
                                  exact: a candidate may miss the shortlist)          */
#define LIDER_SCORE_F16    3   /* tcgen05 tensor cores on FP16 copies of the corpus and
                                  queries (each scaled by a power of two), FP32
                                  accumulation, guard band, exact FP32 re-score      */
#define LIDER_SCORE_FP8    4   /* served form: FP8 e4m3 corpus copy with one scale per
                                  row (max|x|/448), queries likewise, FP32
                                  accumulation, then an FP32 re-rank of a shortlist
                                  of rerank * k (not exact); needs d % 16 == 0      */

/* Implementation caps (checked; LIDER_ELIMIT beyond them). */
#define LIDER_MAX_L        32      /* hashkey arrays per core model (H)     */
#define LIDER_MAX_C        32      /* clusters probed per query (c_0)       */
#define LIDER_MAX_K        1024    /* results per query                     */
#define LIDER_MAX_LR       4096    /* L * R candidates per (query, cluster) */
#define LIDER_MAX_D        4096    /* embedding dimension                   */

typedef struct lider_index lider_index;   /* opaque; owns its device memory */

/* Index parameters, in the paper's notation (Table 1):
 *   L  = H, number of hashkey arrays (LSH repetitions) per core model;
 *   m  = M, hashes per hashkey; p-stable: each packs into floor(64/m) bits
 *        with offset 2^(floor(64/m)-1) and clamping; hyperplane: one bit each
 *        (a 64-bit sortable key either way);
 *   rmi_leaves = width of the RMI second stage (linear models per array);
 *   r0 = expansion factor, R = r0 * k positions per array (Sec. 6.1);
 *   B  = elements read by KD_e in the extended hashkey distance dist_e
 *        (Sec. 4.2); (bits per element) * B must be <= 56;
 *   hash_kind = LIDER_HASH_PSTABLE or LIDER_HASH_HYPERPLANE;
 *   W  = p-stable bucket width (> 0);
 *   score_mode = LIDER_SCORE_TENSOR, LIDER_SCORE_SIMT, LIDER_SCORE_BF16,
 *        LIDER_SCORE_F16 or LIDER_SCORE_FP8 (tensor modes need L <= 16; BF16
 *        and F16 need d % 8 == 0, FP8 d % 16 == 0);
 *   rerank = shortlist factor of LIDER_SCORE_BF16 / FP8: rerank * k candidates per
 *        query are re-scored in FP32 (0 means 4);
 *   route_kind = LIDER_ROUTE_EXACT (0) or LIDER_ROUTE_CORE (1, needs
 *        n_clusters <= 8192);
 *   raw_keys = 0: the RMIs learn re-scaled keys (Sec. 5.1, the method);
 *        1: they learn the raw 64-bit key values converted to FP64, without
 *        re-scaling (the ablation of Sec. 7.4; see rmi_oor below). */
typedef struct {
    int32_t L;
    int32_t m;
    int32_t rmi_leaves;
    int32_t r0;
    int32_t B;
    int32_t hash_kind;
    double  W;
    int32_t score_mode;
    int32_t rerank;
    int32_t route_kind;
    int32_t raw_keys;
} lider_params;

/* Counters of one search (host struct, filled when the call returns). */
typedef struct {
    int64_t n_queries;
    int64_t pairs;             /* (query, probed cluster) pairs searched          */
    int64_t candidates;        /* unique candidates scored, summed over pairs      */
    int64_t qkey_boundary;     /* query hash values within 1e-6*W of a bucket edge */
    int64_t qkey_clamped;      /* query hash values clamped into the element range */
    int64_t locate_fallback;   /* lower bounds found outside the RMI error window  */
    int64_t empty_pairs;       /* probed clusters that hold no point               */
    int64_t tc_tiles;          /* 128 x 256 tensor-core tiles computed (tensor path) */
    int64_t route_fallback;    /* tensor paths: queries whose routing shortlist was
                                  too close to call and were routed by an exact
                                  scan of all centroids                          */
    int64_t select_overflow;   /* guarded tensor paths (TENSOR, F16): queries whose
                                  guard band of near-tied candidates did not fit
                                  the re-score list; their whole band is then
                                  re-scored exactly by a second kernel, so the
                                  top k stays exact (0 in normal operation)      */
    /* RMI diagnostics of Sec. 7.4, over every (query, probed cluster, array):
     * the prediction p^ is out of range (OOR) when it was clamped to 0 or
     * n_c - 1, i.e. it equals either end; it is a large error (LE) when
     * |p^ - p*| > k, p* being the exact lower bound of the query key. */
    int64_t rmi_oor;
    int64_t rmi_le;
    int64_t rmi_oor_le;        /* both */
    int64_t passes;            /* passes the batch was searched in (lider_search) */
} lider_search_stats;

/* Phases of one search, in order; events[i] is recorded when phase i starts
 * and events[LIDER_NUM_PHASES] when the last one ends. */
#define LIDER_PHASE_HASH    0   /* query hashkeys (Sec. 4.1)                        */
#define LIDER_PHASE_ROUTE   1   /* top-c centroids (Sec. 3.3.2)                     */
#define LIDER_PHASE_GROUP   2   /* (query, cluster) pairs bucketed by cluster       */
#define LIDER_PHASE_LOCATE  3   /* re-scale, RMI, bounded search, expansion         */
#define LIDER_PHASE_GATHER  4   /* queries gathered per cluster and candidate
                                   bitmaps marked (tensor modes only)              */
#define LIDER_PHASE_SCORE   5   /* candidate scores (SIMT mode: also per-pair top-k)*/
#define LIDER_PHASE_SELECT  6   /* per-query selection (tensor modes only)          */
#define LIDER_PHASE_MERGE   7   /* SIMT: per-query merge of the c lists (Sec. 6.2);
                                   tensor modes: FP32 re-score of the selection    */
#define LIDER_NUM_PHASES    8

/* Optional per-step outputs of a search, for parity checking and profiling.
 * Every member may be NULL; non-NULL array members are device arrays the
 * caller allocates:
 *   route  [nq*c]    probed clusters of each query, best first;
 *   qkeys  [nq*L]    packed query hashkeys;
 *   pstar  [nq*c*L]  lower bound of the query key in each probed cluster's array
 *                    (cluster-local position);
 *   wstart [nq*c*L]  start of the expansion window (cluster-local);
 *   wlen   [nq*c*L]  its length, min(R, n_c);
 *   ucount [nq*c]    unique candidates scored in each probed cluster;
 *   events           host array of LIDER_NUM_PHASES + 1 cudaEvent_t handles
 *                    (entries may be NULL), recorded on the search stream at
 *                    the phase boundaries; the caller creates and owns them. */
typedef struct {
    int32_t*  route;
    uint64_t* qkeys;
    int32_t*  pstar;
    int32_t*  wstart;
    int32_t*  wlen;
    int32_t*  ucount;
    void* const* events;
} lider_trace;

/* How lider_build clusters the corpus (Sec. 3.2: k-means) and seeds its
 * random draws.
 *   n_clusters    the paper's c, number of k-means clusters (1 .. training rows);
 *   kmeans_iters  Lloyd iterations (0 keeps the initial rows as centroids);
 *   kmeans_sample k-means learns from the first min(kmeans_sample, n) corpus
 *                 rows (0: all n); every row is then partitioned;
 *   seed          the initial centroids are the Forgy rows of the training
 *                 rows that Floyd's sampling algorithm draws from SplitMix64
 *                 started at `seed` (draw i = mix64(seed + (i+1)*0x9E3779B97F4A7C15),
 *                 uniform integer on [0, j] = draw mod (j+1); rows in ascending
 *                 order become centroids 0, 1, ...); when lider_build gets no
 *                 projections it also draws them from `seed`. */
typedef struct {
    int32_t  n_clusters;
    int32_t  kmeans_iters;
    int64_t  kmeans_sample;
    uint64_t seed;
} lider_cluster_params;

/* Build an index from a corpus alone (Sec. 3.3.2 "LIDER is built as follows";
 * Sec. 3.2 for the clustering, Sec. 3.3.1 for one core model; Table 5 stages
 * 1-3), on the device:
 *   1. k-means: Lloyd iterations from the Forgy rows of `cluster`; each round
 *      assigns every training row to the centroid maximising x.mu - |mu|^2/2
 *      (exact up to FP64 rounding: compensated dot products finished in FP64;
 *      ties to the lower index) and moves each centroid to the FP64 mean of its
 *      rows, rounded to FP32 (a cluster left empty keeps its centroid);
 *   2. partition of all n rows by the same nearest-centroid rule;
 *   3. hashing, segment sorts and RMI fits, as for lider_build_centroids.
 *   corpus     device, n x d FP32, the embeddings (n >= 1, d % 4 == 0);
 *   cluster    host, see lider_cluster_params;
 *   A, b       device, (L*m) x d and (L*m) FP32: row l*m+j of A and entry
 *              l*m+j of b define hash j of array l (the LSH draws, Sec. 4.1);
 *              both NULL: drawn on the device from cluster->seed (A ~ N(0,1)
 *              by Box-Muller from SplitMix64 draws, b ~ U[0, W)); the draws
 *              can be read back with lider_export_projections;
 *   params     host, see lider_params;
 *   stream     the build runs on it and is synchronised before returning;
 *   out        host, receives the new index.
 * The caller keeps ownership of its buffers.  Errors: those of
 * lider_build_centroids; LIDER_EINVAL also for a NULL `cluster`, only one of
 * A and b given, kmeans_iters outside [0, 100000], kmeans_sample < 0, or
 * n_clusters above the training rows.  On error *out is NULL. */
int lider_build(const float* corpus, int64_t n, int32_t d, const lider_cluster_params* cluster,
                const float* A, const float* b, const lider_params* params, void* stream,
                lider_index** out);

/* Build an index from given centroids (Sec. 3.3.2; Sec. 3.3.1 for one core
 * model; Table 5 stages 2-3): no clustering runs.
 *   corpus     device, n x d FP32, the embeddings (n >= 1, d % 4 == 0);
 *   centroids  device, n_clusters x d FP32, the k-means centroids; every point
 *              joins the centroid maximising x.mu - |mu|^2/2 (ties: lower index);
 *   A, b       device, (L*m) x d and (L*m) FP32, as for lider_build (required);
 *   params     host, see lider_params;
 *   stream     the build runs on it and is synchronised before returning;
 *   out        host, receives the new index.
 * The corpus, centroids and projections are copied; the caller keeps
 * ownership of its buffers.  Errors: LIDER_EINVAL for null pointers, n < 1,
 * d % 4 != 0, n_clusters < 1, L/m/r0/B/rmi_leaves < 1, W <= 0 (p-stable),
 * an unknown hash_kind, route_kind or raw_keys, or (bits per element)*B > 56;
 * LIDER_ELIMIT past the caps above (and n_clusters > 8192 with
 * LIDER_ROUTE_CORE);
 * LIDER_ENOMEM / LIDER_ECUDA from the device.  On error *out is NULL. */
int lider_build_centroids(const float* corpus, int64_t n, int32_t d,
                          const float* centroids, int32_t n_clusters,
                          const float* A, const float* b,
                          const lider_params* params, void* stream, lider_index** out);

/* How an index was built (host output). */
typedef struct {
    int32_t  clustered;          /* 1: k-means ran in lider_build; 0: centroids given */
    int32_t  projections_drawn;  /* 1: A and b were drawn from the seed               */
    lider_cluster_params cluster;/* the clustering parameters (clustered == 1)         */
    int64_t  train_rows;         /* rows k-means learned from (clustered == 1)         */
    int32_t  empty_clusters;     /* clusters that hold no corpus row                   */
    int32_t  reserved;
    double   kmeans_ms;          /* host wall time of the k-means iterations           */
    double   build_ms;           /* host wall time of the whole build                  */
} lider_build_info;

int lider_get_build_info(const lider_index* index, lider_build_info* info);

/* Copy the index's FP32 centroids (n_clusters x d, host) / the cluster of
 * every corpus row (n int32, host, indexed by corpus row id) / the LSH draws
 * (A: (L*m) x d FP32 and b: L*m FP32, host; either may be NULL).
 * Synchronous. */
int lider_export_centroids(const lider_index* index, float* centroids_host);
int lider_export_assignment(const lider_index* index, int32_t* asg_host);
int lider_export_projections(const lider_index* index, float* A_host, float* b_host);

/* Batched k-NN search (Sec. 3.3.2 "When using LIDER for ANN queries"; Sec. 6).
 *   queries     device, nq x d FP32, starting on a 16-byte boundary;
 *   k           results per query (1..LIDER_MAX_K); R = r0*k, L*R <= LIDER_MAX_LR;
 *   c           clusters probed per query, c_0 (1..min(n_clusters, LIDER_MAX_C));
 *   out_ids     device, nq x k int64: corpus row ids, best first (score
 *               descending, ties by lower id), -1 past the candidates found;
 *   out_scores  device, nq x k FP32: exact inner products, -inf where id = -1;
 *   stats       host or NULL; when non-NULL the call synchronises `stream`
 *               and fills the counters;
 *   stream      the call's work is ordered on it: in the tensor score modes
 *               (default route) independent steps run on a second stream the
 *               index owns, forked from `stream` and joined back to it by
 *               events, so the results are complete in `stream` order, and
 *               under stream capture those steps join the captured graph.
 * Scratch memory comes from a stream-ordered pool owned by the index, so
 * concurrent calls on different streams are safe (their steps on the
 * index's second stream run one after another); the index is read-only.
 * nq == 0 is a no-op.  Errors: LIDER_EINVAL (null index/pointers, nq < 0,
 * k < 1, c < 1 or c > n_clusters), LIDER_ELIMIT (caps), LIDER_ENOMEM,
 * LIDER_ECUDA. */
int lider_search(const lider_index* index, const float* queries, int64_t nq,
                 int32_t k, int32_t c, int64_t* out_ids, float* out_scores,
                 lider_search_stats* stats, void* stream);

/* lider_search plus the optional per-step outputs of `trace` (may be NULL). */
int lider_search_trace(const lider_index* index, const float* queries, int64_t nq,
                       int32_t k, int32_t c, int64_t* out_ids, float* out_scores,
                       const lider_trace* trace, lider_search_stats* stats,
                       void* stream);

/* End-to-end form of lider_search on HOST buffers: copies queries (host,
 * nq x d FP32; pinned memory gives asynchronous copies) to the device,
 * searches, copies ids/scores back into host arrays of nq x k, and
 * synchronises `stream` before returning.  Same arguments, errors and passes
 * as lider_search; the copies of each pass's queries run on a second stream
 * in up to four chunks, each chunk's hash and route starting when it lands.
 * Result arrays in pinned, mapped host memory are written by the search
 * itself (no copy back).  Device memory: the whole batch's queries (and,
 * unless the results are mapped, its results) plus one pass's scratch. */
int lider_search_host(const lider_index* index, const float* queries_host, int64_t nq,
                      int32_t k, int32_t c, int64_t* ids_host, float* scores_host,
                      lider_search_stats* stats, void* stream);

/* Device scratch, in bytes, that lider_search takes from the index's pool for
 * one call of this shape (host computation only; no device is touched).  A
 * server uses it to admit batches against a memory budget.  Writes 0 for
 * nq == 0.  Errors: those of lider_search's argument checks, and
 * LIDER_EINVAL for a NULL `bytes`. */
int lider_search_scratch_bytes(const lider_index* index, int64_t nq, int32_t k,
                               int32_t c, size_t* bytes);

/* Bytes of the fixed device scratch used by lider_search_noalloc. */
#define LIDER_NOALLOC_SCRATCH_BYTES (64u << 20)

/* lider_search without any device allocation (the paper has no counterpart:
 * this serves callers that cannot allocate device memory while they search,
 * e.g. a service that reserved its whole GPU budget up front, or code running
 * while another framework owns the CUDA allocator).
 * Same arguments, results and errors as lider_search, except:
 *   - scratch is one fixed device array of LIDER_NOALLOC_SCRATCH_BYTES that
 *     every GPU loading this library holds until the process exits; a batch
 *     whose scratch would not fit is rejected with LIDER_ELIMIT (search fewer
 *     queries per call; the need grows with nq * c * L * r0 * k);
 *   - the first call on a device (and the first after the device's context
 *     changed, e.g. after a reset) looks up the array's device address; make
 *     it before any stream capture;
 *   - all calls share the array: calls that overlap on the GPU race and must
 *     be serialised by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
int lider_search_noalloc(const lider_index* index, const float* queries, int64_t nq,
                         int32_t k, int32_t c, int64_t* out_ids, float* out_scores,
                         lider_search_stats* stats, void* stream);

/* ---------------------------------------------------------------------------
 * Continuous-batching server (the paper has no counterpart: this serves a
 * stream of independent requests through the batched search above).
 *
 * A request is a block of queries on the host, a k, and host buffers for its
 * results.  A scheduler thread packs pending requests of equal k, oldest first,
 * into batches of at most max_batch queries and launches a batch when one of
 * `slots` execution slots (each a CUDA stream with its own pinned and device
 * staging) is free and the search scratch of the batches in flight, plus this
 * one, stays within mem_budget bytes; while batches are in flight it waits up
 * to max_wait_us for more requests before launching a partly filled batch.  A
 * completion thread finishes batches in launch order, copies each request's
 * rows into its buffers and records its latency (submission to results).
 * A request gets exactly the ids and scores lider_search gives for its queries
 * alone.  All functions are thread-safe.  mem_budget counts search scratch
 * only: the index itself and the fixed LIDER_NOALLOC_SCRATCH_BYTES array that
 * every GPU loading the library holds are outside it. */
typedef struct lider_server lider_server;

typedef struct {
    int32_t c;            /* clusters probed per query (as in lider_search)          */
    int32_t slots;        /* batches in flight, 1..16                                */
    int32_t max_batch;    /* queries per batch; a request may not exceed it          */
    int32_t max_k;        /* largest k a request may ask for (<= LIDER_MAX_K)         */
    int64_t mem_budget;   /* bytes of search scratch the batches in flight may hold  */
    double max_wait_us;   /* batching window while the device is busy, >= 0           */
} lider_server_params;

typedef struct {
    int64_t requests;              /* completed requests                             */
    int64_t queries;               /* completed queries                              */
    int64_t batches;               /* completed batches                              */
    int64_t refused;               /* requests rejected by lider_server_submit       */
    int64_t failed;                /* requests whose batch failed                    */
    int32_t max_inflight_batches;
    int32_t reserved;
    int64_t max_inflight_bytes;    /* largest scratch held by batches in flight      */
    double launch_s;               /* host time gathering and enqueueing batches     */
    double finish_s;               /* host time waiting for and scattering batches   */
} lider_server_counters;

/* Start a server over `index` (which must outlive it).  Allocates the slots'
 * staging (pinned host and device) and starts two host threads.  Errors:
 * LIDER_EINVAL (NULL arguments, c, slots, max_batch, max_k, mem_budget or
 * max_wait_us out of range), LIDER_ELIMIT (a batch of max_batch queries with
 * max_k would exceed lider_search's caps), LIDER_ENOMEM, LIDER_ECUDA. */
int lider_server_create(const lider_index* index, const lider_server_params* params,
                        lider_server** out);

/* Enqueue a request: queries_host nq x d FP32, results into ids_host and
 * scores_host (nq x k each, as lider_search writes them).  The three buffers
 * belong to the server until lider_server_wait reports the request done.
 * *ticket identifies the request.  nq == 0 completes at once.  Errors:
 * LIDER_EINVAL (NULL pointers, nq < 0, k < 1, server stopping), LIDER_ELIMIT
 * (nq > max_batch, k > max_k, or scratch above mem_budget). */
int lider_server_submit(lider_server* server, const float* queries_host, int64_t nq,
                        int32_t k, int64_t* ids_host, float* scores_host, int64_t* ticket);

/* Wait up to timeout_s seconds (< 0: no limit) for a request.  LIDER_OK once
 * its results are in its buffers (each ticket can be waited for once);
 * LIDER_ETIMEDOUT if it is still running; LIDER_EINVAL for an unknown or
 * already waited ticket; the batch's error code if its batch failed. */
int lider_server_wait(lider_server* server, int64_t ticket, double timeout_s);

/* Counters since the server started (host output). */
int lider_server_stats(lider_server* server, lider_server_counters* stats);

/* Copy up to cap per-request latencies in milliseconds (completion order) to
 * out_ms; *total receives how many are recorded.  clear != 0 drops them all
 * afterwards (e.g. after a warm-up). */
int lider_server_latencies(lider_server* server, double* out_ms, int64_t cap,
                           int32_t clear, int64_t* total);

/* Finish every submitted request, stop the threads, free the staging.  NULL
 * is accepted. */
void lider_server_destroy(lider_server* server);

/* ---------------------------------------------------------------------------
 * Launch shapes of the tensor-path kernels (the paper has no counterpart).
 * They change speed only: results are the same for every setting. */
typedef struct {
    int32_t select_threads;   /* per-query select block: 64, 128, 256 or 512           */
    int32_t rescore_threads;  /* per-query re-score block: 64, 128, 256 or 512         */
    int32_t mark_threads;     /* per-pair bitmap block: 32, 64, 128 or 256             */
    int32_t tile_order;       /* tensor tiles of a cluster: 0 query tiles outer, 1 row
                                 tiles outer (a row tile's query tiles run together)   */
    int32_t probe_batch;      /* queries per pass of lider_search (>= 0; 0: the whole
                                 batch); a batch larger than one pass allows (the caps
                                 of LIDER_ELIMIT, or a scratch budget of 48 GiB and at
                                 most 3/4 of the device memory free after the build)
                                 is searched in passes of half as many, halved until
                                 one fits                                           */
} lider_tuning;

/* Current launch shapes of the index (host output). */
int lider_get_tuning(const lider_index* index, lider_tuning* tuning);

/* Set them; LIDER_EINVAL for a value outside the sets above.  Not thread-safe
 * against searches running on the same index. */
int lider_set_tuning(lider_index* index, const lider_tuning* tuning);

/* Pick the launch shapes by measurement: starting from the current ones, each
 * field in turn takes the value whose searches of `queries` (device, nq x d,
 * with k and c) run fastest (median of `reps` timed searches after one
 * warm-up, CUDA events on `stream`), two rounds.  Keeps the best in the index
 * and returns it in *chosen (may be NULL) with its median time in *best_ms
 * (may be NULL).  Synchronous.  Errors: those of lider_search; LIDER_EINVAL
 * for reps < 1. */
int lider_autotune(lider_index* index, const float* queries, int64_t nq, int32_t k, int32_t c,
                   int32_t reps, lider_tuning* chosen, double* best_ms, void* stream);

/* Index shape, host outputs (any may be NULL). */
int lider_index_info(const lider_index* index, int64_t* n, int32_t* d,
                     int32_t* n_clusters, lider_params* params);

/* Cluster sizes as offsets, host array of n_clusters + 1 entries: points of
 * cluster j are rows offsets[j]..offsets[j+1]-1 of the index's reordered copy. */
int lider_cluster_offsets(const lider_index* index, int64_t* offsets_host);

/* Copy one sorted hashkey array of one core model to host memory (parity
 * checks).  keys_host: n_c uint64 keys in SK-LSH order; ids_host: n_c corpus
 * row ids (int64), equal keys ordered by id.  Synchronous. */
int lider_export_array(const lider_index* index, int32_t cluster, int32_t array,
                       uint64_t* keys_host, int64_t* ids_host);

/* Copy the RMI of one (cluster, array) to host memory.  Synchronous.
 *   minmax_host [2]   x_min, x_max of the re-scaling (Sec. 5.1);
 *   root_host   [2]   intercept, slope of the first stage;
 *   leaf_host   [2*F] intercept, slope of each leaf;
 *   err_host    [2*F] error window [lo, hi] of each leaf: for every key of the
 *                     leaf, lo <= first position of that key - prediction <= hi. */
int lider_export_rmi(const lider_index* index, int32_t cluster, int32_t array,
                     uint64_t* minmax_host, double* root_host, double* leaf_host,
                     int32_t* err_host);

/* Self-test of the tensor-core scoring engine (tcgen05 + TMA + TMEM):
 * out[m x n] = A[m x d] . B[n x d]^T for device row-major FP32 A, B, out with
 * 1 <= m <= 128, 1 <= n <= 256.  kind 0: three TF32 products per FP32 product
 * (d % 4 == 0); kind 1: A and B rounded to BF16, one product, FP32
 * accumulation (d % 8 == 0); kind 2: the same with FP16 (values outside
 * FP16's range saturate or flush; no scaling).  Synchronous; allocates its
 * own scratch.
 * LIDER_ECUDA if an internal wait times out (the kernel then exits cleanly). */
int lider_debug_tc_tile(const float* A, int32_t m, const float* B, int32_t n, int32_t d,
                        int32_t kind, float* out, void* stream);

/* Test of the engine's bounded waits (the paper has no counterpart): the same
 * one-tile run as lider_debug_tc_tile, but every wait of the engine gives up
 * after limit_ms milliseconds (0 < limit_ms <= 10000) and the TMA producer
 * leaves the first stage of K unloaded, so the MMA warp's wait for it runs
 * out.  The kernel records the code of the first wait that gave up, raises
 * its abort flag, lets the other warps leave, waits (with the same limit) for
 * the stages it did load, frees its TMEM and returns; the call then returns
 * LIDER_ECUDA with "wait timed out (code N)" in lider_last_error() (N: 1 empty
 * stage, 2 full stage, 3 accumulator full, 4 accumulator empty, 5 drain).  No
 * memory access is skipped or faults; the device stays usable.  Synchronous. */
int lider_debug_tc_wait_expiry(const float* A, int32_t m, const float* B, int32_t n, int32_t d,
                               int32_t kind, float* out, double limit_ms, void* stream);

/* Release the index and its device memory.  NULL is accepted. */
void lider_free(lider_index* index);

/* Message of the last failed call on this thread ("" if none). */
const char* lider_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LIDER_H_ */
