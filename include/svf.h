/*
 * svf.h -- C ABI of the B300 (sm_103a) streaming graph-ANNS hot path of
 * SVFusion (arXiv 2601.08528): Build / Search / Insert / Delete over a
 * vector store X_t and a fixed out-degree proximity graph G_t (Sec. 2.2,
 * Sec. 2.3).
 *
 * Conventions
 *  - Every call returns int: SVF_OK (0) or a negative SVF_E* code; the text
 *    of the last error of the calling thread is svf_last_error().
 *  - Pointers marked "device" are CUDA device pointers on the current
 *    device; "host" pointers are ordinary CPU memory.  `stream` is a
 *    cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Work is enqueued asynchronously on `stream`; outputs are valid once the
 *    stream is synchronised.  Errors found on the device (a bad id in a
 *    delete batch, an exhausted wait) are written to the index's status word
 *    and returned by svf_sync() and by the next call on the index.
 *  - Ownership: every device buffer is allocated by the caller (sizes from
 *    svf_buffer_sizes) and BORROWED by the index, which allocates no device
 *    memory.  The index itself is a small host object freed by svf_destroy.
 *  - A call that fails validation changes nothing.
 *  - Ids are 0-based uint32, assigned densely in insertion order and never
 *    reused (the paper numbers host ids from 1, Sec. 4.2); ids must stay
 *    below 2^30.  SVF_EMPTY marks an unused graph slot / missing result.
 *  - Distances: squared L2, or the negated inner product -<q,x> (so smaller
 *    is nearer in both).  Every order is lexicographic (distance, id).
 */
#ifndef SVF_H
#define SVF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SVF_OK 0
#define SVF_EINVAL (-1)    /* bad argument (sizes, ids, null pointers) */
#define SVF_ECAPACITY (-2) /* n_used + m would exceed n_cap */
#define SVF_ECUDA (-3)     /* a CUDA runtime call failed */
#define SVF_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define SVF_EBOUNDS (-5)   /* a device-side range check failed */
#define SVF_EDEVICE (-6)   /* other device-side error */

#define SVF_EMPTY 0xFFFFFFFFu

enum svf_dtype { SVF_F32 = 0, SVF_U8 = 1, SVF_BF16 = 2, SVF_FP8 = 3 };
enum svf_metric { SVF_L2 = 0, SVF_IP = 1 };
enum svf_prune_mode { SVF_PRUNE_RNG = 0, SVF_PRUNE_RANK = 1 };

/* Index parameters.
 *   d        dimension, a multiple of 16, 16..2048
 *   dtype    primary store: SVF_F32 or SVF_U8 (u8 distances are exact int32)
 *   metric   SVF_L2 or SVF_IP
 *   R        out-degree: 32 or 64 (Sec. 2.3: fixed out-degree KNNG)
 *   n_cap    capacity in vectors (< 2^30)
 *   prune    neighbour reordering rule (Sec. 5.1): SVF_PRUNE_RNG counts
 *            candidates j < i with dist(c_j, c_i) < dist(v, c_i);
 *            SVF_PRUNE_RANK counts j < i whose list contains c_i
 *   repair_c entries taken from each deleted neighbour's list in the
 *            localized repair (Sec. 5.2; the paper uses c = 8)
 *   lowp     bit 0: keep a bfloat16 copy, bit 1: keep an FP8-E4M3 copy with
 *            a per-vector fp32 scale (F32 primary only)
 *   seed     default seed of the random pool initialisation (Alg. 1) */
typedef struct {
    int32_t d;
    int32_t dtype;
    int32_t metric;
    int32_t R;
    int64_t n_cap;
    int32_t prune;
    int32_t repair_c;
    int32_t lowp;
    int32_t reserved0;
    uint64_t seed;
} svf_params;

/* Byte sizes of the caller-allocated device buffers (all 256-byte aligned). */
typedef struct {
    size_t vecs;      /* n_cap rows of d*esize bytes (primary store) */
    size_t vecs_bf16; /* n_cap rows of 2d bytes, 0 unless lowp bit 0 */
    size_t vecs_fp8;  /* n_cap rows of fp8_pitch = roundup(d + 4, 32) bytes: codes, then the fp32 scale */
    size_t graph;     /* n_cap * R uint32 */
    size_t del_bits;  /* ceil(n_cap / 32) uint32 */
    size_t workspace; /* scratch for build / insert / delete of up to max_batch vectors */
    size_t status;    /* status word and counters */
} svf_sizes;

/* Device buffers, borrowed by the index for its lifetime.  vecs, graph,
 * del_bits, workspace and status are required; the low-precision stores
 * are required iff the matching lowp bit is set.  svf_create zeroes
 * del_bits and status and sets every graph slot to SVF_EMPTY. */
typedef struct {
    void *vecs;
    void *vecs_bf16;
    void *vecs_fp8;
    uint32_t *graph;
    uint32_t *del_bits;
    void *workspace;
    size_t ws_bytes;
    void *status;
    size_t status_bytes;
} svf_buffers;

/* Search parameters (Alg. 1 with a fixed iteration count).
 *   k         results per query, 1 <= k <= min(L, 32)
 *   L         candidate pool size (itopk): 32, 64, 128 or 256
 *   T         iterations; one parent (the nearest unexpanded pool entry) is
 *             expanded per iteration; an iteration with none left is a no-op
 *   precision traversal store: SVF_F32/SVF_U8 (primary), SVF_BF16, SVF_FP8
 *   rerank    1: recompute the final pool's distances exactly from the
 *             primary store and re-sort before taking k (low precision only)
 *   mlp       device pointer to a packed stop network (svf_mlp_pack layout)
 *             or NULL; with it the network is evaluated after iteration t
 *             when t+1 >= t_min and (t+1-t_min) % t_every == 0 (t_every 0
 *             means 1), and the query stops there if z >= z_tau (z = logit)
 *   qkeys     device, nq uint64 query keys, or NULL: key = wrapping sum over
 *             the query's 32-bit words w_i of splitmix64((i << 32) | w_i)
 *   seed      pool-initialisation seed (0: the index's seed)
 *   hash_log2 per-query visited-table size, log2 of slots (0: automatic)
 *   trace_feat  device [nq][T][16] float, or NULL: per-iteration features
 *   trace_meta  device [nq][2] int32 (iterations run, last top-k change)
 *   pool_out  device [nq][L] uint64 keys of the final pool, or NULL
 *   W         parents per iteration, 0/1, 2, 4 or 8 (intra-query parallelism,
 *             Sec. 4.4): with W > 1 each query runs on a CTA of W warps and
 *             every iteration expands the W nearest unexpanded pool entries
 *             (an id named by two parents is visited once); T counts
 *             iterations, so a query expands up to W*T parents.  W > 1 does
 *             not combine with mlp / trace_feat / trace_meta (SVF_EINVAL).
 *             Meant for small batches, where one warp per query leaves most
 *             of the GPU idle. */
typedef struct {
    int32_t k;
    int32_t L;
    int32_t T;
    int32_t precision;
    int32_t rerank;
    int32_t t_min;
    const void *mlp;
    float z_tau;
    int32_t hash_log2;
    const uint64_t *qkeys;
    uint64_t seed;
    float *trace_feat;
    int32_t *trace_meta;
    uint64_t *pool_out;
    int32_t t_every;
    int32_t W;
} svf_search_params;

/* Running counters (since svf_create or svf_stats_reset). */
typedef struct {
    int64_t n_used;
    int64_t n_deleted;
    uint64_t search_queries;
    uint64_t search_iters;      /* parents expanded */
    uint64_t search_evals;      /* distance evaluations in traversal */
    uint64_t hash_resets;       /* visited-table resets */
    uint64_t repaired_rows;     /* rows rewritten by localized repair */
    uint64_t reverse_targets;   /* rows whose tail took reverse edges */
    uint64_t cache_hits;        /* tiered store: rows read from the device cache */
    uint64_t cache_misses;      /* tiered store: rows read from host memory */
    uint64_t promoted;          /* tiered store: rows promoted into the cache */
    uint64_t evicted;           /* tiered store: cached rows evicted */
    uint64_t build_fallback;    /* last build: rows whose tensor-core neighbours were recomputed by the exact scan */
    uint64_t build_tensor_core; /* last build: 1 if its exact 2R-NN came from the tensor-core scan, else 0 */
} svf_counters;

typedef struct svf_index svf_index;

const char *svf_last_error(void);

/* Buffer sizes for an index of `p` that builds / inserts / deletes at most
 * max_batch vectors per call (build needs max_batch >= n). */
int svf_buffer_sizes(const svf_params *p, int64_t max_batch, svf_sizes *out);

/* Create an index over caller-allocated device buffers (host handle out). */
int svf_create(const svf_params *p, const svf_buffers *b, svf_index **out);
int svf_destroy(svf_index *h);

/* Declare that the buffers already hold n_used valid rows, graph rows and
 * deletion bits (an index restored from a file or built elsewhere). */
int svf_attach(svf_index *h, int64_t n_used);

/* Build (Sec. 2.2 Build, Sec. 4.2 Index Construction): X is device, n rows
 * of d primary elements (n <= n_cap, n <= max_batch).  Copies X into the
 * store, computes the exact 2R nearest neighbours of every row (self
 * excluded) and prunes each list to R (Sec. 5.1 reordering).  Resets
 * deletions; n_used = n.  With d <= 128 (a multiple of 16), 2R <= 128 and
 * n >= 65,536 the neighbours of an fp32 inner-product store or of a uint8
 * store (either metric) come from the tensor cores: a bf16 tcgen05 scan of the
 * rows against themselves, exact re-scoring of a certified band of candidates
 * (fp32; for uint8 the scan is itself exact and the re-scoring is integer),
 * and the exact scan for rows whose certificate fails; otherwise from the
 * exact SIMT scan.  Every path gives the exact 2R-NN by (distance, id), the
 * distance in fp32 for fp32 stores and in int32 for uint8 stores.  The
 * counters' build_tensor_core tells which path the last build took. */
int svf_build(svf_index *h, const void *X, int64_t n, void *stream);

/* Search (Alg. 1): Q is device, nq rows of d elements (uint8 for a U8
 * index, fp32 otherwise).  out_ids: device [nq][k] uint32; out_dist:
 * device [nq][k], int32 for a U8 index and float otherwise.  Missing
 * results are SVF_EMPTY / +inf (INT32_MAX for U8). */
int svf_search(svf_index *h, const void *Q, int64_t nq, const svf_search_params *sp, uint32_t *out_ids,
               void *out_dist, void *stream);

/* Insert (Sec. 5.1): X is device, m rows.  The new ids are n_used ..
 * n_used+m-1 (written to out_ids, device, if not NULL).  Each new vector
 * searches the pre-call graph (pool L_ins, T_ins iterations), its pool is
 * reordered into its row, and every chosen neighbour u keeps the R/2 best
 * (distance, id) of its tail half [R/2, R) and the new vertices that chose
 * it.  L_ins: 32..256 power of two >= R. */
int svf_insert(svf_index *h, const void *X, int64_t m, int32_t L_ins, int32_t T_ins, uint32_t *out_ids,
               void *stream);

/* Delete (Sec. 5.2): ids is device, m uint32.  Any id >= n_used fails the
 * whole call (SVF_EINVAL reported by svf_sync; nothing changes); ids already
 * deleted are counted no-ops.  Sets the bits, then repairs every live vertex
 * with more than R/2 deleted neighbours from a snapshot of the graph.
 * out_newly (device int64, optional) receives the number newly deleted. */
int svf_delete(svf_index *h, const uint32_t *ids, int64_t m, int64_t *out_newly, void *stream);

/* Global consolidation (Sec. 5.2) under the multi-version mechanism of
 * Sec. 5.3, in three calls; one consolidation at a time, not on a tiered
 * store.
 *   svf_consolidate_sizes: bytes of the caller's consolidation buffer
 *     (device, 256-byte aligned, borrowed until commit / abort): a snapshot
 *     of the graph and deletion bits, repair scratch (about 8 n_cap R bytes
 *     plus 64 MB) and a log of log_rows inserted rows.
 *   svf_consolidate_begin: snapshot the graph rows [0, n_used) and the
 *     deletion bits on `stream`; from now on each svf_insert batch also logs
 *     its new rows and their distances.  More than log_rows logged rows make
 *     the later commit fail with SVF_ECAPACITY (the active graph stays valid).
 *   svf_consolidate_run: on the snapshot only, so it may run on its own
 *     stream while searches and updates continue on the active graph: every
 *     live vertex u with at least one deleted out-neighbour takes as
 *     candidates its live row entries, then every live entry of each deleted
 *     neighbour's row (row order, not u, no repeats; at most `cap` in all,
 *     R <= cap <= 512, 0 meaning 512),
 *     sorted by (distance, id) and reordered by the index's prune (Sec. 5.1);
 *     if fewer than R survive, its deleted entries fill the remaining slots
 *     in their old order.  Synchronises `stream` once (the number of rows),
 *     then queues the rest; out_rows (host, optional) gets that number.
 *   svf_consolidate_commit: in stream order with the updates: each logged
 *     batch's reverse edges are applied, in order, to the consolidated tails
 *     of targets inside the snapshot (as in svf_insert), then the consolidated
 *     rows replace rows [0, n0) of the active graph; rows inserted since the
 *     snapshot are kept (Sec. 5.3 incremental subgraph appending and reverse
 *     edge integration).  Returns after the copy completes.
 *   svf_consolidate_abort: discard a consolidation (waits for a queued run).
 * svf_build and svf_attach discard a consolidation in progress. */
int svf_consolidate_sizes(const svf_params *p, int64_t log_rows, size_t *bytes);
int svf_consolidate_begin(svf_index *h, void *buf, size_t bytes, int64_t log_rows, void *stream);
int svf_consolidate_run(svf_index *h, int32_t cap, int64_t *out_rows, void *stream);
int svf_consolidate_commit(svf_index *h, void *stream);
int svf_consolidate_abort(svf_index *h);

/* Wait for the index's last stream and report any device-side error. */
int svf_sync(svf_index *h);

/* Counters (synchronises). */
int svf_stats(svf_index *h, svf_counters *out);
int svf_stats_reset(svf_index *h);

/* Encode fp32 rows into the low-precision layouts (device to device):
 * bf16 = round-to-nearest-even; FP8 row = E4M3(x_i / s) with satfinite and
 * s = max|x| / 448 (1 if 0) stored as fp32 at byte d. */
int svf_encode_bf16(const float *X, int64_t n, int32_t d, void *out, void *stream);
int svf_encode_fp8(const float *X, int64_t n, int32_t d, void *out, int64_t pitch, void *stream);

/* Exact brute-force k nearest neighbours (ground truth, Sec. 6.1 "exhaustive
 * linear scan"): for each of nq device queries the k <= 128 rows of the
 * device store X (n rows of d elements, dtype F32 or U8, metric as in an
 * index) with the smallest (distance, id), skipping row self[i] if self
 * (device int64 [nq]) is given.  work_keys: device scratch [nq][k] uint64
 * (caller-allocated).  out_ids device [nq][k] uint32, out_dist device
 * [nq][k] (int32 for U8, float otherwise; may be NULL). */
int svf_knn(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t metric, const void *Q, int64_t nq,
            const int64_t *self, int32_t k, uint64_t *work_keys, uint32_t *out_ids, void *out_dist, void *stream);

/* ---- tiered store (serving form, Sec. 4.2-4.3, Alg. 2).
 * After svf_tier_enable the primary (fp32/uint8) rows live in caller-pinned
 * host memory and a device cache of M rows holds the hot ones; every kernel
 * reads a row from its cache slot when mapped and from host memory (mapped,
 * zero-copy) otherwise, so results do not depend on what is cached.  A miss
 * adds to F_recent(x); x is queued for promotion when
 *   F_lambda(x) = alpha * F_recent(x) + beta * log(1 + E_in(x)) > theta
 * (Eq. 2, the threshold form of Eq. 1).  svf_tier_maintain promotes queued
 * rows (highest F_lambda first) into victims chosen by a clock sweep over
 * the cache that skips (and clears) referenced slots and takes the lowest
 * F_lambda among unreferenced ones (Alg. 2), halves F_recent every
 * decay_every misses, and adapts theta to the miss rate (Sec. 4.4).  It must
 * not run while a search or update on the index is in flight.
 * Enable warms the cache with the highest in-degree rows (cold start).  The
 * device copy of the primary store is not read afterwards; low-precision
 * copies (lowp) stay whole in device memory and are encoded from the
 * inserted rows, so BF16/FP8 traversal reads no host memory and only the
 * exact re-rank goes through the tier. */
/* Placement policies (svf_tier_params.policy).  WAVP is the paper's
 * (Alg. 2, Eq. 2); the others are the baselines of its Sec. 6.3 on the same
 * machinery (a maintenance round promotes up to promote_batch queued rows
 * into victims chosen among the sweep * promote_batch slots the clock
 * passes, an empty slot first):
 * CLOCK admits every missed row in miss order and evicts the first
 * unreferenced slots the clock meets (second chance: recency only); LFU
 * admits and evicts by F_recent alone (beta ignored, theta fixed at theta0);
 * STATIC keeps the cold-start cache of the highest in-degree rows; LRU
 * admits every missed row in miss order and evicts the slots whose last hit
 * is oldest (hits are stamped with a counter of the calls that read the
 * tier); LRFU admits every missed row and evicts the slots of lowest
 * combined recency-frequency C = sum over hits of 2^(-lambda * age), age in
 * maintenance rounds (C <- C * 2^-lambda + hits of the round; a promoted row
 * starts at 1 for the miss that admitted it). */
enum svf_tier_policy {
    SVF_TIER_WAVP = 0,
    SVF_TIER_CLOCK = 1,
    SVF_TIER_LFU = 2,
    SVF_TIER_STATIC = 3,
    SVF_TIER_LRU = 4,
    SVF_TIER_LRFU = 5
};

typedef struct {
    int64_t M;              /* cache slots */
    uint32_t qcap;          /* promotion queue capacity (<= 16384) */
    int32_t promote_batch;  /* rows promoted per maintenance (<= 2048) */
    int32_t sweep;          /* clock slots examined per promotion (sweep * batch <= 8192) */
    float alpha, beta;      /* Eq. 2 weights (paper: alpha/(alpha+beta) ~ 0.6) */
    float theta0;           /* initial promotion threshold */
    uint64_t decay_every;   /* halve F_recent after this many misses */
    int32_t policy;         /* svf_tier_policy */
    float lrfu_lambda;      /* LRFU decay per maintenance round (0: 0.5) */
} svf_tier_params;

typedef struct {
    size_t cache, map, owner, ref, freq, ein, queue, scratch; /* device bytes */
    size_t host;                                              /* pinned host bytes */
    size_t slot_stat;                                         /* device bytes: per-slot LRU / LRFU state */
} svf_tier_sizes;

typedef struct {
    void *cache; int32_t *map; int32_t *owner; uint8_t *ref; uint32_t *freq; uint32_t *ein; uint32_t *queue;
    void *scratch;
    void *host;  /* pinned (cudaHostAlloc / page-locked) host memory for n_cap rows */
    void *slot_stat;
} svf_tier_buffers;

int svf_tier_buffer_sizes(const svf_params *p, const svf_tier_params *tp, svf_tier_sizes *out);
/* Copies rows [0, n_used) to the host store, computes E_in, warms the cache. */
int svf_tier_enable(svf_index *h, const svf_tier_params *tp, const svf_tier_buffers *tb, void *stream);
/* One maintenance round; *out_promoted (host, optional) = rows promoted. */
int svf_tier_maintain(svf_index *h, int64_t *out_promoted, void *stream);
/* Current promotion threshold. */
float svf_tier_theta(svf_index *h);
/* Re-initialise a tiered store with new parameters (policy, weights,
 * threshold, and a cache of M slots, at most the M it was enabled with; the
 * buffers stay): miss counts, queue and reference bits are cleared, E_in is
 * recomputed from the current graph and the cache is warmed again with the
 * highest in-degree rows, read from the host store.  Must not run while a
 * search or update on the index is in flight. */
int svf_tier_reset(svf_index *h, const svf_tier_params *tp, void *stream);

/* ---- continuous-batching request loop (Sec. 4.4 real-time coordination,
 * Sec. 5.3 consistency).  A worker thread admits requests in submission
 * order, each no earlier than its t_arrival (svf_serve_now clock; 0 = now).
 * Searches run on n_streams streams with up to max_inflight batches on the
 * GPU at once; inserts and deletes run one at a time on a dedicated update
 * stream.  Every request completes with an epoch: for an update, its number
 * (1, 2, ... in submission order); for a search, the number of updates whose
 * effect it sees -- its result equals the same search run alone on the index
 * state after exactly those updates.  `consistency` says how searches meet
 * updates:
 *   SVF_SERVE_BARRIER           an update waits for the in-flight searches,
 *                               runs alone, and later searches wait for it.
 *   SVF_SERVE_READ_AFTER_WRITE  an update runs while earlier searches are
 *                               still on the GPU; a search sees every update
 *                               submitted before it (its stream waits for the
 *                               last one), the paper's "with sync" mode.
 *   SVF_SERVE_SNAPSHOT          as above, but a search sees the updates that
 *                               have completed when it is admitted and never
 *                               waits for one (the paper's "without sync").
 * The last two keep versions for the searches that overlap an update: the
 * update copies every existing row it rewrites into a shadow row and stamps
 * it, and stamps every vertex it deletes, so that a search of an older epoch
 * reads the row as it was and still treats the vertex as live (vertices an
 * update inserts have ids the older search never names).  One shadow per row
 * is kept: update E+1 starts once every search of an epoch below E has
 * finished.  Searches of the versioned modes run without the stop network
 * or traces (SVF_EINVAL).  An update that rewrites more than shadow_rows existing rows
 * (an insert of m vectors rewrites at most m*R; a delete's repair is counted
 * on the device) runs as a barrier instead.  `versions` is a device buffer of
 * svf_serve_version_bytes(h, shadow_rows) bytes, borrowed until stop.
 * With a tiered store, svf_tier_maintain runs every maintain_every search
 * batches while nothing is in flight.  All request buffers are device memory
 * owned by the caller and must stay valid until the completion for the
 * request has been polled. */
enum svf_op { SVF_OP_SEARCH = 0, SVF_OP_INSERT = 1, SVF_OP_DELETE = 2 };
enum svf_consistency { SVF_SERVE_BARRIER = 0, SVF_SERVE_READ_AFTER_WRITE = 1, SVF_SERVE_SNAPSHOT = 2 };

typedef struct {
    int32_t max_inflight;
    int32_t n_streams;
    int32_t maintain_every;
    int32_t consistency;      /* svf_consistency */
    void *versions;           /* device, svf_serve_version_bytes bytes (consistency 1 or 2), else NULL */
    size_t versions_bytes;
    int64_t shadow_rows;      /* existing rows one update may rewrite concurrently with searches */
} svf_serve_cfg;

/* Bytes of the version buffer for an index (row stamps, deletion stamps and
 * two halves of shadow_rows shadow rows). */
size_t svf_serve_version_bytes(svf_index *h, int64_t shadow_rows);

typedef struct {
    int32_t op;               /* svf_op */
    int32_t count;            /* queries / vectors / ids */
    const void *data;         /* device: queries, vectors or uint32 ids */
    svf_search_params sp;     /* search */
    uint32_t *out_ids;        /* search: device [count][k] */
    void *out_dist;           /* search: device [count][k] */
    uint32_t *out_new_ids;    /* insert: device [count] (optional) */
    int32_t L_ins, T_ins;     /* insert */
    uint64_t tag;             /* caller's request id */
    double t_arrival;         /* arrival time, svf_serve_now() clock */
} svf_request;

typedef struct {
    uint64_t tag;
    int32_t op;
    int32_t status;           /* SVF_OK or an error code */
    uint64_t epoch;           /* updates applied before (search) / after (update) it */
    int64_t count;
    double t_arrival, t_start, t_done;
} svf_completion;

typedef struct svf_server svf_server;

double svf_serve_now(void);
int svf_serve_start(svf_index *h, const svf_serve_cfg *cfg, svf_server **out);
int svf_serve_submit(svf_server *s, const svf_request *r);
int svf_serve_poll(svf_server *s, svf_completion *out, int max, int *n_out);
/* Wait until every submitted request completed (SVF_ETIMEOUT after timeout_s);
 * returns the first request error seen, if any. */
int svf_serve_drain(svf_server *s, double timeout_s);
int svf_serve_stop(svf_server *s);

/* Exact kNN on the tensor cores (fp32 store and queries, d <= 128 multiple
 * of 16, k <= 32): bf16 tcgen05 GEMM tiles with TMEM accumulators select 48
 * approximate candidates per query and database slice, which are re-scored
 * exactly in fp32; a per-query certificate (bf16 error bound) proves that no
 * row was missed, and queries that fail it are recomputed by the SIMT scan.
 * scratch: device, svf_knn_tc_scratch_bytes(n, nq, d, k) bytes.
 * *out_fallback (host, optional) = queries recomputed.  Synchronises. */
size_t svf_knn_tc_scratch_bytes(int64_t n, int64_t nq, int32_t d, int32_t k);
int svf_knn_tc(const float *X, int64_t n, int32_t d, int32_t metric, const float *Q, int64_t nq, int32_t k,
               void *scratch, size_t scratch_bytes, uint32_t *out_ids, float *out_dist, int64_t *out_fallback,
               void *stream);

/* ---- allocation-free variant of svf_knn (the paper has no counterpart).
 * For callers that cannot call cudaMalloc -- a plugin or custom call inside
 * a host framework whose memory manager owns the device's memory, or a
 * latency-critical loop where an allocation could stall -- this computes the
 * same result as svf_knn without the caller's work_keys buffer.  Its scratch
 * is a fixed device array of svf_knn_static_capacity() = 1,048,576 uint64
 * keys (8 MiB) that every GPU loading the library holds until the process
 * exits; nq * k above that capacity is rejected with SVF_EINVAL.  The first
 * call on each device looks up the array's device address (with that device
 * current) and caches it; make that first call before any stream capture.
 * All calls share the array, which keeps the last call's keys: calls that
 * overlap on the GPU (different streams, devices sharing nothing else) race
 * and must be serialised by the caller.  The call allocates nothing.  The
 * cached address belongs to the device's primary context: after that context
 * is destroyed (cudaDeviceReset) it is stale, as is every other device
 * pointer the caller held, and the library must be reloaded.  Errors are
 * described by svf_knn_static_error() and, like every other call's, by
 * svf_last_error(). */
int svf_knn_static(const void *X, int64_t n, int32_t d, int32_t dtype, int32_t metric, const void *Q, int64_t nq,
                   const int64_t *self, int32_t k, uint32_t *out_ids, void *out_dist, void *stream);
int64_t svf_knn_static_capacity(void);
const char *svf_knn_static_error(void);

/* ---- learned early stop (16 -> 64 ReLU -> 1; not in the paper: an added
 * learned part that shortens Alg. 1's fixed iteration count).
 * Parameter vector (fp32, SVF_MLP_PARAMS entries): W1[64][16] row-major,
 * b1[64], w2[64], b2.  The search reads the packed bf16 copy
 * (SVF_MLP_PACKED entries, same order, zero padded). */
#define SVF_MLP_PARAMS 1153
#define SVF_MLP_PACKED 1160

/* Minibatch gradient of the mean binary cross-entropy.  feat: device trace
 * [nq][T][16] float; meta: device [nq][2] int32 (iterations run, last top-k
 * change); idx: device [B] int32 sample ids q*T+t (t < iterations run);
 * label = (t >= last change).  grad: device [SVF_MLP_PARAMS]; partial:
 * device scratch of svf_mlp_partial_floats(B) floats; loss: device float
 * (may be NULL).  Deterministic (fixed reduction order). */
int svf_mlp_grad(const float *feat, const int32_t *meta, int32_t T, const int32_t *idx, int64_t B, const float *params,
                 float *grad, float *partial, float *loss, void *stream);
int64_t svf_mlp_partial_floats(int64_t B);
/* One Adam step (bias-corrected, step >= 1) on device fp32 vectors. */
int svf_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t step, float lr, float beta1,
                 float beta2, float eps, void *stream);
/* fp32 parameters -> packed bf16 (round to nearest even) for svf_search. */
int svf_mlp_pack(const float *params, void *packed, void *stream);
/* Logits of the fp32 network for n feature rows (device [n][16] -> [n]). */
int svf_mlp_forward(const float *params, const float *feat, int64_t n, float *z, void *stream);

/* ---- failure-path self test (no counterpart in the paper).  Every device
 * wait in the library polls an mbarrier at most svf_wait_limit() times, then
 * records SVF_ETIMEOUT (and the poll count as detail) in the status words
 * and returns.  svf_selftest_wait_timeout runs one warp on a barrier nothing
 * arrives at, with the same loop capped at `polls`; status is a caller-owned
 * device buffer of >= 2 uint64 (overwritten).  Returns SVF_ETIMEOUT when the
 * wait gave up and reported it, as it must; *out_seconds (host, optional) is
 * the wall time of the launch. */
uint32_t svf_wait_limit(void);
int svf_selftest_wait_timeout(uint32_t polls, unsigned long long *status, double *out_seconds, void *stream);

/* ---- random-row fetch ceiling (a measurement, no counterpart in the paper).
 * The search fetches rows at ids it cannot predict (Alg. 1's neighbour
 * expansion), so the rate at which the GPU serves independent random rows
 * bounds it.  svf_gather_probe copies about `rows` rows of `row_bytes` bytes,
 * at ids drawn uniformly from [0, n) of a device table whose rows are `pitch`
 * bytes apart, into shared memory with the search kernel's own copy pattern:
 * one 1-D bulk copy per lane, 32 rows per warp batch on one mbarrier, blocks
 * of 4 warps, `warps_per_sm` warps per SM; nothing is computed on the rows.
 * Outputs (host): *out_rows = rows actually copied (`rows` rounded up to whole
 * batches of every warp), *out_ms = device time of the launch (CUDA events on
 * `stream`).  table: device, 16-byte aligned, n * pitch bytes, read only;
 * pitch and row_bytes multiples of 16 with 16 <= row_bytes <= min(pitch,
 * 1024); 1 <= n < 2^31; rows >= 1; warps_per_sm a multiple of 4 in [4, 64];
 * status: caller-owned device buffer of >= 2 uint64 (overwritten).
 * Errors: SVF_EINVAL (arguments), SVF_ETIMEOUT (a bounded wait gave up;
 * recorded in status), SVF_ECUDA. */
int svf_gather_probe(const void *table, int64_t n, int32_t pitch, int32_t row_bytes, int64_t rows, int32_t warps_per_sm,
                     uint64_t seed, unsigned long long *status, int64_t *out_rows, float *out_ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SVF_H */
