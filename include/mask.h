/*
 * mask.h -- C ABI of the GB300 MASK library (libmask_gb300.so).
 *
 * MASK (Ortega, Algar, Martin de Diego, Moguerza, "Unconventional application
 * of k-means for distributed approximate similarity search"):
 *   - build (§3.1, Algorithm 1, global form): level by level, k-means++
 *     seeding (§3.2) and Lloyd iterations (§2.4) over the items of the level
 *     below; the centroids of one level are the data of the next.
 *   - query (§3.3, Algorithm 2): distances from the query to the top level's
 *     centroids, keep the nearest p; at each lower level keep the nearest p
 *     among the children of the kept centroids; scan the points of the kept
 *     leaf clusters and return the k nearest.
 * Metric: Euclidean (§4.2).  Distances are returned SQUARED.
 *
 * Conventions for every entry point:
 *   - Pointers are plain host or device pointers of the current CUDA device;
 *     each is classified per call (cudaPointerGetAttributes).  Host inputs are
 *     copied in and host outputs copied back before the call returns; with
 *     device pointers only, a query is stream-ordered on `stream` and returns
 *     without synchronising.
 *   - Arrays are dense row-major with no padding: a [n x d] float array has
 *     element (i, t) at i*d + t.
 *   - The caller owns every buffer it passes.  The library owns the index
 *     (device memory inside); it is released only by mask_free.
 *   - Errors are returned as mask_status; nothing is thrown across the ABI.
 *     mask_last_error() gives a message for the calling thread's last failure.
 *   - Level numbering: arrays indexed by level are finest first (index 0 =
 *     the centroids directly above the points).
 *   - Random numbers: SplitMix64 (Steele, Lea & Flood 2014); the stream of
 *     level lv starts at seed ^ (0x9E3779B97F4A7C15 * (lv + 1)); a uniform
 *     draw is (next >> 11) * 2^-53.  The paper names no generator.
 */
#ifndef MASK_GB300_H
#define MASK_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MASK_MAX_LEVELS 16

typedef struct mask_index mask_index;

/* A cudaStream_t; NULL is the legacy default stream. */
typedef void *mask_stream;

typedef enum {
    MASK_PENDING = 1,       /* (serving) the request has not finished yet */
    MASK_OK = 0,
    MASK_EINVAL = -1,       /* bad argument (sizes, k > items below, NULL) */
    MASK_ENOMEM = -2,       /* device or host allocation failed */
    MASK_ECUDA = -3,        /* a CUDA call or kernel launch failed */
    MASK_ETIMEOUT = -4,     /* a bounded device-side wait ran out */
    MASK_EUNSUPPORTED = -5  /* valid request this build does not implement */
} mask_status;

typedef enum {
    MASK_FP32 = 0,     /* all distances in FP32 */
    MASK_BF16 = 1,     /* BF16 distance GEMMs + exact FP32 re-rank */
    MASK_FP8E4M3 = 2   /* FP8 e4m3 (per-row scales) + exact FP32 re-rank */
} mask_precision;

typedef struct {
    int64_t n;                               /* indexed points */
    int32_t d;                               /* dimension */
    int32_t n_levels;
    int32_t k_per_level[MASK_MAX_LEVELS];    /* finest first */
    int32_t iters;                           /* Lloyd iterations per level */
    int32_t sparse;                          /* built from CSR rows */
    int64_t device_bytes;                    /* device memory the index holds */
} mask_index_info;

/* Message describing the calling thread's most recent failure ("" if none). */
const char *mask_last_error(void);

/*
 * Build a multilevel k-means index over n dense points (§3.1, Algorithm 1,
 * one group per level).
 *   points       [n x d] float32.
 *   k_per_level  host array [n_levels], finest first; 1 <= k_0 <= n and
 *                1 <= k_l <= k_{l-1}; n_levels <= MASK_MAX_LEVELS.
 *   iters        Lloyd iterations per level (>= 0): iters updates and
 *                iters+1 assignments; ties go to the smallest centroid index;
 *                an empty cluster keeps its centroid.
 *   seed         RNG seed for k-means++ seeding (§3.2).  When n_in * k > 2^32
 *                and 8k < n_in, seeding runs on 8k inputs drawn by a partial
 *                Fisher-Yates shuffle.
 *   out          receives the index (free with mask_free).
 * Synchronises `stream` before returning.
 */
mask_status mask_build(const float *points, int64_t n, int32_t d,
                       const int32_t *k_per_level, int32_t n_levels, int32_t iters,
                       uint64_t seed, mask_stream stream, mask_index **out);

/*
 * As mask_build, for n sparse points in CSR form (the TF-IDF shape of §4.3):
 *   row_ptr [n+1] int64, row_ptr[0] = 0 and nondecreasing; nnz = row_ptr[n];
 *   col     [nnz] int32, each in [0, d) and strictly increasing within a row;
 *   val     [nnz] float32.
 * Centroids are dense ([k_l x d] float32).  Level 0 runs on the CSR rows:
 * k-means++ and the mean update use ||x - c||^2 = sum_{t in x} (x_t - c_t)^2
 * + (||c||^2 - sum_{t in x} c_t^2); the assignment is a CSR-times-dense
 * product with the argmin fused (rows whose best two centroids are closer
 * than the FP32 rounding bound are re-decided in FP64).  The levels above run
 * on the level-0 centroids as dense rows, exactly as in mask_build.
 * d <= 40960 (k-means++ stages a dense row in shared memory), else
 * MASK_EUNSUPPORTED; malformed CSR arrays give MASK_EINVAL.
 * Query the index with mask_query_csr.  Synchronises `stream`.
 */
mask_status mask_build_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                           int64_t n, int32_t d, const int32_t *k_per_level,
                           int32_t n_levels, int32_t iters, uint64_t seed,
                           mask_stream stream, mask_index **out);

/*
 * Approximate k-NN of nq dense queries (§3.3, Algorithm 2, p_l kept centroids
 * per level instead of one).
 *   queries   [nq x d] float32.
 *   k         neighbours per query (1 <= k <= 1024).
 *   probes    host array [n_levels], finest first; p_l >= 1, clamped to k_l.
 *   precision MASK_FP32: every distance in FP32.  MASK_BF16 / MASK_FP8E4M3:
 *             the leaf scan ranks points by distances between BF16 (or FP8
 *             e4m3 with a per-row scale max|x|/448) copies of the points and
 *             the query, keeps the max(4k, 16) nearest, and re-ranks those by exact
 *             FP32 distances (k <= 16 and d <= 256, else MASK_EUNSUPPORTED);
 *             the quantised copy is made on the first such query (the index
 *             grows by 2 or 1 bytes per coordinate plus 4-8 bytes per point).
 *   ids_out   [nq x k] int64 original point ids, ascending by (distance, id);
 *             -1 where fewer than k points were reached.
 *   dists_out [nq x k] float32 squared distances; +inf where ids_out is -1.
 * Each query's result does not depend on the other queries in the batch.
 */
mask_status mask_query(const mask_index *index, const float *queries, int64_t nq,
                       int32_t k, const int32_t *probes, mask_precision precision,
                       int64_t *ids_out, float *dists_out, mask_stream stream);

/*
 * As mask_query, for nq CSR queries (row_ptr [nq+1], col, val as for
 * mask_build_csr) against an index built by mask_build_csr (a dense index
 * gives MASK_EINVAL, as does mask_query on a CSR index).  Distances to a
 * level's centroids: sum_{t in q} (q_t - c_t)^2 + (||c||^2 - sum_{t in q}
 * c_t^2); to a leaf point: sum_{t in x} (x_t - q_t)^2 + (||q||^2 -
 * sum_{t in x} q_t^2), so a point equal to the query is at distance 0.
 * MASK_FP32 only, and at most 8192 nonzeros per query; otherwise
 * MASK_EUNSUPPORTED.  Synchronises `stream`.
 */
mask_status mask_query_csr(const mask_index *index, const int64_t *row_ptr,
                           const int32_t *col, const float *val, int64_t nq, int32_t k,
                           const int32_t *probes, mask_precision precision,
                           int64_t *ids_out, float *dists_out, mask_stream stream);

/* Release an index (NULL is ignored). */
void mask_free(mask_index *index);

/* Sizes of an index. */
mask_status mask_index_get_info(const mask_index *index, mask_index_info *out);

/*
 * Copy one level of an index out (level 0 = finest).
 *   centroids_out [k_level x d] float32 in k-means cluster order (may be NULL).
 *   labels_out    [n_below] int32: the level's centroid of every item one level
 *                 below (points for level 0), in item order (may be NULL).
 *   chosen_out    [k_level] int64: the inputs k-means++ picked as initial
 *                 centres, as indices into the level's inputs (may be NULL).
 *   objective_out [iters+1] double: k-means objective sum ||x - c_label||^2
 *                 after each assignment (may be NULL).
 * Synchronises `stream`.
 */
mask_status mask_index_export_level(const mask_index *index, int32_t level,
                                    float *centroids_out, int32_t *labels_out,
                                    int64_t *chosen_out, double *objective_out,
                                    mask_stream stream);

/*
 * Assemble an index from given centroids and labels instead of building it
 * (used to query an index built elsewhere, e.g. loaded from disk).
 *   points         [n x d] float32.
 *   centroids[l]   [k_l x d] float32 (host array of n_levels pointers).
 *   labels[l]      [n_below(l)] int32, each in [0, k_l) (host array of pointers).
 * The structure (membership lists, cluster-major leaf layout) is derived on
 * the device exactly as mask_build derives it.  Synchronises `stream`.
 */
mask_status mask_index_load(const float *points, int64_t n, int32_t d, int32_t n_levels,
                            const int32_t *k_per_level, const float *const *centroids,
                            const int32_t *const *labels, mask_stream stream,
                            mask_index **out);

/* ---- the grouped build of §3.1 and the point query of §3.3 ------------ */

/*
 * Level sizes of the grouped build (Algorithm 1 as printed): at each level the
 * m items are split into floor(m / length_group) groups of nCentroids
 * centroids each; the loop ends when that count drops below one.
 *   sizes_out    host [MASK_MAX_LEVELS]: centroids per level, finest first.
 *   n_levels_out number of levels (0 when n < length_group).
 * Needs 1 <= n_centroids <= length_group (MASK_EINVAL otherwise).  Host only.
 */
mask_status mask_grouped_levels(int64_t n, int32_t length_group, int32_t n_centroids,
                                int64_t *sizes_out, int32_t *n_levels_out);

/*
 * Grouped multilevel index (§3.1, Algorithm 1 as printed): at every level the
 * items (points, then the centroids of the level below) are split at random
 * into floor(m / length_group) groups whose sizes differ by at most one (a
 * Fisher-Yates shuffle from the level's SplitMix64 stream, then consecutive
 * parts, the first m mod G parts one larger); every group is clustered into
 * n_centroids centroids by its own k-means (k-means++ seeding from the state
 * level_state(seed, lv) ^ (0xD1B54A32D192ED03 * (group + 1)), then `iters`
 * Lloyd iterations with the conventions of mask_build), over its items in
 * ascending index.  Centroid j of group g is centroid g * n_centroids + j of
 * the level.  Levels as mask_grouped_levels gives them (at most
 * MASK_MAX_LEVELS, else MASK_EUNSUPPORTED).
 *   points  [n x d] float32, n >= length_group.
 *   group0  [n] int32 (host or device, may be NULL): the level-0 group of
 *           every point, each in [0, n / length_group) and each group with
 *           at least n_centroids points, instead of the random split (the
 *           relocation of §4.1, see mask_relocate); levels above are split
 *           at random as usual.
 * A group's items (times the padded dimension) must fit shared memory (about
 * 50,000 floats), else MASK_EINVAL.  The result is an ordinary index: query
 * it with mask_query, mask_descend or mask_range_query.  Synchronises
 * `stream`.
 */
mask_status mask_build_grouped(const float *points, int64_t n, int32_t d, int32_t length_group,
                               int32_t n_centroids, int32_t iters, uint64_t seed,
                               const int32_t *group0, mask_stream stream, mask_index **out);

/*
 * The descent of §3.3 (Algorithm 2 with p_l kept centroids per level) down to
 * the leaf clusters, without the leaf scan: leaf_out [nq x probes[0]] int32
 * receives the kept leaf clusters (level-0 centroid ids), nearest first, -1
 * past the clusters that exist.  probes as for mask_query; all ones is the
 * greedy descent of the paper's point query.  Synchronises `stream`.
 */
mask_status mask_descend(const mask_index *index, const float *queries, int64_t nq,
                         const int32_t *probes, int32_t *leaf_out, mask_stream stream);

/*
 * One relocation pass of §4.1 on a grouped index of `points` (the same
 * [n x d] points it was built from): every point is searched for by the
 * greedy point query (one kept centroid per level); a point is missed when the
 * leaf cluster reached is not its own.  A missed point moves to the level-0
 * group of the reached cluster (its id / n_centroids), in ascending point
 * order, unless its current group would fall below n_centroids points.
 *   group0      HOST [n] int32, in/out: the level-0 groups the index was
 *               built with; updated in place for the next mask_build_grouped.
 *   missed_out  points the greedy point query missed (may be NULL).
 *   moved_out   points moved (may be NULL).
 * The level-0 group of point i in an index built by mask_build_grouped is
 * labels_0[i] / n_centroids (mask_index_export_level, level 0).
 * Synchronises `stream`.
 */
mask_status mask_relocate(const mask_index *index, const float *points, int32_t n_centroids,
                          int32_t *group0, int64_t *missed_out, int64_t *moved_out,
                          mask_stream stream);

/*
 * Range search (§3.3, Algorithm 3): from the top level down, the candidate
 * centroids within distance `radius` of the query are kept and their
 * children become the next candidates; the result is the points of the kept
 * leaf clusters within `radius`, ascending by (squared distance, id).  A
 * point whose ancestors lie outside the ball is not found: the search is
 * approximate, as the paper's.  Distances are FP32 sums of squared
 * differences and are returned squared.
 *   counts_out [nq] int64: results per query (always written).
 *   ids_out / dists_out: [capacity] int64 / float32 (may be NULL: counts
 *   only); results are written query after query (the first counts_out[0]
 *   entries belong to query 0, ...).  When their total exceeds `capacity`
 *   nothing else is written and MASK_EINVAL is returned with counts_out
 *   filled, so the caller can retry with a larger buffer.
 * Synchronises `stream`.
 */
mask_status mask_range_query(const mask_index *index, const float *queries, int64_t nq,
                             float radius, int64_t *counts_out, int64_t capacity,
                             int64_t *ids_out, float *dists_out, mask_stream stream);

/*
 * Insertion (§3.3, last paragraph): each new point descends greedily (one
 * kept centroid per level) and joins the leaf cluster it reaches; the
 * centroids are not changed.  The new points get the ids index->n .. n +
 * n_new - 1 in order; leaf_out [n_new] int32 (may be NULL) receives the leaf
 * cluster each joined.  Dense indexes only (MASK_EUNSUPPORTED for CSR).  The
 * BF16/FP8 copies of the points are dropped and made again on their next use.
 * Not safe while a server or another call uses the index.  Synchronises
 * `stream`.
 */
mask_status mask_insert(mask_index *index, const float *points, int64_t n_new,
                        int32_t *leaf_out, mask_stream stream);

/*
 * The exchange step of the distributed design (§3.4): each of n_parts nodes
 * answers the same queries on its own partition with its own index; their
 * results, gathered, are merged into the k nearest over all partitions.
 *   ids, dists  [n_parts x nq x k] int64 / float32, partition-major (the
 *               layout of an all-gather of each node's [nq x k] mask_query
 *               output); ids -1 (with dists +inf) are padding.
 *   id_offset   [n_parts] int64 (may be NULL): added to partition g's ids,
 *               turning partition-local ids into global ones.
 *   ids_out, dists_out [nq x k]: ascending by (distance, global id), padded
 *               with (-1, +inf).
 * n_parts * k <= 16384 (one block sorts a query's candidates in shared
 * memory), else MASK_EUNSUPPORTED.  Synchronises `stream`.
 */
mask_status mask_merge_topk(const int64_t *ids, const float *dists, int32_t n_parts, int64_t nq,
                            int32_t k, const int64_t *id_offset, int64_t *ids_out,
                            float *dists_out, mask_stream stream);

/* ---- k-means steps (the build's kernels, callable on their own) -------- */

/*
 * k-means++ seeding (§3.2) of k centres from the n rows of X, with the
 * random stream of `level` under `seed` (subsampling rule as in mask_build).
 *   centroids_out [k x d] float32: copies of the chosen rows.
 *   chosen_out    [k] int64 indices into X (may be NULL).
 * Synchronises `stream`.
 */
mask_status mask_kmeanspp(const float *X, int64_t n, int32_t d, int32_t k, uint64_t seed,
                          int32_t level, float *centroids_out, int64_t *chosen_out,
                          mask_stream stream);

/*
 * Lloyd assignment half-step (§2.4): labels_out[i] = argmin_j ||x_i - c_j||^2,
 * ties to the smallest j.  dist_out[i] (may be NULL) = the minimum squared
 * distance, evaluated as sum_t (x_it - c_jt)^2 in FP32.
 *   X [n x d], C [k x d] float32; labels_out [n] int32.
 */
mask_status mask_kmeans_assign(const float *X, int64_t n, int32_t d, const float *C,
                               int32_t k, int32_t *labels_out, float *dist_out,
                               mask_stream stream);

/*
 * Lloyd update half-step (§2.4): C_out[j] = mean of the rows of X with
 * label j; an empty cluster copies C_prev[j].  counts_out [k] (may be NULL)
 * receives the cluster sizes.  Sums are FP32, FP64 for clusters with more
 * than 2^20 members.
 */
mask_status mask_kmeans_update(const float *X, int64_t n, int32_t d, const int32_t *labels,
                               int32_t k, const float *C_prev, float *C_out,
                               int64_t *counts_out, mask_stream stream);

/*
 * CSR forms of the three steps above (rows as for mask_build_csr; centroids
 * dense [k x d]).  mask_kmeanspp_csr needs d <= 40960.  dist_out of
 * mask_kmeans_assign_csr is sum_{t in x} (x_t - c_t)^2 + (||c||^2 -
 * sum_{t in x} c_t^2) in FP32 for the chosen centroid.
 */
mask_status mask_kmeanspp_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                              int64_t n, int32_t d, int32_t k, uint64_t seed, int32_t level,
                              float *centroids_out, int64_t *chosen_out, mask_stream stream);
mask_status mask_kmeans_assign_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                                   int64_t n, int32_t d, const float *C, int32_t k,
                                   int32_t *labels_out, float *dist_out, mask_stream stream);
mask_status mask_kmeans_update_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                                   int64_t n, int32_t d, const int32_t *labels, int32_t k,
                                   const float *C_prev, float *C_out, int64_t *counts_out,
                                   mask_stream stream);

/*
 * Allocation-free variant of mask_kmeans_assign, for callers that cannot let
 * this library allocate device memory: frameworks that reserve the GPU's
 * memory up front and hand it out only through their own allocator (a
 * cudaMalloc from inside the library could fail or fragment their pool), and
 * latency-critical loops that cannot absorb the device-wide synchronisation
 * cudaMalloc/cudaFree may cause.  The paper has no counterpart: this is an
 * interface convenience, not part of the method.
 *
 * Same result as mask_kmeans_assign (same kernels), but it calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its temporaries live in
 * one file-scope device array of 2.36 MB that every GPU which loads the
 * library holds until the process exits.
 *   X [n x d], C [k x d] float32, labels_out [n] int32, dist_out [n] float32
 *   (may be NULL): all DEVICE memory of the current device; X and C 16-byte
 *   aligned.  The C side cannot see array lengths: the caller guarantees
 *   that C has d columns and the outputs hold n elements.
 *   d must be a multiple of 8 (rows are used in place, not padded).
 *   1 <= k <= 65536 (the array holds at most 65536 centroid norms); any n
 *   (rows are processed 262,144 at a time).
 * Larger k, host pointers, another device's pointers or other d return
 * MASK_EINVAL with a message.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array: calls whose
 * work overlaps on the GPU (different streams or host threads without
 * ordering between them) race and give wrong labels.  Calls ordered on one
 * stream are safe; each call clears what it needs.
 */
mask_status mask_kmeans_assign_noalloc(const float *X, int64_t n, int32_t d, const float *C,
                                       int32_t k, int32_t *labels_out, float *dist_out,
                                       mask_stream stream);

/* ---- observability ---------------------------------------------------- */

/*
 * Per-kernel device timing.  The paper reports wall-clock build and search
 * times only (§4.2, Tables 3-6); these split the device time by kernel.
 * While enabled, the library brackets its main kernels with CUDA events on
 * the launching stream.  Region names: "assign_tc" (tensor-core distance
 * GEMM), "assign_gemm" (CUDA-core distance GEMM), "assign_recheck",
 * "label_sort", "centroid_update", "kmeanspp", "scan_topk_level",
 * "scan_topk_leaf".  Off by default.
 */
void mask_profile_enable(int32_t on);

/* Drop all recorded timings. */
void mask_profile_reset(void);

/*
 * Totals for one region since the last reset: launches, summed device time
 * in ms, summed algorithmic work (useful flop 2*n*k*d for "assign_tc" and
 * "assign_gemm", bytes for the others).  Waits for the recorded events.  Returns 1, or 0 if nothing was
 * recorded under that name.  Any output pointer may be NULL.
 */
int32_t mask_profile_read(const char *name, int64_t *launches, double *total_ms,
                          double *work);

/* Kernel launches the library has issued since it was loaded. */
int64_t mask_launch_count(void);

/*
 * Device and pinned-host allocations the library has made since it was
 * loaded (stream-ordered scratch, index arrays, serving staging buffers).
 * A test hook: it lets a caller check that a call allocated nothing.
 */
int64_t mask_test_alloc_count(void);

/*
 * Test of the failure-detection contract of the library's device-side waits
 * (every spin on a flag or barrier is bounded and reports instead of hanging):
 * one GPU thread polls a device flag, set before the launch when flag_set is
 * nonzero and never otherwise, for at most limit_us microseconds of GPU timer
 * time.  Returns MASK_OK if it saw the flag, MASK_ETIMEOUT if the wait ran out
 * (the context stays usable), MASK_EINVAL if limit_us is outside
 * [0, 10,000,000].  Synchronises `stream`.
 */
mask_status mask_test_bounded_wait(int32_t flag_set, int32_t limit_us, mask_stream stream);

/*
 * Timing probe of the 5th-generation tensor-core MMA behind the tensor-core
 * assignment's tile width (the paper has no counterpart: this measures the
 * hardware).  One CTA on the current device issues rounds x 12
 * tcgen05.mma.cta_group::1.kind::f16 instructions (M = 128, N = n, K = 16,
 * zero operands: 4 K-steps x 3 products, the assignment's pattern) into
 * n_acc accumulators used round-robin, with A in tensor memory (a_in_tmem
 * nonzero) or shared memory and B in shared memory.  cycles_out[0] = SM
 * cycles spent issuing them, cycles_out[1] = cycles until the last one
 * completed.  n: a multiple of 16 in [16, 256]; n_acc * n <= 448 with A in
 * tensor memory, else 512; rounds in [1, 65536].  MASK_EINVAL outside these,
 * MASK_ETIMEOUT if completion does not arrive within the library's wait
 * limit.  Synchronous.
 */
mask_status mask_test_tc_mma_cycles(int32_t n, int32_t a_in_tmem, int32_t n_acc, int32_t rounds,
                                    int64_t *cycles_out);

/* ---- serving: continuous batching over a resident index ----------------
 *
 * The paper answers queries one at a time (§3.3); a service takes a stream
 * of requests (batches of queries of any size, each with its own k, probes
 * and precision) against one resident dense index.  The paper has no
 * counterpart: this is the interface of the query path as a service.
 *
 * A worker thread merges pending requests with equal probes and precision
 * (low precision: also equal k) into one launch of up to max_batch queries
 * (a larger request is split), replays the captured CUDA graph of that batch
 * shape on one of max_slots streams, and admits a batch only while the
 * device bytes of the batches in flight (graph buffers and kernel scratch,
 * estimated per shape) stay within mem_budget.  Requests arriving while
 * others run join the next batch as slots and memory free up.  A request's
 * result is the same as mask_query's on its queries alone (bit for bit).
 * For FP32 shapes where both leaf scans apply, the first batch of a shape
 * (probes, precision, batch bucket, k) times five captured graphs: the
 * query-major scan, and the cluster-major scan with 16 or 8 queries per work
 * item at all the blocks per SM that fit or at one.  It keeps the fastest
 * and releases the others (autotuning; results are identical).  The graphs
 * captured while autotuning hold buffers outside the mem_budget accounting
 * (the budget covers the batches admitted to run).
 *
 * The index must stay alive until mask_server_close.  Queries and outputs
 * are HOST memory: queries are copied at submit; ids_out / dists_out are
 * written by the worker and must stay valid until poll or wait returns
 * something other than MASK_PENDING for the ticket.
 */
typedef struct mask_server mask_server;

typedef struct {
    int64_t requests_done, requests_failed, queries_done;
    int64_t batches;              /* launches (graph replays) of merged batches */
    int64_t graph_launches;
    int64_t graph_captures;       /* batch shapes captured so far */
    int64_t autotuned_shapes;
    double mean_batch_queries;    /* queries per batch (before padding) */
    double latency_mean_ms, latency_p50_ms, latency_p99_ms, latency_max_ms;  /* submit -> done */
    double elapsed_s;             /* first submit -> last completion */
    int64_t peak_inflight_bytes;  /* most estimated device bytes in flight at once */
    int64_t mem_budget;
} mask_server_info;

/* Opens a server on a dense index: mem_budget (> 0) device bytes for batches
 * in flight, max_slots in [1, 64] concurrent batches (streams), max_batch in
 * [8, 2^20] queries per launch (rounded up to a power of two). */
mask_status mask_server_open(const mask_index *index, int64_t mem_budget, int32_t max_slots,
                             int32_t max_batch, mask_server **out);

/* Queues a request (arguments as mask_query, host pointers only) and returns
 * its ticket; errors in the arguments are returned here. */
mask_status mask_server_submit(mask_server *server, const float *queries, int64_t nq, int32_t k,
                               const int32_t *probes, mask_precision precision,
                               int64_t *ids_out, float *dists_out, uint64_t *ticket_out);

/* MASK_PENDING while the request runs; otherwise its final status (MASK_OK:
 * outputs written), after which the ticket is forgotten. */
mask_status mask_server_poll(mask_server *server, uint64_t ticket);

/* As poll, waiting up to timeout_ms (< 0: no limit). */
mask_status mask_server_wait(mask_server *server, uint64_t ticket, int32_t timeout_ms);

/* Counters and latency percentiles since open (or the last reset). */
mask_status mask_server_stats(mask_server *server, mask_server_info *out, int32_t reset);

/* Finishes every queued request, then releases the server (NULL is ignored). */
void mask_server_close(mask_server *server);

#ifdef __cplusplus
}
#endif

#endif /* MASK_GB300_H */
