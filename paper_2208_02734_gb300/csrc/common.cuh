// common.cuh -- internal declarations shared by the CUDA translation units of
// libmask_gb300.so (not part of the C ABI; see include/mask.h for that).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "mask.h"

namespace mask {

// ------------------------------------------------------------------ errors

struct Error : std::runtime_error {
    mask_status status;
    Error(mask_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] void fail(mask_status s, const std::string &msg);
// Sets the calling thread's mask_last_error() message.
void set_last_error(const std::string &msg);

// ------------------------------------------------------------- profiling

// Counts one kernel launch (called by MASK_LAUNCHED at every launch site).
void count_launch();
// True while mask_profile_enable(1) is in effect (kernels then also count
// the bytes their scans read).
bool profiling_enabled();
// Counts n launches at once (the kernel nodes of a replayed graph).
void count_launches(long long n);
// Counts one device or pinned-host allocation (Scratch, DevArray, server
// staging); read through mask_test_alloc_count().
void count_alloc();

// While profiling is enabled, brackets its scope with CUDA events on stream s
// and books the elapsed device time and `work` (flop or bytes) under `name`.
class ProfRegion {
  public:
    ProfRegion(const char *name, cudaStream_t s, double work);
    ~ProfRegion();
    ProfRegion(const ProfRegion &) = delete;
    ProfRegion &operator=(const ProfRegion &) = delete;

  private:
    const char *name_;
    cudaStream_t s_;
    double work_;
    cudaEvent_t a_{}, b_{};
    bool active_ = false;
};

#define MASK_CUDA(call)                                                             \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess)                                                      \
            ::mask::fail(e_ == cudaErrorMemoryAllocation ? MASK_ENOMEM : MASK_ECUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

#define MASK_LAUNCHED(what)                                                          \
    do {                                                                             \
        ::mask::count_launch();                                                      \
        cudaError_t e_ = cudaGetLastError();                                         \
        if (e_ != cudaSuccess)                                                       \
            ::mask::fail(MASK_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define MASK_REQUIRE(cond, msg)                                   \
    do {                                                          \
        if (!(cond)) ::mask::fail(MASK_EINVAL, std::string(msg)); \
    } while (0)

// --------------------------------------------------------- device buffers

// Stream-ordered allocation from the library's memory pool of the current
// device (kept warm between calls: up to kScratchKeepBytes stay reserved
// after a synchronisation instead of going back to the driver); inside a
// stream capture, from the device's default pool (graph memory nodes).
void *scratch_alloc(size_t bytes, cudaStream_t s);
constexpr unsigned long long kScratchKeepBytes = 4ull << 30;

// Stream-ordered scratch (scratch_alloc / cudaFreeAsync on one stream).
template <class T>
struct Scratch {
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    Scratch() = default;
    Scratch(size_t count, cudaStream_t st) { alloc(count, st); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    Scratch(Scratch &&o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    Scratch &operator=(Scratch &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
        return *this;
    }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count) {
            count_alloc();
            p = static_cast<T *>(scratch_alloc(count * sizeof(T), st));
        }
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    ~Scratch() { release(); }
    T *get() const { return p; }
};

// Long-lived device array (cudaMalloc), owned by an index.
template <class T>
struct DevArray {
    T *p = nullptr;
    size_t n = 0;
    DevArray() = default;
    DevArray(const DevArray &) = delete;
    DevArray &operator=(const DevArray &) = delete;
    DevArray(DevArray &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevArray &operator=(DevArray &&o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) {
            count_alloc();
            MASK_CUDA(cudaMalloc((void **)&p, count * sizeof(T)));
        }
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevArray() { release(); }
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------- constants

// Internal row stride: dimensions are zero-padded to a multiple of 8 floats
// (32 bytes) so every row starts 16-byte aligned and splits into float4s.
inline int padded_dim(int d) { return (d + 7) / 8 * 8; }

// Lanes cooperating on one row: the largest power of two <= min(32, dp/4).
inline int lanes_per_row(int dp) {
    int c = dp / 4, l = 1;
    while (l * 2 <= c && l * 2 <= 32) l *= 2;
    return l;
}

constexpr uint64_t kNoKey = ~0ull;

// Largest dimension of CSR inputs: k-means++ holds one dense row of it in
// shared memory.
constexpr int kCsrMaxDim = 40960;

// ------------------------------------------------------- random numbers

// R1: SplitMix64 (Steele, Lea & Flood 2014), host side: every draw of the
// library is taken on the host from this generator.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
};

// The stream of level lv (0-based) under `seed`.
inline uint64_t level_state(uint64_t seed, int lv) {
    return seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(lv + 1));
}

// ------------------------------------------------------ kernel launchers

// kmeans.cu
void pad_rows(const float *src, int64_t n, int d, float *dst, int dp, cudaStream_t s);
void unpad_rows(const float *src, int64_t n, int dp, float *dst, int d, cudaStream_t s);
void row_sqnorm(const float *X, int64_t n, int dp, float *out, cudaStream_t s);
void max_reduce(const float *v, int64_t n, float *out, cudaStream_t s);
template <class I>
void gather_rows(const float *src, int dp, const I *idx, int64_t m, float *dst, cudaStream_t s);
void iota_i32(int32_t *p, int64_t n, cudaStream_t s);
// k-means++ over the m rows of Xs; chosen[0] must be set; fills chosen[1..k).
// a53[t] (device) is the t-th draw as the generator's 53-bit integer
// (u_t = a53[t] * 2^-53).
void kmeanspp_steps(const float *Xs, int64_t m, int dp, int k, const unsigned long long *a53,
                    int64_t *chosen, cudaStream_t s);
// the same over CSR rows (dense row of dp <= kCsrMaxDim in shared memory)
void kmeanspp_steps_csr(const int64_t *rp, const int32_t *col, const float *val, int64_t m,
                        int64_t nnz, int dp, int k, const unsigned long long *a53,
                        int64_t *chosen, cudaStream_t s);
// counting sort of labels in [0,k): off[k+1] (int64), perm[n] (item ids by label)
void label_sort(const int32_t *labels, int64_t n, int k, int64_t *off, int32_t *perm,
                cudaStream_t s);
// per-cluster mean (write=true) and sum of squared distances to C_prev
void centroid_update(const float *X, int dp, const int32_t *perm, const int64_t *off, int k,
                     const float *C_prev, float *C_new, float *sse, bool write,
                     cudaStream_t s);
// dist[i] = ||x_i - c_{labels[i]}||^2, difference form
void label_dist(const float *X, int64_t n, int dp, const float *C, const int32_t *labels,
                float *dist, cudaStream_t s);
void off_to_counts(const int64_t *off, int k, int64_t *counts, cudaStream_t s);
void count_bad_labels(const int32_t *labels, int64_t n, int k, int *bad, cudaStream_t s);

// sparse.cu -- CSR rows (row_ptr int64 [n+1], col int32, val float32)
// bad[0] = malformed rows (row_ptr decreasing, columns not strictly
// increasing), bad[1] = column ids outside [0, d), bad[2] = longest row;
// bad must hold 3 ints
void csr_validate(const int64_t *rp, const int32_t *col, int64_t n, int64_t nnz, int d, int *bad,
                  cudaStream_t s);
void csr_row_sqnorm(const int64_t *rp, const float *val, int64_t n, float *xn, cudaStream_t s);
void inclusive_scan_i64(int64_t *v, int64_t n, cudaStream_t s);
// rows idx[0..m) of a CSR matrix as a new CSR matrix (synchronises s)
template <class I>
void csr_gather_rows(const int64_t *rp, const int32_t *col, const float *val, const I *idx,
                     int64_t m, DevArray<int64_t> &orp, DevArray<int32_t> &ocol,
                     DevArray<float> &oval, cudaStream_t s);
// out [m x dp] = dense copies of rows rows[i] (rows == null: rows 0..m)
void csr_densify_rows(const int64_t *rp, const int32_t *col, const float *val,
                      const int64_t *rows, int64_t m, int dp, float *out, cudaStream_t s);
// cn [kp] = ||c_j||^2 (float-float sum rounded; +inf for j >= k), cn_lo [k]
// the remainders (cn + cn_lo = the float-float sums)
void centroid_norms(const float *C, int k, int dp, int kp, float *cn, float *cn_lo,
                    cudaStream_t s);
// labels = argmin_j ||x_i - c_j||^2 for CSR rows and dense C [k x dp] (ties to
// the smallest j); cn_out (optional, [k]) receives ||c_j||^2
void csr_assign(const int64_t *rp, const int32_t *col, const float *val, int64_t n,
                int64_t nnz, const float *xn, const float *C, int k, int dp, int32_t *labels,
                float *cn_out, cudaStream_t s);
// dist[i] = ||x_i - c_{labels[i]}||^2 (cn = ||c_j||^2)
void csr_label_dist(const int64_t *rp, const int32_t *col, const float *val, int64_t n,
                    const float *C, int dp, const float *cn, const int32_t *labels, float *dist,
                    cudaStream_t s);
// C_new = per-cluster means of CSR rows (C_prev kept for empty clusters; C_new
// may be null), sse[j] = sum over members of ||x_i - c_prev_j||^2 (cn_prev =
// ||c_prev_j||^2)
void csr_centroid_update(const int64_t *rp, const int32_t *col, const float *val,
                         const int32_t *perm, const int64_t *off, int64_t n_rows, int k, int dp,
                         const float *C_prev, const float *cn_prev, float *C_new, float *sse,
                         cudaStream_t s);

// query_csr.cu -- the descent for CSR queries over a CSR index
// level scan: dense centroid rows R (norms rcn) against the query nonzeros
// (at most qcap per query, staged in shared memory)
size_t csr_level_scan_smem(int K, int P, int qcap);
void csr_level_scan(const float *R, int dp, const float *rcn, const int32_t *rid,
                    const int64_t *off, const int32_t *sel, int P, int64_t root_end,
                    const int64_t *qrp, const int32_t *qcol, const float *qval, int qcap,
                    int64_t nq, int K, int32_t *out32, cudaStream_t s);
// cluster-major leaf scan for large CSR batches (K <= 64): same keys as
// csr_leaf_scan; queries longer than csr_cm_longest_query() nonzeros come out
// empty and must be served by csr_leaf_scan(..., min_nnz = that length)
bool csr_cm_supported(int K);
int csr_cm_longest_query();
void csr_cm_leaf_scan(const int64_t *xrp, const int32_t *xcol, const float *xval,
                      const int32_t *xids, const int64_t *leaf_off, int k0, const int32_t *sel,
                      int P, const int64_t *qrp, const int32_t *qcol, const float *qval,
                      int64_t nq, int K, int64_t *out64, float *out_d, cudaStream_t s);
// bytes the CSR scans read since the last reset ([0] levels, [1] leaf)
double csr_scan_bytes(int which);
void csr_scan_bytes_reset();
// leaf scan: CSR point rows (cluster-major) against the query's nonzeros held
// in a shared-memory table sized for the longest query (`longest` nonzeros)
size_t csr_leaf_scan_smem(int K, int P, int longest);
void csr_leaf_scan(const int64_t *xrp, const int32_t *xcol, const float *xval,
                   const int32_t *xids, const int64_t *off, const int32_t *sel, int P,
                   const int64_t *qrp, const int32_t *qcol, const float *qval, int longest,
                   int64_t nq, int K, int64_t *out64, float *out_d, cudaStream_t s,
                   int64_t min_nnz = -1);  // only queries with more nonzeros than this

// assign.cu -- labels[i] = argmin_j ||x_i - c_j||^2 (ties to the smallest j)
void assign_labels(const float *X, const float *xn, int64_t n, int dp, const float *C, int k,
                   int32_t *labels, cudaStream_t s);

// re-decide the listed rows exactly over all k centroids (difference form)
void assign_recheck_rows(const float *X, int dp, const float *C, int k, const int32_t *rows,
                         const int *count, int32_t *labels, cudaStream_t s);

// assign_tc.cu -- the same assignment on tcgen05 (FP16 three-product split), for dp <= 64
struct TcAssign;
bool tc_assign_enabled(int dp);
// Splits X (padded, [n x dp]) into scaled FP16 hi/lo parts once; null if unsupported.
std::shared_ptr<TcAssign> tc_assign_prepare(const float *X, int64_t n, int dp, cudaStream_t s);
// seeded: labels holds the previous assignment's labels on entry (the
// kernel starts each row's search threshold from its previous centroid).
void tc_assign(TcAssign &p, const float *xn, const float *C, int k, int32_t *labels,
               bool seeded, cudaStream_t s);
// Raises MASK_ETIMEOUT if a kernel of this plan hit a wait limit (synchronises).
void tc_assign_check(TcAssign &p, cudaStream_t s);

// grouped.cu -- the grouped build of Algorithm 1 (random split into groups of
// lengthGroup items, nCentroids centroids per group by its own k-means)
uint64_t group_state(uint64_t seed, int lv, int64_t g);
std::vector<int64_t> grouped_sizes(int64_t n, int lg, int nc);
std::vector<int32_t> split_groups(int64_t m, int64_t G, SplitMix64 &rng);
void grouped_level(const float *X, int64_t m, int dp, const std::vector<int32_t> &group_of,
                   int64_t G, int nc, int iters, uint64_t seed, int lv, float *C,
                   int32_t *labels, cudaStream_t s);

// range.cu -- range search (Algorithm 3) over a dense index: counts_out
// (host) [nq] = results per query; when ids_out is given and the total fits
// `capacity`, the results (ascending by (distance, id), query after query)
// go to ids_out / dists_out (device).  Returns the total.
int64_t range_search(const mask_index &idx, const float *Qp, int64_t nq, float radius,
                     int64_t *counts_out, int64_t capacity, int64_t *ids_out, float *dists_out,
                     cudaStream_t s);

// merge.cu -- the distributed exchange (§3.4): ids/dists [G x nq x k] from G
// partitions -> the k smallest (distance, global id) per query
size_t merge_topk_smem(int G, int k);
void merge_topk(const int64_t *ids, const float *dists, int G, int64_t nq, int k,
                const int64_t *id_offset, int64_t *ids_out, float *dists_out, cudaStream_t s);

// query.cu -- the greedy descent (one kept centroid per level) for a whole
// batch in one launch: per level, the parent-major centroid rows, their ids
// and off[l] = the child ranges of level l's centroids in level l-1's rows
// (level 0: in the points).  leaf (may be null) gets the reached leaf cluster;
// ids/dists (may be null) the nearest point of that cluster.
struct GreedyLevels {
    const float4 *Cs[MASK_MAX_LEVELS];
    const int32_t *ids[MASK_MAX_LEVELS];
    const int64_t *off[MASK_MAX_LEVELS];
    int64_t k_top;
};
void greedy_descent(const GreedyLevels &lv, int L, const float *Xs, const int32_t *xids, int dp,
                    const float *Qp, int64_t nq, int32_t *leaf, int64_t *ids, float *dists,
                    cudaStream_t s);

// query.cu -- keep the K nearest rows among the children of each query's parents
struct ScanArgs {
    const float *R = nullptr;     // [M x dp] rows (parent-major)
    const int32_t *rid = nullptr; // [M] id of each row (used in the ordering key)
    const int64_t *off = nullptr; // [n_parents+1] child ranges, or null for the root range
    const int32_t *sel = nullptr; // [Q x P] parent ids (-1 = none), or null for the root
    int P = 0;
    int64_t root_end = 0;         // root range [0, root_end) when off == null
    const float *Q = nullptr;     // [nq x dp] padded queries
    int64_t nq = 0;
    int dp = 0;
    int K = 0;
    int32_t *out_ids32 = nullptr; // [nq x K] (levels) ...
    int64_t *out_ids64 = nullptr; // ... or int64 (leaf)
    float *out_d = nullptr;       // [nq x K] (may be null)
    // centroid levels: false when only the first (nearest) key's place
    // matters to the caller, who reads the rest as a set
    bool sorted = true;
};
void scan_topk(const ScanArgs &a, cudaStream_t s);
// bytes streamed by the scans since the last reset ([0] levels, [1] leaf)
double scan_bytes(int which);
void scan_bytes_reset();

// query_cm.cu -- cluster-major leaf scan for large batches (K <= 32, dp <= 128)
bool cm_leaf_supported(int dp, int K);
// ids/dists [nq x K] = each query's K smallest keys over its P per-pair lists
// (pair_out [nq*P x K], keys = distance bits << 32 | original id)
void cm_merge(const unsigned long long *pair_out, int64_t nq, int P, int K, int64_t *ids,
              float *dists, cudaStream_t s);
// seed_d [nq x K] = each query's K nearest exact (FP32, per-query scan)
// distances within its nearest kept cluster (the first of its kept list);
// the K-th bounds the query's final K-th distance from above (+inf if short)
void leaf_seed(const float *Xs, const int32_t *xids, const int64_t *leaf_off, int dp,
               const float *Qp, int64_t nq, const int32_t *sel, int P, int K, float *seed_d,
               cudaStream_t s);
// probe_tc.cu: cycles to issue (cycles[0]) and to complete (cycles[1])
// rounds x 12 tcgen05 kind::f16 MMAs of M = 128, K = 16 and the given N
void probe_tc_mma(int n, int a_in_tmem, int n_acc, int rounds, int64_t *cycles_out);

// Work-item shape of the cluster-major scans, chosen by the serving loop's
// autotuner: queries per item (0: the kernel's widest, cm_item_queries), the
// kernel (the tensor-core scan where it applies, or the mma.sync scan), and
// for the latter blocks per SM (0: as many as fit).
struct CmTile {
    int qpi = 0;
    int bps = 0;
    bool legacy = false;
};

// The tensor-core cluster-major scan (query_cm_tc.cu): rows of 32 or 64
// floats, K <= 32, in two passes (a tensor-core filter against T_q that
// appends candidates per query, then one warp per query for the exact keys
// and the top-K, written to ids / dists).  A bounded pipeline wait that ran
// out raises a device error word; cm_tc_check (synchronising) reports it as
// MASK_ETIMEOUT and clears it, cm_tc_error_word gives its device address.
bool cm_tc_supported(int dp, int K);
// widest work item of the tensor-core scan: 32 queries for K <= 16, else 16
int cm_tc_item_queries(int K);
// candidates kept per query (beyond them a query is scanned in full)
int cm_tc_cand_cap(int64_t nq);
// qs: queries per item slot of meta / qid (16 or 32; the filter's MMA N);
// ccount [nq] (preset 0) and cand [nq x cap]: the candidate lists
void cm_tc_scan(const float *Xs, int64_t n, const float *xn, int dp, const int32_t *xids,
                const int64_t *leaf_off, int k0, const float *Qp, int64_t nq, const int32_t *sel,
                int P, const float *qn, const float *seed_d, float mcoef, const int4 *meta,
                const int32_t *qid, const int64_t *item_off, int K, int qs, unsigned *ccount,
                uint32_t *cand, int cap, int64_t *ids, float *dists,
                unsigned long long *bytes_ctr, cudaStream_t s);
int *cm_tc_error_word();
void cm_tc_check(cudaStream_t s);
// Whether cm_tc_scan was called on this thread since the last call (clears).
bool cm_tc_take_launched();
void cm_leaf_scan(const float *Xs, int64_t n, const float *xn, int dp, const int32_t *xids,
                  const int64_t *leaf_off, int k0, const float *Qp, int64_t nq,
                  const int32_t *sel, int P, int K, int64_t *ids, float *dists, cudaStream_t s,
                  CmTile tile = CmTile{});
double cm_bytes();
void cm_bytes_reset();
// groups the (query, kept leaf) pairs by leaf cluster; item_off[k0] = work items
void cm_group_pairs(const int32_t *sel, int64_t nq, int P, int k0, Scratch<int32_t> &pairs,
                    Scratch<int64_t> &poff, Scratch<int64_t> &item_off, cudaStream_t s,
                    int qpi = 16);
// queries per work item of the cluster-major scans (the tensor-core scan
// also takes items of up to kCmTcItemQueries)
constexpr int kCmItemQueries = 16;
constexpr int kCmTcItemQueries = 32;
// per work item i of cm_group_pairs (cluster c, up to qpi <= qs of its
// pairs): meta[i] = {first row (lo, hi), rows of c, pairs in the item};
// pid/qid[i * qs + q] = the item's q-th pair (-1 past the last) and its
// query (0 past the last)
void cm_item_meta(const int32_t *pairs, const int64_t *poff, const int64_t *item_off,
                  const int64_t *leaf_off, int64_t npairs, int P, int k0, Scratch<int4> &meta,
                  Scratch<int32_t> &pid, Scratch<int32_t> &qid, cudaStream_t s,
                  int qpi = kCmItemQueries, int qs = kCmItemQueries);

// Asynchronous global -> shared copies (cp.async); a false `valid` writes
// zeros (the source is then not read, but must still be a valid address).
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// query_lp.cu -- BF16 / FP8 leaf scan with exact FP32 re-rank of a 4k shortlist
int lp_padded_dim(int dp);
int lp_shortlist(int k);  // max(4k, 16)
bool lp_supported(int dp, int k);
// quantised copy ([rows x lp_padded_dim] BF16 or e4m3), per-row scale (FP8) and
// squared norm of every quantised row
void lp_quantize(const float *src, int64_t rows, int dp, bool fp8, void *dst, float *scale,
                 float *norm2, cudaStream_t s);
void lp_leaf_scan(bool fp8, const void *Xl, const float *xn2, const float *xscale, const float *Xs,
                  int64_t leaf_rows, int dp, const int32_t *xids, const int64_t *leaf_off, int k0,
                  const float *Qp, int64_t nq, const int32_t *sel, int P, int k, int64_t *ids,
                  float *dists, cudaStream_t s);

}  // namespace mask
