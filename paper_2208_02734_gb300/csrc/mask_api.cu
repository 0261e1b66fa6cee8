// mask_api.cu -- host orchestration and the C ABI of libmask_gb300.so.
//
// Build (§3.1, Algorithm 1, one group per level): for each level, k-means++
// seeding (§3.2), Lloyd iterations (§2.4) as assign -> label sort -> mean
// update, a final assignment, then the level's centroids are the next
// level's data.  Afterwards every level is laid out parent-major (children of
// a centroid contiguous) and the points cluster-major, so the query (§3.3,
// Algorithm 2) is a chain of scan_topk launches over contiguous row ranges.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "index.cuh"

namespace mask {

namespace {
thread_local std::string g_err;
}

void fail(mask_status s, const std::string &msg) { throw Error(s, msg); }

void set_last_error(const std::string &msg) { g_err = msg; }

namespace {


// ------------------------------------------------------- pointer staging

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A caller input as a device pointer (host data copied in on the stream).
template <class T>
struct In {
    const T *p = nullptr;
    Scratch<T> tmp;
    In(const T *src, size_t count, cudaStream_t s) {
        if (src == nullptr || count == 0 || on_device(src)) {
            p = src;
            return;
        }
        tmp.alloc(count, s);
        MASK_CUDA(cudaMemcpyAsync(tmp.get(), src, count * sizeof(T), cudaMemcpyHostToDevice, s));
        p = tmp.get();
    }
};

// A caller output as a device pointer (copied back to host memory by finish()).
template <class T>
struct Out {
    T *user = nullptr, *p = nullptr;
    size_t count = 0;
    bool host = false;
    Scratch<T> tmp;
    Out(T *dst, size_t c, cudaStream_t s) : user(dst), count(c) {
        if (dst == nullptr || c == 0 || on_device(dst)) {
            p = dst;
            return;
        }
        host = true;
        tmp.alloc(c, s);
        p = tmp.get();
    }
    void finish(cudaStream_t s) {
        if (host)
            MASK_CUDA(cudaMemcpyAsync(user, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
};

template <class T>
void to_host(std::vector<T> &v, const T *dev, size_t count, cudaStream_t s) {
    v.resize(count);
    if (count == 0) return;
    MASK_CUDA(cudaMemcpyAsync(v.data(), dev, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    MASK_CUDA(cudaStreamSynchronize(s));
}

template <class T>
void copy_out_host_vec(const std::vector<T> &v, T *dst, cudaStream_t s) {
    if (dst == nullptr || v.empty()) return;
    if (on_device(dst)) {
        MASK_CUDA(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        MASK_CUDA(cudaStreamSynchronize(s));
    } else {
        std::memcpy(dst, v.data(), v.size() * sizeof(T));
    }
}

template <class F>
mask_status guard(F &&f) {
    try {
        f();
        return MASK_OK;
    } catch (const Error &e) {
        g_err = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return MASK_ENOMEM;
    } catch (const std::exception &e) {
        g_err = e.what();
        return MASK_ECUDA;
    }
}

int current_device() {
    int dev = 0;
    MASK_CUDA(cudaGetDevice(&dev));
    return dev;
}

// ---------------------------------------------------- seeding (§3.2, R2-R3)

// Number of inputs k-means++ runs on: all of them, or 8k when the n*k
// distance evaluations of full seeding exceed 2^32 and 8k < n.
int64_t seed_sample_size(int64_t n, int k) {
    if ((double)n * (double)k > 4294967296.0 && 8 * (int64_t)k < n) return 8 * (int64_t)k;
    return n;
}

// The partial Fisher-Yates draws of a seeding subsample of m of n inputs.
std::vector<int64_t> draw_subsample(SplitMix64 &rng, int64_t n, int64_t m) {
    std::vector<int64_t> idx((size_t)n);
    for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = i;
    for (int64_t j = 0; j < m; ++j) {
        int64_t r = j + (int64_t)std::floor(rng.uniform() * (double)(n - j));
        if (r > n - 1) r = n - 1;
        std::swap(idx[(size_t)j], idx[(size_t)r]);
    }
    idx.resize((size_t)m);
    return idx;
}

// One draw per centre: a53 [k] on the device holds each draw as the
// generator's 53-bit integer a (u = a * 2^-53, so the device decides the
// pick rule in integers), and chosen[0] = floor(u_0 m).
void draw_centres(SplitMix64 &rng, int64_t m, int k, Scratch<unsigned long long> &a53,
                  Scratch<int64_t> &ch, cudaStream_t s) {
    std::vector<unsigned long long> a((size_t)k);
    for (int t = 0; t < k; ++t) a[(size_t)t] = rng.next() >> 11;
    int64_t first = (int64_t)std::floor((double)a[0] * 0x1.0p-53 * (double)m);
    if (first > m - 1) first = m - 1;
    a53.alloc(k, s);
    ch.alloc(k, s);
    MASK_CUDA(cudaMemcpyAsync(a53.get(), a.data(), k * sizeof(unsigned long long),
                              cudaMemcpyHostToDevice, s));
    MASK_CUDA(cudaMemcpyAsync(ch.get(), &first, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MASK_CUDA(cudaStreamSynchronize(s));  // a and first are host temporaries
}

// k-means++ for one level: C_out [k x dp] = the chosen rows of X; `chosen`
// receives their indices into X.  Random draws on the host (R1): first the
// partial Fisher-Yates draws of the subsample (if any), then one per centre.
void seed_level(const float *X, int64_t n, int dp, int k, uint64_t seed, int lv, float *C_out,
                std::vector<int64_t> &chosen, cudaStream_t s) {
    SplitMix64 rng{level_state(seed, lv)};
    const int64_t m = seed_sample_size(n, k);
    std::vector<int64_t> sample;
    Scratch<float> Xsub;
    const float *S = X;
    if (m < n) {
        sample = draw_subsample(rng, n, m);
        Scratch<int64_t> sidx(m, s);
        MASK_CUDA(cudaMemcpyAsync(sidx.get(), sample.data(), m * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
        Xsub.alloc((size_t)m * dp, s);
        gather_rows<int64_t>(X, dp, sidx.get(), m, Xsub.get(), s);
        S = Xsub.get();
        MASK_CUDA(cudaStreamSynchronize(s));  // sidx and sample are released below
    }
    Scratch<unsigned long long> ud;
    Scratch<int64_t> ch;
    draw_centres(rng, m, k, ud, ch, s);
    kmeanspp_steps(S, m, dp, k, ud.get(), ch.get(), s);
    gather_rows<int64_t>(S, dp, ch.get(), k, C_out, s);
    to_host(chosen, ch.get(), (size_t)k, s);
    if (m < n)
        for (auto &c : chosen) c = sample[(size_t)c];
}

// The same for CSR rows; C_out receives dense copies of the chosen rows.
void seed_level_csr(const int64_t *rp, const int32_t *col, const float *val, int64_t n, int dp,
                    int k, uint64_t seed, int lv, float *C_out, std::vector<int64_t> &chosen,
                    cudaStream_t s) {
    SplitMix64 rng{level_state(seed, lv)};
    const int64_t m = seed_sample_size(n, k);
    std::vector<int64_t> sample;
    DevArray<int64_t> srp;
    DevArray<int32_t> scol;
    DevArray<float> sval;
    const int64_t *Rp = rp;
    const int32_t *Cl = col;
    const float *Vl = val;
    if (m < n) {
        sample = draw_subsample(rng, n, m);
        Scratch<int64_t> sidx(m, s);
        MASK_CUDA(cudaMemcpyAsync(sidx.get(), sample.data(), m * sizeof(int64_t),
                                  cudaMemcpyHostToDevice, s));
        csr_gather_rows<int64_t>(rp, col, val, sidx.get(), m, srp, scol, sval, s);
        Rp = srp.get();
        Cl = scol.get();
        Vl = sval.get();
    }
    Scratch<unsigned long long> ud;
    Scratch<int64_t> ch;
    draw_centres(rng, m, k, ud, ch, s);
    int64_t nnz = 0;
    MASK_CUDA(cudaMemcpyAsync(&nnz, Rp + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MASK_CUDA(cudaStreamSynchronize(s));
    kmeanspp_steps_csr(Rp, Cl, Vl, m, nnz, dp, k, ud.get(), ch.get(), s);
    csr_densify_rows(Rp, Cl, Vl, ch.get(), k, dp, C_out, s);
    to_host(chosen, ch.get(), (size_t)k, s);
    if (m < n)
        for (auto &c : chosen) c = sample[(size_t)c];
}

// ------------------------------------------------------- Lloyd (§2.4, R4)

// The objective after each assignment: the k per-cluster sums of squared
// distances (FP32, one row per assignment) are kept on the device and summed
// on the host in FP64, in cluster order, once the iterations are done.
struct ObjectiveTrace {
    Scratch<float> rows;
    int k = 0, count = 0;
    ObjectiveTrace(int k_, int count_, cudaStream_t s) : rows((size_t)k_ * count_, s), k(k_), count(count_) {}
    void record(int i, const float *sse, cudaStream_t s) {
        MASK_CUDA(cudaMemcpyAsync(rows.get() + (size_t)i * k, sse, sizeof(float) * k,
                                  cudaMemcpyDeviceToDevice, s));
    }
    void finish(std::vector<double> &out, cudaStream_t s) {
        std::vector<float> h;
        to_host(h, rows.get(), (size_t)k * count, s);
        out.assign((size_t)count, 0.0);
        for (int i = 0; i < count; ++i)
            for (int j = 0; j < k; ++j) out[(size_t)i] += (double)h[(size_t)i * k + j];
    }
};

// Lloyd iterations on the n_in rows of X (padded) from the centres in C
// (k x dp, updated in place).  Writes the final labels, the membership list
// of the final assignment (off [k+1], perm [n_in]) and the objective after
// each assignment (iters+1 values).
void lloyd(const float *X, int64_t n_in, int dp, int k, int iters, float *C, int32_t *labels,
           int64_t *off, int32_t *perm, std::vector<double> &objective, cudaStream_t s) {
    Scratch<float> xn(n_in, s), Cn((size_t)k * dp, s), sse(k, s);
    ObjectiveTrace J(k, iters + 1, s);
    row_sqnorm(X, n_in, dp, xn.get(), s);
    // tensor-core assignment when the row fits (X split into FP16 hi/lo
    // parts once); from the second assignment on, each row's search starts
    // from its previous label
    auto tc = tc_assign_prepare(X, n_in, dp, s);
    bool have_labels = false;
    auto assign = [&](const float *Cc) {
        if (tc) tc_assign(*tc, xn.get(), Cc, k, labels, have_labels, s);
        else assign_labels(X, xn.get(), n_in, dp, Cc, k, labels, s);
        have_labels = true;
    };
    float *cur = C, *nxt = Cn.get();
    for (int it = 0; it < iters; ++it) {
        assign(cur);
        label_sort(labels, n_in, k, off, perm, s);
        centroid_update(X, dp, perm, off, k, cur, nxt, sse.get(), true, s);
        J.record(it, sse.get(), s);
        std::swap(cur, nxt);
    }
    assign(cur);
    label_sort(labels, n_in, k, off, perm, s);
    centroid_update(X, dp, perm, off, k, cur, nullptr, sse.get(), false, s);
    if (tc) tc_assign_check(*tc, s);
    J.record(iters, sse.get(), s);
    if (cur != C)
        MASK_CUDA(cudaMemcpyAsync(C, cur, sizeof(float) * k * dp, cudaMemcpyDeviceToDevice, s));
    J.finish(objective, s);
}

// Lloyd iterations on CSR rows (dense centroids C [k x dp], updated in place);
// the same outputs as lloyd().
void lloyd_csr(const int64_t *rp, const int32_t *col, const float *val, int64_t n, int64_t nnz,
               int dp, int k, int iters, float *C, int32_t *labels, int64_t *off, int32_t *perm,
               std::vector<double> &objective, cudaStream_t s) {
    Scratch<float> xn(n, s), Cn((size_t)k * dp, s), sse(k, s), cn(k, s);
    ObjectiveTrace J(k, iters + 1, s);
    csr_row_sqnorm(rp, val, n, xn.get(), s);
    float *cur = C, *nxt = Cn.get();
    for (int it = 0; it < iters; ++it) {
        csr_assign(rp, col, val, n, nnz, xn.get(), cur, k, dp, labels, cn.get(), s);
        label_sort(labels, n, k, off, perm, s);
        csr_centroid_update(rp, col, val, perm, off, n, k, dp, cur, cn.get(), nxt, sse.get(), s);
        J.record(it, sse.get(), s);
        std::swap(cur, nxt);
    }
    csr_assign(rp, col, val, n, nnz, xn.get(), cur, k, dp, labels, cn.get(), s);
    label_sort(labels, n, k, off, perm, s);
    csr_centroid_update(rp, col, val, perm, off, n, k, dp, cur, cn.get(), nullptr, sse.get(), s);
    J.record(iters, sse.get(), s);
    if (cur != C)
        MASK_CUDA(cudaMemcpyAsync(C, cur, sizeof(float) * k * dp, cudaMemcpyDeviceToDevice, s));
    J.finish(objective, s);
}

// ------------------------------------------------------------ index layout

// Given every level's centroids C, labels and membership lists (level lv's
// off, and the perm of its items, stored as the ids of the level below),
// lay out the parent-major arrays: points cluster-major (Xs), and each
// non-top level's centroids in the order of their parents (Cs).
void finish_levels(mask_index &idx, cudaStream_t s) {
    const int dp = idx.dp;
    for (int lv = 0; lv < idx.L; ++lv) {
        auto &L = idx.lv[(size_t)lv];
        L.Cs.alloc((size_t)L.k * dp);
        if (lv == idx.L - 1) {
            L.ids.alloc((size_t)L.k);
            iota_i32(L.ids.get(), L.k, s);
            MASK_CUDA(cudaMemcpyAsync(L.Cs.get(), L.C.get(), sizeof(float) * L.k * dp,
                                      cudaMemcpyDeviceToDevice, s));
        } else {
            gather_rows<int32_t>(L.C.get(), dp, L.ids.get(), L.k, L.Cs.get(), s);
        }
        if (idx.sparse) {
            L.cns.alloc((size_t)L.k);
            Scratch<float> nlo(L.k, s);
            centroid_norms(L.Cs.get(), L.k, dp, L.k, L.cns.get(), nlo.get(), s);
            MASK_CUDA(cudaStreamSynchronize(s));
        }
    }
    MASK_CUDA(cudaStreamSynchronize(s));
}

void finish_layout(mask_index &idx, const float *Xp, cudaStream_t s) {
    idx.Xs.alloc((size_t)idx.n * idx.dp);
    gather_rows<int32_t>(Xp, idx.dp, idx.xids.get(), idx.n, idx.Xs.get(), s);
    idx.xn.alloc((size_t)idx.n);
    row_sqnorm(idx.Xs.get(), idx.n, idx.dp, idx.xn.get(), s);
    finish_levels(idx, s);
}

// CSR index: the points' rows cluster-major (row i = point xids[i]).
void finish_layout_csr(mask_index &idx, const int64_t *rp, const int32_t *col, const float *val,
                       cudaStream_t s) {
    csr_gather_rows<int32_t>(rp, col, val, idx.xids.get(), idx.n, idx.xrp, idx.xcol, idx.xval, s);
    finish_levels(idx, s);
}

void check_common(int64_t n, int d, const int32_t *k_per_level, int n_levels, mask_index **out) {
    MASK_REQUIRE(out != nullptr, "out is NULL");
    MASK_REQUIRE(n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31)");
    MASK_REQUIRE(d >= 1, "d must be >= 1");
    MASK_REQUIRE(n_levels >= 1 && n_levels <= MASK_MAX_LEVELS, "n_levels out of range");
    MASK_REQUIRE(k_per_level != nullptr, "k_per_level is NULL");
    int64_t below = n;
    for (int l = 0; l < n_levels; ++l) {
        MASK_REQUIRE(k_per_level[l] >= 1 && (int64_t)k_per_level[l] <= below,
                     "k_per_level[" + std::to_string(l) + "] must be in [1, items below]");
        below = k_per_level[l];
    }
}

std::unique_ptr<mask_index> new_index(int64_t n, int d, const int32_t *kpl, int L) {
    auto idx = std::make_unique<mask_index>();
    idx->device = current_device();
    idx->n = n;
    idx->d = d;
    idx->dp = padded_dim(d);
    idx->L = L;
    idx->lv.resize((size_t)L);
    for (int l = 0; l < L; ++l) idx->lv[(size_t)l].k = kpl[l];
    return idx;
}

// Level-l items' ids array (the perm of level l's membership lists): the
// point ids for l = 0, else the ids of level l-1's parent-major rows.
int32_t *below_ids(mask_index &idx, int lv, int64_t n_in) {
    if (lv == 0) {
        idx.xids.alloc((size_t)n_in);
        return idx.xids.get();
    }
    auto &B = idx.lv[(size_t)lv - 1];
    B.ids.alloc((size_t)n_in);
    return B.ids.get();
}

// Levels lv0.. of the build on the n_in dense rows `in` (level lv0's items).
void build_dense_levels(mask_index &idx, int lv0, const float *in, int64_t n_in, uint64_t seed,
                        cudaStream_t s) {
    for (int lv = lv0; lv < idx.L; ++lv) {
        auto &L = idx.lv[(size_t)lv];
        L.C.alloc((size_t)L.k * idx.dp);
        L.labels.alloc((size_t)n_in);
        L.off.alloc((size_t)L.k + 1);
        int32_t *perm = below_ids(idx, lv, n_in);
        seed_level(in, n_in, idx.dp, L.k, seed, lv, L.C.get(), L.chosen, s);
        lloyd(in, n_in, idx.dp, L.k, idx.iters, L.C.get(), L.labels.get(), L.off.get(), perm,
              L.objective, s);
        in = L.C.get();
        n_in = L.k;
    }
}

void build_dense(mask_index &idx, const float *Xp, uint64_t seed, cudaStream_t s) {
    build_dense_levels(idx, 0, Xp, idx.n, seed, s);
    finish_layout(idx, Xp, s);
}

// CSR points: level 0 on the sparse rows (dense centroids), the levels above
// on those centroids as dense rows.
void build_csr(mask_index &idx, const int64_t *rp, const int32_t *col, const float *val,
               int64_t nnz, uint64_t seed, cudaStream_t s) {
    auto &L = idx.lv[0];
    const int64_t n = idx.n;
    L.C.alloc((size_t)L.k * idx.dp);
    L.labels.alloc((size_t)n);
    L.off.alloc((size_t)L.k + 1);
    int32_t *perm = below_ids(idx, 0, n);
    seed_level_csr(rp, col, val, n, idx.dp, L.k, seed, 0, L.C.get(), L.chosen, s);
    lloyd_csr(rp, col, val, n, nnz, idx.dp, L.k, idx.iters, L.C.get(), L.labels.get(),
              L.off.get(), perm, L.objective, s);
    build_dense_levels(idx, 1, L.C.get(), L.k, seed, s);
    finish_layout_csr(idx, rp, col, val, s);
}

// A value of a caller array that may live on the host or the device.
template <class T>
T read_value(const T *p, cudaStream_t s) {
    T v{};
    if (on_device(p)) {
        MASK_CUDA(cudaMemcpyAsync(&v, p, sizeof(T), cudaMemcpyDeviceToHost, s));
        MASK_CUDA(cudaStreamSynchronize(s));
    } else {
        v = *p;
    }
    return v;
}

// Stages and checks caller CSR arrays of `rows` rows over d columns; returns
// the nonzero count and (optionally) the longest row.
struct CsrIn {
    int64_t nnz = 0;
    int longest = 0;
    std::unique_ptr<In<int64_t>> rp;
    std::unique_ptr<In<int32_t>> col;
    std::unique_ptr<In<float>> val;
    CsrIn(const int64_t *row_ptr, const int32_t *c, const float *v, int64_t rows, int d,
          cudaStream_t s) {
        MASK_REQUIRE(row_ptr != nullptr, "row_ptr is NULL");
        const int64_t r0 = read_value(row_ptr, s), rn = read_value(row_ptr + rows, s);
        MASK_REQUIRE(r0 == 0, "row_ptr[0] must be 0");
        MASK_REQUIRE(rn >= 0, "row_ptr[rows] must be >= 0");
        nnz = rn;
        MASK_REQUIRE(nnz == 0 || (c != nullptr && v != nullptr), "col or val is NULL");
        rp = std::make_unique<In<int64_t>>(row_ptr, (size_t)rows + 1, s);
        col = std::make_unique<In<int32_t>>(c, (size_t)nnz, s);
        val = std::make_unique<In<float>>(v, (size_t)nnz, s);
        Scratch<int> bad(3, s);
        csr_validate(rp->p, col->p, rows, nnz, d, bad.get(), s);
        int h[3] = {0, 0, 0};
        MASK_CUDA(cudaMemcpyAsync(h, bad.get(), sizeof(h), cudaMemcpyDeviceToHost, s));
        MASK_CUDA(cudaStreamSynchronize(s));
        MASK_REQUIRE(h[0] == 0, std::to_string(h[0]) +
                                    " CSR rows malformed (row_ptr decreasing or column ids not "
                                    "strictly increasing within a row)");
        MASK_REQUIRE(h[1] == 0, std::to_string(h[1]) + " CSR column ids outside [0, d)");
        longest = h[2];
    }
};

}  // namespace

void ensure_lowp(const mask_index &idx, bool fp8, cudaStream_t s) {
    const int slot = fp8 ? 1 : 0;
    std::lock_guard<std::mutex> lk(idx.lp_mu);
    if (idx.Xlp[slot].p != nullptr) return;
    const int dpl = lp_padded_dim(idx.dp);
    idx.Xlp[slot].alloc((size_t)idx.n * dpl * (fp8 ? 1 : 2));
    idx.xn_lp[slot].alloc((size_t)idx.n);
    if (fp8) idx.xscale_fp8.alloc((size_t)idx.n);
    lp_quantize(idx.Xs.get(), idx.n, idx.dp, fp8, idx.Xlp[slot].get(),
                fp8 ? idx.xscale_fp8.get() : nullptr, idx.xn_lp[slot].get(), s);
    MASK_CUDA(cudaStreamSynchronize(s));
}

// inv[perm[i]] = i for a permutation of [0, n).
__global__ void invert_perm_kernel(const int32_t *__restrict__ perm, int64_t n,
                                   int32_t *__restrict__ inv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        inv[perm[i]] = (int32_t)i;
}

// The index's levels for the one-launch greedy descent.
GreedyLevels greedy_levels(const mask_index &idx) {
    GreedyLevels g{};
    for (int l = 0; l < idx.L; ++l) {
        g.Cs[l] = reinterpret_cast<const float4 *>(idx.lv[(size_t)l].Cs.get());
        g.ids[l] = idx.lv[(size_t)l].ids.get();
        g.off[l] = idx.lv[(size_t)l].off.get();
    }
    g.k_top = idx.lv[(size_t)idx.L - 1].k;
    return g;
}

bool all_ones(const std::vector<int> &p) {
    for (int v : p)
        if (v != 1) return false;
    return true;
}

// The descent of Algorithm 2 down to the leaf clusters: sel[l] [nq x p_l]
// receives each level's kept centroids (cluster ids), nearest first.
void descend_levels(const mask_index &idx, const float *Qp, int64_t nq, const std::vector<int> &p,
                    std::vector<Scratch<int32_t>> &sel, cudaStream_t s, bool sorted_last) {
    const int L = idx.L, dp = idx.dp;
    sel.resize((size_t)L);
    for (int l = 0; l < L; ++l) sel[(size_t)l].alloc((size_t)nq * p[(size_t)l], s);
    ScanArgs a;
    a.Q = Qp;
    a.nq = nq;
    a.dp = dp;
    const int top = L - 1;
    a.R = idx.lv[(size_t)top].Cs.get();
    a.rid = idx.lv[(size_t)top].ids.get();
    a.root_end = idx.lv[(size_t)top].k;
    a.K = p[(size_t)top];
    a.out_ids32 = sel[(size_t)top].get();
    // the kept parents of a level are read as a set; the last level's list
    // only needs its nearest entry first, unless the caller wants it sorted
    a.sorted = top == 0 ? sorted_last : false;
    scan_topk(a, s);
    for (int l = top; l >= 1; --l) {
        ScanArgs b = a;
        b.R = idx.lv[(size_t)l - 1].Cs.get();
        b.rid = idx.lv[(size_t)l - 1].ids.get();
        b.off = idx.lv[(size_t)l].off.get();
        b.sel = sel[(size_t)l].get();
        b.P = p[(size_t)l];
        b.K = p[(size_t)l - 1];
        b.out_ids32 = sel[(size_t)l - 1].get();
        b.sorted = l == 1 ? sorted_last : false;
        scan_topk(b, s);
    }
}

void query_dense(const mask_index &idx, const float *Qp, int64_t nq, int k,
                 const std::vector<int> &p, mask_precision prec, LeafMode mode, int64_t *ids,
                 float *dists, cudaStream_t s, CmTile tile) {
    if (nq == 0) return;
    const int dp = idx.dp;
    if (k == 1 && prec == MASK_FP32 && all_ones(p)) {
        // the paper's point query / nearest neighbour: one launch for the
        // whole descent (same results as the general path)
        greedy_descent(greedy_levels(idx), idx.L, idx.Xs.get(), idx.xids.get(), dp, Qp, nq,
                       nullptr, ids, dists, s);
        return;
    }
    std::vector<Scratch<int32_t>> sel;
    descend_levels(idx, Qp, nq, p, sel, s, false);
    ScanArgs a;
    a.Q = Qp;
    a.nq = nq;
    a.dp = dp;
    const int k0 = idx.lv[0].k;
    if (prec != MASK_FP32) {
        // BF16 / FP8 distances for a max(4k, 16) shortlist, exact FP32 re-rank
        const bool fp8 = prec == MASK_FP8E4M3;
        const int slot = fp8 ? 1 : 0;
        MASK_REQUIRE(idx.Xlp[slot].p != nullptr, "low-precision copy missing");
        lp_leaf_scan(fp8, idx.Xlp[slot].get(), idx.xn_lp[slot].get(),
                     fp8 ? idx.xscale_fp8.get() : nullptr, idx.Xs.get(), idx.n, dp, idx.xids.get(),
                     idx.lv[0].off.get(), k0, Qp, nq, sel[0].get(), p[0], k, ids, dists, s);
        return;
    }
    // Leaf scan: cluster-major when the batch keeps each leaf cluster several
    // times on average, else query by query (same arithmetic, same results).
    bool cluster_major = cm_leaf_supported(dp, k) && nq * (int64_t)p[0] >= 4 * (int64_t)k0;
    if (mode == LeafMode::Cluster) cluster_major = cm_leaf_supported(dp, k);
    if (mode == LeafMode::Query) cluster_major = false;
    if (cluster_major) {
        cm_leaf_scan(idx.Xs.get(), idx.n, idx.xn.get(), dp, idx.xids.get(), idx.lv[0].off.get(),
                     k0, Qp, nq, sel[0].get(), p[0], k, ids, dists, s, tile);
    } else {
        ScanArgs c = a;
        c.R = idx.Xs.get();
        c.rid = idx.xids.get();
        c.off = idx.lv[0].off.get();
        c.sel = sel[0].get();
        c.P = p[0];
        c.K = k;
        c.out_ids32 = nullptr;
        c.out_ids64 = ids;
        c.out_d = dists;
        scan_topk(c, s);
    }
}

}  // namespace mask

using namespace mask;

// ===================================================================== C ABI

extern "C" {

const char *mask_last_error(void) { return g_err.c_str(); }

mask_status mask_build(const float *points, int64_t n, int32_t d, const int32_t *k_per_level,
                       int32_t n_levels, int32_t iters, uint64_t seed, mask_stream stream,
                       mask_index **out) {
    return guard([&] {
        check_common(n, d, k_per_level, n_levels, out);
        MASK_REQUIRE(points != nullptr, "points is NULL");
        MASK_REQUIRE(iters >= 0, "iters must be >= 0");
        cudaStream_t s = (cudaStream_t)stream;
        auto idx = new_index(n, d, k_per_level, n_levels);
        idx->iters = iters;
        In<float> P(points, (size_t)n * d, s);
        Scratch<float> Xp((size_t)n * idx->dp, s);
        pad_rows(P.p, n, d, Xp.get(), idx->dp, s);
        build_dense(*idx, Xp.get(), seed, s);
        MASK_CUDA(cudaStreamSynchronize(s));
        *out = idx.release();
    });
}

mask_status mask_build_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                           int64_t n, int32_t d, const int32_t *k_per_level, int32_t n_levels,
                           int32_t iters, uint64_t seed, mask_stream stream, mask_index **out) {
    return guard([&] {
        check_common(n, d, k_per_level, n_levels, out);
        MASK_REQUIRE(iters >= 0, "iters must be >= 0");
        if (d > kCsrMaxDim)
            fail(MASK_EUNSUPPORTED, "CSR inputs need d <= " + std::to_string(kCsrMaxDim));
        cudaStream_t s = (cudaStream_t)stream;
        CsrIn in(row_ptr, col, val, n, d, s);
        auto idx = new_index(n, d, k_per_level, n_levels);
        idx->iters = iters;
        idx->sparse = true;
        build_csr(*idx, in.rp->p, in.col->p, in.val->p, in.nnz, seed, s);
        MASK_CUDA(cudaStreamSynchronize(s));
        *out = idx.release();
    });
}

mask_status mask_index_load(const float *points, int64_t n, int32_t d, int32_t n_levels,
                            const int32_t *k_per_level, const float *const *centroids,
                            const int32_t *const *labels, mask_stream stream,
                            mask_index **out) {
    return guard([&] {
        check_common(n, d, k_per_level, n_levels, out);
        MASK_REQUIRE(points && centroids && labels, "NULL array");
        cudaStream_t s = (cudaStream_t)stream;
        auto idx = new_index(n, d, k_per_level, n_levels);
        In<float> P(points, (size_t)n * d, s);
        Scratch<float> Xp((size_t)n * idx->dp, s);
        pad_rows(P.p, n, d, Xp.get(), idx->dp, s);
        Scratch<int> bad(1, s);
        int64_t n_in = n;
        for (int lv = 0; lv < n_levels; ++lv) {
            auto &L = idx->lv[(size_t)lv];
            MASK_REQUIRE(centroids[lv] && labels[lv], "NULL level array");
            In<float> Cin(centroids[lv], (size_t)L.k * d, s);
            In<int32_t> Lin(labels[lv], (size_t)n_in, s);
            L.C.alloc((size_t)L.k * idx->dp);
            pad_rows(Cin.p, L.k, d, L.C.get(), idx->dp, s);
            L.labels.alloc((size_t)n_in);
            MASK_CUDA(cudaMemcpyAsync(L.labels.get(), Lin.p, sizeof(int32_t) * n_in,
                                      cudaMemcpyDeviceToDevice, s));
            count_bad_labels(L.labels.get(), n_in, L.k, bad.get(), s);
            int nbad = 0;
            MASK_CUDA(cudaMemcpyAsync(&nbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
            MASK_CUDA(cudaStreamSynchronize(s));
            MASK_REQUIRE(nbad == 0, "labels of level " + std::to_string(lv) + " out of range");
            L.off.alloc((size_t)L.k + 1);
            label_sort(L.labels.get(), n_in, L.k, L.off.get(), below_ids(*idx, lv, n_in), s);
            n_in = L.k;
        }
        finish_layout(*idx, Xp.get(), s);
        *out = idx.release();
    });
}

void mask_free(mask_index *index) {
    if (index == nullptr) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(index->device);
    delete index;
    cudaSetDevice(prev);
}

mask_status mask_index_get_info(const mask_index *index, mask_index_info *out) {
    return guard([&] {
        MASK_REQUIRE(index && out, "NULL argument");
        std::memset(out, 0, sizeof(*out));
        out->n = index->n;
        out->d = index->d;
        out->n_levels = index->L;
        out->iters = index->iters;
        out->sparse = index->sparse ? 1 : 0;
        int64_t bytes = (int64_t)(index->Xs.bytes() + index->xids.bytes() + index->xn.bytes() +
                                  index->xrp.bytes() +
                                  index->xcol.bytes() + index->xval.bytes());
        for (int q = 0; q < 2; ++q) bytes += (int64_t)(index->Xlp[q].bytes() + index->xn_lp[q].bytes());
        bytes += (int64_t)index->xscale_fp8.bytes();
        for (int l = 0; l < index->L; ++l) {
            const auto &L = index->lv[(size_t)l];
            out->k_per_level[l] = L.k;
            bytes += (int64_t)(L.C.bytes() + L.Cs.bytes() + L.ids.bytes() + L.off.bytes() +
                               L.labels.bytes() + L.cns.bytes());
        }
        out->device_bytes = bytes;
    });
}

mask_status mask_index_export_level(const mask_index *index, int32_t level, float *centroids_out,
                                    int32_t *labels_out, int64_t *chosen_out,
                                    double *objective_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr, "index is NULL");
        MASK_REQUIRE(level >= 0 && level < index->L, "level out of range");
        cudaStream_t s = (cudaStream_t)stream;
        const auto &L = index->lv[(size_t)level];
        const int64_t n_below = level == 0 ? index->n : index->lv[(size_t)level - 1].k;
        if (centroids_out) {
            Out<float> C(centroids_out, (size_t)L.k * index->d, s);
            unpad_rows(L.C.get(), L.k, index->dp, C.p, index->d, s);
            C.finish(s);
        }
        if (labels_out) {
            Out<int32_t> lb(labels_out, (size_t)n_below, s);
            MASK_CUDA(cudaMemcpyAsync(lb.p, L.labels.get(), sizeof(int32_t) * n_below,
                                      cudaMemcpyDeviceToDevice, s));
            lb.finish(s);
        }
        MASK_CUDA(cudaStreamSynchronize(s));
        copy_out_host_vec(L.chosen, chosen_out, s);
        copy_out_host_vec(L.objective, objective_out, s);
    });
}

mask_status mask_query(const mask_index *index, const float *queries, int64_t nq, int32_t k,
                       const int32_t *probes, mask_precision precision, int64_t *ids_out,
                       float *dists_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr, "index is NULL");
        MASK_REQUIRE(nq >= 0, "nq must be >= 0");
        MASK_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
        MASK_REQUIRE(probes != nullptr, "probes is NULL");
        MASK_REQUIRE(current_device() == index->device, "index lives on another device");
        MASK_REQUIRE(!index->sparse, "index built from CSR points: query it with mask_query_csr");
        MASK_REQUIRE(precision == MASK_FP32 || precision == MASK_BF16 ||
                         precision == MASK_FP8E4M3, "unknown precision");
        const bool lowp = precision != MASK_FP32;
        if (lowp && !lp_supported(index->dp, k))
            fail(MASK_EUNSUPPORTED, "BF16/FP8 modes keep a 4k shortlist: k <= 16 and d <= 256");
        if (nq == 0) return;
        MASK_REQUIRE(queries && ids_out, "NULL queries or ids_out");
        cudaStream_t s = (cudaStream_t)stream;
        const int L = index->L, dp = index->dp;
        std::vector<int> p((size_t)L);
        for (int l = 0; l < L; ++l) {
            MASK_REQUIRE(probes[l] >= 1, "probes must be >= 1");
            p[(size_t)l] = std::min<int>(probes[l], index->lv[(size_t)l].k);
        }
        if (lowp) ensure_lowp(*index, precision == MASK_FP8E4M3, s);
        // MASK_LEAF_SCAN = query | cluster[:queries per item:blocks per SM]
        // pins the leaf scan (and the cluster-major tile) for tests
        LeafMode mode = LeafMode::Auto;
        CmTile tile;
        if (const char *m = std::getenv("MASK_LEAF_SCAN")) {
            if (std::strncmp(m, "cluster", 7) == 0) {
                mode = LeafMode::Cluster;
                int qpi = 0, bps = 0;
                if (std::sscanf(m + 7, ":%d:%d", &qpi, &bps) == 2) {
                    MASK_REQUIRE(qpi >= 1 && qpi <= kCmTcItemQueries && bps >= 0,
                                 "MASK_LEAF_SCAN tile out of range");
                    tile = CmTile{qpi, bps};
                }
            }
            if (std::strcmp(m, "query") == 0) mode = LeafMode::Query;
        }
        In<float> Qin(queries, (size_t)nq * index->d, s);
        Scratch<float> Qp((size_t)nq * dp, s);
        pad_rows(Qin.p, nq, index->d, Qp.get(), dp, s);
        Out<int64_t> ids(ids_out, (size_t)nq * k, s);
        Out<float> dd(dists_out, (size_t)nq * k, s);
        cm_tc_take_launched();
        query_dense(*index, Qp.get(), nq, k, p, precision, mode, ids.p, dd.p, s, tile);
        ids.finish(s);
        dd.finish(s);
        if (cm_tc_take_launched()) cm_tc_check(s);   // synchronises; MASK_ETIMEOUT on a stall
        if (ids.host || dd.host) MASK_CUDA(cudaStreamSynchronize(s));
    });
}

mask_status mask_query_csr(const mask_index *index, const int64_t *row_ptr, const int32_t *col,
                           const float *val, int64_t nq, int32_t k, const int32_t *probes,
                           mask_precision precision, int64_t *ids_out, float *dists_out,
                           mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr, "index is NULL");
        MASK_REQUIRE(nq >= 0, "nq must be >= 0");
        MASK_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
        MASK_REQUIRE(probes != nullptr, "probes is NULL");
        MASK_REQUIRE(current_device() == index->device, "index lives on another device");
        MASK_REQUIRE(index->sparse, "index built from dense points: query it with mask_query");
        MASK_REQUIRE(precision == MASK_FP32 || precision == MASK_BF16 ||
                         precision == MASK_FP8E4M3, "unknown precision");
        if (precision != MASK_FP32) fail(MASK_EUNSUPPORTED, "CSR queries run in FP32 only");
        if (nq == 0) return;
        MASK_REQUIRE(ids_out != nullptr, "ids_out is NULL");
        cudaStream_t s = (cudaStream_t)stream;
        const int L = index->L, dp = index->dp;
        std::vector<int> p((size_t)L);
        for (int l = 0; l < L; ++l) {
            MASK_REQUIRE(probes[l] >= 1, "probes must be >= 1");
            p[(size_t)l] = std::min<int>(probes[l], index->lv[(size_t)l].k);
        }
        CsrIn in(row_ptr, col, val, nq, index->d, s);
        constexpr int kQueryNnzMax = 8192;
        if (in.longest > kQueryNnzMax)
            fail(MASK_EUNSUPPORTED, "a CSR query has more than " + std::to_string(kQueryNnzMax) +
                                        " nonzeros");
        const int qcap = std::max(1, in.longest);
        Out<int64_t> ids(ids_out, (size_t)nq * k, s);
        Out<float> dd(dists_out, (size_t)nq * k, s);
        std::vector<Scratch<int32_t>> sel((size_t)L);
        for (int l = 0; l < L; ++l) sel[(size_t)l].alloc((size_t)nq * p[(size_t)l], s);
        const int top = L - 1;
        const auto &T = index->lv[(size_t)top];
        csr_level_scan(T.Cs.get(), dp, T.cns.get(), T.ids.get(), nullptr, nullptr, 1, T.k,
                       in.rp->p, in.col->p, in.val->p, qcap, nq, p[(size_t)top],
                       sel[(size_t)top].get(), s);
        for (int l = top; l >= 1; --l) {
            const auto &B = index->lv[(size_t)l - 1];
            csr_level_scan(B.Cs.get(), dp, B.cns.get(), B.ids.get(), index->lv[(size_t)l].off.get(),
                           sel[(size_t)l].get(), p[(size_t)l], 0, in.rp->p, in.col->p, in.val->p,
                           qcap, nq, p[(size_t)l - 1], sel[(size_t)l - 1].get(), s);
        }
        // leaf scan: cluster-major when the batch keeps each leaf cluster several
        // times on average (same keys), else query by query
        const int k0 = index->lv[0].k;
        bool cluster_major = csr_cm_supported(k) && nq * (int64_t)p[0] >= 4 * (int64_t)k0;
        if (const char *m = std::getenv("MASK_LEAF_SCAN")) {
            if (std::strcmp(m, "cluster") == 0) cluster_major = csr_cm_supported(k);
            if (std::strcmp(m, "query") == 0) cluster_major = false;
        }
        if (cluster_major) {
            csr_cm_leaf_scan(index->xrp.get(), index->xcol.get(), index->xval.get(),
                             index->xids.get(), index->lv[0].off.get(), k0, sel[0].get(), p[0],
                             in.rp->p, in.col->p, in.val->p, nq, k, ids.p, dd.p, s);
            // queries too long for the cluster-major tables, query by query
            if (in.longest > csr_cm_longest_query())
                csr_leaf_scan(index->xrp.get(), index->xcol.get(), index->xval.get(),
                              index->xids.get(), index->lv[0].off.get(), sel[0].get(), p[0],
                              in.rp->p, in.col->p, in.val->p, qcap, nq, k, ids.p, dd.p, s,
                              csr_cm_longest_query());
        } else
            csr_leaf_scan(index->xrp.get(), index->xcol.get(), index->xval.get(),
                          index->xids.get(), index->lv[0].off.get(), sel[0].get(), p[0], in.rp->p,
                          in.col->p, in.val->p, qcap, nq, k, ids.p, dd.p, s);
        ids.finish(s);
        dd.finish(s);
        MASK_CUDA(cudaStreamSynchronize(s));  // the staged CSR copies are released on return
    });
}

mask_status mask_kmeanspp(const float *X, int64_t n, int32_t d, int32_t k, uint64_t seed,
                          int32_t level, float *centroids_out, int64_t *chosen_out,
                          mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(X && centroids_out, "NULL argument");
        MASK_REQUIRE(n >= 1 && n <= INT32_MAX && d >= 1, "bad n or d");
        MASK_REQUIRE(k >= 1 && k <= n, "k must be in [1, n]");
        MASK_REQUIRE(level >= 0, "level must be >= 0");
        cudaStream_t s = (cudaStream_t)stream;
        const int dp = padded_dim(d);
        In<float> Xin(X, (size_t)n * d, s);
        Scratch<float> Xp((size_t)n * dp, s), Cp((size_t)k * dp, s);
        pad_rows(Xin.p, n, d, Xp.get(), dp, s);
        std::vector<int64_t> chosen;
        seed_level(Xp.get(), n, dp, k, seed, level, Cp.get(), chosen, s);
        Out<float> C(centroids_out, (size_t)k * d, s);
        unpad_rows(Cp.get(), k, dp, C.p, d, s);
        C.finish(s);
        MASK_CUDA(cudaStreamSynchronize(s));
        copy_out_host_vec(chosen, chosen_out, s);
    });
}

mask_status mask_kmeans_assign(const float *X, int64_t n, int32_t d, const float *C, int32_t k,
                               int32_t *labels_out, float *dist_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(X && C && labels_out, "NULL argument");
        MASK_REQUIRE(n >= 0 && n <= INT32_MAX && d >= 1 && k >= 1, "bad sizes");
        if (n == 0) return;
        cudaStream_t s = (cudaStream_t)stream;
        const int dp = padded_dim(d);
        In<float> Xin(X, (size_t)n * d, s), Cin(C, (size_t)k * d, s);
        Scratch<float> Xp((size_t)n * dp, s), Cp((size_t)k * dp, s), xn(n, s);
        pad_rows(Xin.p, n, d, Xp.get(), dp, s);
        pad_rows(Cin.p, k, d, Cp.get(), dp, s);
        row_sqnorm(Xp.get(), n, dp, xn.get(), s);
        Out<int32_t> lb(labels_out, (size_t)n, s);
        if (auto tc = tc_assign_prepare(Xp.get(), n, dp, s)) {
            tc_assign(*tc, xn.get(), Cp.get(), k, lb.p, false, s);
            tc_assign_check(*tc, s);
        } else {
            assign_labels(Xp.get(), xn.get(), n, dp, Cp.get(), k, lb.p, s);
        }
        if (dist_out) {
            Out<float> dist(dist_out, (size_t)n, s);
            label_dist(Xp.get(), n, dp, Cp.get(), lb.p, dist.p, s);
            dist.finish(s);
            lb.finish(s);
            MASK_CUDA(cudaStreamSynchronize(s));
        } else {
            lb.finish(s);
            if (lb.host) MASK_CUDA(cudaStreamSynchronize(s));
        }
    });
}

namespace mask {
namespace {
// One thread polls *flag until it is nonzero or limit_ns of GPU timer time
// have passed (a cap on the number of polls bounds it even without the
// timer); *seen = 1 if the flag was seen, 0 if the wait ran out.
__global__ void bounded_wait_kernel(const int *flag, unsigned long long limit_ns, int *seen) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long t0, now;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
    for (unsigned i = 0; i < (1u << 26); ++i) {
        if (*(const volatile int *)flag != 0) {
            *seen = 1;
            return;
        }
        if ((i & 63u) == 63u) {
            asm volatile("mov.u64 %0, %globaltimer;" : "=l"(now));
            if (now - t0 > limit_ns) break;
        }
    }
    *seen = 0;
}
}  // namespace
}  // namespace mask

mask_status mask_test_bounded_wait(int32_t flag_set, int32_t limit_us, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(limit_us >= 0 && limit_us <= 10000000, "limit_us out of range");
        cudaStream_t s = (cudaStream_t)stream;
        Scratch<int> buf(2, s);  // [0] the flag, [1] what the wait saw
        const int init[2] = {flag_set ? 1 : 0, -1};
        MASK_CUDA(cudaMemcpyAsync(buf.get(), init, sizeof(init), cudaMemcpyHostToDevice, s));
        mask::bounded_wait_kernel<<<1, 32, 0, s>>>(buf.get(), (unsigned long long)limit_us * 1000ull,
                                                   buf.get() + 1);
        MASK_LAUNCHED("bounded_wait");
        int seen = -1;
        MASK_CUDA(cudaMemcpyAsync(&seen, buf.get() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        MASK_CUDA(cudaStreamSynchronize(s));
        if (seen != 1) fail(MASK_ETIMEOUT, "bounded device wait ran out (the flag was never set)");
    });
}

mask_status mask_test_tc_mma_cycles(int32_t n, int32_t a_in_tmem, int32_t n_acc, int32_t rounds,
                                    int64_t *cycles_out) {
    return guard([&] { probe_tc_mma(n, a_in_tmem, n_acc, rounds, cycles_out); });
}

mask_status mask_kmeans_update(const float *X, int64_t n, int32_t d, const int32_t *labels,
                               int32_t k, const float *C_prev, float *C_out,
                               int64_t *counts_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(X && labels && C_prev && C_out, "NULL argument");
        MASK_REQUIRE(n >= 0 && n <= INT32_MAX && d >= 1 && k >= 1, "bad sizes");
        cudaStream_t s = (cudaStream_t)stream;
        const int dp = padded_dim(d);
        In<float> Xin(X, (size_t)n * d, s), Cin(C_prev, (size_t)k * d, s);
        In<int32_t> Lin(labels, (size_t)n, s);
        Scratch<int> bad(1, s);
        count_bad_labels(Lin.p, n, k, bad.get(), s);
        int nbad = 0;
        MASK_CUDA(cudaMemcpyAsync(&nbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        MASK_CUDA(cudaStreamSynchronize(s));
        MASK_REQUIRE(nbad == 0, "labels out of range");
        Scratch<float> Xp((size_t)n * dp, s), Cp((size_t)k * dp, s), Cn((size_t)k * dp, s), sse(k, s);
        Scratch<int64_t> off((size_t)k + 1, s);
        Scratch<int32_t> perm((size_t)n, s);
        pad_rows(Xin.p, n, d, Xp.get(), dp, s);
        pad_rows(Cin.p, k, d, Cp.get(), dp, s);
        label_sort(Lin.p, n, k, off.get(), perm.get(), s);
        centroid_update(Xp.get(), dp, perm.get(), off.get(), k, Cp.get(), Cn.get(), sse.get(), true, s);
        Out<float> Co(C_out, (size_t)k * d, s);
        unpad_rows(Cn.get(), k, dp, Co.p, d, s);
        Co.finish(s);
        if (counts_out) {
            Out<int64_t> cnt(counts_out, (size_t)k, s);
            off_to_counts(off.get(), k, cnt.p, s);
            cnt.finish(s);
        }
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

mask_status mask_kmeanspp_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                              int64_t n, int32_t d, int32_t k, uint64_t seed, int32_t level,
                              float *centroids_out, int64_t *chosen_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(centroids_out != nullptr, "centroids_out is NULL");
        MASK_REQUIRE(n >= 1 && n <= INT32_MAX && d >= 1, "bad n or d");
        MASK_REQUIRE(k >= 1 && k <= n, "k must be in [1, n]");
        MASK_REQUIRE(level >= 0, "level must be >= 0");
        if (d > kCsrMaxDim)
            fail(MASK_EUNSUPPORTED, "CSR inputs need d <= " + std::to_string(kCsrMaxDim));
        cudaStream_t s = (cudaStream_t)stream;
        CsrIn in(row_ptr, col, val, n, d, s);
        const int dp = padded_dim(d);
        Scratch<float> Cp((size_t)k * dp, s);
        std::vector<int64_t> chosen;
        seed_level_csr(in.rp->p, in.col->p, in.val->p, n, dp, k, seed, level, Cp.get(), chosen, s);
        Out<float> C(centroids_out, (size_t)k * d, s);
        unpad_rows(Cp.get(), k, dp, C.p, d, s);
        C.finish(s);
        MASK_CUDA(cudaStreamSynchronize(s));
        copy_out_host_vec(chosen, chosen_out, s);
    });
}

mask_status mask_kmeans_assign_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                                   int64_t n, int32_t d, const float *C, int32_t k,
                                   int32_t *labels_out, float *dist_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(C && labels_out, "NULL argument");
        MASK_REQUIRE(n >= 0 && n <= INT32_MAX && d >= 1 && k >= 1, "bad sizes");
        if (n == 0) return;
        cudaStream_t s = (cudaStream_t)stream;
        CsrIn in(row_ptr, col, val, n, d, s);
        const int dp = padded_dim(d);
        In<float> Cin(C, (size_t)k * d, s);
        Scratch<float> Cp((size_t)k * dp, s), xn(n, s), cn(k, s);
        pad_rows(Cin.p, k, d, Cp.get(), dp, s);
        csr_row_sqnorm(in.rp->p, in.val->p, n, xn.get(), s);
        Out<int32_t> lb(labels_out, (size_t)n, s);
        csr_assign(in.rp->p, in.col->p, in.val->p, n, in.nnz, xn.get(), Cp.get(), k, dp, lb.p,
                   cn.get(), s);
        if (dist_out) {
            Out<float> dist(dist_out, (size_t)n, s);
            csr_label_dist(in.rp->p, in.col->p, in.val->p, n, Cp.get(), dp, cn.get(), lb.p, dist.p,
                           s);
            dist.finish(s);
            lb.finish(s);
        } else {
            lb.finish(s);
        }
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

mask_status mask_kmeans_update_csr(const int64_t *row_ptr, const int32_t *col, const float *val,
                                   int64_t n, int32_t d, const int32_t *labels, int32_t k,
                                   const float *C_prev, float *C_out, int64_t *counts_out,
                                   mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(labels && C_prev && C_out, "NULL argument");
        MASK_REQUIRE(n >= 0 && n <= INT32_MAX && d >= 1 && k >= 1, "bad sizes");
        cudaStream_t s = (cudaStream_t)stream;
        CsrIn in(row_ptr, col, val, n, d, s);
        const int dp = padded_dim(d);
        In<float> Cin(C_prev, (size_t)k * d, s);
        In<int32_t> Lin(labels, (size_t)n, s);
        Scratch<int> bad(1, s);
        count_bad_labels(Lin.p, n, k, bad.get(), s);
        int nbad = 0;
        MASK_CUDA(cudaMemcpyAsync(&nbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        MASK_CUDA(cudaStreamSynchronize(s));
        MASK_REQUIRE(nbad == 0, "labels out of range");
        Scratch<float> Cp((size_t)k * dp, s), Cn((size_t)k * dp, s), sse(k, s), cn(k, s);
        Scratch<float> cn_lo(k, s);
        Scratch<int64_t> off((size_t)k + 1, s);
        Scratch<int32_t> perm((size_t)(n > 0 ? n : 1), s);
        pad_rows(Cin.p, k, d, Cp.get(), dp, s);
        centroid_norms(Cp.get(), k, dp, k, cn.get(), cn_lo.get(), s);
        label_sort(Lin.p, n, k, off.get(), perm.get(), s);
        csr_centroid_update(in.rp->p, in.col->p, in.val->p, perm.get(), off.get(), n, k, dp,
                            Cp.get(), cn.get(), Cn.get(), sse.get(), s);
        Out<float> Co(C_out, (size_t)k * d, s);
        unpad_rows(Cn.get(), k, dp, Co.p, d, s);
        Co.finish(s);
        if (counts_out) {
            Out<int64_t> cnt(counts_out, (size_t)k, s);
            off_to_counts(off.get(), k, cnt.p, s);
            cnt.finish(s);
        }
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

// ------------------------------------------------ grouped build (§3.1, A1)

mask_status mask_grouped_levels(int64_t n, int32_t length_group, int32_t n_centroids,
                                int64_t *sizes_out, int32_t *n_levels_out) {
    return guard([&] {
        MASK_REQUIRE(sizes_out && n_levels_out, "NULL output");
        MASK_REQUIRE(length_group >= 1 && n_centroids >= 1 && n_centroids <= length_group,
                     "need 1 <= nCentroids <= lengthGroup");
        MASK_REQUIRE(n >= 0, "n must be >= 0");
        const auto sizes = grouped_sizes(n, length_group, n_centroids);
        MASK_REQUIRE((int)sizes.size() <= MASK_MAX_LEVELS, "more than MASK_MAX_LEVELS levels");
        for (size_t l = 0; l < sizes.size(); ++l) sizes_out[l] = sizes[l];
        *n_levels_out = (int32_t)sizes.size();
    });
}

mask_status mask_build_grouped(const float *points, int64_t n, int32_t d, int32_t length_group,
                               int32_t n_centroids, int32_t iters, uint64_t seed,
                               const int32_t *group0, mask_stream stream, mask_index **out) {
    return guard([&] {
        MASK_REQUIRE(out != nullptr, "out is NULL");
        MASK_REQUIRE(points != nullptr, "points is NULL");
        MASK_REQUIRE(n >= 1 && n <= INT32_MAX, "n must be in [1, 2^31)");
        MASK_REQUIRE(d >= 1, "d must be >= 1");
        MASK_REQUIRE(length_group >= 1 && n_centroids >= 1 && n_centroids <= length_group,
                     "need 1 <= nCentroids <= lengthGroup");
        MASK_REQUIRE(n >= length_group, "fewer points than lengthGroup: no level to build");
        MASK_REQUIRE(iters >= 0, "iters must be >= 0");
        const auto sizes = grouped_sizes(n, length_group, n_centroids);
        const int L = (int)sizes.size();
        if (L > MASK_MAX_LEVELS) fail(MASK_EUNSUPPORTED, "more than MASK_MAX_LEVELS levels");
        std::vector<int32_t> kpl((size_t)L);
        for (int l = 0; l < L; ++l) {
            MASK_REQUIRE(sizes[(size_t)l] <= INT32_MAX, "too many centroids at one level");
            kpl[(size_t)l] = (int32_t)sizes[(size_t)l];
        }
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t G0 = n / length_group;
        std::vector<int32_t> g0;
        if (group0) {
            g0.resize((size_t)n);
            if (on_device(group0)) {
                MASK_CUDA(cudaMemcpyAsync(g0.data(), group0, sizeof(int32_t) * n,
                                          cudaMemcpyDeviceToHost, s));
                MASK_CUDA(cudaStreamSynchronize(s));
            } else {
                std::copy(group0, group0 + n, g0.begin());
            }
            for (int32_t v : g0) MASK_REQUIRE(v >= 0 && v < G0, "group0 value outside [0, n / lengthGroup)");
        }
        auto idx = new_index(n, d, kpl.data(), L);
        idx->iters = iters;
        In<float> P(points, (size_t)n * d, s);
        Scratch<float> Xp((size_t)n * idx->dp, s);
        pad_rows(P.p, n, d, Xp.get(), idx->dp, s);
        const float *in = Xp.get();
        int64_t m = n;
        for (int lv = 0; lv < L; ++lv) {
            auto &Lv = idx->lv[(size_t)lv];
            const int64_t G = m / length_group;
            std::vector<int32_t> group_of;
            if (lv == 0 && group0) {
                group_of = g0;
            } else {
                SplitMix64 rng{level_state(seed, lv)};
                group_of = split_groups(m, G, rng);
            }
            Lv.C.alloc((size_t)Lv.k * idx->dp);
            Lv.labels.alloc((size_t)m);
            Lv.off.alloc((size_t)Lv.k + 1);
            grouped_level(in, m, idx->dp, group_of, G, n_centroids, iters, seed, lv, Lv.C.get(),
                          Lv.labels.get(), s);
            label_sort(Lv.labels.get(), m, Lv.k, Lv.off.get(), below_ids(*idx, lv, m), s);
            in = Lv.C.get();
            m = Lv.k;
        }
        finish_layout(*idx, Xp.get(), s);
        MASK_CUDA(cudaStreamSynchronize(s));
        *out = idx.release();
    });
}

// ------------------------------------------------- descent (§3.3, A2)

mask_status mask_descend(const mask_index *index, const float *queries, int64_t nq,
                         const int32_t *probes, int32_t *leaf_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr, "index is NULL");
        MASK_REQUIRE(nq >= 0, "nq must be >= 0");
        MASK_REQUIRE(probes != nullptr, "probes is NULL");
        MASK_REQUIRE(current_device() == index->device, "index lives on another device");
        MASK_REQUIRE(!index->sparse, "index built from CSR points");
        if (nq == 0) return;
        MASK_REQUIRE(queries && leaf_out, "NULL queries or leaf_out");
        cudaStream_t s = (cudaStream_t)stream;
        const int L = index->L, dp = index->dp;
        std::vector<int> p((size_t)L);
        for (int l = 0; l < L; ++l) {
            MASK_REQUIRE(probes[l] >= 1, "probes must be >= 1");
            p[(size_t)l] = std::min<int>(probes[l], index->lv[(size_t)l].k);
        }
        In<float> Qin(queries, (size_t)nq * index->d, s);
        Scratch<float> Qp((size_t)nq * dp, s);
        pad_rows(Qin.p, nq, index->d, Qp.get(), dp, s);
        Out<int32_t> lo(leaf_out, (size_t)nq * probes[0], s);
        std::vector<Scratch<int32_t>> sel;
        if (all_ones(p) && probes[0] == 1) {
            greedy_descent(greedy_levels(*index), L, index->Xs.get(), index->xids.get(), dp,
                           Qp.get(), nq, lo.p, nullptr, nullptr, s);
        } else {
            descend_levels(*index, Qp.get(), nq, p, sel, s, true);
        }
        if (!sel.empty() && p[0] == probes[0]) {
            MASK_CUDA(cudaMemcpyAsync(lo.p, sel[0].get(), sizeof(int32_t) * nq * p[0],
                                      cudaMemcpyDeviceToDevice, s));
        } else if (!sel.empty()) {
            // more probes than leaf clusters: pad each row with -1
            MASK_CUDA(cudaMemsetAsync(lo.p, 0xFF, sizeof(int32_t) * nq * probes[0], s));
            MASK_CUDA(cudaMemcpy2DAsync(lo.p, sizeof(int32_t) * probes[0], sel[0].get(),
                                        sizeof(int32_t) * p[0], sizeof(int32_t) * p[0], nq,
                                        cudaMemcpyDeviceToDevice, s));
        }
        lo.finish(s);
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

// -------------------------------------------- relocation (§4.1), R20

mask_status mask_relocate(const mask_index *index, const float *points, int32_t n_centroids,
                          int32_t *group0, int64_t *missed_out, int64_t *moved_out,
                          mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr && points != nullptr && group0 != nullptr, "NULL argument");
        MASK_REQUIRE(!on_device(group0), "group0 must be host memory");
        MASK_REQUIRE(n_centroids >= 1, "n_centroids must be >= 1");
        MASK_REQUIRE(current_device() == index->device, "index lives on another device");
        MASK_REQUIRE(!index->sparse, "index built from CSR points");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n = index->n;
        std::vector<int32_t> leaf((size_t)n), own((size_t)n);
        // the greedy point query of every indexed point (one kept centroid per level)
        {
            In<float> P(points, (size_t)n * index->d, s);
            Scratch<float> Qp((size_t)n * index->dp, s);
            pad_rows(P.p, n, index->d, Qp.get(), index->dp, s);
            Scratch<int32_t> dleaf((size_t)n, s);
            greedy_descent(greedy_levels(*index), index->L, index->Xs.get(), index->xids.get(),
                           index->dp, Qp.get(), n, dleaf.get(), nullptr, nullptr, s);
            MASK_CUDA(cudaMemcpyAsync(leaf.data(), dleaf.get(), sizeof(int32_t) * n,
                                      cudaMemcpyDeviceToHost, s));
            MASK_CUDA(cudaMemcpyAsync(own.data(), index->lv[0].labels.get(), sizeof(int32_t) * n,
                                      cudaMemcpyDeviceToHost, s));
            MASK_CUDA(cudaStreamSynchronize(s));
        }
        int64_t G = 0;
        for (int64_t i = 0; i < n; ++i) {
            MASK_REQUIRE(group0[i] >= 0, "group0 value < 0");
            G = std::max<int64_t>(G, (int64_t)group0[i] + 1);
        }
        std::vector<int64_t> size((size_t)G, 0);
        for (int64_t i = 0; i < n; ++i) size[(size_t)group0[i]] += 1;
        int64_t missed = 0, moved = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (leaf[(size_t)i] == own[(size_t)i]) continue;
            ++missed;
            const int64_t tgt = leaf[(size_t)i] / n_centroids, src = group0[i];
            if (leaf[(size_t)i] < 0 || tgt == src || tgt >= G || size[(size_t)src] <= n_centroids)
                continue;
            size[(size_t)src] -= 1;
            size[(size_t)tgt] += 1;
            group0[i] = (int32_t)tgt;
            ++moved;
        }
        if (missed_out) *missed_out = missed;
        if (moved_out) *moved_out = moved;
    });
}

// ------------------------------------------------ range search (§3.3, A3)

mask_status mask_range_query(const mask_index *index, const float *queries, int64_t nq,
                             float radius, int64_t *counts_out, int64_t capacity,
                             int64_t *ids_out, float *dists_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr, "index is NULL");
        MASK_REQUIRE(nq >= 0 && nq <= INT32_MAX, "nq must be in [0, 2^31)");
        MASK_REQUIRE(radius >= 0.f && std::isfinite(radius), "radius must be finite and >= 0");
        MASK_REQUIRE(capacity >= 0, "capacity must be >= 0");
        MASK_REQUIRE(current_device() == index->device, "index lives on another device");
        MASK_REQUIRE(!index->sparse, "index built from CSR points");
        if (nq == 0) return;
        MASK_REQUIRE(queries && counts_out, "NULL queries or counts_out");
        cudaStream_t s = (cudaStream_t)stream;
        In<float> Qin(queries, (size_t)nq * index->d, s);
        Scratch<float> Qp((size_t)nq * index->dp, s);
        pad_rows(Qin.p, nq, index->d, Qp.get(), index->dp, s);
        std::vector<int64_t> counts((size_t)nq);
        Out<int64_t> ids(ids_out, (size_t)(ids_out ? capacity : 0), s);
        Out<float> dd(dists_out, (size_t)(dists_out ? capacity : 0), s);
        const int64_t total = range_search(*index, Qp.get(), nq, radius, counts.data(), capacity,
                                           ids_out ? ids.p : nullptr, dists_out ? dd.p : nullptr,
                                           s);
        copy_out_host_vec(counts, counts_out, s);
        if (ids_out && total > capacity)
            fail(MASK_EINVAL, "capacity " + std::to_string(capacity) + " < " +
                                  std::to_string(total) + " results (counts_out is filled)");
        if (ids_out) {
            // only the first `total` entries are results
            if (ids.host)
                MASK_CUDA(cudaMemcpyAsync(ids_out, ids.p, sizeof(int64_t) * total,
                                          cudaMemcpyDeviceToHost, s));
            if (dists_out && dd.host)
                MASK_CUDA(cudaMemcpyAsync(dists_out, dd.p, sizeof(float) * total,
                                          cudaMemcpyDeviceToHost, s));
        }
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

// ---------------------------------------------- insertion (§3.3, end)

mask_status mask_insert(mask_index *index, const float *points, int64_t n_new,
                        int32_t *leaf_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(index != nullptr, "index is NULL");
        MASK_REQUIRE(n_new >= 0, "n_new must be >= 0");
        MASK_REQUIRE(current_device() == index->device, "index lives on another device");
        if (index->sparse) fail(MASK_EUNSUPPORTED, "insertion into a CSR index is not built");
        if (n_new == 0) return;
        MASK_REQUIRE(points != nullptr, "points is NULL");
        MASK_REQUIRE(index->n + n_new <= INT32_MAX, "index would exceed 2^31 points");
        cudaStream_t s = (cudaStream_t)stream;
        mask_index &idx = *index;
        const int dp = idx.dp;
        const int64_t n0 = idx.n, n1 = n0 + n_new;
        auto &L0 = idx.lv[0];
        // the greedy descent of each new point (one kept centroid per level)
        In<float> P(points, (size_t)n_new * idx.d, s);
        Scratch<float> Xall((size_t)n1 * dp, s);
        pad_rows(P.p, n_new, idx.d, Xall.get() + (size_t)n0 * dp, dp, s);
        std::vector<Scratch<int32_t>> sel(1);
        sel[0].alloc((size_t)n_new, s);
        greedy_descent(greedy_levels(idx), idx.L, idx.Xs.get(), idx.xids.get(), dp,
                       Xall.get() + (size_t)n0 * dp, n_new, sel[0].get(), nullptr, nullptr, s);
        // the points in id order (old ones back out of the cluster-major
        // layout), then every point's leaf cluster: the old labels and the
        // reached clusters of the new points
        Scratch<int32_t> inv((size_t)n0, s);
        invert_perm_kernel<<<(unsigned)std::min<int64_t>((n0 + 255) / 256, 152 * 16), 256, 0, s>>>(
            idx.xids.get(), n0, inv.get());
        MASK_LAUNCHED("invert_perm");
        gather_rows<int32_t>(idx.Xs.get(), dp, inv.get(), n0, Xall.get(), s);
        DevArray<int32_t> labels;
        labels.alloc((size_t)n1);
        MASK_CUDA(cudaMemcpyAsync(labels.get(), L0.labels.get(), sizeof(int32_t) * n0,
                                  cudaMemcpyDeviceToDevice, s));
        MASK_CUDA(cudaMemcpyAsync(labels.get() + n0, sel[0].get(), sizeof(int32_t) * n_new,
                                  cudaMemcpyDeviceToDevice, s));
        if (leaf_out) {
            Out<int32_t> lo(leaf_out, (size_t)n_new, s);
            MASK_CUDA(cudaMemcpyAsync(lo.p, sel[0].get(), sizeof(int32_t) * n_new,
                                      cudaMemcpyDeviceToDevice, s));
            lo.finish(s);
        }
        // the new leaf layout: membership lists, points cluster-major, norms;
        // the centroids stay as they are (the paper assigns the point to the
        // reached group)
        L0.labels = std::move(labels);
        idx.xids.alloc((size_t)n1);
        label_sort(L0.labels.get(), n1, L0.k, L0.off.get(), idx.xids.get(), s);
        idx.n = n1;
        idx.Xs.alloc((size_t)n1 * dp);
        gather_rows<int32_t>(Xall.get(), dp, idx.xids.get(), n1, idx.Xs.get(), s);
        idx.xn.alloc((size_t)n1);
        row_sqnorm(idx.Xs.get(), n1, dp, idx.xn.get(), s);
        {
            // the low-precision copies describe the old layout: made again on use
            std::lock_guard<std::mutex> lk(idx.lp_mu);
            for (int i = 0; i < 2; ++i) {
                idx.Xlp[i].release();
                idx.xn_lp[i].release();
            }
            idx.xscale_fp8.release();
        }
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

// ------------------------------------------ distributed merge (§3.4)

mask_status mask_merge_topk(const int64_t *ids, const float *dists, int32_t n_parts, int64_t nq,
                            int32_t k, const int64_t *id_offset, int64_t *ids_out,
                            float *dists_out, mask_stream stream) {
    return guard([&] {
        MASK_REQUIRE(n_parts >= 1 && k >= 1 && nq >= 0, "need n_parts >= 1, k >= 1, nq >= 0");
        if ((size_t)merge_topk_smem(n_parts, k) > 200 * 1024)
            fail(MASK_EUNSUPPORTED, "n_parts * k too large for one block (at most 16384)");
        if (nq == 0) return;
        MASK_REQUIRE(ids && dists && ids_out && dists_out, "NULL array");
        cudaStream_t s = (cudaStream_t)stream;
        const size_t total = (size_t)n_parts * nq * k;
        In<int64_t> I(ids, total, s);
        In<float> D(dists, total, s);
        In<int64_t> off(id_offset, id_offset ? (size_t)n_parts : 0, s);
        Out<int64_t> io(ids_out, (size_t)nq * k, s);
        Out<float> dout(dists_out, (size_t)nq * k, s);
        merge_topk(I.p, D.p, n_parts, nq, k, id_offset ? off.p : nullptr, io.p, dout.p, s);
        io.finish(s);
        dout.finish(s);
        MASK_CUDA(cudaStreamSynchronize(s));
    });
}

}  // extern "C"
