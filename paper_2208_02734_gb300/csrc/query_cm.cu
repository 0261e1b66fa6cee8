// query_cm.cu -- cluster-major leaf scan: the last step of the k-NN descent
// (§3.3, Algorithm 2: rank the points of the reached leaf clusters, keep the
// k nearest) for large query batches.
//
// With many queries and many probes per query, the same leaf cluster is kept
// by many queries.  Scanning query by query reads the cluster once per query;
// here the (query, kept cluster) pairs are grouped by cluster, each cluster's
// rows are read once per group of up to 16 of its queries, and all distances
// of the group are computed from shared memory.  Each pair leaves its K best
// keys; a merge pass then keeps every query's K best over its kept clusters.
//
// Every key that can enter a result is computed with the arithmetic of
// query.cu (one thread per (row, query) pair, sum_t (r_t - q_t)^2 in
// increasing t with FMAs), so a query's result is the same whichever kernel
// served it and whatever else is in the batch.  The scan first ranks rows by
// the cheaper expanded form ||x||^2 + ||q||^2 - 2 x.q (one FMA per dimension)
// and evaluates a row exactly only where that value, less its rounding bound,
// can reach the smaller of the pair's current K-th distance and T_q -- the K-th
// exact distance within the query's nearest kept cluster (a seed pass), which
// bounds the query's final K-th from above.  Rows the test drops cannot be
// among the query's K nearest, so the result equals the full exact scan's.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace mask {

// Bytes the cluster-major scan streams (rows x (row + id), per work item).
__device__ unsigned long long g_cm_bytes;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int CM_THREADS = 256;
constexpr int CM_QB = 16;   // queries per work item
constexpr int CM_R = 128;   // cluster rows per shared-memory chunk

__device__ __forceinline__ unsigned long long umin64(unsigned long long a,
                                                     unsigned long long b) {
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v = umin64(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// out[q] = sel[q * P] (each query's nearest kept cluster, or -1)
__global__ void first_col_kernel(const int32_t *__restrict__ sel, int64_t nq, int P,
                                 int32_t *__restrict__ out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = sel[q * P];
}

// labels for grouping: the kept cluster of each pair, or k0 for "none"
__global__ void pair_labels_kernel(const int32_t *__restrict__ sel, int64_t npairs, int k0,
                                   int32_t *__restrict__ lab) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npairs;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = sel[e];
        lab[e] = (c >= 0 && c < k0) ? c : k0;
    }
}

// item_off[c] = sum over clusters < c of ceil(pairs_c / CM_QB); item_off[k0]
// is the number of work items (one block of 1024 threads).
__global__ void __launch_bounds__(1024) item_scan_kernel(const int64_t *__restrict__ poff, int k0,
                                                         int64_t *__restrict__ item_off) {
    __shared__ long long part[1024];
    const int tid = threadIdx.x;
    const int per = (k0 + 1023) / 1024;
    const int b = tid * per, e = min(k0, b + per);
    long long s = 0;
    for (int c = b; c < e; ++c) s += (poff[c + 1] - poff[c] + CM_QB - 1) / CM_QB;
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    long long run = part[tid] - s;
    for (int c = b; c < e; ++c) {
        item_off[c] = run;
        run += (poff[c + 1] - poff[c] + CM_QB - 1) / CM_QB;
    }
    if (tid == 1023) item_off[k0] = part[1023];
}

// One work item = (cluster c, up to CM_QB of its pairs).  xn: row norms;
// qn: query norms; seed_d [nq x K]: each query's K nearest distances within
// its nearest kept cluster (the K-th is T_q); mcoef: rounding bound of
// |expanded form - exact key| per unit of ||x||^2 + ||q||^2.
__global__ __launch_bounds__(CM_THREADS) void cm_scan_kernel(
    const float4 *__restrict__ Xs, const float *__restrict__ xn, int dp4,
    const int32_t *__restrict__ xids, const int64_t *__restrict__ leaf_off,
    const float4 *__restrict__ Qp, const float *__restrict__ qn,
    const float *__restrict__ seed_d, float mcoef, int P, const int64_t *__restrict__ poff,
    const int32_t *__restrict__ pairs, const int64_t *__restrict__ item_off, int k0, int K,
    unsigned long long *__restrict__ pair_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int dp = dp4 * 4;
    float *xs = reinterpret_cast<float *>(smem);                 // [dp][CM_R] rows, transposed
    float *qs = xs + (size_t)dp * CM_R;                          // [dp][CM_QB] queries, transposed
    float *D = qs + (size_t)dp * CM_QB;                          // [CM_QB][CM_R] expanded-form distances
    int32_t *ids = reinterpret_cast<int32_t *>(D + CM_QB * CM_R);// [CM_R] row ids
    unsigned long long *top = reinterpret_cast<unsigned long long *>(ids + CM_R);  // [CM_QB][K]
    __shared__ int s_c;
    __shared__ int64_t s_pb, s_pe;
    __shared__ __align__(16) float s_xn[CM_R];  // read as float4
    __shared__ float s_qn[CM_QB], s_tq[CM_QB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_items = item_off[k0];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        if (tid == 0) {
            // the cluster holding this item: last c with item_off[c] <= item
            int lo = 0, hi = k0 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (item_off[mid] <= item) lo = mid; else hi = mid - 1;
            }
            s_c = lo;
            s_pb = poff[lo] + (item - item_off[lo]) * CM_QB;
            s_pe = min(poff[lo + 1], s_pb + CM_QB);
        }
        __syncthreads();
        const int c = s_c;
        const int64_t pb = s_pb;
        const int nqb = (int)(s_pe - pb);
        // queries of the item, transposed; missing ones are zero
        for (int i = tid; i < CM_QB * dp4; i += CM_THREADS) {
            const int qb = i % CM_QB, c4 = i / CM_QB;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (qb < nqb) v = Qp[(int64_t)(pairs[pb + qb] / P) * dp4 + c4];
            qs[(c4 * 4 + 0) * CM_QB + qb] = v.x;
            qs[(c4 * 4 + 1) * CM_QB + qb] = v.y;
            qs[(c4 * 4 + 2) * CM_QB + qb] = v.z;
            qs[(c4 * 4 + 3) * CM_QB + qb] = v.w;
        }
        for (int i = tid; i < CM_QB * K; i += CM_THREADS) top[i] = kNoKey;
        if (tid < CM_QB) {
            float qv = 0.f, tv = -1.f;  // missing queries: nothing passes the test
            if (tid < nqb) {
                const int64_t qq = pairs[pb + tid] / P;
                qv = qn[qq];
                tv = seed_d[qq * K + K - 1];  // +inf when the seed cluster has < K rows
            }
            s_qn[tid] = qv;
            s_tq[tid] = tv;
        }
        const int64_t rb = leaf_off[c], re = leaf_off[c + 1];
        if (tid == 0)
            atomicAdd(&g_cm_bytes, (unsigned long long)(re - rb) * (dp4 * 16ull + 4ull));
        for (int64_t r0 = rb; r0 < re; r0 += CM_R) {
            const int nr = (int)((re - r0) < (int64_t)CM_R ? (re - r0) : (int64_t)CM_R);
            __syncthreads();
            for (int i = tid; i < CM_R * dp4; i += CM_THREADS) {
                const int rr = i % CM_R, c4 = i / CM_R;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (rr < nr) v = Xs[(r0 + rr) * dp4 + c4];
                xs[(c4 * 4 + 0) * CM_R + rr] = v.x;
                xs[(c4 * 4 + 1) * CM_R + rr] = v.y;
                xs[(c4 * 4 + 2) * CM_R + rr] = v.z;
                xs[(c4 * 4 + 3) * CM_R + rr] = v.w;
            }
            for (int i = tid; i < CM_R; i += CM_THREADS) {
                ids[i] = i < nr ? xids[r0 + i] : -1;
                s_xn[i] = i < nr ? xn[r0 + i] : 0.f;
            }
            __syncthreads();
            // expanded-form distances: warp w -> queries 2w, 2w+1; lane -> rows 4*lane .. +3
            {
                float acc[2][4];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
                const int q0 = warp * 2;
#pragma unroll 8
                for (int t = 0; t < dp; ++t) {
                    const float4 xv = *reinterpret_cast<const float4 *>(&xs[t * CM_R + lane * 4]);
                    const float qa = qs[t * CM_QB + q0], qb2 = qs[t * CM_QB + q0 + 1];
                    acc[0][0] = fmaf(xv.x, qa, acc[0][0]);
                    acc[0][1] = fmaf(xv.y, qa, acc[0][1]);
                    acc[0][2] = fmaf(xv.z, qa, acc[0][2]);
                    acc[0][3] = fmaf(xv.w, qa, acc[0][3]);
                    acc[1][0] = fmaf(xv.x, qb2, acc[1][0]);
                    acc[1][1] = fmaf(xv.y, qb2, acc[1][1]);
                    acc[1][2] = fmaf(xv.z, qb2, acc[1][2]);
                    acc[1][3] = fmaf(xv.w, qb2, acc[1][3]);
                }
                const float4 xr = *reinterpret_cast<const float4 *>(&s_xn[lane * 4]);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float qv = s_qn[q0 + i];
                    *reinterpret_cast<float4 *>(&D[(q0 + i) * CM_R + lane * 4]) =
                        make_float4(fmaf(-2.f, acc[i][0], xr.x + qv), fmaf(-2.f, acc[i][1], xr.y + qv),
                                    fmaf(-2.f, acc[i][2], xr.z + qv), fmaf(-2.f, acc[i][3], xr.w + qv));
                }
            }
            __syncthreads();
            // merge the chunk into each query's K best: warp w owns queries 2w, 2w+1
            for (int qi = 0; qi < 2; ++qi) {
                const int qb = warp * 2 + qi;
                if (qb >= nqb) break;
                unsigned long long *tq = top + qb * K;
                const unsigned long long th = tq[K - 1];
                // distance bound a row must be able to reach (key of the list's K-th, or T_q)
                const float lim = fminf(s_tq[qb], th == kNoKey ? __int_as_float(0x7f800000)
                                                               : __uint_as_float((unsigned)(th >> 32)));
                const float qv = s_qn[qb];
                unsigned long long cand[CM_R / 32];
                bool any = false;
#pragma unroll
                for (int i = 0; i < CM_R / 32; ++i) {
                    const int rr = lane + 32 * i;
                    cand[i] = kNoKey;
                    if (rr < nr && D[qb * CM_R + rr] <= lim + mcoef * (s_xn[rr] + qv)) {
                        // exact key, the arithmetic of the per-query scan
                        float e2 = 0.f;
#pragma unroll 4
                        for (int t = 0; t < dp; ++t) {
                            const float e = xs[t * CM_R + rr] - qs[t * CM_QB + qb];
                            e2 = fmaf(e, e, e2);
                        }
                        const unsigned long long key =
                            ((unsigned long long)__float_as_uint(e2) << 32) | (unsigned)ids[rr];
                        if (key < th) { cand[i] = key; any = true; }
                    }
                }
                if (!__any_sync(kFull, any)) continue;
                // K rounds of warp-wide minimum over (current list, candidates)
                unsigned long long old = lane < K ? tq[lane] : kNoKey;
                unsigned long long out = kNoKey;
                for (int r = 0; r < K; ++r) {
                    unsigned long long mine = old;
#pragma unroll
                    for (int i = 0; i < CM_R / 32; ++i) mine = umin64(mine, cand[i]);
                    const unsigned long long w = warp_min64(mine);
                    if (lane == r) out = w;
                    if (w == kNoKey) break;
                    // the unique owner of w drops it (keys are distinct: ids differ)
                    if (old == w) old = kNoKey;
#pragma unroll
                    for (int i = 0; i < CM_R / 32; ++i)
                        if (cand[i] == w) cand[i] = kNoKey;
                }
                __syncwarp();
                if (lane < K) tq[lane] = out;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = tid; i < nqb * K; i += CM_THREADS) {
            const int qb = i / K, j = i % K;
            pair_out[(int64_t)pairs[pb + qb] * K + j] = top[qb * K + j];
        }
        __syncthreads();
    }
}

// Per query: the K best keys over its P kept clusters (P*K keys), one warp each.
__global__ __launch_bounds__(256) void cm_merge_kernel(const unsigned long long *__restrict__ pair_out,
                                                       int64_t nq, int P, int K,
                                                       int64_t *__restrict__ ids,
                                                       float *__restrict__ dists) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (q >= nq) return;
    const unsigned long long *src = pair_out + q * (int64_t)P * K;
    const int total = P * K;
    unsigned long long last = 0;  // keys already emitted are <= last
    bool first = true;
    for (int r = 0; r < K; ++r) {
        unsigned long long mine = kNoKey;
        for (int i = lane; i < total; i += 32) {
            const unsigned long long v = src[i];
            if ((first || v > last) && v < mine) mine = v;
        }
        const unsigned long long w = warp_min64(mine);
        if (lane == 0) {
            const bool ok = w != kNoKey;
            ids[q * K + r] = ok ? (int64_t)(int32_t)(w & 0xffffffffu) : -1;
            if (dists) dists[q * K + r] = ok ? __uint_as_float((unsigned)(w >> 32)) : __int_as_float(0x7f800000);
        }
        if (w == kNoKey) {
            for (int rr = r + 1 + lane; rr < K; rr += 32) {
                ids[q * K + rr] = -1;
                if (dists) dists[q * K + rr] = __int_as_float(0x7f800000);
            }
            break;
        }
        last = w;
        first = false;
    }
}

int grid_cap(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

bool cm_leaf_supported(int dp, int K) { return dp <= 128 && K >= 1 && K <= 32; }

void cm_group_pairs(const int32_t *sel, int64_t nq, int P, int k0, Scratch<int32_t> &pairs,
                    Scratch<int64_t> &poff, Scratch<int64_t> &item_off, cudaStream_t s) {
    const int64_t npairs = nq * P;
    ProfRegion pr("leaf_group", s, 0.0);
    Scratch<int32_t> lab(npairs, s);
    pairs.alloc(npairs, s);
    poff.alloc((size_t)k0 + 2, s);
    item_off.alloc((size_t)k0 + 1, s);
    pair_labels_kernel<<<grid_cap(npairs, 256), 256, 0, s>>>(sel, npairs, k0, lab.get());
    MASK_LAUNCHED("pair_labels");
    label_sort(lab.get(), npairs, k0 + 1, poff.get(), pairs.get(), s);
    item_scan_kernel<<<1, 1024, 0, s>>>(poff.get(), k0, item_off.get());
    MASK_LAUNCHED("item_scan");
}

void cm_merge(const unsigned long long *pair_out, int64_t nq, int P, int K, int64_t *ids,
              float *dists, cudaStream_t s) {
    if (nq == 0) return;
    ProfRegion pr("leaf_merge", s, 0.0);
    cm_merge_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(pair_out, nq, P, K, ids, dists);
    MASK_LAUNCHED("cm_merge");
}

void leaf_seed(const float *Xs, const int32_t *xids, const int64_t *leaf_off, int dp,
               const float *Qp, int64_t nq, const int32_t *sel, int P, int K, float *seed_d,
               cudaStream_t s) {
    if (nq == 0) return;
    Scratch<int64_t> seed_i((size_t)nq * K, s);
    Scratch<int32_t> sel0(nq, s);
    first_col_kernel<<<grid_cap(nq, 256), 256, 0, s>>>(sel, nq, P, sel0.get());
    MASK_LAUNCHED("first_col");
    ScanArgs a;
    a.R = Xs;
    a.rid = xids;
    a.off = leaf_off;
    a.sel = sel0.get();
    a.P = 1;
    a.Q = Qp;
    a.nq = nq;
    a.dp = dp;
    a.K = K;
    a.out_ids64 = seed_i.get();
    a.out_d = seed_d;
    scan_topk(a, s);
}

void cm_leaf_scan(const float *Xs, const float *xn, int dp, const int32_t *xids,
                  const int64_t *leaf_off, int k0, const float *Qp, int64_t nq,
                  const int32_t *sel, int P, int K, int64_t *ids, float *dists, cudaStream_t s) {
    if (nq == 0) return;
    const int64_t npairs = nq * P;
    Scratch<float> qn(nq, s), seed_d((size_t)nq * K, s);
    row_sqnorm(Qp, nq, dp, qn.get(), s);
    leaf_seed(Xs, xids, leaf_off, dp, Qp, nq, sel, P, K, seed_d.get(), s);
    // |expanded form - exact key| <= (4 dp + 8) 2^-24 (||x||^2 + ||q||^2):
    // FP32 norms (dp terms each), the dot product (dp FMAs of products bounded
    // by (||x||^2 + ||q||^2) / 2, times 2), three roundings of the combination,
    // and the exact key's own dp FMAs over a distance <= 2 (||x||^2 + ||q||^2);
    // widened by 1/8
    const float mcoef = (float)((4.0 * dp + 8.0) * 0x1.0p-24 * 1.125);
    Scratch<int32_t> pairs;
    Scratch<int64_t> poff, item_off;
    Scratch<unsigned long long> pair_out((size_t)npairs * K, s);
    // pairs of an absent parent (sel = -1, fewer children than probes) are in
    // no work item: their lists stay empty
    MASK_CUDA(cudaMemsetAsync(pair_out.get(), 0xFF, sizeof(unsigned long long) * npairs * K, s));
    cm_group_pairs(sel, nq, P, k0, pairs, poff, item_off, s);
    {
        ProfRegion pr("scan_leaf_cm", s, 0.0);
        const size_t smem = ((size_t)dp * CM_R + (size_t)dp * CM_QB + CM_QB * CM_R) * 4 +
                            CM_R * 4 + (size_t)CM_QB * K * 8 + 16;
        MASK_CUDA(cudaFuncSetAttribute(cm_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        cm_scan_kernel<<<152 * 4, CM_THREADS, smem, s>>>(
            reinterpret_cast<const float4 *>(Xs), xn, dp / 4, xids, leaf_off,
            reinterpret_cast<const float4 *>(Qp), qn.get(), seed_d.get(), mcoef, P, poff.get(),
            pairs.get(), item_off.get(), k0, K, pair_out.get());
        MASK_LAUNCHED("cm_scan");
    }
    cm_merge(pair_out.get(), nq, P, K, ids, dists, s);
}

double cm_bytes() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_cm_bytes, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return (double)v;
}

void cm_bytes_reset() {
    const unsigned long long z = 0;
    if (cudaMemcpyToSymbol(g_cm_bytes, &z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}

}  // namespace mask
