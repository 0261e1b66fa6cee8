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
// (Rows of 32 or 64 floats go to the tensor-core scan of query_cm_tc.cu,
// which shares this file's pair grouping, work items and seed pass.)
//
// Every key that can enter a result is computed with the arithmetic of
// query.cu (one thread per (row, query) pair, sum_t (r_t - q_t)^2 in
// increasing t with FMAs), so a query's result is the same whichever kernel
// served it and whatever else is in the batch.  The scan first ranks rows by
// the cheaper expanded form ||x||^2 + ||q||^2 - 2 x.q (the dot products on the
// tensor cores, 3xTF32) and evaluates a row exactly only where that value,
// less its rounding bound, can reach the smaller of the pair's current K-th
// distance and T_q -- the K-th exact distance within the query's nearest kept
// cluster, extended over the next kept clusters while those hold fewer than
// K rows (a seed pass), which bounds the query's final K-th from above.  Rows
// the test drops cannot be among the query's K nearest, so the result equals
// the full exact scan's.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace mask {

// Bytes the cluster-major scan streams (rows x (row + id), per work item).
__device__ unsigned long long g_cm_bytes;

// Device address of a byte counter while profiling is on; null otherwise, so
// the kernels skip the count (one uniform test, no atomic) in normal runs.
unsigned long long *cm_bytes_counter() {
    if (!profiling_enabled()) return nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cm_bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned long long *>(p);
}

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int CM_THREADS = 256;
constexpr int CM_QB = kCmItemQueries;   // queries per work item
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

// The seed of the leaf scans, one warp per query: the K smallest exact
// distances among the rows of the query's nearest kept cluster sel[q * P]
// and, while those hold fewer than K rows, the next kept clusters of the
// list (ascending, +inf past the rows seen).  Rows one per lane with the
// arithmetic of the per-query leaf scan (sum over t of (x_t - q_t)^2, FMAs, t
// ascending); each lane keeps its 32 smallest in registers (an insertion
// network), and K rounds of warp minimum take the K smallest of all lanes.
constexpr int kSeedK = 32;
__global__ __launch_bounds__(256) void leaf_seed_warp_kernel(
    const float4 *__restrict__ Xs, int dp4, const int64_t *__restrict__ leaf_off,
    const float4 *__restrict__ Q, int64_t nq, const int32_t *__restrict__ sel, int P, int K,
    float *__restrict__ seed_d) {
    __shared__ __align__(16) float4 qs[8][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * 8 + w;
    if (q >= nq) return;   // whole warps leave together
    for (int c = lane; c < dp4; c += 32) qs[w][c] = Q[q * dp4 + c];
    __syncwarp();
    const float inf = __int_as_float(0x7f800000);
    float t[kSeedK];
#pragma unroll
    for (int j = 0; j < kSeedK; ++j) t[j] = inf;
    int64_t seen = 0;   // warp-uniform
    for (int p = 0; p < P && seen < K; ++p) {
        const int32_t c0 = sel[q * P + p];
        if (c0 < 0) continue;
        const int64_t b = leaf_off[c0], e = leaf_off[c0 + 1];
        seen += e - b;
        for (int64_t row = b + lane; row < e; row += 32) {
            const float4 *r = Xs + row * dp4;
            float acc = 0.f;
#pragma unroll 4
            for (int c = 0; c < dp4; ++c) {
                const float4 v = r[c], x = qs[w][c];
                float d = v.x - x.x;
                acc = fmaf(d, d, acc);
                d = v.y - x.y;
                acc = fmaf(d, d, acc);
                d = v.z - x.z;
                acc = fmaf(d, d, acc);
                d = v.w - x.w;
                acc = fmaf(d, d, acc);
            }
#pragma unroll
            for (int j = kSeedK - 1; j > 0; --j)
                t[j] = t[j - 1] > acc ? t[j - 1] : (t[j] > acc ? acc : t[j]);
            t[0] = fminf(t[0], acc);
        }
    }
    for (int rd = 0; rd < K; ++rd) {
        float m = t[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(kFull, m, o));
        // one lane holding the minimum at its head pops it
        const unsigned bal = __ballot_sync(kFull, t[0] == m);
        if (lane == __ffs(bal) - 1) {
#pragma unroll
            for (int j = 0; j < kSeedK - 1; ++j) t[j] = t[j + 1];
            t[kSeedK - 1] = inf;
        }
        if (lane == 0) seed_d[q * K + rd] = m;
    }
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

// item_off[c] = sum over clusters < c of ceil(pairs_c / qpi); item_off[k0]
// is the number of work items (one block of 1024 threads).
__global__ void __launch_bounds__(1024) item_scan_kernel(const int64_t *__restrict__ poff, int k0,
                                                         int qpi, int64_t *__restrict__ item_off) {
    __shared__ long long part[1024];
    const int tid = threadIdx.x;
    const int per = (k0 + 1023) / 1024;
    const int b = tid * per, e = min(k0, b + per);
    long long s = 0;
    for (int c = b; c < e; ++c) s += (poff[c + 1] - poff[c] + qpi - 1) / qpi;
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
        run += (poff[c + 1] - poff[c] + qpi - 1) / qpi;
    }
    if (tid == 1023) item_off[k0] = part[1023];
}

// Per work item i (cluster c, up to qpi <= qs of its pairs):
//   meta[i] = {first row lo, first row hi, rows of c, pairs in the item}
//   pid[i * qs + q] = the item's q-th pair (-1 past the last),
//   qid[i * qs + q] = that pair's query.
__global__ void item_meta_kernel(const int64_t *__restrict__ item_off, const int64_t *__restrict__ poff,
                                 const int64_t *__restrict__ leaf_off,
                                 const int32_t *__restrict__ pairs, int P, int k0, int qpi, int qs,
                                 int4 *__restrict__ meta, int32_t *__restrict__ pid,
                                 int32_t *__restrict__ qid) {
    // one warp per cluster; lanes over the cluster's (item, slot) entries
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < k0; c += gridDim.x * wpb) {
        const int64_t rb = leaf_off[c], rows = leaf_off[c + 1] - rb;
        const int64_t i0 = item_off[c], ni = item_off[c + 1] - i0;
        const int64_t p0 = poff[c], np = poff[c + 1] - p0;
        for (int64_t e = lane; e < ni * qs; e += 32) {
            const int64_t i = i0 + e / qs;
            const int q = (int)(e % qs);
            const int64_t pe = (e / qs) * qpi + q;  // pair offset within the cluster
            const int32_t pp = (q < qpi && pe < np) ? pairs[p0 + pe] : -1;
            pid[i * qs + q] = pp;
            qid[i * qs + q] = pp >= 0 ? pp / P : 0;
            if (q == 0) {
                const int nqb = (int)min((int64_t)qpi, np - pe);
                meta[i] = make_int4((int)(rb & 0xffffffff), (int)(rb >> 32), (int)rows, nqb);
            }
        }
    }
}

// hi = x rounded to TF32, lo = x - hi (exact in FP32; the MMA reads its TF32 part)
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    hi = h;
    lo = __float_as_uint(x - __uint_as_float(h));
}

// D += A (16 x 8, row-major) * B (8 x 8, column-major), TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                                uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Floats per staged row: dp + 4 or dp + 8, so the row stride is an odd number
// of float4s and the 8 lanes of each 128-bit shared-memory phase that read 8
// consecutive rows hit 8 different bank groups (and the MMA fragment loads,
// 8 rows x 4 consecutive columns, hit 32 different banks).  The padding
// columns hold zeros: the MMA's last k-step may read them.
__host__ __device__ inline int cm_stride(int dp4) { return 4 * (dp4 + ((dp4 & 1) ? 2 : 1)); }

// One work item = (cluster c, up to CM_QB of its pairs).  xn: row norms;
// qn: query norms; seed_d [nq x K]: each query's K nearest distances within
// its nearest kept cluster (the K-th is T_q); mcoef: rounding bound of
// |expanded form - exact key| per unit of ||x||^2 + ||q||^2.
//
// A block walks its items' chunks (up to CM_R rows of the item's cluster) in
// order; the rows and norms of the next chunk (and the queries of the next
// item) are copied asynchronously into the other half of double-buffered
// shared memory while the current chunk is ranked, and the next item's
// metadata is read one item ahead.  Rows are staged row-major (stride
// cm_stride floats).  The expanded-form dot products run on the tensor cores
// (mma.sync, 3xTF32: x.q ~ x_hi.q_hi + x_hi.q_lo + x_lo.q_hi); mcoef covers
// their error.  An item of an empty cluster is one chunk of no rows.
__global__ __launch_bounds__(CM_THREADS, 2) void cm_scan_kernel(
    const float4 *__restrict__ Xs, const float *__restrict__ xn, int dp4,
    const int32_t *__restrict__ xids, const float4 *__restrict__ Qp,
    const float *__restrict__ qn, const float *__restrict__ seed_d, float mcoef,
    const int4 *__restrict__ meta, const int32_t *__restrict__ pid,
    const int32_t *__restrict__ qid, const int64_t *__restrict__ item_off, int k0, int K,
    unsigned long long *__restrict__ pair_out, unsigned long long *__restrict__ bytes_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int XS = cm_stride(dp4), XS4 = XS / 4;
    float *xs = reinterpret_cast<float *>(smem);                 // [2][CM_R][XS] rows
    float *qs = xs + 2 * CM_R * XS;                              // [2][CM_QB][XS] queries
    float *xnb = qs + 2 * CM_QB * XS;                            // [2][CM_R] row norms
    unsigned long long *top = reinterpret_cast<unsigned long long *>(xnb + 2 * CM_R);  // [CM_QB][K]
    unsigned long long *cbuf = top + CM_QB * K;                  // [CM_QB][CM_R] chunk candidates
    __shared__ float s_qn[2][CM_QB], s_tq[2][CM_QB];
    __shared__ int32_t s_pid[2][CM_QB];
    __shared__ int s_ncand[CM_QB];                  // candidates of the chunk, per query
    __shared__ unsigned long long s_th[CM_QB];      // each list's K-th key (kNoKey: not full)
    // per warp: the (query, row) pairs of its tile that pass the filter,
    // query << 8 | row (a warp's tile holds 16 rows x 16 queries)
    __shared__ unsigned short s_pass[CM_THREADS / 32][256];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_items = item_off[k0];
    const int64_t G = gridDim.x;
    int64_t item = blockIdx.x;
    if (item >= n_items) return;

    // thread -> (row offset, float4 column) of the staging copies; a copier
    // stages queries rfirst and rfirst + rstep (rstep >= 8 since dp4 <= 32)
    const int rstep = CM_THREADS / dp4, rfirst = tid / dp4, c4 = tid - rfirst * dp4;
    const bool copier = rfirst < rstep;
    const int q0c = rfirst, q1c = rfirst + rstep;
    const int qt = tid < CM_QB ? tid : 0;

    // an item's metadata and the query ids this thread stages
    struct Item {
        int64_t rb;
        int rows, nqb, qa, qb, qn;
    };
    auto load_item = [&](int64_t it) {
        Item r;
        const int4 m = meta[it];
        r.rb = (int64_t)(uint32_t)m.x | ((int64_t)m.y << 32);
        r.rows = m.z;
        r.nqb = m.w;
        r.qa = (copier && q0c < CM_QB) ? qid[it * CM_QB + q0c] : 0;
        r.qb = (copier && q1c < CM_QB) ? qid[it * CM_QB + q1c] : 0;
        r.qn = qid[it * CM_QB + qt];
        return r;
    };
    // stage rows [r0, r0 + nr) of the current cluster into row buffer b and,
    // for an item's first chunk, its queries into query buffer qb
    auto prefetch = [&](const Item &im, int64_t it, int64_t r0, int nr, bool first, int b, int qb) {
        float *xsb = xs + b * CM_R * XS;
        if (copier)
            for (int rr = rfirst; rr < CM_R; rr += rstep) {
                const bool v = rr < nr;
                cp_async16(xsb + rr * XS + c4 * 4,
                           v ? (const void *)(Xs + (r0 + rr) * dp4 + c4) : (const void *)Xs, v);
            }
        if (tid < CM_R) {
            const bool v = tid < nr;
            cp_async4(xnb + b * CM_R + tid, v ? xn + r0 + tid : xn, v);
        }
        if (first) {
            float *qsb = qs + qb * CM_QB * XS;
            if (copier && q0c < CM_QB)
                cp_async16(qsb + q0c * XS + c4 * 4, Qp + (int64_t)im.qa * dp4 + c4, q0c < im.nqb);
            if (copier && q1c < CM_QB)
                cp_async16(qsb + q1c * XS + c4 * 4, Qp + (int64_t)im.qb * dp4 + c4, q1c < im.nqb);
            if (tid < CM_QB) {
                const bool v = tid < im.nqb;
                cp_async4(&s_qn[qb][tid], qn + im.qn, v);
                cp_async4(&s_tq[qb][tid], seed_d + (int64_t)im.qn * K + K - 1, v);  // +inf: < K rows
                cp_async4(&s_pid[qb][tid], pid + it * CM_QB + tid, true);
            }
        }
        cp_commit();
    };

    for (int i = tid; i < CM_QB * K; i += CM_THREADS) top[i] = kNoKey;
    if (tid < CM_QB) {
        s_ncand[tid] = 0;
        s_th[tid] = kNoKey;
    }
    {
        const int padw = XS - 4 * dp4;  // zero padding columns of every staged row and query
        for (int i = tid; i < (2 * CM_R + 2 * CM_QB) * padw; i += CM_THREADS)
            xs[(i / padw) * XS + 4 * dp4 + i % padw] = 0.f;
    }
    Item cur = load_item(item), nit;
    const bool has_next0 = item + G < n_items;
    if (has_next0) nit = load_item(item + G);
    int64_t r0 = cur.rb;
    int nr = min(CM_R, cur.rows);
    int buf = 0, qbuf = 0;
    prefetch(cur, item, r0, nr, true, 0, 0);
    for (;;) {
        cp_wait_all();
        __syncthreads();  // the chunk is staged; every warp is done with the other buffers
        // the next chunk: the rest of this cluster, else the block's next item
        const bool more = r0 + CM_R < cur.rb + cur.rows;
        const bool has_next = more || item + G < n_items;
        const int nbuf = buf ^ 1, nqbuf = more ? qbuf : (qbuf ^ 1);
        if (more) {
            const int64_t r1 = r0 + CM_R;
            prefetch(cur, item, r1, (int)min((int64_t)CM_R, cur.rb + cur.rows - r1), false, nbuf,
                     nqbuf);
        } else if (has_next) {
            prefetch(nit, item + G, nit.rb, min(CM_R, nit.rows), true, nbuf, nqbuf);
        }

        const float *xsb = xs + buf * CM_R * XS;
        const float *qsb = qs + qbuf * CM_QB * XS;
        const float *xnc = xnb + buf * CM_R;
        const int nqb = cur.nqb;
        // expanded-form distances on the tensor cores: warp w -> rows 16w ..
        // 16w+15 (two 8-row tiles) x all 16 queries; k-steps of 8 columns
        {
            const int g = lane >> 2, t = lane & 3;
            // hi.hi and the two cross terms accumulate separately (shorter
            // dependent MMA chains); they are added once at the end
            float acc[2][4], acx[2][4];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[j][e] = acx[j][e] = 0.f;
            const float *qa = qsb + g * XS + t, *qb8 = qa + 8 * XS;
            const float *xb0 = xsb + (16 * warp + g) * XS + t, *xb1 = xb0 + 8 * XS;
            const int ksteps = (dp4 + 1) >> 1;
            for (int ks = 0; ks < ksteps; ++ks) {
                const int k0 = ks * 8;
                uint32_t ah[4], al[4];
                tf32_split(qa[k0], ah[0], al[0]);
                tf32_split(qb8[k0], ah[1], al[1]);
                tf32_split(qa[k0 + 4], ah[2], al[2]);
                tf32_split(qb8[k0 + 4], ah[3], al[3]);
                uint32_t bh0, bl0, bh1, bl1;
                tf32_split(xb0[k0], bh0, bl0);
                tf32_split(xb0[k0 + 4], bh1, bl1);
                mma_tf32_16x8x8(acc[0], ah, bh0, bh1);
                mma_tf32_16x8x8(acx[0], ah, bl0, bl1);
                mma_tf32_16x8x8(acx[0], al, bh0, bh1);
                tf32_split(xb1[k0], bh0, bl0);
                tf32_split(xb1[k0 + 4], bh1, bl1);
                mma_tf32_16x8x8(acc[1], ah, bh0, bh1);
                mma_tf32_16x8x8(acx[1], ah, bl0, bl1);
                mma_tf32_16x8x8(acx[1], al, bh0, bh1);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[j][e] += acx[j][e];
            // accumulator (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1) of each
            // tile.  A (query, row) whose expanded form, less its rounding
            // bound, can reach the smaller of the list's K-th and T_q gets its
            // exact key (the arithmetic of the per-query scan); keys below the
            // list's K-th at the start of the chunk become candidates.
            // The pairs that pass are first collected (ballots give each its
            // slot), then evaluated one per lane, so the exact loop runs once
            // per 32 survivors instead of once per slot any lane needs.
            int npass = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = g + 8 * h;
                const unsigned long long th = q < nqb ? s_th[q] : kNoKey;
                const float qv = q < nqb ? s_qn[qbuf][q] : 0.f;
                const float lim = fminf(q < nqb ? s_tq[qbuf][q] : 0.f,
                                        th == kNoKey ? __int_as_float(0x7f800000)
                                                     : __uint_as_float((unsigned)(th >> 32)));
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int row = 16 * warp + 8 * j + 2 * t + e;
                        bool pass = false;
                        if (q < nqb && row < nr) {
                            const float xv = xnc[row];
                            const float dv = fmaf(-2.f, acc[j][2 * h + e], xv + qv);
                            pass = dv <= lim + mcoef * (xv + qv);
                        }
                        const unsigned bal = __ballot_sync(kFull, pass);
                        if (pass)
                            s_pass[warp][npass + __popc(bal & ((1u << lane) - 1u))] =
                                (unsigned short)((q << 8) | row);
                        npass += __popc(bal);
                    }
            }
            __syncwarp();
            for (int i = lane; i < npass; i += 32) {
                const int pr = s_pass[warp][i];
                const int q = pr >> 8, row = pr & 255;
                const float4 *x4 = reinterpret_cast<const float4 *>(xsb) + row * XS4;
                const float4 *q4 = reinterpret_cast<const float4 *>(qsb) + q * XS4;
                float e2 = 0.f;
                for (int t4 = 0; t4 < dp4; ++t4) {
                    const float4 a4 = x4[t4], b4 = q4[t4];
                    float d = a4.x - b4.x;
                    e2 = fmaf(d, d, e2);
                    d = a4.y - b4.y;
                    e2 = fmaf(d, d, e2);
                    d = a4.z - b4.z;
                    e2 = fmaf(d, d, e2);
                    d = a4.w - b4.w;
                    e2 = fmaf(d, d, e2);
                }
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(e2) << 32) | (unsigned)xids[r0 + row];
                if (key < s_th[q]) cbuf[q * CM_R + atomicAdd(&s_ncand[q], 1)] = key;
            }
        }
        __syncthreads();
        // merge each query's candidates into its K best: warp w owns queries 2w, 2w+1
        for (int qi = 0; qi < 2; ++qi) {
            const int qb = warp * 2 + qi;
            const int total = qb < nqb ? s_ncand[qb] : 0;
            if (total == 0) continue;
            unsigned long long *tq = top + qb * K;
            const unsigned long long *cq = cbuf + qb * CM_R;
            unsigned long long old = lane < K ? tq[lane] : kNoKey;
            if (total <= 8) {
                // few candidates: insert each into the sorted list held one
                // entry per lane (keys are distinct: ids differ)
                for (int i = 0; i < total; ++i) {
                    const unsigned long long key = cq[i];
                    const int pos = __popc(__ballot_sync(kFull, lane < K && old < key));
                    const unsigned long long up = __shfl_up_sync(kFull, old, 1);
                    if (pos < K) old = lane < pos ? old : (lane == pos ? key : up);
                }
            } else {
                // K rounds of warp-wide minimum over (current list, candidates)
                unsigned long long cand[CM_R / 32];
#pragma unroll
                for (int i = 0; i < CM_R / 32; ++i)
                    cand[i] = lane + 32 * i < total ? cq[lane + 32 * i] : kNoKey;
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
                old = out;
            }
            if (lane < K) tq[lane] = old;
            const unsigned long long kth = __shfl_sync(kFull, old, K - 1);
            if (lane == 0) {
                s_th[qb] = kth;
                s_ncand[qb] = 0;
            }
        }
        if (!more) {
            // the item is done: write its pair lists and clear them for the next item
            if (bytes_ctr != nullptr && tid == 0)
                atomicAdd(bytes_ctr, (unsigned long long)cur.rows * (dp4 * 16ull + 4ull));
            __syncthreads();
            for (int i = tid; i < nqb * K; i += CM_THREADS) {
                const int qb = i / K, j = i % K;
                pair_out[(int64_t)s_pid[qbuf][qb] * K + j] = top[i];
                top[i] = kNoKey;
            }
            for (int i = nqb * K + tid; i < CM_QB * K; i += CM_THREADS) top[i] = kNoKey;
            if (tid < CM_QB) s_th[tid] = kNoKey;
        }
        if (!has_next) break;
        if (more) {
            r0 += CM_R;
        } else {
            item += G;
            cur = nit;
            r0 = cur.rb;
            if (item + G < n_items) nit = load_item(item + G);  // read one item ahead
        }
        nr = (int)min((int64_t)CM_R, cur.rb + cur.rows - r0);
        buf = nbuf;
        qbuf = nqbuf;
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
                    Scratch<int64_t> &poff, Scratch<int64_t> &item_off, cudaStream_t s,
                    int qpi) {
    MASK_REQUIRE(qpi >= 1 && qpi <= kCmTcItemQueries, "queries per item out of range");
    const int64_t npairs = nq * P;
    ProfRegion pr("leaf_group", s, 0.0);
    Scratch<int32_t> lab(npairs, s);
    pairs.alloc(npairs, s);
    poff.alloc((size_t)k0 + 2, s);
    item_off.alloc((size_t)k0 + 1, s);
    pair_labels_kernel<<<grid_cap(npairs, 256), 256, 0, s>>>(sel, npairs, k0, lab.get());
    MASK_LAUNCHED("pair_labels");
    label_sort(lab.get(), npairs, k0 + 1, poff.get(), pairs.get(), s);
    item_scan_kernel<<<1, 1024, 0, s>>>(poff.get(), k0, qpi, item_off.get());
    MASK_LAUNCHED("item_scan");
}

void cm_item_meta(const int32_t *pairs, const int64_t *poff, const int64_t *item_off,
                  const int64_t *leaf_off, int64_t npairs, int P, int k0, Scratch<int4> &meta,
                  Scratch<int32_t> &pid, Scratch<int32_t> &qid, cudaStream_t s, int qpi,
                  int qs) {
    MASK_REQUIRE(qpi >= 1 && qpi <= qs && (qs == kCmItemQueries || qs == kCmTcItemQueries),
                 "queries per item out of range");
    // a cluster with m pairs has ceil(m / qpi) <= m / qpi + 1 items, and at most m
    const int64_t max_items = std::max<int64_t>(
        1, std::min(npairs, (npairs + qpi - 1) / qpi + (int64_t)k0));
    meta.alloc(max_items, s);
    pid.alloc((size_t)max_items * qs, s);
    qid.alloc((size_t)max_items * qs, s);
    item_meta_kernel<<<(k0 + 7) / 8, 256, 0, s>>>(item_off, poff, leaf_off, pairs, P, k0, qpi, qs,
                                                  meta.get(), pid.get(), qid.get());
    MASK_LAUNCHED("item_meta");
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
    if (K <= kSeedK && dp <= 128) {
        ProfRegion pr("scan_topk_leaf", s, 0.0);
        leaf_seed_warp_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(
            reinterpret_cast<const float4 *>(Xs), dp / 4, leaf_off,
            reinterpret_cast<const float4 *>(Qp), nq, sel, P, K, seed_d);
        MASK_LAUNCHED("leaf_seed");
        return;
    }
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

void cm_leaf_scan(const float *Xs, int64_t n, const float *xn, int dp, const int32_t *xids,
                  const int64_t *leaf_off, int k0, const float *Qp, int64_t nq,
                  const int32_t *sel, int P, int K, int64_t *ids, float *dists, cudaStream_t s,
                  CmTile tile) {
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
    // the tensor-core dot product (3xTF32) adds: the split (the dropped
    // lo x lo products and the TF32 truncation of the lo parts, 2.5 * 2^-21
    // relative to sum |x_t q_t|) and its FP32 accumulation over 3 ceil(dp/8)
    // MMAs (in two chains, added once) plus 8 in-MMA additions, counted at one
    // ulp (2^-22) each; times 2 for the factor -2 and
    // sum |x_t q_t| <= (||x||^2 + ||q||^2) / 2
    const float mcoef_tc =
        mcoef + (float)((2.5 * 0x1.0p-21 + (3.0 * ((dp + 7) / 8) + 8.0) * 0x1.0p-22) * 1.125);
    Scratch<int32_t> pairs;
    Scratch<int64_t> poff, item_off;
    // queries per work item: the tile's, at most the kernel's widest; the
    // tensor-core scan's items of more than 16 queries use 32-query slots
    const bool tc = !tile.legacy && cm_tc_supported(dp, K);
    const int qmax = tc ? cm_tc_item_queries(K) : kCmItemQueries;
    const int qpi = tile.qpi > 0 ? std::min(tile.qpi, qmax) : qmax;
    const int qs = qpi > kCmItemQueries ? kCmTcItemQueries : kCmItemQueries;
    cm_group_pairs(sel, nq, P, k0, pairs, poff, item_off, s, qpi);
    Scratch<int4> meta;
    Scratch<int32_t> ipid, iqid;
    cm_item_meta(pairs.get(), poff.get(), item_off.get(), leaf_off, npairs, P, k0, meta, ipid, iqid,
                 s, qpi, qs);
    if (tc) {
        // the tensor-core scan (kind::tf32): the rows are read as TF32
        // (|x - x_tf32| <= 2^-10 |x|), the queries split into an exact TF32
        // part and a remainder read as TF32 (2^-20 |q|), which leaves
        // (2^-10 + 2^-20 + 2^-30) of sum |x_t q_t| in the units above;
        // accumulation: 2 ceil(dp/8) MMAs plus 8 in-MMA additions at 2^-22
        const float mcoef_t =
            mcoef + (float)((0x1.0p-10 + 0x1.0p-20 + 0x1.0p-30 + (2.0 * ((dp + 7) / 8) + 8.0) *
                                                                    0x1.0p-22) * 1.125);
        // candidate lists of the filter pass; the exact pass writes ids / dists
        const int cap = cm_tc_cand_cap(nq);
        Scratch<unsigned> ccount(nq, s);
        Scratch<uint32_t> cand((size_t)nq * cap, s);
        MASK_CUDA(cudaMemsetAsync(ccount.get(), 0, sizeof(unsigned) * nq, s));
        cm_tc_scan(Xs, n, xn, dp, xids, leaf_off, k0, Qp, nq, sel, P, qn.get(), seed_d.get(),
                   mcoef_t, meta.get(), iqid.get(), item_off.get(), K, qs, ccount.get(),
                   cand.get(), cap, ids, dists, cm_bytes_counter(), s);
        return;
    }
    {
        // pairs of an absent parent (sel = -1, fewer children than probes) are in
        // no work item: their lists stay empty
        Scratch<unsigned long long> pair_out((size_t)npairs * K, s);
        MASK_CUDA(cudaMemsetAsync(pair_out.get(), 0xFF, sizeof(unsigned long long) * npairs * K, s));
        {
            ProfRegion pr("scan_leaf_cm", s, 0.0);
            const int XS = cm_stride(dp / 4);
            const size_t smem = ((size_t)2 * CM_R * XS + (size_t)2 * CM_QB * XS + 2 * CM_R) * 4 +
                                (size_t)CM_QB * K * 8 + (size_t)CM_QB * CM_R * 8 + 16;
            MASK_CUDA(cudaFuncSetAttribute(cm_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
            int per_sm = 0;
            MASK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cm_scan_kernel,
                                                                    CM_THREADS, smem));
            int dev = 0, sms = 0;
            MASK_CUDA(cudaGetDevice(&dev));
            MASK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            if (tile.bps > 0) per_sm = std::min(per_sm, tile.bps);
            cm_scan_kernel<<<std::max(1, per_sm) * sms, CM_THREADS, smem, s>>>(
                reinterpret_cast<const float4 *>(Xs), xn, dp / 4, xids,
                reinterpret_cast<const float4 *>(Qp), qn.get(), seed_d.get(), mcoef_tc, meta.get(),
                ipid.get(), iqid.get(), item_off.get(), k0, K, pair_out.get(), cm_bytes_counter());
            MASK_LAUNCHED("cm_scan");
        }
        cm_merge(pair_out.get(), nq, P, K, ids, dists, s);
    }
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
