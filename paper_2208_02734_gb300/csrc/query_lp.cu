// query_lp.cu -- low-precision leaf scan with exact FP32 re-rank (the BF16 and
// FP8 e4m3 query modes; not in the paper, which states no precision).
//
// The leaf scan of the k-NN descent (§3.3, Algorithm 2) ranks the points of
// the kept leaf clusters.  In these modes the index also holds the points in
// BF16, or in FP8 e4m3 with a per-row scale s = max|x| / 448, with the squared
// norm of each quantised row.  Queries are grouped by cluster as in the FP32
// cluster-major scan; the distances of a group are
//     ||x~||^2 + ||q~||^2 - 2 x~.q~    (x~, q~ the quantised vectors)
// with x~.q~ from warp-level tensor-core MMAs (FP32 accumulation).  Every
// (query, cluster) pair keeps its max(k, 4) nearest by these distances; every query
// keeps a shortlist of the K' = max(4k, 16) nearest of those, which is then
// re-ranked with exact FP32 distances sum_t (x_t - q_t)^2 of the FP32 rows; the
// k best of the shortlist are returned.  Shortlist keys carry row positions in
// the cluster-major point array, so the re-rank reads those rows directly.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <climits>

#include "common.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int LP_THREADS = 256;
constexpr int LP_QB = kCmItemQueries;   // queries per work item (two n8 MMA tiles)
constexpr int LP_R = 128;   // rows per chunk (eight m16 MMA tiles, one per warp)
constexpr int LP_KMAX = 64; // shortlist length limit

__device__ __forceinline__ unsigned long long umin64(unsigned long long a,
                                                     unsigned long long b) {
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v = umin64(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// ------------------------------------------------------------- quantisers

// BF16 copy of padded rows (dpl >= dp columns, zero beyond dp) and the
// squared norm of every quantised row.
__global__ void quant_bf16_kernel(const float *__restrict__ src, int64_t rows, int dp, int dpl,
                                  __nv_bfloat16 *__restrict__ dst, float *__restrict__ norm2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); r < rows;
         r += warps) {
        float acc = 0.f;
        for (int c = lane; c < dpl; c += 32) {
            const float x = c < dp ? src[r * dp + c] : 0.f;
            const __nv_bfloat16 b = __float2bfloat16_rn(x);
            dst[r * dpl + c] = b;
            const float y = __bfloat162float(b);
            acc = fmaf(y, y, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) norm2[r] = acc;
    }
}

// FP8 e4m3 copy with a per-row scale s = max|x| / 448 (x = s * x~), and the
// squared norm of every dequantised row s^2 ||x~||^2.
__global__ void quant_fp8_kernel(const float *__restrict__ src, int64_t rows, int dp, int dpl,
                                 __nv_fp8_e4m3 *__restrict__ dst, float *__restrict__ scale,
                                 float *__restrict__ norm2) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); r < rows;
         r += warps) {
        float mx = 0.f;
        for (int c = lane; c < dp; c += 32) mx = fmaxf(mx, fabsf(src[r * dp + c]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(kFull, mx, o));
        const float s = mx > 0.f ? mx / 448.f : 1.f;
        float acc = 0.f;
        for (int c = lane; c < dpl; c += 32) {
            const float x = c < dp ? src[r * dp + c] / s : 0.f;
            const __nv_fp8_e4m3 q(x);
            dst[r * dpl + c] = q;
            const float y = float(q);
            acc = fmaf(y, y, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) {
            scale[r] = s;
            norm2[r] = acc * s * s;
        }
    }
}

// ------------------------------------------------------- tensor-core MMA

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_e4m3_16832(float (&d)[4], const uint32_t (&a)[4],
                                               const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One work item = (leaf cluster c, up to LP_QB of its (query, cluster) pairs).
// FP8 = false: BF16 elements (2 bytes), MMA k = 16; true: e4m3 (1 byte), k = 32.
//
// A block walks its items' chunks (up to LP_R rows of the item's cluster) in
// order; the next chunk's rows, norms and scales (and the next item's
// queries) are copied asynchronously into the other half of double-buffered
// shared memory while the current chunk is ranked, and the next item's
// metadata is read one item ahead (cm_item_meta).  Each thread tests the
// quantised distances it holds in MMA accumulators against the seed bound and
// the pair's current list and appends the passing keys to per-query candidate
// lists, which each query's warp merges.  An item of an empty cluster is one
// chunk of no rows.
template <bool FP8>
__global__ __launch_bounds__(LP_THREADS, 2) void lp_scan_kernel(
    const uint8_t *__restrict__ Xl, int dpl, const float *__restrict__ xn2,
    const float *__restrict__ xscale, const uint8_t *__restrict__ Ql,
    const float *__restrict__ qn2, const float *__restrict__ qscale,
    const float *__restrict__ seed_d, int kseed, float eta, float rslack,
    const int4 *__restrict__ meta, const int32_t *__restrict__ pid, const int32_t *__restrict__ qid,
    const int64_t *__restrict__ item_off, int k0, int K, unsigned long long *__restrict__ pair_out) {
    constexpr int ES = FP8 ? 1 : 2;                   // bytes per element
    constexpr int KSTEP = FP8 ? 32 : 16;              // elements per MMA k-step
    extern __shared__ __align__(16) unsigned char smem[];
    const int rowb = dpl * ES + 16;                   // padded row stride in bytes
    unsigned char *rows = smem;                                        // [2][LP_R][rowb]
    unsigned char *qs = rows + 2 * (size_t)LP_R * rowb;                // [2][LP_QB][rowb]
    float *rn = reinterpret_cast<float *>(qs + 2 * (size_t)LP_QB * rowb);  // [2][LP_R] norms
    float *rsc = rn + 2 * LP_R;                                        // [2][LP_R] scales (FP8)
    unsigned long long *top = reinterpret_cast<unsigned long long *>(rsc + 2 * LP_R);  // [LP_QB][K]
    unsigned long long *cbuf = top + LP_QB * K;                        // [LP_QB][LP_R] candidates
    __shared__ float s_qn[2][LP_QB], s_qsc[2][LP_QB], s_sd[2][LP_QB];
    __shared__ int32_t s_pid[2][LP_QB];
    __shared__ int s_ncand[LP_QB];
    __shared__ unsigned long long s_th[LP_QB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const int c16 = dpl * ES / 16;                    // 16-byte chunks per row
    const int64_t n_items = item_off[k0];
    const int64_t G = gridDim.x;
    int64_t item = blockIdx.x;
    if (item >= n_items) return;

    // thread -> (row offset, 16-byte chunk) of the staging copies; a copier
    // stages queries rfirst and rfirst + rstep (rstep >= 8 since c16 <= 32)
    const int rstep = LP_THREADS / c16, rfirst = tid / c16, cc = tid - rfirst * c16;
    const bool copier = rfirst < rstep;
    const int q0c = rfirst, q1c = rfirst + rstep;
    const int qt = tid < LP_QB ? tid : 0;
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
        r.qa = (copier && q0c < LP_QB) ? qid[it * LP_QB + q0c] : 0;
        r.qb = (copier && q1c < LP_QB) ? qid[it * LP_QB + q1c] : 0;
        r.qn = qid[it * LP_QB + qt];
        return r;
    };
    auto prefetch = [&](const Item &im, int64_t it, int64_t r0, int nr, bool first, int b, int qb) {
        unsigned char *rb_ = rows + (size_t)b * LP_R * rowb;
        if (copier)
            for (int rr = rfirst; rr < LP_R; rr += rstep) {
                const bool v = rr < nr;
                cp_async16(rb_ + rr * rowb + cc * 16,
                           v ? (const void *)(Xl + (r0 + rr) * dpl * ES + cc * 16) : (const void *)Xl,
                           v);
            }
        if (tid < LP_R) {
            const bool v = tid < nr;
            cp_async4(rn + b * LP_R + tid, v ? xn2 + r0 + tid : xn2, v);
            if (FP8) cp_async4(rsc + b * LP_R + tid, v ? xscale + r0 + tid : xscale, v);
        }
        if (first) {
            unsigned char *qb_ = qs + (size_t)qb * LP_QB * rowb;
            if (copier && q0c < LP_QB)
                cp_async16(qb_ + q0c * rowb + cc * 16, Ql + (int64_t)im.qa * dpl * ES + cc * 16,
                           q0c < im.nqb);
            if (copier && q1c < LP_QB)
                cp_async16(qb_ + q1c * rowb + cc * 16, Ql + (int64_t)im.qb * dpl * ES + cc * 16,
                           q1c < im.nqb);
            if (tid < LP_QB) {
                const bool v = tid < im.nqb;
                cp_async4(&s_qn[qb][tid], qn2 + im.qn, v);
                if (FP8) cp_async4(&s_qsc[qb][tid], qscale + im.qn, v);
                cp_async4(&s_sd[qb][tid], seed_d + (int64_t)im.qn * kseed + kseed - 1, v);
                cp_async4(&s_pid[qb][tid], pid + it * LP_QB + tid, true);
            }
        }
        cp_commit();
    };

    for (int i = tid; i < LP_QB * K; i += LP_THREADS) top[i] = kNoKey;
    if (tid < LP_QB) {
        s_ncand[tid] = 0;
        s_th[tid] = kNoKey;
        if (!FP8) s_qsc[0][tid] = s_qsc[1][tid] = 1.f;
    }
    if (!FP8)
        for (int i = tid; i < 2 * LP_R; i += LP_THREADS) rsc[i] = 1.f;
    Item cur = load_item(item), nit;
    if (item + G < n_items) nit = load_item(item + G);
    int64_t r0 = cur.rb;
    int nr = min(LP_R, cur.rows);
    int buf = 0, qbuf = 0;
    prefetch(cur, item, r0, nr, true, 0, 0);
    for (;;) {
        cp_wait_all();
        __syncthreads();  // the chunk is staged; every warp is done with the other buffers
        const bool more = r0 + LP_R < cur.rb + cur.rows;
        const bool has_next = more || item + G < n_items;
        const int nbuf = buf ^ 1, nqbuf = more ? qbuf : (qbuf ^ 1);
        if (more) {
            const int64_t r1 = r0 + LP_R;
            prefetch(cur, item, r1, (int)min((int64_t)LP_R, cur.rb + cur.rows - r1), false, nbuf,
                     nqbuf);
        } else if (has_next) {
            prefetch(nit, item + G, nit.rb, min(LP_R, nit.rows), true, nbuf, nqbuf);
        }
        const unsigned char *rws = rows + (size_t)buf * LP_R * rowb;
        const unsigned char *qss = qs + (size_t)qbuf * LP_QB * rowb;
        const float *rnc = rn + buf * LP_R, *rsc_c = rsc + buf * LP_R;
        const int nqb = cur.nqb;
        // warp w: rows 16w .. 16w+15 against the 16 queries (two n8 tiles)
        {
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            const unsigned char *ra = rws + (16 * warp + g) * rowb;
            const unsigned char *rb8 = ra + 8 * rowb;
            for (int kk = 0; kk < dpl / KSTEP; ++kk) {
                const int e0 = kk * KSTEP + tig * (FP8 ? 4 : 2);   // first element, low half
                const int e1 = e0 + KSTEP / 2;                       // high half
                uint32_t a[4];
                a[0] = *reinterpret_cast<const uint32_t *>(ra + e0 * ES);
                a[1] = *reinterpret_cast<const uint32_t *>(rb8 + e0 * ES);
                a[2] = *reinterpret_cast<const uint32_t *>(ra + e1 * ES);
                a[3] = *reinterpret_cast<const uint32_t *>(rb8 + e1 * ES);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const unsigned char *qb = qss + (nt * 8 + g) * rowb;
                    uint32_t b[2];
                    b[0] = *reinterpret_cast<const uint32_t *>(qb + e0 * ES);
                    b[1] = *reinterpret_cast<const uint32_t *>(qb + e1 * ES);
                    if (FP8) mma_e4m3_16832(acc[nt], a, b);
                    else mma_bf16_16816(acc[nt], a, b);
                }
            }
            // accumulator h of tile nt: row 16w + g (+8 for h >= 2), query
            // nt * 8 + 2 tig + (h & 1).  A row whose quantised distance
            // exceeds sqrt(T_q) + eta (|x| + |q|) is farther than T_q exactly
            // and cannot be among the k nearest; rslack covers the rounding
            // of the FP32 expanded form itself.
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int rr = 16 * warp + g + (h >= 2 ? 8 : 0);
                    const int qb = nt * 8 + tig * 2 + (h & 1);
                    if (rr >= nr || qb >= nqb) continue;
                    const float rnv = rnc[rr], qnv = s_qn[qbuf][qb];
                    const float dot = acc[nt][h] * rsc_c[rr] * s_qsc[qbuf][qb];
                    const float dq = fmaxf(rnv + qnv - 2.f * dot, 0.f);
                    const float lim = sqrtf(s_sd[qbuf][qb]) + eta * (sqrtf(rnv) + sqrtf(qnv));
                    const float slack = rslack * (rnv + qnv);
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(dq) << 32) | (unsigned)(r0 + rr);
                    if (key < s_th[qb] && dq <= fmaf(lim, lim, slack))
                        cbuf[qb * LP_R + atomicAdd(&s_ncand[qb], 1)] = key;
                }
        }
        __syncthreads();
        // merge each query's candidates into its list: warp w owns queries 2w, 2w+1
        for (int qi = 0; qi < 2; ++qi) {
            const int qb = warp * 2 + qi;
            const int total = qb < nqb ? s_ncand[qb] : 0;
            if (total == 0) continue;
            unsigned long long *tq = top + qb * K;
            const unsigned long long *cq = cbuf + qb * LP_R;
            unsigned long long old = lane < K ? tq[lane] : kNoKey;
            if (total <= 8) {
                // few candidates: insert each into the sorted list held one
                // entry per lane (keys are distinct: positions differ)
                for (int i = 0; i < total; ++i) {
                    const unsigned long long key = cq[i];
                    const int pos = __popc(__ballot_sync(kFull, lane < K && old < key));
                    const unsigned long long up = __shfl_up_sync(kFull, old, 1);
                    if (pos < K) old = lane < pos ? old : (lane == pos ? key : up);
                }
            } else {
                // K rounds of warp-wide minimum over (current list, candidates)
                unsigned long long cand[LP_R / 32];
#pragma unroll
                for (int i = 0; i < LP_R / 32; ++i)
                    cand[i] = lane + 32 * i < total ? cq[lane + 32 * i] : kNoKey;
                unsigned long long out = kNoKey;
                for (int r = 0; r < K; ++r) {
                    unsigned long long mine = old;
#pragma unroll
                    for (int i = 0; i < LP_R / 32; ++i) mine = umin64(mine, cand[i]);
                    const unsigned long long w = warp_min64(mine);
                    if (lane == r) out = w;
                    if (w == kNoKey) break;
                    if (old == w) old = kNoKey;
#pragma unroll
                    for (int i = 0; i < LP_R / 32; ++i)
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
            __syncthreads();
            for (int i = tid; i < nqb * K; i += LP_THREADS) {
                const int qb = i / K, j = i % K;
                pair_out[(int64_t)s_pid[qbuf][qb] * K + j] = top[i];
                top[i] = kNoKey;
            }
            for (int i = nqb * K + tid; i < LP_QB * K; i += LP_THREADS) top[i] = kNoKey;
            if (tid < LP_QB) s_th[tid] = kNoKey;
        }
        if (!has_next) break;
        if (more) {
            r0 += LP_R;
        } else {
            item += G;
            cur = nit;
            r0 = cur.rb;
            if (item + G < n_items) nit = load_item(item + G);  // read one item ahead
        }
        nr = (int)min((int64_t)LP_R, cur.rb + cur.rows - r0);
        buf = nbuf;
        qbuf = nqbuf;
    }
}

// Per query: the Kp best approximate keys among the P x Kpair keys of its
// (query, cluster) pairs; their row positions form the shortlist (-1 where
// fewer exist).  One warp per query; the keys stay in registers when they fit.
__global__ __launch_bounds__(256) void lp_shortlist_kernel(
    const unsigned long long *__restrict__ pair_out, int64_t nq, int P, int Kpair, int Kp,
    int32_t *__restrict__ shortlist) {
    constexpr int REG = 32;  // keys per lane held in registers
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (q >= nq) return;
    const unsigned long long *src = pair_out + q * (int64_t)P * Kpair;
    const int total = P * Kpair;
    if (total <= 32 * REG) {
        unsigned long long v[REG];
#pragma unroll
        for (int i = 0; i < REG; ++i) v[i] = lane + 32 * i < total ? src[lane + 32 * i] : kNoKey;
        for (int r = 0; r < Kp; ++r) {
            unsigned long long mine = kNoKey;
#pragma unroll
            for (int i = 0; i < REG; ++i) mine = umin64(mine, v[i]);
            const unsigned long long w = warp_min64(mine);
            if (lane == 0) shortlist[q * Kp + r] = w == kNoKey ? -1 : (int32_t)(w & 0xffffffffu);
            if (w == kNoKey) {
                for (int rr = r + 1 + lane; rr < Kp; rr += 32) shortlist[q * Kp + rr] = -1;
                return;
            }
#pragma unroll
            for (int i = 0; i < REG; ++i)
                if (v[i] == w) v[i] = kNoKey;
        }
        return;
    }
    unsigned long long last = 0;
    bool first = true;
    for (int r = 0; r < Kp; ++r) {
        unsigned long long mine = kNoKey;
        for (int i = lane; i < total; i += 32) {
            const unsigned long long v = src[i];
            if ((first || v > last) && v < mine) mine = v;
        }
        const unsigned long long w = warp_min64(mine);
        if (lane == 0) shortlist[q * Kp + r] = w == kNoKey ? -1 : (int32_t)(w & 0xffffffffu);
        if (w == kNoKey) {
            for (int rr = r + 1 + lane; rr < Kp; rr += 32) shortlist[q * Kp + rr] = -1;
            break;
        }
        last = w;
        first = false;
    }
}

// Exact FP32 re-rank of the shortlist: sum_t (x_t - q_t)^2 of the FP32 rows
// (t ascending, FMA per term, as in the FP32 leaf scans); the k smallest
// (distance, original id).  One warp per query.
__global__ __launch_bounds__(256) void lp_rerank_kernel(
    const float4 *__restrict__ Xs, int dp4, const int32_t *__restrict__ xids,
    const float4 *__restrict__ Qp, const int32_t *__restrict__ shortlist, int64_t nq, int Kp,
    int k, int64_t n_rows, int64_t *__restrict__ ids, float *__restrict__ dists) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (q >= nq) return;
    const float4 *qv = Qp + q * dp4;
    unsigned long long key[2] = {kNoKey, kNoKey};  // entries lane and lane + 32
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h;
        if (j >= Kp) continue;
        const int32_t p = shortlist[q * Kp + j];
        if (p < 0 || p >= n_rows) continue;
        const float4 *row = Xs + (int64_t)p * dp4;
        float acc = 0.f;
        for (int c = 0; c < dp4; ++c) {
            const float4 v = row[c], w = qv[c];
            float e = v.x - w.x;
            acc = fmaf(e, e, acc);
            e = v.y - w.y;
            acc = fmaf(e, e, acc);
            e = v.z - w.z;
            acc = fmaf(e, e, acc);
            e = v.w - w.w;
            acc = fmaf(e, e, acc);
        }
        key[h] = ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)xids[p];
    }
    for (int r = 0; r < k; ++r) {
        const unsigned long long w = warp_min64(umin64(key[0], key[1]));
        if (lane == 0) {
            const bool ok = w != kNoKey;
            ids[q * k + r] = ok ? (int64_t)(int32_t)(w & 0xffffffffu) : -1;
            if (dists) dists[q * k + r] = ok ? __uint_as_float((unsigned)(w >> 32)) : __int_as_float(0x7f800000);
        }
        if (key[0] == w) key[0] = kNoKey;
        if (key[1] == w) key[1] = kNoKey;
    }
}

int grid_cap(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

int lp_padded_dim(int dp) { return (dp + 31) / 32 * 32; }

int lp_shortlist(int k) { return std::max(4 * k, 16); }

bool lp_supported(int dp, int k) { return k >= 1 && 4 * k <= LP_KMAX && lp_padded_dim(dp) <= 256; }

void lp_quantize(const float *src, int64_t rows, int dp, bool fp8, void *dst, float *scale,
                 float *norm2, cudaStream_t s) {
    if (rows == 0) return;
    const int dpl = lp_padded_dim(dp);
    const int grid = grid_cap(rows * 32, 256);
    if (fp8)
        quant_fp8_kernel<<<grid, 256, 0, s>>>(src, rows, dp, dpl,
                                              static_cast<__nv_fp8_e4m3 *>(dst), scale, norm2);
    else
        quant_bf16_kernel<<<grid, 256, 0, s>>>(src, rows, dp, dpl,
                                               static_cast<__nv_bfloat16 *>(dst), norm2);
    MASK_LAUNCHED("lp_quantize");
}

void lp_leaf_scan(bool fp8, const void *Xl, const float *xn2, const float *xscale, const float *Xs,
                  int64_t leaf_rows, int dp, const int32_t *xids, const int64_t *leaf_off, int k0, const float *Qp,
                  int64_t nq, const int32_t *sel, int P, int k, int64_t *ids, float *dists,
                  cudaStream_t s) {
    if (nq == 0) return;
    const int dpl = lp_padded_dim(dp);
    const int Kp = lp_shortlist(k);
    // every (query, cluster) pair keeps its max(k, 4) best by approximate
    // distance (a floor, so a near-tie inside one cluster cannot drop the
    // nearest point at k = 1); the shortlist is the Kp best of their union
    const int Kpair = std::min(Kp, std::max(k, 4));
    Scratch<unsigned char> Ql((size_t)nq * dpl * (fp8 ? 1 : 2), s);
    Scratch<float> qn2(nq, s), qsc(fp8 ? nq : 1, s);
    lp_quantize(Qp, nq, dp, fp8, Ql.get(), qsc.get(), qn2.get(), s);
    Scratch<int32_t> pairs;
    Scratch<int64_t> poff, item_off;
    cm_group_pairs(sel, nq, P, k0, pairs, poff, item_off, s);
    // the FP32 seed: each query's k-th exact distance within its nearest kept
    // cluster bounds the distance of its k nearest
    Scratch<float> seed_d((size_t)nq * k, s);
    leaf_seed(Xs, xids, leaf_off, dp, Qp, nq, sel, P, k, seed_d.get(), s);
    // element-wise quantisation error relative to the element: BF16 rounds to
    // 8 significant bits (2^-8; 2x margin), e4m3 to 4 (2^-4, and |x| <=
    // |x~| / (1 - 2^-4): 2^-4 x 1.125; the subnormals of the per-row scaled
    // range add at most 2^-10 x max|x| / 448 per element)
    const float eta = fp8 ? 0x1.2p-4f : 0x1.0p-7f;
    // |FP32 expanded form - exact distance of the quantised rows| per unit of
    // their squared norms (dot over dpl terms x 2, norms, final roundings), x2
    const float rslack = (float)((4.0 * dpl + 16.0) * 0x1.0p-24);
    Scratch<unsigned long long> pair_out((size_t)nq * P * Kpair, s);
    // pairs of an absent parent (sel = -1, fewer children than probes) are in
    // no work item: their lists stay empty
    MASK_CUDA(cudaMemsetAsync(pair_out.get(), 0xFF, sizeof(unsigned long long) * nq * P * Kpair, s));
    Scratch<int32_t> shortlist((size_t)nq * Kp, s);
    Scratch<int4> meta;
    Scratch<int32_t> ipid, iqid;
    cm_item_meta(pairs.get(), poff.get(), item_off.get(), leaf_off, nq * (int64_t)P, P, k0, meta,
                 ipid, iqid, s);
    {
        ProfRegion pr(fp8 ? "scan_leaf_fp8" : "scan_leaf_bf16", s, 0.0);
        MASK_REQUIRE(Kpair <= 32, "per-pair list longer than a warp");
        const int rowb = dpl * (fp8 ? 1 : 2) + 16;
        const size_t smem = 2 * (size_t)(LP_R + LP_QB) * rowb + (size_t)4 * LP_R * 4 +
                            (size_t)LP_QB * Kpair * 8 + (size_t)LP_QB * LP_R * 8 + 16;
        int dev = 0, sms = 0;
        MASK_CUDA(cudaGetDevice(&dev));
        MASK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int per_sm = 0;
        if (fp8) {
            MASK_CUDA(cudaFuncSetAttribute(lp_scan_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            MASK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lp_scan_kernel<true>,
                                                                    LP_THREADS, smem));
            lp_scan_kernel<true><<<std::max(1, per_sm) * sms, LP_THREADS, smem, s>>>(
                static_cast<const uint8_t *>(Xl), dpl, xn2, xscale, Ql.get(), qn2.get(), qsc.get(),
                seed_d.get(), k, eta, rslack, meta.get(), ipid.get(), iqid.get(), item_off.get(), k0,
                Kpair, pair_out.get());
        } else {
            MASK_CUDA(cudaFuncSetAttribute(lp_scan_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            MASK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lp_scan_kernel<false>,
                                                                    LP_THREADS, smem));
            lp_scan_kernel<false><<<std::max(1, per_sm) * sms, LP_THREADS, smem, s>>>(
                static_cast<const uint8_t *>(Xl), dpl, xn2, nullptr, Ql.get(), qn2.get(), nullptr,
                seed_d.get(), k, eta, rslack, meta.get(), ipid.get(), iqid.get(), item_off.get(), k0,
                Kpair, pair_out.get());
        }
        MASK_LAUNCHED("lp_scan");
    }
    {
        ProfRegion pr("leaf_rerank", s, 0.0);
        const unsigned blocks = (unsigned)((nq + 7) / 8);
        lp_shortlist_kernel<<<blocks, 256, 0, s>>>(pair_out.get(), nq, P, Kpair, Kp,
                                                   shortlist.get());
        MASK_LAUNCHED("lp_shortlist");
        lp_rerank_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(Xs), dp / 4, xids,
                                                reinterpret_cast<const float4 *>(Qp),
                                                shortlist.get(), nq, Kp, k, leaf_rows, ids,
                                                dists);
        MASK_LAUNCHED("lp_rerank");
    }
}

}  // namespace mask
