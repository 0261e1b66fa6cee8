// query_cm_tc.cu -- the cluster-major leaf scan (§3.3, Algorithm 2: rank the
// points of the kept leaf clusters, keep the k nearest) on the 5th-generation
// tensor cores, for rows of 32 or 64 floats.
//
// Same work items, same filter and same exact keys as cm_scan_kernel
// (query_cm.cu): a work item is a leaf cluster and up to 16 of the queries
// that kept it; each 128-row chunk of the cluster is ranked by the expanded
// form ||x||^2 + ||q||^2 - 2 x.q, and only (query, row) pairs whose value,
// less a proven rounding bound, can reach the smaller of the pair's current
// K-th key and the query's seed bound T_q get the exact difference-form key
// sum_t (x_t - q_t)^2 (increasing t, FMAs).  So the results are bit-identical
// to the per-query scan's.
//
// The dot products x.q run on tcgen05 (kind::tf32, M = 128 rows, N = 16
// queries, FP32 accumulation in tensor memory).  The rows go to the MMA as
// they were staged (FP32 containers, read as TF32, |x - x_tf32| <= 2^-10 |x|);
// each query is cut into q_hi = q with its low 13 mantissa bits cleared (a
// TF32 value, read exactly) and q_lo = q - q_hi (exact in FP32), and
//     x.q ~= x.q_hi + x.q_lo
// (two MMAs per K-step).  The filter's rounding bound covers the TF32 reading
// of x; it admits a few more pairs to the exact evaluation than an FP32
// product would, and the evaluation is exact either way.
//
// Warp roles (one CTA per SM, persistent over the items of a grid stride):
//   warp 0      TMA producer: each chunk's rows (FP32, 128-byte swizzled
//               boxes of 32 columns) into a 4-stage shared-memory ring;
//   warp 1      MMA issuer (and tensor-memory owner: four accumulators);
//   warps 2-5   queries: each item's 16 queries into shared memory (FP32 for
//               the exact keys, swizzled hi/lo parts for the MMA), loaded
//               one item ahead; and, once the epilogue is done with an item,
//               the merge of its lists into each pair's K best (three items
//               in flight);
//   warps 6-13  epilogue: two warps per tensor-memory lane quadrant, each
//               one row per thread and 8 of the 16 query columns; the filter,
//               exact keys one per lane for the pairs that pass, and a top-K
//               list per (warp, query).  No block-wide barrier: stages,
//               accumulators and item buffers are handed back through
//               mbarriers.
// Every wait is bounded (tc_common.cuh); a stalled pipeline raises the error
// word that the host turns into MASK_ETIMEOUT.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "tc_common.cuh"

namespace mask {

// Raised by a CTA of the tensor-core leaf scan whose bounded wait ran out.
__device__ int g_cm_tc_err;

namespace {

using namespace tc;

constexpr unsigned kFull = 0xffffffffu;
constexpr int CT_R = 128;                  // rows per chunk (MMA M)
constexpr int CT_QB = kCmItemQueries;      // queries per work item (MMA N)
constexpr int CT_S = 4;                    // chunks in flight
constexpr int CT_NACC = 4;                 // accumulators in tensor memory
constexpr int CT_NQ = 3;                   // items in flight (query and list buffers)
constexpr int CT_QW0 = 2;                  // first query warp (four)
constexpr int CT_EPI0 = 6;                 // first epilogue warp
constexpr int CT_EPI_WARPS = 8;            // two per TMEM lane quadrant (8 query columns each)
constexpr int CT_EPI_COLS = CT_QB / 2;
constexpr int CT_THREADS = (CT_EPI0 + CT_EPI_WARPS) * 32;
constexpr uint32_t CT_BOX = CT_R * 128;    // 128 rows x 32 floats: 16 KB
constexpr uint32_t CT_QBOX = CT_QB * 128;  // 16 queries x 32 floats: 2 KB
constexpr uint32_t CT_TMEM_COLS = 64;      // the four accumulators

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 16, M = 128
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) |
                                ((uint32_t)(CT_QB >> 3) << 17) | ((uint32_t)(CT_R >> 4) << 24);

// D (+)= A.B^T, kind::tf32, A and B in shared memory (descriptors).
__device__ __forceinline__ void mma_tf32_ss(uint32_t d_tmem, uint64_t a, uint64_t b,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdescTf32), "r"(accumulate)
        : "memory");
}

// Named barrier 2 over the four query warps, ANDing a flag across them.
__device__ __forceinline__ bool ct_q_bar_and(bool v) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)v)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void ct_q_bar() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

// hi = v with the low 13 mantissa bits cleared (exact in TF32), lo = v - hi.
__device__ __forceinline__ void split_tf32(float v, uint32_t &hi, uint32_t &lo) {
    const uint32_t h = __float_as_uint(v) & 0xFFFFE000u;
    hi = h;
    lo = __float_as_uint(v - __uint_as_float(h));
}

// One work item's metadata.
struct CtItem {
    int64_t rb;   // first row of the cluster
    int rows;     // rows of the cluster
    int nqb;      // queries of the item
};

__device__ __forceinline__ CtItem ct_item(const int4 *meta, int64_t it) {
    const int4 m = meta[it];
    CtItem r;
    r.rb = (int64_t)(uint32_t)m.x | ((int64_t)m.y << 32);
    r.rows = m.z;
    r.nqb = m.w;
    return r;
}

// Shared-memory layout (dynamic part, 1024-byte aligned base), NB = dp / 32
// boxes per row:
//   rows  [CT_S][NB][CT_BOX]            FP32 rows, 128-byte swizzle (TMA)
//   qhi   [NQ][NB][CT_QBOX]             query hi parts, 128-byte swizzle
//   qlo   [NQ][NB][CT_QBOX]             query lo parts
//   qraw  [NQ][CT_QB][dp + 4]           FP32 queries (exact keys)
//   lists [NQ][8][8][K]                 per item buffer, epilogue warp and query column: K best keys
//   mrg   [4][32]                       per query warp: merge scratch
//   pass  [8][32 * 8] u16               per epilogue warp: (query, row) that pass
//   bars  full[S] sfree[S] accfull[NACC] accempty[NACC] qready[NQ] ldone[NQ]
struct CtLayout {
    uint32_t rows, qhi, qlo, qraw, lists, mrg, pass, bars, total;
    __host__ __device__ CtLayout(int dp, int K) {
        const uint32_t nb = (uint32_t)dp / 32;
        rows = 0;
        qhi = rows + CT_S * nb * CT_BOX;
        qlo = qhi + CT_NQ * nb * CT_QBOX;
        qraw = qlo + CT_NQ * nb * CT_QBOX;
        lists = qraw + (uint32_t)CT_NQ * CT_QB * (uint32_t)(dp + 4) * 4u;
        lists = (lists + 15u) & ~15u;
        mrg = lists + (uint32_t)CT_NQ * CT_EPI_WARPS * CT_EPI_COLS * (uint32_t)K * 8u;
        pass = mrg + 4u * 32u * 8u;
        bars = pass + (uint32_t)CT_EPI_WARPS * 32u * CT_EPI_COLS * 2u;
        bars = (bars + 7u) & ~7u;
        total = bars + (2 * CT_S + 2 * CT_NACC + 2 * CT_NQ) * 8u;
    }
};

// The kernel.  xn: row norms of the index's points; qn: query norms;
// seed_d [nq x K]: each query's K nearest distances within its nearest kept
// cluster (the K-th is T_q); mcoef: the filter's rounding bound per unit of
// ||x||^2 + ||q||^2; meta / pid / qid / item_off: the work items
// (cm_item_meta); pair_out [pairs x K]: each pair's K best keys, preset to
// kNoKey (items of empty clusters are skipped, and so are pair lists that
// receive nothing).
template <int NB>
__global__ __launch_bounds__(CT_THREADS, 1) void cm_tc_scan_kernel(
    const __grid_constant__ CUtensorMap tmX, const float *__restrict__ xn,
    const int32_t *__restrict__ xids, const float *__restrict__ Qp, const float *__restrict__ qn,
    const float *__restrict__ seed_d, float mcoef, const int4 *__restrict__ meta,
    const int32_t *__restrict__ pid, const int32_t *__restrict__ qid,
    const int64_t *__restrict__ item_off, int k0, int K,
    unsigned long long *__restrict__ pair_out, unsigned long long *__restrict__ bytes_ctr,
    int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;   // swizzled tiles need 1 KB alignment
    unsigned char *basep = smem_raw + (base - raw);
    constexpr int dp = 32 * NB, nb = NB, dp4 = dp / 4, QS = dp + 4;   // NB boxes of 32 floats
    const CtLayout lay(dp, K);
    float *qraw = reinterpret_cast<float *>(basep + lay.qraw);
    unsigned long long *lists = reinterpret_cast<unsigned long long *>(basep + lay.lists);
    unsigned long long *mrg = reinterpret_cast<unsigned long long *>(basep + lay.mrg);
    unsigned short *pass = reinterpret_cast<unsigned short *>(basep + lay.pass);
    __shared__ __align__(16) float s_qn[CT_NQ][CT_QB];
    __shared__ __align__(16) float s_tq[CT_NQ][CT_QB];
    __shared__ int32_t s_pid[CT_NQ][CT_QB];
    __shared__ int s_nqb[CT_NQ];       // per item buffer: the item's query count
    __shared__ int s_rows[CT_NQ];      // per item buffer: the item's row count
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;

    const uint32_t bar0 = base + lay.bars;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto sfree = [&](int s) { return bar0 + 8u * (CT_S + s); };
    auto accfull = [&](int a) { return bar0 + 8u * (2 * CT_S + a); };
    auto accempty = [&](int a) { return bar0 + 8u * (2 * CT_S + CT_NACC + a); };
    auto qready = [&](int b) { return bar0 + 8u * (2 * CT_S + 2 * CT_NACC + b); };
    auto ldone = [&](int b) { return bar0 + 8u * (2 * CT_S + 2 * CT_NACC + CT_NQ + b); };
    auto rows_at = [&](int s) { return base + lay.rows + (uint32_t)s * (uint32_t)nb * CT_BOX; };
    auto qhi_at = [&](int b) { return base + lay.qhi + (uint32_t)b * (uint32_t)nb * CT_QBOX; };
    auto qlo_at = [&](int b) { return base + lay.qlo + (uint32_t)b * (uint32_t)nb * CT_QBOX; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n_items = item_off[k0];
    const int64_t G = gridDim.x;
    if (*(volatile int *)err != 0) return;   // the grid already gave up

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < CT_S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(sfree(s), CT_EPI_WARPS);
        }
        for (int a = 0; a < CT_NACC; ++a) {
            mbar_init(accfull(a), 1);
            mbar_init(accempty(a), CT_EPI_WARPS);
        }
        for (int b = 0; b < CT_NQ; ++b) {
            mbar_init(qready(b), 4);
            mbar_init(ldone(b), CT_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < CT_NQ * CT_EPI_WARPS * CT_EPI_COLS * K; i += CT_THREADS)
        lists[i] = kNoKey;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "n"(CT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int64_t j = 0, armed = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; ok && it < n_items; it += G) {
                const CtItem im = ct_item(meta, it);
                for (int64_t r0 = im.rb; r0 < im.rb + im.rows; r0 += CT_R, ++j) {
                    const int s = (int)(j % CT_S);
                    const int64_t u = j / CT_S;
                    if (u > 0 && !mbar_wait(sfree(s), (uint32_t)((u - 1) & 1), err)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(full(s), (uint32_t)nb * CT_BOX);
                    for (int h = 0; h < nb; ++h)
                        tma_load_2d(rows_at(s) + (uint32_t)h * CT_BOX, &tmX, 32 * h, (int)r0,
                                    full(s));
                    armed = j + 1;
                }
            }
            // every load issued must land before the CTA may exit
            for (int64_t jj = (armed > CT_S ? armed - CT_S : 0); jj < armed; ++jj)
                mbar_wait(full((int)(jj % CT_S)), (uint32_t)((jj / CT_S) & 1), err, true);
            if (!ok) s_err = 1;
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int64_t j = 0, iseq = -1, last = -1;
            bool ok = true;
            constexpr int ksteps = dp / 8;
            for (int64_t it = blockIdx.x; ok && it < n_items; it += G) {
                const CtItem im = ct_item(meta, it);
                if (im.rows == 0) continue;
                ++iseq;
                const int b = (int)(iseq % CT_NQ);
                ok = mbar_wait(qready(b), (uint32_t)((iseq / CT_NQ) & 1), err);
                const uint64_t dQh = sw128_desc(qhi_at(b)), dQl = sw128_desc(qlo_at(b));
                for (int64_t r0 = im.rb; ok && r0 < im.rb + im.rows; r0 += CT_R, ++j) {
                    const int s = (int)(j % CT_S), a = (int)(j % CT_NACC);
                    ok = mbar_wait(full(s), (uint32_t)((j / CT_S) & 1), err);
                    if (ok && j >= CT_NACC)
                        ok = mbar_wait(accempty(a), (uint32_t)((j / CT_NACC - 1) & 1), err);
                    if (!ok) break;
                    fence_after();
                    const uint32_t d = tmem + (uint32_t)(16 * a);
                    const uint64_t dX = sw128_desc(rows_at(s));
                    // K-step ks covers columns 8ks..8ks+7: box ks / 4, 32 bytes
                    // into each 128-byte row per step (+2 in 16-byte units)
#pragma unroll
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t step = (uint64_t)((ks & 3) * 2);
                        const uint64_t ox = (uint64_t)((ks >> 2) * (CT_BOX >> 4)) + step;
                        const uint64_t oq = (uint64_t)((ks >> 2) * (CT_QBOX >> 4)) + step;
                        mma_tf32_ss(d, dX + ox, dQh + oq, ks > 0 ? 1u : 0u);
                        mma_tf32_ss(d, dX + ox, dQl + oq, 1u);
                    }
                    mma_commit(accfull(a));   // the accumulator is ready
                    last = j;
                }
            }
            // the MMAs must be complete before tensor memory is released
            if (last >= 0)
                mbar_wait(accfull((int)(last % CT_NACC)), (uint32_t)((last / CT_NACC) & 1), err,
                          true);
            if (!ok) s_err = 1;
        }
    } else if (warp < CT_EPI0) {
        // ---------------- queries (loaded one item ahead) and merges ----------------
        const int tq = (warp - CT_QW0) * 32 + lane;   // 0..127
        const int q = tq >> 3, c = tq & 7;            // query, 16-byte column group of a box
        const int qw = warp - CT_QW0;                 // 0..3
        const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
        float4 nx[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
        float nqn = 0.f, ntq = 0.f;
        int32_t npid = -1;
        auto fetch = [&](int64_t it, const CtItem &im) {
            const bool v = q < im.nqb;
            const int32_t qq = v ? qid[it * CT_QB + q] : 0;
#pragma unroll
            for (int h = 0; h < nb; ++h)
                nx[h] = v ? Q4[(int64_t)qq * dp4 + 8 * h + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (tq < CT_QB) {
                const bool vv = tq < im.nqb;
                const int32_t q2 = vv ? qid[it * CT_QB + tq] : 0;
                nqn = vv ? qn[q2] : 0.f;
                ntq = vv ? seed_d[(int64_t)q2 * K + K - 1] : 0.f;
                npid = vv ? pid[it * CT_QB + tq] : -1;
            }
        };
        auto next_item = [&](int64_t it) {   // the next item of this CTA with rows
            while (it < n_items && meta[it].z == 0) it += G;
            return it;
        };
        // The item that last used buffer b is done in the epilogue: merge
        // each of its queries' four lists (one per lane quadrant) into the
        // pair's K best, write it, and clear the lists.  Query warp qw takes
        // queries qw, qw + 4, ...
        unsigned long long *wm = mrg + qw * 32;
        auto merge_item = [&](int b) {
            const int nqb = s_nqb[b];
            for (int qb = qw; qb < nqb; qb += 4) {
                const int half = qb / CT_EPI_COLS, col = qb % CT_EPI_COLS;
                unsigned long long *L0 =
                    lists + (((size_t)b * CT_EPI_WARPS + half * 4) * CT_EPI_COLS + col) * K;
                unsigned long long e[4];
                int cnt[4], tot = 0;
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    e[w] = lane < K ? L0[(size_t)w * CT_EPI_COLS * K + lane] : kNoKey;
                    cnt[w] = __popc(__ballot_sync(kFull, e[w] != kNoKey));
                    tot += cnt[w];
                }
                if (tot == 0) continue;   // the pair list stays empty (preset)
                unsigned long long *dst = pair_out + (int64_t)s_pid[b][qb] * K;
                if (tot <= 32) {
                    // gather the valid keys (each list holds its valid keys
                    // first); each lane writes its key at its rank among them
                    // (keys are distinct: ids differ)
                    int off = 0;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        if (e[w] != kNoKey) wm[off + lane] = e[w];
                        off += cnt[w];
                    }
                    __syncwarp();
                    const unsigned long long key = lane < tot ? wm[lane] : kNoKey;
                    int rank = 0;
                    for (int i = 0; i < tot; ++i) rank += wm[i] < key ? 1 : 0;
                    if (lane < tot && rank < K) dst[rank] = key;
                    __syncwarp();
                } else {
                    // K rounds of warp-wide minimum over the four lists
                    unsigned long long out = kNoKey;
                    unsigned long long f[4] = {e[0], e[1], e[2], e[3]};
                    for (int rd = 0; rd < K; ++rd) {
                        unsigned long long mine = f[0];
#pragma unroll
                        for (int i = 1; i < 4; ++i) mine = f[i] < mine ? f[i] : mine;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const unsigned long long v = __shfl_xor_sync(kFull, mine, o);
                            mine = v < mine ? v : mine;
                        }
                        if (lane == rd) out = mine;
                        if (mine == kNoKey) break;
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (f[i] == mine) f[i] = kNoKey;
                    }
                    if (lane < K) dst[lane] = out;
                }
                // this query's lists are read: clear them for the buffer's next item
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (e[w] != kNoKey) L0[(size_t)w * CT_EPI_COLS * K + lane] = kNoKey;
            }
            if (bytes_ctr != nullptr && qw == 0 && lane == 0)
                atomicAdd(bytes_ctr, (unsigned long long)s_rows[b] * (dp * 4ull + 4ull));
        };
        int64_t it = next_item(blockIdx.x), iseq = -1;
        if (it < n_items) fetch(it, ct_item(meta, it));
        bool ok = true;
        while (it < n_items) {
            ++iseq;
            const int b = (int)(iseq % CT_NQ);
            const int64_t nit = next_item(it + G);
            if (iseq >= CT_NQ) {
                // the buffer's previous item: the epilogue is done with it;
                // the four query warps agree, merge it, and all have merged
                // before the buffer is overwritten
                const bool lok = __all_sync(
                    kFull, mbar_wait(ldone(b), (uint32_t)((iseq / CT_NQ - 1) & 1), err));
                ok = ct_q_bar_and(lok);
                if (!ok) break;
                merge_item(b);
                ct_q_bar();
            }
            const CtItem im = ct_item(meta, it);
#pragma unroll
            for (int h = 0; h < nb; ++h) {
                const float4 x = nx[h];
                reinterpret_cast<float4 *>(qraw + (b * CT_QB + q) * QS)[8 * h + c] = x;
                uint4 hv, lv;
                split_tf32(x.x, hv.x, lv.x);
                split_tf32(x.y, hv.y, lv.y);
                split_tf32(x.z, hv.z, lv.z);
                split_tf32(x.w, hv.w, lv.w);
                const uint32_t o = (uint32_t)h * CT_QBOX + (uint32_t)q * 128u +
                                   (uint32_t)((c ^ (q & 7)) << 4);
                *reinterpret_cast<uint4 *>(basep + (qhi_at(b) - base) + o) = hv;
                *reinterpret_cast<uint4 *>(basep + (qlo_at(b) - base) + o) = lv;
            }
            if (tq < CT_QB) {
                s_qn[b][tq] = nqn;
                s_tq[b][tq] = ntq;
                s_pid[b][tq] = npid;
            }
            if (tq == 0) {
                s_nqb[b] = im.nqb;
                s_rows[b] = im.rows;
            }
            fence_proxy_async();   // the MMA reads the swizzled parts through the async proxy
            __syncwarp();
            if (lane == 0) mbar_arrive(qready(b));
            if (nit < n_items) fetch(nit, ct_item(meta, nit));   // in flight during the next wait
            it = nit;
        }
        // the last items in flight
        for (int64_t k = (iseq >= CT_NQ ? iseq - CT_NQ + 1 : 0); ok && k <= iseq; ++k) {
            const int b = (int)(k % CT_NQ);
            const bool lok =
                __all_sync(kFull, mbar_wait(ldone(b), (uint32_t)((k / CT_NQ) & 1), err));
            ok = ct_q_bar_and(lok);
            if (!ok) break;
            merge_item(b);
        }
        if (!ok && lane == 0) s_err = 1;
    } else {
        // ------- epilogue: one chunk row per thread, 8 of the 16 query columns -------
        const int quad = warp & 3;
        const int r = quad * 32 + lane;             // the chunk row (TMEM lane) of this thread
        const int ew = warp - CT_EPI0;              // 0..7
        const int q0 = (ew >> 2) * CT_EPI_COLS;     // first query column of this warp
        unsigned short *wpass = pass + ew * 32 * CT_EPI_COLS;
        const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
        int64_t j = 0, iseq = -1;
        bool ok = true;
        for (int64_t it = blockIdx.x; ok && it < n_items; it += G) {
            const CtItem im = ct_item(meta, it);
            if (im.rows == 0) continue;
            ++iseq;
            const int b = (int)(iseq % CT_NQ);
            const int nqb = im.nqb;
            const float *qrb = qraw + b * CT_QB * QS;
            // a failed wait ends the warp's work (the others learn of it
            // through their own wait limits and the abort word)
            bool wok = __all_sync(kFull, mbar_wait(qready(b), (uint32_t)((iseq / CT_NQ) & 1), err));
            // this warp's [8][K] lists of the item: the query warps merged and
            // cleared them (item iseq - NQ) before staging the item's queries,
            // so they start empty
            unsigned long long *wl = lists + ((size_t)b * CT_EPI_WARPS + ew) * CT_EPI_COLS * K;
            // the item's per-query constants of this warp's columns
            float qv[CT_EPI_COLS], tqv[CT_EPI_COLS];
            if (wok) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&s_qn[b][q0]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&s_qn[b][q0 + 4]);
                const float4 t0 = *reinterpret_cast<const float4 *>(&s_tq[b][q0]);
                const float4 t1 = *reinterpret_cast<const float4 *>(&s_tq[b][q0 + 4]);
                qv[0] = a0.x; qv[1] = a0.y; qv[2] = a0.z; qv[3] = a0.w;
                qv[4] = a1.x; qv[5] = a1.y; qv[6] = a1.z; qv[7] = a1.w;
                tqv[0] = t0.x; tqv[1] = t0.y; tqv[2] = t0.z; tqv[3] = t0.w;
                tqv[4] = t1.x; tqv[5] = t1.y; tqv[6] = t1.z; tqv[7] = t1.w;
            }
            for (int64_t r0 = im.rb; wok && r0 < im.rb + im.rows; r0 += CT_R, ++j) {
                const int s = (int)(j % CT_S), a = (int)(j % CT_NACC);
                const int nr = (int)min((int64_t)CT_R, im.rb + im.rows - r0);
                // this row's norm and id, read ahead of the waits
                const bool rv = r < nr;
                const float xv = rv ? xn[r0 + r] : 0.f;
                const int32_t xid = rv ? xids[r0 + r] : 0;
                wok = mbar_wait(full(s), (uint32_t)((j / CT_S) & 1), err) &&
                      mbar_wait(accfull(a), (uint32_t)((j / CT_NACC) & 1), err);
                if (!__all_sync(kFull, wok)) {
                    wok = false;
                    break;
                }
                fence_after();
                uint32_t acc[CT_EPI_COLS];
                tmem_ld8(lane_addr + (uint32_t)(16 * a + q0), acc);
                // each list's K-th key bounds its pair's candidates (broadcast loads)
                float lim[CT_EPI_COLS];
#pragma unroll
                for (int cc = 0; cc < CT_EPI_COLS; ++cc) {
                    const unsigned long long th = wl[cc * K + K - 1];
                    lim[cc] = fminf(tqv[cc], th == kNoKey ? __int_as_float(0x7f800000)
                                                          : __uint_as_float((unsigned)(th >> 32)));
                }
                tmem_wait();
                // the accumulator is in registers: hand it back to the MMA warp
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(accempty(a));
                // A (query, row) whose expanded form, less its rounding bound,
                // can reach the smaller of its list's K-th and T_q gets its
                // exact key.  The tests are independent; the rare passes are
                // then collected per warp (ballots give each its slot).
                uint32_t mask = 0;
#pragma unroll
                for (int cc = 0; cc < CT_EPI_COLS; ++cc) {
                    const float dv = fmaf(-2.f, __uint_as_float(acc[cc]), xv + qv[cc]);
                    const bool p = rv && q0 + cc < nqb && dv <= lim[cc] + mcoef * (xv + qv[cc]);
                    mask |= p ? (1u << cc) : 0u;
                }
                if (__any_sync(kFull, mask != 0)) {
                    int npass = 0;
#pragma unroll
                    for (int cc = 0; cc < CT_EPI_COLS; ++cc) {
                        const bool p = (mask >> cc) & 1u;
                        const unsigned bal = __ballot_sync(kFull, p);
                        if (p)
                            wpass[npass + __popc(bal & ((1u << lane) - 1u))] =
                                (unsigned short)((cc << 8) | lane);
                        npass += __popc(bal);
                    }
                    __syncwarp();
                    // exact keys, one (query, row) per lane: the arithmetic of
                    // the per-query scan (sum over t of (x_t - q_t)^2, FMAs, t
                    // ascending); then each key goes into its list
                    const unsigned char *rows = basep + (rows_at(s) - base);
                    for (int i0 = 0; i0 < npass; i0 += 32) {
                        const int i = i0 + lane;
                        const int pr = i < npass ? wpass[i] : 0;
                        const int cc = pr >> 8, rl = pr & 31, rr = quad * 32 + rl;
                        const int32_t id = __shfl_sync(kFull, xid, rl);
                        unsigned long long key = kNoKey;
                        if (i < npass) {
                            const unsigned char *xr = rows + (uint32_t)rr * 128u;
                            const float4 *q4 = reinterpret_cast<const float4 *>(qrb + (q0 + cc) * QS);
                            float e2 = 0.f;
#pragma unroll
                            for (int t4 = 0; t4 < dp4; ++t4) {
                                const int h = t4 >> 3, cq = t4 & 7;
                                const float4 x4 = *reinterpret_cast<const float4 *>(
                                    xr + (uint32_t)h * CT_BOX + (uint32_t)((cq ^ (rr & 7)) << 4));
                                const float4 b4 = q4[t4];
                                float d = x4.x - b4.x;
                                e2 = fmaf(d, d, e2);
                                d = x4.y - b4.y;
                                e2 = fmaf(d, d, e2);
                                d = x4.z - b4.z;
                                e2 = fmaf(d, d, e2);
                                d = x4.w - b4.w;
                                e2 = fmaf(d, d, e2);
                            }
                            key = ((unsigned long long)__float_as_uint(e2) << 32) | (unsigned)id;
                        }
                        // insert the round's keys into this warp's lists, one
                        // at a time (a list is held one entry per lane; keys
                        // are distinct: ids differ)
                        unsigned m = __ballot_sync(kFull, key != kNoKey);
                        while (m) {
                            const int src = __ffs(m) - 1;
                            m &= m - 1u;
                            const unsigned long long k1 = __shfl_sync(kFull, key, src);
                            const int c1 = __shfl_sync(kFull, cc, src);
                            unsigned long long old = lane < K ? wl[c1 * K + lane] : kNoKey;
                            const int pos = __popc(__ballot_sync(kFull, lane < K && old < k1));
                            if (pos < K) {
                                const unsigned long long up = __shfl_up_sync(kFull, old, 1);
                                old = lane < pos ? old : (lane == pos ? k1 : up);
                                if (lane < K) wl[c1 * K + lane] = old;
                            }
                            __syncwarp();
                        }
                    }
                }
                // the chunk's rows are no longer needed: hand the stage back
                __syncwarp();
                if (lane == 0) mbar_arrive(sfree(s));
            }
            // the item is done for this warp; the query warps merge its lists
            // once all eight epilogue warps are done
            if (!__all_sync(kFull, wok)) {
                ok = false;
                break;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(ldone(b));
        }
        if (!ok && lane == 0) s_err = 1;
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "n"(CT_TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && s_err) atomicExch(err, 1);
}

}  // namespace

// ================================================================= host side

namespace {
thread_local bool t_cm_tc_launched = false;   // set by cm_tc_scan on the calling thread
}

bool cm_tc_take_launched() {
    const bool v = t_cm_tc_launched;
    t_cm_tc_launched = false;
    return v;
}

bool cm_tc_supported(int dp, int K) {
    const char *e = std::getenv("MASK_CM_KERNEL");
    if (e && std::strcmp(e, "simt") == 0) return false;
    return (dp == 32 || dp == 64) && K >= 1 && K <= 32 && encode_fn() != nullptr;
}

int *cm_tc_error_word() {
    void *p = nullptr;
    MASK_CUDA(cudaGetSymbolAddress(&p, g_cm_tc_err));
    return static_cast<int *>(p);
}

void cm_tc_check(cudaStream_t s) {
    int e = 0;
    MASK_CUDA(cudaMemcpyFromSymbolAsync(&e, g_cm_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    MASK_CUDA(cudaStreamSynchronize(s));
    if (e) {
        const int z = 0;
        MASK_CUDA(cudaMemcpyToSymbol(g_cm_tc_err, &z, sizeof(int)));
        fail(MASK_ETIMEOUT, "cluster-major leaf scan: a bounded pipeline wait ran out");
    }
}

void cm_tc_scan(const float *Xs, int64_t n, const float *xn, int dp, const int32_t *xids,
                const float *Qp, const float *qn, const float *seed_d, float mcoef,
                const int4 *meta, const int32_t *pid, const int32_t *qid, const int64_t *item_off,
                int k0, int K, unsigned long long *pair_out, unsigned long long *bytes_ctr,
                cudaStream_t s) {
    const CUtensorMap tmX = make_map_2d(Xs, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n, dp, CT_R, 32);
    const CtLayout lay(dp, K);
    const size_t smem = (size_t)lay.total + 1024;
    auto kfn = dp == 32 ? cm_tc_scan_kernel<1> : cm_tc_scan_kernel<2>;
    MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    MASK_CUDA(cudaGetDevice(&dev));
    MASK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MASK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, CT_THREADS, smem));
    kfn<<<std::max(1, per_sm) * sms, CT_THREADS, smem, s>>>(tmX, xn, xids, Qp, qn, seed_d, mcoef,
                                                            meta, pid, qid, item_off, k0, K,
                                                            pair_out, bytes_ctr,
                                                            cm_tc_error_word());
    MASK_LAUNCHED("cm_tc_scan");
    t_cm_tc_launched = true;
}

}  // namespace mask
