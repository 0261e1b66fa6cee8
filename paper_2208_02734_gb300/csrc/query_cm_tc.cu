// query_cm_tc.cu -- the cluster-major leaf scan (§3.3, Algorithm 2: rank the
// points of the kept leaf clusters, keep the k nearest) on the 5th-generation
// tensor cores, for rows of 32 or 64 floats.
//
// Same work items, same filter and same exact keys as cm_scan_kernel
// (query_cm.cu): a work item is a leaf cluster and up to QB (16 or 32) of
// the queries that kept it; each 128-row chunk of the cluster is ranked by the expanded
// form ||x||^2 + ||q||^2 - 2 x.q, and only (query, row) pairs whose value,
// less a proven rounding bound, can reach the smaller of the pair's current
// K-th key and the query's seed bound T_q get the exact difference-form key
// sum_t (x_t - q_t)^2 (increasing t, FMAs).  So the results are bit-identical
// to the per-query scan's.
//
// The dot products x.q run on tcgen05 (kind::tf32, M = 128 rows, N = QB
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
//   warps 2-5   queries: each item's QB queries into shared memory (FP32 for
//               the exact keys, swizzled hi/lo parts for the MMA), loaded
//               one item ahead; and, once the epilogue is done with an item,
//               the merge of its lists into each pair's K best (three items
//               in flight at QB = 16, two at QB = 32);
//   warps 6-13  epilogue: two warps per tensor-memory lane quadrant, each
//               one row per thread and QB / 2 of the query columns; the filter,
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
constexpr int CT_S = 4;                    // chunks in flight
constexpr int CT_NACC = 4;                 // accumulators in tensor memory
constexpr int CT_QW0 = 2;                  // first query warp (four)
constexpr int CT_EPI0 = 6;                 // first epilogue warp
constexpr int CT_EPI_WARPS = 8;            // two per TMEM lane quadrant (QB / 2 query columns each)
constexpr int CT_THREADS = (CT_EPI0 + CT_EPI_WARPS) * 32;
constexpr uint32_t CT_BOX = CT_R * 128;    // 128 rows x 32 floats: 16 KB
constexpr int kCmTcWideMaxK = 16;          // largest K of the 32-query items (shared memory)
// Row norms and ids of a chunk come with its rows, as 1-D TMA boxes that
// start at the chunk's first row rounded down to a multiple of 4 (16 bytes):
// 128 + 4 elements, each box at a 128-byte aligned slot of 160 elements (a
// tensor copy's shared-memory destination is 128-byte aligned).
constexpr int CT_NBOX = CT_R + 4;
constexpr int CT_NSLOT = 160;

// The shapes that depend on the item width QB (queries per work item, the
// MMA's N: 16 or 32).
template <int QB>
struct CtShape {
    static_assert(QB == 16 || QB == 32, "items of 16 or 32 queries");
    static constexpr int NQ = QB == 16 ? 3 : 2;           // items in flight (query and list buffers)
    static constexpr int EC = QB / 2;                     // query columns per epilogue warp
    static constexpr uint32_t QBOX = QB * 128u;           // QB queries x 32 floats
    static constexpr uint32_t TMEM_COLS = CT_NACC * QB;   // the four accumulators (64 or 128)
    // instruction descriptor: D = F32, A = B = TF32, both K-major, N = QB, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) |
                                      ((uint32_t)(QB >> 3) << 17) | ((uint32_t)(CT_R >> 4) << 24);
};

// D (+)= A.B^T, kind::tf32, A and B in shared memory (descriptors).
__device__ __forceinline__ void mma_tf32_ss(uint32_t d_tmem, uint64_t a, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
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
// boxes per row, EC = QB / 2:
//   rows  [CT_S][NB][CT_BOX]            FP32 rows, 128-byte swizzle (TMA)
//   qhi   [NQ][NB][QBOX]                query hi parts, 128-byte swizzle
//   qlo   [NQ][NB][QBOX]                query lo parts
//   qraw  [NQ][QB][dp + 4]              FP32 queries (exact keys)
//   lists [NQ][8][EC][K]                per item buffer, epilogue warp and query column: K best keys
//   mrg   [4][32]                       per query warp: merge scratch
//   pass  [8][32 * EC] u16              per epilogue warp: (query, row) that pass
//   bars  full[S] sfree[S] accfull[NACC] accempty[NACC] qready[NQ] ldone[NQ] lfree[NQ]
template <int QB>
struct CtLayout {
    using SH = CtShape<QB>;
    uint32_t rows, qhi, qlo, qraw, lists, mrg, pass, bars, total;
    __host__ __device__ CtLayout(int dp, int K) {
        const uint32_t nb = (uint32_t)dp / 32;
        rows = 0;
        qhi = rows + CT_S * nb * CT_BOX;
        qlo = qhi + SH::NQ * nb * SH::QBOX;
        qraw = qlo + SH::NQ * nb * SH::QBOX;
        lists = qraw + (uint32_t)SH::NQ * QB * (uint32_t)(dp + 4) * 4u;
        lists = (lists + 15u) & ~15u;
        mrg = lists + (uint32_t)SH::NQ * CT_EPI_WARPS * SH::EC * (uint32_t)K * 8u;
        pass = mrg + 4u * 32u * 8u;
        bars = pass + (uint32_t)CT_EPI_WARPS * 32u * SH::EC * 2u;
        bars = (bars + 7u) & ~7u;
        total = bars + (2 * CT_S + 2 * CT_NACC + 3 * SH::NQ) * 8u;
    }
};

// The kernel.  xn: row norms of the index's points; qn: query norms;
// seed_d [nq x K]: each query's K nearest distances within its nearest kept
// cluster (the K-th is T_q); mcoef: the filter's rounding bound per unit of
// ||x||^2 + ||q||^2; meta / pid / qid / item_off: the work items
// (cm_item_meta); pair_out [pairs x K]: each pair's K best keys, preset to
// kNoKey (items of empty clusters are skipped, and so are pair lists that
// receive nothing); qbound [nq]: each query's running bound on its K-th
// distance (FP32 bits, preset to a huge value), lowered by the merges.
template <int NB, int QB>
__global__ __launch_bounds__(CT_THREADS, 1) void cm_tc_scan_kernel(
    const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmXn,
    const __grid_constant__ CUtensorMap tmXid, const float *__restrict__ Qp, const float *__restrict__ qn,
    const float *__restrict__ seed_d, float mcoef, const int4 *__restrict__ meta,
    const int32_t *__restrict__ pid, const int32_t *__restrict__ qid,
    const int64_t *__restrict__ item_off, int k0, int K,
    unsigned long long *__restrict__ pair_out, unsigned *__restrict__ qbound,
    unsigned long long *__restrict__ bytes_ctr, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;   // swizzled tiles need 1 KB alignment
    unsigned char *basep = smem_raw + (base - raw);
    constexpr int dp = 32 * NB, nb = NB, dp4 = dp / 4, QS = dp + 4;   // NB boxes of 32 floats
    using SH = CtShape<QB>;
    constexpr int NQ = SH::NQ, EC = SH::EC;
    constexpr uint32_t QBOX = SH::QBOX;
    const CtLayout<QB> lay(dp, K);
    float *qraw = reinterpret_cast<float *>(basep + lay.qraw);
    unsigned long long *lists = reinterpret_cast<unsigned long long *>(basep + lay.lists);
    unsigned long long *mrg = reinterpret_cast<unsigned long long *>(basep + lay.mrg);
    unsigned short *pass = reinterpret_cast<unsigned short *>(basep + lay.pass);
    __shared__ __align__(16) float s_qn[NQ][QB];
    __shared__ __align__(16) float s_tq[NQ][QB];
    __shared__ int32_t s_pid[NQ][QB];
    __shared__ int32_t s_qid[NQ][QB];
    __shared__ __align__(128) float s_xn[CT_S][CT_NSLOT];     // per stage: the chunk's row norms
    __shared__ __align__(128) int32_t s_xid[CT_S][CT_NSLOT];  // and ids
    __shared__ int s_nqb[NQ];       // per item buffer: the item's query count
    __shared__ int s_rows[NQ];      // per item buffer: the item's row count
    __shared__ uint32_t s_tmem;
    __shared__ int s_err;

    const uint32_t bar0 = base + lay.bars;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto sfree = [&](int s) { return bar0 + 8u * (CT_S + s); };
    auto accfull = [&](int a) { return bar0 + 8u * (2 * CT_S + a); };
    auto accempty = [&](int a) { return bar0 + 8u * (2 * CT_S + CT_NACC + a); };
    auto qready = [&](int b) { return bar0 + 8u * (2 * CT_S + 2 * CT_NACC + b); };
    auto ldone = [&](int b) { return bar0 + 8u * (2 * CT_S + 2 * CT_NACC + NQ + b); };
    auto lfree = [&](int b) { return bar0 + 8u * (2 * CT_S + 2 * CT_NACC + 2 * NQ + b); };
    auto rows_at = [&](int s) { return base + lay.rows + (uint32_t)s * (uint32_t)nb * CT_BOX; };
    auto qhi_at = [&](int b) { return base + lay.qhi + (uint32_t)b * (uint32_t)nb * QBOX; };
    auto qlo_at = [&](int b) { return base + lay.qlo + (uint32_t)b * (uint32_t)nb * QBOX; };

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
        for (int b = 0; b < NQ; ++b) {
            mbar_init(qready(b), 4);
            mbar_init(ldone(b), CT_EPI_WARPS);
            mbar_init(lfree(b), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < NQ * CT_EPI_WARPS * EC * K; i += CT_THREADS)
        lists[i] = kNoKey;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "n"(SH::TMEM_COLS)
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
                    mbar_expect_tx(full(s), (uint32_t)nb * CT_BOX + 2u * CT_NBOX * 4u);
                    for (int h = 0; h < nb; ++h)
                        tma_load_2d(rows_at(s) + (uint32_t)h * CT_BOX, &tmX, 32 * h, (int)r0,
                                    full(s));
                    tma_load_1d(smem_u32(&s_xn[s][0]), &tmXn, (int)(r0 & ~3ll), full(s));
                    tma_load_1d(smem_u32(&s_xid[s][0]), &tmXid, (int)(r0 & ~3ll), full(s));
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
                const int b = (int)(iseq % NQ);
                ok = mbar_wait(qready(b), (uint32_t)((iseq / NQ) & 1), err);
                const uint64_t dQh = sw128_desc(qhi_at(b)), dQl = sw128_desc(qlo_at(b));
                for (int64_t r0 = im.rb; ok && r0 < im.rb + im.rows; r0 += CT_R, ++j) {
                    const int s = (int)(j % CT_S), a = (int)(j % CT_NACC);
                    ok = mbar_wait(full(s), (uint32_t)((j / CT_S) & 1), err);
                    if (ok && j >= CT_NACC)
                        ok = mbar_wait(accempty(a), (uint32_t)((j / CT_NACC - 1) & 1), err);
                    if (!ok) break;
                    fence_after();
                    const uint32_t d = tmem + (uint32_t)(QB * a);
                    const uint64_t dX = sw128_desc(rows_at(s));
                    // K-step ks covers columns 8ks..8ks+7: box ks / 4, 32 bytes
                    // into each 128-byte row per step (+2 in 16-byte units)
#pragma unroll
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint64_t step = (uint64_t)((ks & 3) * 2);
                        const uint64_t ox = (uint64_t)((ks >> 2) * (CT_BOX >> 4)) + step;
                        const uint64_t oq = (uint64_t)((ks >> 2) * (QBOX >> 4)) + step;
                        mma_tf32_ss(d, dX + ox, dQh + oq, SH::IDESC, ks > 0 ? 1u : 0u);
                        mma_tf32_ss(d, dX + ox, dQl + oq, SH::IDESC, 1u);
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
        constexpr int QR = QB / 16;                   // queries per thread (rounds of 16)
        const int tq = (warp - CT_QW0) * 32 + lane;   // 0..127
        const int q = tq >> 3, c = tq & 7;            // query (+ 16 per round), 16-byte column group of a box
        const int qw = warp - CT_QW0;                 // 0..3
        const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
        float4 nx[QR][NB];
#pragma unroll
        for (int rq = 0; rq < QR; ++rq)
#pragma unroll
            for (int h = 0; h < nb; ++h) nx[rq][h] = make_float4(0.f, 0.f, 0.f, 0.f);
        float nqn = 0.f, ntq = 0.f;
        int32_t npid = -1, nqid = -1;
        auto fetch = [&](int64_t it, const CtItem &im) {
#pragma unroll
            for (int rq = 0; rq < QR; ++rq) {
                const int qr = q + 16 * rq;
                const bool v = qr < im.nqb;
                const int32_t qq = v ? qid[it * QB + qr] : 0;
#pragma unroll
                for (int h = 0; h < nb; ++h)
                    nx[rq][h] =
                        v ? Q4[(int64_t)qq * dp4 + 8 * h + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            if (tq < QB) {
                const bool vv = tq < im.nqb;
                const int32_t q2 = vv ? qid[it * QB + tq] : 0;
                nqn = vv ? qn[q2] : 0.f;
                // T_q, or the query's running bound if already tighter
                ntq = vv ? fminf(seed_d[(int64_t)q2 * K + K - 1], __uint_as_float(__ldcg(qbound + q2)))
                         : 0.f;
                npid = vv ? pid[it * QB + tq] : -1;
                nqid = vv ? q2 : -1;
            }
        };
        auto next_item = [&](int64_t it) {   // the next item of this CTA with rows
            while (it < n_items && meta[it].z == 0) it += G;
            return it;
        };
        // The item that last used buffer b is done in the epilogue: merge
        // each of its queries' four lists (one per lane quadrant) into the
        // pair's K best, write it, and clear the lists.  Query warp qw takes
        // queries qw, qw + 4, ... (lane l holds the pair and query of
        // qw + 4 l, read before the next item overwrites the buffer).  The
        // K-th of a merged list is an exact distance of K rows of the query,
        // so it bounds the query's K-th: it tightens the query's running
        // bound, which later items take as T_q where it is smaller.
        struct MergeMeta {
            int nqb, rows;
            int32_t pid, qid;
        };
        auto take_meta = [&](int b) {
            MergeMeta m;
            m.nqb = s_nqb[b];
            m.rows = s_rows[b];
            const int qb = qw + 4 * lane;
            const bool v = lane < QB / 4 && qb < m.nqb;
            m.pid = v ? s_pid[b][qb] : -1;
            m.qid = v ? s_qid[b][qb] : -1;
            return m;
        };
        unsigned long long *wm = mrg + qw * 32;
        auto merge_item = [&](int b, const MergeMeta &m) {
            const int nqb = m.nqb;
            for (int qb = qw, l = 0; qb < nqb; qb += 4, ++l) {
                const int32_t mpid = __shfl_sync(kFull, m.pid, l);
                const int32_t mqid = __shfl_sync(kFull, m.qid, l);
                const int half = qb / EC, col = qb % EC;
                unsigned long long *L0 =
                    lists + (((size_t)b * CT_EPI_WARPS + half * 4) * EC + col) * K;
                unsigned long long e[4];
                int cnt[4], tot = 0;
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    e[w] = lane < K ? L0[(size_t)w * EC * K + lane] : kNoKey;
                    cnt[w] = __popc(__ballot_sync(kFull, e[w] != kNoKey));
                    tot += cnt[w];
                }
                if (tot == 0) continue;   // the pair list stays empty (preset)
                unsigned long long *dst = pair_out + (int64_t)mpid * K;
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
                    if (lane < tot && rank == K - 1) atomicMin(qbound + mqid, (unsigned)(key >> 32));
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
                    if (lane == K - 1 && out != kNoKey) atomicMin(qbound + mqid, (unsigned)(out >> 32));
                }
                // this query's lists are read: clear them for the buffer's next item
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    if (e[w] != kNoKey) L0[(size_t)w * EC * K + lane] = kNoKey;
            }
            if (bytes_ctr != nullptr && qw == 0 && lane == 0)
                atomicAdd(bytes_ctr, (unsigned long long)m.rows * (dp * 4ull + 4ull));
        };
        int64_t it = next_item(blockIdx.x), iseq = -1;
        if (it < n_items) fetch(it, ct_item(meta, it));
        bool ok = true;
        while (it < n_items) {
            ++iseq;
            const int b = (int)(iseq % NQ);
            const int64_t nit = next_item(it + G);
            MergeMeta mm{0, 0, -1, -1};
            if (iseq >= NQ) {
                // the buffer's previous item: the epilogue is done with it;
                // the four query warps agree and take its merge metadata
                // before the buffer is overwritten (its lists stay until
                // merged: the epilogue waits for lfree before using them)
                const bool lok = __all_sync(
                    kFull, mbar_wait(ldone(b), (uint32_t)((iseq / NQ - 1) & 1), err));
                ok = ct_q_bar_and(lok);
                if (!ok) break;
                mm = take_meta(b);
                ct_q_bar();
            }
            const CtItem im = ct_item(meta, it);
#pragma unroll
            for (int rq = 0; rq < QR; ++rq) {
                const int qr = q + 16 * rq;
#pragma unroll
                for (int h = 0; h < nb; ++h) {
                    const float4 x = nx[rq][h];
                    reinterpret_cast<float4 *>(qraw + (b * QB + qr) * QS)[8 * h + c] = x;
                    uint4 hv, lv;
                    split_tf32(x.x, hv.x, lv.x);
                    split_tf32(x.y, hv.y, lv.y);
                    split_tf32(x.z, hv.z, lv.z);
                    split_tf32(x.w, hv.w, lv.w);
                    const uint32_t o = (uint32_t)h * QBOX + (uint32_t)qr * 128u +
                                       (uint32_t)((c ^ (qr & 7)) << 4);
                    *reinterpret_cast<uint4 *>(basep + (qhi_at(b) - base) + o) = hv;
                    *reinterpret_cast<uint4 *>(basep + (qlo_at(b) - base) + o) = lv;
                }
            }
            if (tq < QB) {
                s_qn[b][tq] = nqn;
                s_tq[b][tq] = ntq;
                s_pid[b][tq] = npid;
                s_qid[b][tq] = nqid;
            }
            if (tq == 0) {
                s_nqb[b] = im.nqb;
                s_rows[b] = im.rows;
            }
            fence_proxy_async();   // the MMA reads the swizzled parts through the async proxy
            __syncwarp();
            if (lane == 0) mbar_arrive(qready(b));
            if (nit < n_items) fetch(nit, ct_item(meta, nit));   // in flight during the merge
            if (iseq >= NQ) {
                // the previous item of the buffer, while the MMAs of this one run
                merge_item(b, mm);
                __syncwarp();
                if (lane == 0) mbar_arrive(lfree(b));
            }
            it = nit;
        }
        // the last items in flight
        for (int64_t k = (iseq >= NQ ? iseq - NQ + 1 : 0); ok && k <= iseq; ++k) {
            const int b = (int)(k % NQ);
            const bool lok =
                __all_sync(kFull, mbar_wait(ldone(b), (uint32_t)((k / NQ) & 1), err));
            ok = ct_q_bar_and(lok);
            if (!ok) break;
            merge_item(b, take_meta(b));
        }
        if (!ok && lane == 0) s_err = 1;
    } else {
        // ------- epilogue: one chunk row per thread, 8 of the 16 query columns -------
        const int quad = warp & 3;
        const int r = quad * 32 + lane;             // the chunk row (TMEM lane) of this thread
        const int ew = warp - CT_EPI0;              // 0..7
        const int q0 = (ew >> 2) * EC;              // first query column of this warp
        unsigned short *wpass = pass + ew * 32 * EC;
        const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
        int64_t j = 0, iseq = -1;
        bool ok = true;
        for (int64_t it = blockIdx.x; ok && it < n_items; it += G) {
            const CtItem im = ct_item(meta, it);
            if (im.rows == 0) continue;
            ++iseq;
            const int b = (int)(iseq % NQ);
            const int nqb = im.nqb;
            const float *qrb = qraw + b * QB * QS;
            // a failed wait ends the warp's work (the others learn of it
            // through their own wait limits and the abort word)
            bool wok = __all_sync(kFull, mbar_wait(qready(b), (uint32_t)((iseq / NQ) & 1), err));
            // the lists of the buffer's previous item are merged and cleared
            if (iseq >= NQ)
                wok = __all_sync(kFull, wok && mbar_wait(lfree(b), (uint32_t)((iseq / NQ - 1) & 1), err));
            // this warp's [EC][K] lists of the item: the query warps merged and
            // cleared them (item iseq - NQ, lfree above), so they start empty
            unsigned long long *wl = lists + ((size_t)b * CT_EPI_WARPS + ew) * EC * K;
            // the item's per-query constants of this warp's columns
            float qv[EC], tqv[EC];
            if (wok) {
#pragma unroll
                for (int c4 = 0; c4 < EC / 4; ++c4) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(&s_qn[b][q0 + 4 * c4]);
                    const float4 t4 = *reinterpret_cast<const float4 *>(&s_tq[b][q0 + 4 * c4]);
                    qv[4 * c4] = a4.x; qv[4 * c4 + 1] = a4.y; qv[4 * c4 + 2] = a4.z;
                    qv[4 * c4 + 3] = a4.w;
                    tqv[4 * c4] = t4.x; tqv[4 * c4 + 1] = t4.y; tqv[4 * c4 + 2] = t4.z;
                    tqv[4 * c4 + 3] = t4.w;
                }
            }
            for (int64_t r0 = im.rb; wok && r0 < im.rb + im.rows; r0 += CT_R, ++j) {
                const int s = (int)(j % CT_S), a = (int)(j % CT_NACC);
                const int nr = (int)min((int64_t)CT_R, im.rb + im.rows - r0);
                const bool rv = r < nr;
                wok = mbar_wait(full(s), (uint32_t)((j / CT_S) & 1), err) &&
                      mbar_wait(accfull(a), (uint32_t)((j / CT_NACC) & 1), err);
                if (!__all_sync(kFull, wok)) {
                    wok = false;
                    break;
                }
                // this row's norm and id (staged with the rows)
                const float xv = rv ? s_xn[s][(int)(r0 & 3) + r] : 0.f;
                const int32_t xid = rv ? s_xid[s][(int)(r0 & 3) + r] : 0;
                fence_after();
                uint32_t acc[EC];
                if constexpr (EC == 8)
                    tmem_ld8(lane_addr + (uint32_t)(QB * a + q0), acc);
                else
                    tmem_ld16(lane_addr + (uint32_t)(QB * a + q0), acc);
                // each list's K-th key bounds its pair's candidates (broadcast loads)
                float lim[EC];
#pragma unroll
                for (int cc = 0; cc < EC; ++cc) {
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
                for (int cc = 0; cc < EC; ++cc) {
                    const float dv = fmaf(-2.f, __uint_as_float(acc[cc]), xv + qv[cc]);
                    const bool p = rv && q0 + cc < nqb && dv <= lim[cc] + mcoef * (xv + qv[cc]);
                    mask |= p ? (1u << cc) : 0u;
                }
                if (__any_sync(kFull, mask != 0)) {
                    int npass = 0;
#pragma unroll
                    for (int cc = 0; cc < EC; ++cc) {
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
                     "n"(SH::TMEM_COLS)
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

int cm_tc_item_queries(int K) { return K <= kCmTcWideMaxK ? kCmTcItemQueries : kCmItemQueries; }

namespace {
template <int QB>
void launch_cm_tc(const CUtensorMap &tmX, const CUtensorMap &tmXn, const CUtensorMap &tmXid, int dp,
                  const float *Qp, const float *qn, const float *seed_d, float mcoef,
                  const int4 *meta, const int32_t *pid, const int32_t *qid,
                  const int64_t *item_off, int k0, int K, unsigned long long *pair_out,
                  unsigned *qbound, unsigned long long *bytes_ctr, cudaStream_t s) {
    const CtLayout<QB> lay(dp, K);
    const size_t smem = (size_t)lay.total + 1024;
    auto kfn = dp == 32 ? cm_tc_scan_kernel<1, QB> : cm_tc_scan_kernel<2, QB>;
    cudaFuncAttributes fa;
    MASK_CUDA(cudaFuncGetAttributes(&fa, kfn));
    MASK_REQUIRE(smem + fa.sharedSizeBytes <= 227u * 1024u,
                 "tensor-core leaf scan: shared memory over 227 KB");
    MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    MASK_CUDA(cudaGetDevice(&dev));
    MASK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MASK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, CT_THREADS, smem));
    kfn<<<std::max(1, per_sm) * sms, CT_THREADS, smem, s>>>(tmX, tmXn, tmXid, Qp, qn, seed_d, mcoef,
                                                            meta, pid, qid, item_off, k0, K,
                                                            pair_out, qbound, bytes_ctr,
                                                            cm_tc_error_word());
    MASK_LAUNCHED("cm_tc_scan");
}
}  // namespace

void cm_tc_scan(const float *Xs, int64_t n, const float *xn, int dp, const int32_t *xids,
                const float *Qp, const float *qn, const float *seed_d, float mcoef,
                const int4 *meta, const int32_t *pid, const int32_t *qid, const int64_t *item_off,
                int k0, int K, int qs, unsigned long long *pair_out, unsigned *qbound,
                unsigned long long *bytes_ctr, cudaStream_t s) {
    MASK_REQUIRE(qs == kCmItemQueries || (qs == kCmTcItemQueries && K <= kCmTcWideMaxK),
                 "tensor-core leaf scan: unsupported item width");
    const CUtensorMap tmX = make_map_2d(Xs, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n, dp, CT_R, 32);
    const CUtensorMap tmXn = make_map_1d(xn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n, CT_NBOX);
    const CUtensorMap tmXid = make_map_1d(xids, CU_TENSOR_MAP_DATA_TYPE_INT32, 4, n, CT_NBOX);
    if (qs == kCmTcItemQueries)
        launch_cm_tc<32>(tmX, tmXn, tmXid, dp, Qp, qn, seed_d, mcoef, meta, pid, qid, item_off,
                         k0, K, pair_out, qbound, bytes_ctr, s);
    else
        launch_cm_tc<16>(tmX, tmXn, tmXid, dp, Qp, qn, seed_d, mcoef, meta, pid, qid, item_off,
                         k0, K, pair_out, qbound, bytes_ctr, s);
    t_cm_tc_launched = true;
}

}  // namespace mask
