// query_cm_tc.cu -- the cluster-major leaf scan (§3.3, Algorithm 2: rank the
// points of the kept leaf clusters, keep the k nearest) on the 5th-generation
// tensor cores, for rows of 32 or 64 floats, in two passes.
//
// 1. Filter (cm_tc_filter_kernel).  The work items of cm_scan_kernel
//    (query_cm.cu): a leaf cluster and up to QB (16 or 32) of the queries
//    that kept it.  Each 128-row chunk of the cluster is ranked by the
//    expanded form ||x||^2 + ||q||^2 - 2 x.q, and every (query, row) pair
//    whose value, less a proven rounding bound, can reach T_q (the K-th exact
//    distance within the query's nearest kept cluster, from the seed pass)
//    is appended to the query's candidate list.
// 2. Exact top-K (cm_exact_topk_kernel).  One warp per query takes the exact
//    difference-form key sum_t (x_t - q_t)^2 (increasing t, FMAs: the
//    arithmetic of the per-query scan) of each candidate and keeps the K
//    smallest keys.  Every row of the true K nearest passes the filter, so
//    the answer is the full exact scan's, bit for bit.  A query with more
//    candidates than its list holds is answered by the same warp from all
//    rows of its kept clusters.
//
// The dot products x.q run on tcgen05 (kind::tf32, M = 128 rows, N = QB
// queries, FP32 accumulation in tensor memory).  The rows go to the MMA as
// they were staged (FP32 containers, read as TF32, |x - x_tf32| <= 2^-10 |x|);
// each query is cut into q_hi = q with its low 13 mantissa bits cleared (a
// TF32 value, read exactly) and q_lo = q - q_hi (exact in FP32), and
//     x.q ~= x.q_hi + x.q_lo
// (two MMAs per K-step).  The filter's rounding bound covers the TF32 reading
// of x; it admits a few more pairs to the exact pass than an FP32 product
// would, and that pass is exact either way.
//
// Warp roles of the filter (one CTA per SM, persistent over the items of a
// grid stride):
//   warp 0      TMA producer: each chunk's rows (FP32, 128-byte swizzled
//               boxes of 32 columns) and their norms (a 1-D box) into a
//               4-stage shared-memory ring;
//   warp 1      MMA issuer (and tensor-memory owner: four accumulators);
//   warps 2-5   queries: each item's QB queries into shared memory (swizzled
//               hi/lo parts for the MMA), their norms, T_q and query ids,
//               one item ahead (three items in flight);
//   warps 6-13  epilogue: two warps per tensor-memory lane quadrant, each
//               one row per thread and QB / 2 of the query columns: the
//               filter and the appends.  No block-wide barrier: stages,
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
constexpr int CT_NQ = 3;                   // items in flight (query buffers)
constexpr int CT_QW0 = 2;                  // first query warp (four)
constexpr int CT_EPI0 = 6;                 // first epilogue warp
constexpr int CT_EPI_WARPS = 8;            // two per TMEM lane quadrant (QB / 2 query columns each)
constexpr int CT_THREADS = (CT_EPI0 + CT_EPI_WARPS) * 32;
constexpr uint32_t CT_BOX = CT_R * 128;    // 128 rows x 32 floats: 16 KB
constexpr int kCmTcWideMaxK = 16;          // largest K of the 32-query items
// Row norms of a chunk come with its rows, as a 1-D TMA box that starts at
// the chunk's first row rounded down to a multiple of 4 (16 bytes): 128 + 4
// elements, in a 128-byte aligned slot of 160 (a tensor copy's shared-memory
// destination is 128-byte aligned).
constexpr int CT_NBOX = CT_R + 4;
constexpr int CT_NSLOT = 160;

// The shapes that depend on the item width QB (queries per work item, the
// MMA's N: 16 or 32).
template <int QB>
struct CtShape {
    static_assert(QB == 16 || QB == 32, "items of 16 or 32 queries");
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
//   qhi   [NQ][NB][QBOX]                query hi parts, 128-byte swizzle
//   qlo   [NQ][NB][QBOX]                query lo parts
//   bars  full[S] sfree[S] accfull[NACC] accempty[NACC] qready[NQ] ldone[NQ]
template <int QB>
struct CtLayout {
    using SH = CtShape<QB>;
    uint32_t rows, qhi, qlo, bars, total;
    __host__ __device__ explicit CtLayout(int dp) {
        const uint32_t nb = (uint32_t)dp / 32;
        rows = 0;
        qhi = rows + CT_S * nb * CT_BOX;
        qlo = qhi + CT_NQ * nb * SH::QBOX;
        bars = qlo + CT_NQ * nb * SH::QBOX;
        total = bars + (2 * CT_S + 2 * CT_NACC + 2 * CT_NQ) * 8u;
    }
};

// The filter.  qn: query norms; seed_d [nq x K]: each query's K nearest
// distances within its nearest kept cluster (the K-th is T_q); mcoef: the
// filter's rounding bound per unit of ||x||^2 + ||q||^2; meta / qid /
// item_off: the work items (cm_item_meta, QB query slots per item);
// ccount [nq] (preset 0) / cand [nq x cap]: per query, the number of pairs
// that passed and the first cap of their rows (indices into the
// cluster-major rows).
template <int NB, int QB>
__global__ __launch_bounds__(CT_THREADS, 1) void cm_tc_filter_kernel(
    const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmXn,
    const float *__restrict__ Qp, const float *__restrict__ qn, const float *__restrict__ seed_d,
    float mcoef, const int4 *__restrict__ meta, const int32_t *__restrict__ qid,
    const int64_t *__restrict__ item_off, int k0, int K, unsigned *__restrict__ ccount,
    uint32_t *__restrict__ cand, int cap, unsigned long long *__restrict__ bytes_ctr,
    int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;   // swizzled tiles need 1 KB alignment
    unsigned char *basep = smem_raw + (base - raw);
    constexpr int dp = 32 * NB, nb = NB, dp4 = dp / 4;   // NB boxes of 32 floats
    using SH = CtShape<QB>;
    constexpr int EC = SH::EC;
    constexpr uint32_t QBOX = SH::QBOX;
    const CtLayout<QB> lay(dp);
    __shared__ __align__(16) float s_qn[CT_NQ][QB];
    __shared__ __align__(16) float s_tq[CT_NQ][QB];
    __shared__ int32_t s_qid[CT_NQ][QB];
    __shared__ __align__(128) float s_xn[CT_S][CT_NSLOT];   // per stage: the chunk's row norms
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
        for (int b = 0; b < CT_NQ; ++b) {
            mbar_init(qready(b), 4);
            mbar_init(ldone(b), CT_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
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
                    mbar_expect_tx(full(s), (uint32_t)nb * CT_BOX + CT_NBOX * 4u);
                    for (int h = 0; h < nb; ++h)
                        tma_load_2d(rows_at(s) + (uint32_t)h * CT_BOX, &tmX, 32 * h, (int)r0,
                                    full(s));
                    tma_load_1d(smem_u32(&s_xn[s][0]), &tmXn, (int)(r0 & ~3ll), full(s));
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
        // ---------------- queries (loaded one item ahead) ----------------
        constexpr int QR = QB / 16;                   // queries per thread (rounds of 16)
        const int tq = (warp - CT_QW0) * 32 + lane;   // 0..127
        const int q = tq >> 3, c = tq & 7;            // query (+ 16 per round), 16-byte column group of a box
        const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
        float4 nx[QR][NB];
#pragma unroll
        for (int rq = 0; rq < QR; ++rq)
#pragma unroll
            for (int h = 0; h < nb; ++h) nx[rq][h] = make_float4(0.f, 0.f, 0.f, 0.f);
        float nqn = 0.f, ntq = 0.f;
        int32_t nqid = 0;
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
                ntq = vv ? seed_d[(int64_t)q2 * K + K - 1] : 0.f;
                nqid = q2;
            }
        };
        auto next_item = [&](int64_t it) {   // the next item of this CTA with rows
            while (it < n_items && meta[it].z == 0) it += G;
            return it;
        };
        int64_t it = next_item(blockIdx.x), iseq = -1;
        if (it < n_items) fetch(it, ct_item(meta, it));
        bool ok = true;
        while (it < n_items) {
            ++iseq;
            const int b = (int)(iseq % CT_NQ);
            const int64_t nit = next_item(it + G);
            if (iseq >= CT_NQ) {
                // the buffer's previous item: the epilogue is done with it (and
                // so are its MMAs, whose results it read); the four query warps
                // agree before any of them overwrites the buffer
                const bool lok = __all_sync(
                    kFull, mbar_wait(ldone(b), (uint32_t)((iseq / CT_NQ - 1) & 1), err));
                ok = ct_q_bar_and(lok);
                if (!ok) break;
            }
            const CtItem im = ct_item(meta, it);
#pragma unroll
            for (int rq = 0; rq < QR; ++rq) {
                const int qr = q + 16 * rq;
#pragma unroll
                for (int h = 0; h < nb; ++h) {
                    const float4 x = nx[rq][h];
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
                s_qid[b][tq] = nqid;
            }
            if (bytes_ctr != nullptr && tq == 0)
                atomicAdd(bytes_ctr, (unsigned long long)im.rows * (dp * 4ull + 4ull));
            fence_proxy_async();   // the MMA reads the swizzled parts through the async proxy
            __syncwarp();
            if (lane == 0) mbar_arrive(qready(b));
            if (nit < n_items) fetch(nit, ct_item(meta, nit));   // in flight during the next wait
            it = nit;
        }
        if (!ok && lane == 0) s_err = 1;
    } else {
        // ------- epilogue: one chunk row per thread, QB / 2 of the query columns -------
        const int quad = warp & 3;
        const int r = quad * 32 + lane;             // the chunk row (TMEM lane) of this thread
        const int ew = warp - CT_EPI0;              // 0..7
        const int q0 = (ew >> 2) * EC;              // first query column of this warp
        const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
        int64_t j = 0, iseq = -1;
        bool ok = true;
        for (int64_t it = blockIdx.x; ok && it < n_items; it += G) {
            const CtItem im = ct_item(meta, it);
            if (im.rows == 0) continue;
            ++iseq;
            const int b = (int)(iseq % CT_NQ);
            const int nqb = im.nqb;
            // a failed wait ends the warp's work (the others learn of it
            // through their own wait limits and the abort word)
            bool wok = __all_sync(kFull, mbar_wait(qready(b), (uint32_t)((iseq / CT_NQ) & 1), err));
            // the item's per-query constants of this warp's columns: norms and
            // T_q (a pair passes where its expanded form can reach T_q)
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
                fence_after();
                uint32_t acc[EC];
                if constexpr (EC == 8)
                    tmem_ld8(lane_addr + (uint32_t)(QB * a + q0), acc);
                else
                    tmem_ld16(lane_addr + (uint32_t)(QB * a + q0), acc);
                // this row's norm (staged with the rows)
                const float xv = rv ? s_xn[s][(int)(r0 & 3) + r] : 0.f;
                tmem_wait();
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(accempty(a));   // the accumulator is in registers
                    mbar_arrive(sfree(s));      // the stage's rows were read by the MMAs, its norms here
                }
                // A (query, row) whose expanded form, less its rounding bound,
                // can reach T_q joins the query's candidates.
                uint32_t mask = 0;
#pragma unroll
                for (int cc = 0; cc < EC; ++cc) {
                    const float dv = fmaf(-2.f, __uint_as_float(acc[cc]), xv + qv[cc]);
                    const bool p = rv && q0 + cc < nqb && dv <= tqv[cc] + mcoef * (xv + qv[cc]);
                    mask |= p ? (1u << cc) : 0u;
                }
                while (mask) {
                    const int cc = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const int32_t qq = s_qid[b][q0 + cc];
                    const unsigned slot = atomicAdd(ccount + qq, 1u);
                    if (slot < (unsigned)cap) cand[(int64_t)qq * cap + slot] = (uint32_t)(r0 + r);
                }
            }
            // the item is done for this warp; its query buffer may be reused
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

// The exact pass: one warp per query.  Each lane keeps the KMAX smallest
// keys (exact distance bits << 32 | point id) of the rows it evaluates, in a
// sorted register list; K rounds of a warp-wide minimum then give the
// query's K nearest (missing places: id -1, distance +inf).  The rows are
// the query's candidates, or, where they overflowed (ccount > cap), every
// row of its kept leaf clusters.
template <int KMAX, int DP4>
__global__ __launch_bounds__(256) void cm_exact_topk_kernel(
    const float4 *__restrict__ Xs, const int32_t *__restrict__ xids,
    const int64_t *__restrict__ leaf_off, int k0, const float4 *__restrict__ Qp, int64_t nq,
    const int32_t *__restrict__ sel, int P, const unsigned *__restrict__ ccount,
    const uint32_t *__restrict__ cand, int cap, int K, int64_t *__restrict__ ids,
    float *__restrict__ dists) {
    constexpr int kWarps = 8, dp4 = DP4;
    __shared__ __align__(16) float4 s_q[kWarps][DP4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * kWarps + w;
    if (q >= nq) return;
    for (int c = lane; c < dp4; c += 32) s_q[w][c] = Qp[q * dp4 + c];
    __syncwarp();
    const float4 *qs = s_q[w];
    unsigned long long t[KMAX];
#pragma unroll
    for (int i = 0; i < KMAX; ++i) t[i] = kNoKey;
    // the key of a row (the arithmetic of the per-query scan), into the list;
    // the row's loads are all issued before its FMA chain
    auto eval = [&](int64_t row) {
        const float4 *xr = Xs + row * dp4;
        float4 xv[DP4];
#pragma unroll
        for (int c = 0; c < dp4; ++c) xv[c] = xr[c];
        const int32_t id = xids[row];
        float e2 = 0.f;
#pragma unroll
        for (int c = 0; c < dp4; ++c) {
            const float4 x4 = xv[c], b4 = qs[c];
            float d = x4.x - b4.x;
            e2 = fmaf(d, d, e2);
            d = x4.y - b4.y;
            e2 = fmaf(d, d, e2);
            d = x4.z - b4.z;
            e2 = fmaf(d, d, e2);
            d = x4.w - b4.w;
            e2 = fmaf(d, d, e2);
        }
        const unsigned long long key = ((unsigned long long)__float_as_uint(e2) << 32) | (uint32_t)id;
#pragma unroll
        for (int i = KMAX - 1; i > 0; --i)
            t[i] = t[i - 1] > key ? t[i - 1] : (t[i] > key ? key : t[i]);
        t[0] = t[0] < key ? t[0] : key;
    };
    const unsigned nc = ccount[q];
    if (nc <= (unsigned)cap) {
        const uint32_t *cq = cand + q * cap;
        for (unsigned i = lane; i < nc; i += 32) eval((int64_t)cq[i]);
    } else {
        for (int p = 0; p < P; ++p) {
            const int32_t cl = sel[q * P + p];
            if (cl < 0 || cl >= k0) continue;
            for (int64_t row = leaf_off[cl] + lane; row < leaf_off[cl + 1]; row += 32) eval(row);
        }
    }
    for (int rd = 0; rd < K; ++rd) {
        unsigned long long m = t[0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(kFull, m, o);
            m = v < m ? v : m;
        }
        // the lane holding the minimum at its head pops it (keys are distinct)
        if (t[0] == m && m != kNoKey) {
#pragma unroll
            for (int i = 0; i < KMAX - 1; ++i) t[i] = t[i + 1];
            t[KMAX - 1] = kNoKey;
        }
        if (lane == 0) {
            const bool ok = m != kNoKey;
            ids[q * K + rd] = ok ? (int64_t)(int32_t)(m & 0xffffffffu) : -1;
            if (dists)
                dists[q * K + rd] =
                    ok ? __uint_as_float((unsigned)(m >> 32)) : __int_as_float(0x7f800000);
        }
    }
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

int cm_tc_item_queries(int K) { return K <= kCmTcWideMaxK ? kCmTcItemQueries : kCmItemQueries; }

// MASK_CM_CAND_CAP overrides the capacity (tests of the overflow path)
int cm_tc_cand_cap(int64_t nq) {
    if (const char *e = std::getenv("MASK_CM_CAND_CAP")) {
        const int v = std::atoi(e);
        if (v >= 1) return v;
    }
    return nq <= 16384 ? 4096 : (nq <= 65536 ? 1024 : 256);
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

namespace {
template <int QB>
void launch_cm_tc_filter(const CUtensorMap &tmX, const CUtensorMap &tmXn, int dp, const float *Qp,
                         const float *qn, const float *seed_d, float mcoef, const int4 *meta,
                         const int32_t *qid, const int64_t *item_off, int k0, int K,
                         unsigned *ccount, uint32_t *cand, int cap,
                         unsigned long long *bytes_ctr, cudaStream_t s) {
    const CtLayout<QB> lay(dp);
    const size_t smem = (size_t)lay.total + 1024;
    auto kfn = dp == 32 ? cm_tc_filter_kernel<1, QB> : cm_tc_filter_kernel<2, QB>;
    cudaFuncAttributes fa;
    MASK_CUDA(cudaFuncGetAttributes(&fa, kfn));
    MASK_REQUIRE(smem + fa.sharedSizeBytes <= 227u * 1024u,
                 "tensor-core leaf scan: shared memory over 227 KB");
    MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    MASK_CUDA(cudaGetDevice(&dev));
    MASK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MASK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, CT_THREADS, smem));
    kfn<<<std::max(1, per_sm) * sms, CT_THREADS, smem, s>>>(tmX, tmXn, Qp, qn, seed_d, mcoef, meta,
                                                            qid, item_off, k0, K, ccount, cand,
                                                            cap, bytes_ctr, cm_tc_error_word());
    MASK_LAUNCHED("cm_tc_filter");
}
}  // namespace

void cm_tc_scan(const float *Xs, int64_t n, const float *xn, int dp, const int32_t *xids,
                const int64_t *leaf_off, int k0, const float *Qp, int64_t nq, const int32_t *sel,
                int P, const float *qn, const float *seed_d, float mcoef, const int4 *meta,
                const int32_t *qid, const int64_t *item_off, int K, int qs, unsigned *ccount,
                uint32_t *cand, int cap, int64_t *ids, float *dists,
                unsigned long long *bytes_ctr, cudaStream_t s) {
    MASK_REQUIRE(qs == kCmItemQueries || (qs == kCmTcItemQueries && K <= kCmTcWideMaxK),
                 "tensor-core leaf scan: unsupported item width");
    MASK_REQUIRE(K >= 1 && K <= 32 && (dp == 32 || dp == 64),
                 "tensor-core leaf scan: K or d out of range");
    MASK_REQUIRE(n < ((int64_t)1 << 31), "tensor-core leaf scan: at most 2^31 - 1 rows");
    const CUtensorMap tmX = make_map_2d(Xs, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n, dp, CT_R, 32);
    const CUtensorMap tmXn = make_map_1d(xn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, n, CT_NBOX);
    {
        ProfRegion pr("scan_leaf_cm", s, 0.0);
        if (qs == kCmTcItemQueries)
            launch_cm_tc_filter<32>(tmX, tmXn, dp, Qp, qn, seed_d, mcoef, meta, qid, item_off, k0,
                                    K, ccount, cand, cap, bytes_ctr, s);
        else
            launch_cm_tc_filter<16>(tmX, tmXn, dp, Qp, qn, seed_d, mcoef, meta, qid, item_off, k0,
                                    K, ccount, cand, cap, bytes_ctr, s);
    }
    {
        ProfRegion pr("leaf_exact", s, 0.0);
        const unsigned blocks = (unsigned)((nq + 7) / 8);
        const float4 *X4 = reinterpret_cast<const float4 *>(Xs);
        const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
        auto kfn = K <= 16 ? (dp == 32 ? cm_exact_topk_kernel<16, 8> : cm_exact_topk_kernel<16, 16>)
                           : (dp == 32 ? cm_exact_topk_kernel<32, 8> : cm_exact_topk_kernel<32, 16>);
        kfn<<<blocks, 256, 0, s>>>(X4, xids, leaf_off, k0, Q4, nq, sel, P, ccount, cand, cap, K,
                                   ids, dists);
        MASK_LAUNCHED("cm_exact_topk");
    }
    t_cm_tc_launched = true;
}

}  // namespace mask
