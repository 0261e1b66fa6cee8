// assign_tc.cu -- Lloyd assignment half-step (§2.4) on the 5th-generation
// tensor cores: labels[i] = argmin_j ||x_i - c_j||^2, ties to the smallest j.
//
// Distances in the expanded form ||x||^2 - 2 x.c + ||c||^2.  The cross term
// x.c is a GEMM on tcgen05 (kind::f16: FP16 operands, FP32 accumulation in
// tensor memory) made FP32-accurate by a three-product split (the scheme of
// Ootomo & Yokota 2022, "Recovering single precision accuracy from Tensor
// Cores while surpassing the FP32 theoretical peak performance", on FP16):
// every row of X is scaled by a power of two s_i that puts its largest
// coordinate in [2^14, 2^15), C by one power of two s_c for all of it, and a
// scaled value v = x*s splits into v_hi = fp16(v) and v_lo = fp16(v - v_hi),
//     (x.c) s_i s_c ~= x_hi.c_hi + x_hi.c_lo + x_lo.c_hi,
// with each fp16 x fp16 product exact in FP32.  The scales are powers of two,
// so undoing them in the epilogue is exact; FP16 runs the tensor pipe at
// twice the TF32 rate, and the split keeps 22 bits of each operand.
//
// One CTA owns 128 rows of X.  Their hi/lo parts sit in tensor memory as
// the MMAs' A operand (so shared memory feeds only the B operand) while
// 192-centroid tiles of C stream through a TMA pipeline; the accumulator is
// double-buffered in TMEM so the epilogue of tile j overlaps the MMAs of the
// next one.  An M = 128 kind::f16 MMA takes about as long at N = 192 as at
// N = 128 (its issue cost, not its arithmetic, bounds it below N ~ 200), so
// the wider tile does 1.5x the work per MMA; 2 x 192 accumulator columns and
// the rows' 64 leave room in the 512 columns of tensor memory.
// Warp roles: warp 0 = TMA producer (C tiles and their norms), warp 1 = MMA
// issuer, warp 2 = TMEM allocator, warps 4-11 = epilogue (one thread per row
// and half of each tile's columns, TMEM lane = row), which keeps the four
// smallest distances of its row over all k centroids.
//
// A row's label is certain when its best and second-best distances differ by
// more than twice the error bound of the expanded form; otherwise the row is
// re-decided exactly in the difference form sum_t (x_t - c_t)^2, over its
// three best candidates when the fourth is clear of the bound, else over all
// centroids.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cfloat>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc_common.cuh"

namespace mask {
namespace {

using namespace tc;

constexpr unsigned kFull = 0xffffffffu;
constexpr int TC_M = 128, TC_N = 192;   // MMA tile: 128 rows x 192 centroids
constexpr int TC_EPI_PARTS = 2;         // epilogue warps per TMEM lane quadrant (column parts)
constexpr int TC_EPI_WARPS = 4 * TC_EPI_PARTS;
constexpr int TC_THREADS = (4 + TC_EPI_WARPS) * 32;
constexpr int TC_EPI_COLS = TC_N / TC_EPI_PARTS;   // columns per epilogue thread per tile
constexpr int TC_EPI_LD = TC_EPI_COLS / 32;        // 32-column TMEM loads per thread per tile
constexpr int TC_EPI_G = TC_EPI_COLS / 8;          // groups of 8 columns per thread per tile
constexpr int TC_DK = 64;               // fp16 columns of the split copies (dp <= 64)
constexpr int TC_CBOX_BYTES = TC_N * TC_DK * 2;     // one C tile part, 128-byte rows: 24 KB
constexpr int TC_NRING = 8;             // slots of the centroid-norm ring
constexpr int TC_NACC = 2;              // accumulator buffers in tensor memory
constexpr uint32_t TC_ACOL = TC_NACC * TC_N;  // tensor-memory column of the rows' hi/lo parts
static_assert(TC_ACOL + TC_DK <= 512, "accumulators and rows fit the 512 TMEM columns");

// instruction descriptor: D = F32, A = B = F16, both K-major, N = 192, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(TC_N >> 3) << 17) |
                            ((uint32_t)(TC_M >> 4) << 24);

// D (+)= A.B^T on tcgen05 (kind::f16, FP32 accumulation in tensor memory),
// with the A operand in tensor memory (row i in lane i, two fp16 values of
// consecutive K per 32-bit column, lower K in the low half) and B in shared
// memory (descriptor).
__device__ __forceinline__ void mma_f16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// Named barrier 1 over the epilogue threads (warps 4 and up) that also ANDs a
// flag across them, so every epilogue warp takes the same exit decision.
__device__ __forceinline__ bool epi_bar_and(bool v) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)v), "n"(TC_EPI_WARPS * 32)
        : "memory");
    return out != 0;
}

// Keep the four smallest values (v0 <= v1 <= v2 <= v3) and the indices of
// the first three; strict comparisons keep the earliest index on ties.
struct Top4 {
    float v0, v1, v2, v3;
    int i0, i1, i2;
    __device__ void init() {
        v0 = v1 = v2 = v3 = FLT_MAX;
        i0 = i1 = i2 = -1;
    }
    __device__ __forceinline__ void push(float d, int j) {
        if (d < v3) {
            if (d < v2) {
                v3 = v2;
                if (d < v1) {
                    v2 = v1; i2 = i1;
                    if (d < v0) { v1 = v0; i1 = i0; v0 = d; i0 = j; }
                    else { v1 = d; i1 = j; }
                } else { v2 = d; i2 = j; }
            } else { v3 = d; }
        }
    }
    // The same insertion without branches (a no-op when d >= v3): with the
    // list sorted, d < v0 implies d < v1 implies d < v2.
    __device__ __forceinline__ void push_nb(float d, int j) {
        const bool c0 = d < v0, c1 = d < v1, c2 = d < v2;
        v3 = c2 ? v2 : fminf(v3, d);
        v2 = c1 ? v1 : (c2 ? d : v2);
        i2 = c1 ? i1 : (c2 ? j : i2);
        v1 = c0 ? v0 : (c1 ? d : v1);
        i1 = c0 ? i0 : (c1 ? j : i1);
        v0 = c0 ? d : v0;
        i0 = c0 ? j : i0;
    }
};

// ------------------------------------------------------------- main kernel

// ksteps = K-steps of 16 fp16 columns (ceil(dp / 16)); xinv[i] = 1 / s_i,
// cinv[0] = 1 / s_c (the scales of the split copies).  When `seeded`, labels
// holds each row's previous label on entry (Xf, Cf: the padded FP32 rows and
// centroids, dp4 float4s each).
template <int S>
__global__ __launch_bounds__(TC_THREADS, 1) void assign_tc_kernel(
    const uint4 *__restrict__ Xh, const uint4 *__restrict__ Xl, const float4 *__restrict__ Xf,
    const float4 *__restrict__ Cf, int dp4, int seeded,
    const __grid_constant__ CUtensorMap tmCh, const __grid_constant__ CUtensorMap tmCl,
    const float *__restrict__ xn, const float *__restrict__ xinv, const float *__restrict__ cinv,
    int64_t n, int ksteps, const float *__restrict__ cn_pad, int k,
    const float *__restrict__ cn_max, float margin_coef, int32_t *__restrict__ labels,
    int4 *__restrict__ list3, int *__restrict__ n3, int32_t *__restrict__ listF,
    int *__restrict__ nF, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr uint32_t kStage = 2u * TC_CBOX_BYTES;      // hi + lo tiles of one C tile
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;        // swizzled tiles need 1 KB alignment
    unsigned char *basep = smem_raw + (base - raw);
    const uint32_t B0 = base;
    uint64_t *bars = reinterpret_cast<uint64_t *>(basep + S * kStage);
    uint32_t *tmem_slot =
        reinterpret_cast<uint32_t *>(bars + 2 * S + 1 + 2 * TC_NACC + 2 * TC_NRING);
    __shared__ int s_err;
    __shared__ __align__(16) float s_cn[TC_NRING][TC_N];   // norms of the C tiles in flight
    __shared__ float s_top[TC_EPI_PARTS - 1][TC_M][4];   // parts 1.. top-4 lists, merged at the end
    __shared__ int s_topi[TC_EPI_PARTS - 1][TC_M][3];
    __shared__ float s_thr[TC_EPI_PARTS][TC_M];          // each part's current fourth value

    // barriers: a_full | b_full[S] | b_empty[S] | acc_full[TC_NACC] |
    //           acc_empty[TC_NACC] | n_full[TC_NRING] | n_empty[TC_NRING]
    const uint32_t bar0 = smem_u32(bars);
    const uint32_t a_full = bar0;
    auto b_full = [&](int s) { return bar0 + 8u * (1 + s); };
    auto b_empty = [&](int s) { return bar0 + 8u * (1 + S + s); };
    auto acc_full = [&](int a) { return bar0 + 8u * (1 + 2 * S + a); };
    auto acc_empty = [&](int a) { return bar0 + 8u * (1 + TC_NACC + 2 * S + a); };
    auto n_full = [&](int q) { return bar0 + 8u * (1 + 2 * TC_NACC + 2 * S + q); };
    auto n_empty = [&](int q) { return bar0 + 8u * (1 + 2 * TC_NACC + 2 * S + TC_NRING + q); };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;
    const int ntiles = (k + TC_N - 1) / TC_N;

    // a CTA that starts after the grid aborted does nothing
    if (*(volatile int *)err != 0) return;
    for (int i = threadIdx.x; i < TC_EPI_PARTS * TC_M; i += TC_THREADS)
        (&s_thr[0][0])[i] = FLT_MAX;
    if (threadIdx.x == 0) {
        s_err = 0;
        mbar_init(a_full, 4);   // the four warps that write the rows into tensor memory
        for (int s = 0; s < S; ++s) {
            mbar_init(b_full(s), 1);
            mbar_init(b_empty(s), 1);
        }
        for (int a = 0; a < TC_NACC; ++a) {
            mbar_init(acc_full(a), 1);
            mbar_init(acc_empty(a), TC_EPI_WARPS);
        }
        for (int q = 0; q < TC_NRING; ++q) {
            mbar_init(n_full(q), 1);
            mbar_init(n_empty(q), TC_EPI_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        int armed = 0, armedN = 0;
        bool ok = true;
        for (int j = 0; j < ntiles; ++j) {
            const int s = j % S, u = j / S;
            if (u > 0 && !mbar_wait(b_empty(s), (u - 1) & 1, err)) { ok = false; break; }
            const uint32_t bh = B0 + s * kStage, bl = bh + TC_CBOX_BYTES;
            mbar_expect_tx(b_full(s), kStage);
            tma_load_2d(bh, &tmCh, 0, j * TC_N, b_full(s));
            tma_load_2d(bl, &tmCl, 0, j * TC_N, b_full(s));
            armed = j + 1;
            // the tile's 128 norms (the ring is 8 tiles deep, far ahead of the epilogue)
            const int q = j % TC_NRING, w = j / TC_NRING;
            if (w > 0 && !mbar_wait(n_empty(q), (w - 1) & 1, err)) { ok = false; break; }
            mbar_expect_tx(n_full(q), TC_N * 4u);
            bulk_load(smem_u32(&s_cn[q][0]), cn_pad + (int64_t)j * TC_N, TC_N * 4u, n_full(q));
            armedN = j + 1;
        }
        // every load this thread issued must land before the CTA may exit
        for (int j = (armed > S ? armed - S : 0); j < armed; ++j)
            mbar_wait(b_full(j % S), (j / S) & 1, err, true);
        for (int j = (armedN > TC_NRING ? armedN - TC_NRING : 0); j < armedN; ++j)
            mbar_wait(n_full(j % TC_NRING), (j / TC_NRING) & 1, err, true);
        if (!ok) s_err = 1;
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        // the CTA's rows are in tensor memory (columns TC_ACOL..): hi parts
        // first, then lo parts, 8 columns (16 fp16 values) per K-step
        bool ok = mbar_wait(a_full, 0, err);
        fence_after();
        const uint32_t tAh = tmem + TC_ACOL, tAl = tmem + TC_ACOL + TC_DK / 2;
        int last = -1;
        for (int j = 0; ok && j < ntiles; ++j) {
            const int s = j % S, u = j / S, a = j % TC_NACC, v = j / TC_NACC;
            ok = mbar_wait(b_full(s), u & 1, err);
            if (ok && v > 0) ok = mbar_wait(acc_empty(a), (v - 1) & 1, err);
            if (!ok) break;
            fence_after();
            const uint32_t d = tmem + (uint32_t)(a * TC_N);
            const uint32_t bh = B0 + s * kStage, bl = bh + TC_CBOX_BYTES;
            const uint64_t dBh = sw128_desc(bh), dBl = sw128_desc(bl);
            // K-step kk covers fp16 columns 16kk..16kk+15: 32 bytes into each
            // 128-byte row, i.e. +2 in the descriptor's 16-byte address units
#pragma unroll
            for (int kk = 0; kk < TC_DK / 16; ++kk) {
                if (kk < ksteps) {
                    const uint64_t off = (uint64_t)(kk * 2);
                    const uint32_t ta = (uint32_t)(kk * 8);
                    mma_f16_ta(d, tAh + ta, dBh + off, kk > 0 ? 1u : 0u);
                    mma_f16_ta(d, tAh + ta, dBl + off, 1u);
                    mma_f16_ta(d, tAl + ta, dBh + off, 1u);
                }
            }
            mma_commit(b_empty(s));    // the C tile's stage is free once these MMAs finish
            mma_commit(acc_full(a));   // accumulator a is ready for the epilogue
            last = j;
        }
        // the MMAs must be complete before tensor memory is released
        if (last >= 0) mbar_wait(acc_full(last % TC_NACC), (last / TC_NACC) & 1, err, true);
        if (!ok) s_err = 1;
    } else if (warp >= 4) {
        // ------------ epilogue: one row per thread, half of each tile's columns ------------
        // Rows are ranked by key = ||c||^2 - 2 x.c (the row's ||x||^2 is
        // added back at the end); the norms of each C tile arrive in a ring
        // of shared-memory slots filled by the producer.  The accumulator
        // holds (x.c) s_i s_c: the factor -2 / (s_i s_c) is a power of two,
        // so the scaling costs no rounding.
        const int quad = warp & 3;                  // TMEM lane quadrant of this warp
        const int part = (warp - 4) >> 2;           // column part of each tile
        const int col = part * TC_EPI_COLS;
        const int r = quad * 32 + lane;
        const int64_t row = row0 + r;
        const float xr = row < n ? xn[row] : 0.f;
        const float mul = row < n ? -2.f * xinv[row] * cinv[0] : 0.f;
        if (part == 0) {
            // the row's hi and lo parts into its tensor-memory lane (rows
            // past n are zero)
            const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16) + TC_ACOL;
            uint32_t hv[32];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 *src = (h == 0 ? Xh : Xl) + row * (TC_DK / 8);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint4 w = row < n ? src[c] : make_uint4(0u, 0u, 0u, 0u);
                    hv[4 * c] = w.x; hv[4 * c + 1] = w.y; hv[4 * c + 2] = w.z; hv[4 * c + 3] = w.w;
                }
                tmem_st32(lane_addr + (uint32_t)(h * (TC_DK / 2)), hv);
            }
            tmem_wait_st();
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(a_full);
        }
        // Seed of the row's threshold from its previous label j': only keys
        // below key(j') + 2 * margin can decide the label, its gap test or
        // its re-decision list (a key above it is more than a margin behind
        // the best, which is at most key(j')).  key(j') is taken in the exact
        // difference form; its FP32 error and that of the tensor-core key are
        // each within a quarter and three quarters of one margin.
        float T0 = FLT_MAX;
        if (seeded && row < n) {
            const int jp = labels[row];
            if (jp >= 0 && jp < k) {
                const float4 *xa = Xf + row * dp4, *ca = Cf + (int64_t)jp * dp4;
                float acc = 0.f;
                for (int c = 0; c < dp4; ++c) {
                    const float4 e = xa[c], f = ca[c];
                    const float e0 = e.x - f.x, e1 = e.y - f.y, e2 = e.z - f.z, e3 = e.w - f.w;
                    acc = fmaf(e0, e0, acc);
                    acc = fmaf(e1, e1, acc);
                    acc = fmaf(e2, e2, acc);
                    acc = fmaf(e3, e3, acc);
                }
                T0 = (acc - xr) + 2.f * margin_coef * (xr + *cn_max);
            }
        }
        Top4 t4;
        t4.init();
        bool ok = true;
        for (int j = 0; j < ntiles; ++j) {
            const int a = j % TC_NACC, v = j / TC_NACC;
            const int q = j % TC_NRING, w = j / TC_NRING;
            ok = mbar_wait(acc_full(a), v & 1, err) && mbar_wait(n_full(q), w & 1, err);
            if (!__all_sync(kFull, ok)) { ok = false; break; }  // the warp leaves as one
            fence_after();
            const uint32_t taddr =
                tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * TC_N + col);
            uint32_t u[TC_EPI_LD][32];
#pragma unroll
            for (int h = 0; h < TC_EPI_LD; ++h) tmem_ld32(taddr + 32 * h, u[h]);
            tmem_wait();
            // the accumulator is in registers: hand the buffer back to the MMA warp
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(a));
            // keys of this thread's columns, with the minimum of each group
            // of 8; columns past k have norm +inf, so their keys never enter
            // the list
            // (computed in place: key 8g + e lives in u's register of its column)
            const float4 *cn4 = reinterpret_cast<const float4 *>(&s_cn[q][col]);
            float gm[TC_EPI_G];
#pragma unroll
            for (int g = 0; g < TC_EPI_G; ++g) {
                uint32_t *uu = u[g >> 2] + (g & 3) * 8;
                const float4 c0v = cn4[2 * g], c1v = cn4[2 * g + 1];
                float kk[8];
                kk[0] = fmaf(mul, __uint_as_float(uu[0]), c0v.x);
                kk[1] = fmaf(mul, __uint_as_float(uu[1]), c0v.y);
                kk[2] = fmaf(mul, __uint_as_float(uu[2]), c0v.z);
                kk[3] = fmaf(mul, __uint_as_float(uu[3]), c0v.w);
                kk[4] = fmaf(mul, __uint_as_float(uu[4]), c1v.x);
                kk[5] = fmaf(mul, __uint_as_float(uu[5]), c1v.y);
                kk[6] = fmaf(mul, __uint_as_float(uu[6]), c1v.z);
                kk[7] = fmaf(mul, __uint_as_float(uu[7]), c1v.w);
#pragma unroll
                for (int e = 0; e < 8; ++e) uu[e] = __float_as_uint(kk[e]);
                gm[g] = fminf(fminf(fminf(kk[0], kk[1]), fminf(kk[2], kk[3])),
                              fminf(fminf(kk[4], kk[5]), fminf(kk[6], kk[7])));
            }
            auto key = [&](int c) { return __uint_as_float(u[c >> 5][c & 31]); };
            // the norms are in registers: hand the ring slot back
            __syncwarp();
            if (lane == 0) mbar_arrive(n_empty(q));
            float mn = gm[0];
#pragma unroll
            for (int g = 1; g < TC_EPI_G; ++g) mn = fminf(mn, gm[g]);
            // A key enters only below the row's threshold: the smallest of
            // the parts' fourth values (each is at least the fourth smallest
            // key over all columns seen, so no key of the final four is lost).
            float T = fminf(T0, t4.v3);
#pragma unroll
            for (int pp = 0; pp < TC_EPI_PARTS; ++pp)
                if (pp != part) T = fminf(T, s_thr[pp][r]);
            // insertions in column order (ties keep the earliest column),
            // under warp-uniform branches only.  A group is visited when some
            // lane has a key in it below that lane's threshold; when no lane
            // has more than one such key, each lane inserts just its group
            // minimum (a no-op where it is not below the fourth), otherwise
            // all eight keys go through the branch-free insertion.
            if (__any_sync(kFull, mn < T)) {
                const int cb = j * TC_N + col;
#pragma unroll
                for (int g = 0; g < TC_EPI_G; ++g) {
                    if (__any_sync(kFull, gm[g] < T)) {
                        int cnt = 0, first = 7;
#pragma unroll
                        for (int e = 7; e >= 0; --e) {
                            cnt += key(8 * g + e) < T ? 1 : 0;
                            first = key(8 * g + e) == gm[g] ? e : first;
                        }
                        if (__any_sync(kFull, cnt > 1)) {
#pragma unroll
                            for (int e = 0; e < 8; ++e)
                                if (key(8 * g + e) < T) t4.push_nb(key(8 * g + e), cb + 8 * g + e);
                        } else if (gm[g] < T) {
                            t4.push_nb(gm[g], cb + 8 * g + first);
                        }
                    }
                }
                s_thr[part][r] = t4.v3;
            }
        }
        // merge the row's part lists: parts 1.. hand their lists to part 0.
        // A part's fourth value enters after its first three, so it can only
        // land in the fourth place (whose index is never used).
        if (part > 0) {
            float *t = s_top[part - 1][r];
            int *ti = s_topi[part - 1][r];
            t[0] = t4.v0; t[1] = t4.v1; t[2] = t4.v2; t[3] = t4.v3;
            ti[0] = t4.i0; ti[1] = t4.i1; ti[2] = t4.i2;
        }
        ok = epi_bar_and(ok);
        if (part > 0) {
            // nothing more to do
        } else if (!ok) {
            s_err = 1;
        } else {
#pragma unroll
            for (int pp = 0; pp < TC_EPI_PARTS - 1; ++pp) {
                t4.push(s_top[pp][r][0], s_topi[pp][r][0]);
                t4.push(s_top[pp][r][1], s_topi[pp][r][1]);
                t4.push(s_top[pp][r][2], s_topi[pp][r][2]);
                t4.push(s_top[pp][r][3], -1);
            }
        }
        if (part == 0 && ok && row < n) {
            labels[row] = t4.i0;
            // gaps are the same in key and distance units
            const float margin = margin_coef * (xr + *cn_max);
            if (k > 1 && !(t4.v1 - t4.v0 > margin)) {
                if (k <= 3 || t4.v3 - t4.v0 > margin) {
                    const int slot = atomicAdd(n3, 1);
                    list3[slot] = make_int4((int)row, t4.i0, t4.i1, t4.i2);
                } else {
                    listF[atomicAdd(nF, 1)] = (int32_t)row;
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
    if (threadIdx.x == 0 && s_err) atomicExch(err, 1);
}

// Exact re-decision among a row's three best candidates (difference form).
template <int LPR>
__global__ __launch_bounds__(256) void recheck3_kernel(const float4 *__restrict__ X, int dp4,
                                                       const float4 *__restrict__ C,
                                                       const int4 *__restrict__ list,
                                                       const int *__restrict__ count,
                                                       int32_t *__restrict__ labels) {
    constexpr int GPW = 32 / LPR;  // lane groups per warp
    const int lane = threadIdx.x & 31, g = lane / LPR, gl = lane % LPR;
    const int wpb = blockDim.x / 32;
    const int cnt = *count;
    for (int e = blockIdx.x * wpb + (threadIdx.x >> 5); e < cnt; e += gridDim.x * wpb) {
        const int4 it = list[e];
        const float4 *xr = X + (int64_t)it.x * dp4;
        unsigned long long best = kNoKey;
        for (int c0 = 0; c0 < 3; c0 += GPW) {
            const int ci = c0 + g;
            const int j = ci == 0 ? it.y : (ci == 1 ? it.z : (ci == 2 ? it.w : -1));
            float acc = 0.f;
            if (j >= 0) {
                const float4 *cr = C + (int64_t)j * dp4;
                for (int c = gl; c < dp4; c += LPR) {
                    const float4 a = xr[c], b = cr[c];
                    const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
                    acc = fmaf(e0, e0, acc);
                    acc = fmaf(e1, e1, acc);
                    acc = fmaf(e2, e2, acc);
                    acc = fmaf(e3, e3, acc);
                }
            }
            for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if (j >= 0)
                best = min(best, ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)j);
        }
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
        if (lane == 0) labels[it.x] = (int32_t)(best & 0xffffffffu);
    }
}

// Exponent e of a positive finite float m with 2^e <= m < 2^(e+1); values
// below the normal range count as 2^-127.
__device__ __forceinline__ int exponent_of(float m) {
    const int b = (int)((__float_as_uint(m) >> 23) & 0xffu);
    return b == 0 ? -127 : b - 127;
}

// 2^e as a float, for e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Split copies for the FP16 three-product scheme: v = x * s with s a power of
// two that puts m (the row's largest |x|, or *global_max for all rows) in
// [2^14, 2^15); hi = fp16(v), lo = fp16(v - hi) (v - hi is exact in FP32).
// hi, lo are [rows x 64] (columns dp..63 zero); inv_scale[row] = 1 / s (one
// value, inv_scale[0], when global_max is given).  Eight lanes per row, eight
// columns each.
__global__ void split_f16_kernel(const float *__restrict__ src, int64_t rows, int dp,
                                 const unsigned *__restrict__ global_max, __half *__restrict__ hi,
                                 __half *__restrict__ lo, float *__restrict__ inv_scale) {
    const int l = threadIdx.x & 7;
    // the loop runs warp-uniformly (the shuffles below need all 32 lanes);
    // a warp covers 4 rows per pass, lanes past the last row idle
    const int64_t warp_rows = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32 * 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x / 32 * 4;
    for (int64_t rb = warp_rows; rb < rows; rb += stride) {
        const int64_t r = rb + (threadIdx.x & 31) / 8;
        const bool live = r < rows;
        float v[8];
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int col = l * 8 + c;
            v[c] = live && col < dp ? src[r * dp + col] : 0.f;
            m = fmaxf(m, fabsf(v[c]));
        }
        if (global_max != nullptr) {
            m = __uint_as_float(*global_max);
        } else {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1, 8));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2, 8));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4, 8));
        }
        int e = m > 0.f ? 14 - exponent_of(m) : 0;
        e = e < -126 ? -126 : (e > 126 ? 126 : e);
        const float sc = pow2f(e);
        alignas(16) __half h8[8], l8[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float x = v[c] * sc;
            const __half h = __float2half_rn(x);
            h8[c] = h;
            l8[c] = __float2half_rn(x - __half2float(h));
        }
        if (!live) continue;
        *reinterpret_cast<uint4 *>(hi + r * TC_DK + l * 8) = *reinterpret_cast<const uint4 *>(h8);
        *reinterpret_cast<uint4 *>(lo + r * TC_DK + l * 8) = *reinterpret_cast<const uint4 *>(l8);
        if (l == 0 && (global_max == nullptr || r == 0)) inv_scale[global_max ? 0 : r] = pow2f(-e);
    }
}

// *out = max |v| (as float bits; *out must start at 0).
__global__ void absmax_kernel(const float *__restrict__ v, int64_t count, unsigned *out) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(v[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// Norms of the padding columns of the last C tile: +inf, so their
// keys (-2 * 0 + inf) never enter a row's list.
__global__ void pad_inf_kernel(float *__restrict__ cn, int k, int total) {
    const int i = k + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) cn[i] = __int_as_float(0x7f800000);
}

// 2-D tensor map of a [rows x 64] fp16 array, boxes of TC_N rows x 64 columns
// (one 128-byte row each), 128-byte swizzle, zero fill out of bounds.
CUtensorMap make_map(const __half *base, int64_t rows) {
    return tc::make_map_2d(base, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, rows, TC_DK, TC_N, TC_DK);
}

int grid_cap(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

template <int S>
size_t tc_smem_bytes() {
    return 1024 + (size_t)S * 2u * TC_CBOX_BYTES + (2 * S + 1 + 2 * TC_NACC + 2 * TC_NRING) * 8 +
           16;
}

constexpr int TC_STAGES = 4;   // C tiles in flight (48 KB each)

}  // namespace

// ================================================================= host side

struct TcAssign {
    int64_t n = 0;
    int dp = 0;
    const float *X = nullptr;      // padded points [n x dp]
    Scratch<__half> Xh, Xl;        // [n x 64] scaled FP16 hi / lo parts
    Scratch<float> xinv;           // [n] 1 / s_i (powers of two)
    Scratch<int> err;              // set by a kernel whose bounded wait ran out
};

bool tc_assign_enabled(int dp) {
    const char *e = std::getenv("MASK_ASSIGN_KERNEL");
    if (e && std::strcmp(e, "simt") == 0) return false;
    return dp <= 64 && encode_fn() != nullptr;
}

std::shared_ptr<TcAssign> tc_assign_prepare(const float *X, int64_t n, int dp, cudaStream_t s) {
    if (n == 0 || !tc_assign_enabled(dp)) return nullptr;
    auto p = std::make_shared<TcAssign>();
    p->n = n;
    p->dp = dp;
    p->X = X;
    p->Xh.alloc((size_t)n * TC_DK, s);
    p->Xl.alloc((size_t)n * TC_DK, s);
    p->xinv.alloc((size_t)n, s);
    split_f16_kernel<<<grid_cap(n * 8), 256, 0, s>>>(X, n, dp, nullptr, p->Xh.get(), p->Xl.get(),
                                                     p->xinv.get());
    MASK_LAUNCHED("split_f16");
    p->err.alloc(1, s);
    MASK_CUDA(cudaMemsetAsync(p->err.get(), 0, sizeof(int), s));
    return p;
}

template <int S>
void launch_tc(const TcAssign &p, const CUtensorMap &mCh, const CUtensorMap &mCl, const float *C,
               bool seeded, const float *xn, const float *cinv, const float *cn, int k,
               const float *cmax, float coef, int32_t *labels, int4 *list3, int *n3,
               int32_t *listF, int *nF, cudaStream_t s) {
    const size_t smem = tc_smem_bytes<S>();
    auto kfn = assign_tc_kernel<S>;
    MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned blocks = (unsigned)((p.n + TC_M - 1) / TC_M);
    kfn<<<blocks, TC_THREADS, smem, s>>>(reinterpret_cast<const uint4 *>(p.Xh.get()),
                                        reinterpret_cast<const uint4 *>(p.Xl.get()),
                                        reinterpret_cast<const float4 *>(p.X),
                                        reinterpret_cast<const float4 *>(C), p.dp / 4,
                                        seeded ? 1 : 0, mCh, mCl, xn, p.xinv.get(), cinv, p.n,
                                        (p.dp + 15) / 16, cn, k, cmax, coef, labels, list3, n3,
                                        listF, nF, p.err.get());
}

void tc_assign(TcAssign &p, const float *xn, const float *C, int k, int32_t *labels,
               bool seeded, cudaStream_t s) {
    const int dp = p.dp;
    const int ntiles = (k + TC_N - 1) / TC_N;
    // centroid norms padded to whole C tiles (+inf past k)
    Scratch<float> cn((size_t)ntiles * TC_N, s), cmax(1, s), cinv(1, s);
    Scratch<__half> Ch((size_t)k * TC_DK, s), Cl((size_t)k * TC_DK, s);
    Scratch<unsigned> cabs(1, s);
    Scratch<int4> list3(p.n, s);
    Scratch<int32_t> listF(p.n, s);
    Scratch<int> counts(2, s);
    row_sqnorm(C, k, dp, cn.get(), s);
    if (ntiles * TC_N > k) {
        pad_inf_kernel<<<1, TC_N, 0, s>>>(cn.get(), k, ntiles * TC_N);
        MASK_LAUNCHED("pad_inf");
    }
    max_reduce(cn.get(), k, cmax.get(), s);
    MASK_CUDA(cudaMemsetAsync(cabs.get(), 0, sizeof(unsigned), s));
    absmax_kernel<<<grid_cap((int64_t)k * dp), 256, 0, s>>>(C, (int64_t)k * dp, cabs.get());
    MASK_LAUNCHED("absmax");
    split_f16_kernel<<<grid_cap((int64_t)k * 8), 256, 0, s>>>(C, k, dp, cabs.get(), Ch.get(),
                                                              Cl.get(), cinv.get());
    MASK_LAUNCHED("split_f16");
    const CUtensorMap mCh = make_map(Ch.get(), k), mCl = make_map(Cl.get(), k);
    MASK_CUDA(cudaMemsetAsync(counts.get(), 0, 2 * sizeof(int), s));
    // Error bound of one expanded-form distance, relative to ||x||^2 + ||c||^2
    // (the factor 2 of -2 x.c cancels against sum|x_t c_t| <= (||x||^2 +
    // ||c||^2) / 2):
    //  - the split: with u = 2^-11 (FP16 rounding), v - hi is within u|v| and
    //    lo within u|v - hi| of it, so the dropped lo*lo product and the two
    //    rounded lo factors leave (3 + 3u) * 2^-22 of sum |x_t c_t|; lo values
    //    below the FP16 normal range add at most 2^-24 (scaled units) each,
    //    which after unscaling is below 2^-27 of ||x||^2 + ||c||^2;
    //  - FP32 accumulation in the tensor core: 3 * ceil(dp/16) MMAs into one
    //    accumulator plus 16 additions inside an MMA, counted at 2^-23 each
    //    (truncating adders);
    //  - the FP32 norms (dp * 2^-24) and two final roundings (4 * 2^-24).
    // A label is certain when the best two differ by more than twice the
    // bound; the coefficient is widened 2x beyond that.
    const double per = (3.0 + 3.0 * 0x1.0p-11) * 0x1.0p-22 + 0x1.0p-27 +
                       (3.0 * ((dp + 15) / 16) + 16.0) * 0x1.0p-23 + (dp + 4.0) * 0x1.0p-24;
    const float coef = (float)(2.0 * 2.0 * per);
    {
        ProfRegion pr("assign_tc", s, 2.0 * (double)p.n * (double)k * (double)dp);
        launch_tc<TC_STAGES>(p, mCh, mCl, C, seeded, xn, cinv.get(), cn.get(), k, cmax.get(), coef,
                             labels,
                             list3.get(), counts.get(), listF.get(), counts.get() + 1, s);
        MASK_LAUNCHED("assign_tc");
    }
    {
        ProfRegion pr("assign_recheck", s, 0.0);
        const int lpr = lanes_per_row(dp);
        const float4 *X4 = reinterpret_cast<const float4 *>(p.X);
        const float4 *C4 = reinterpret_cast<const float4 *>(C);
        switch (lpr) {
        case 1: recheck3_kernel<1><<<152 * 4, 256, 0, s>>>(X4, dp / 4, C4, list3.get(), counts.get(), labels); break;
        case 2: recheck3_kernel<2><<<152 * 4, 256, 0, s>>>(X4, dp / 4, C4, list3.get(), counts.get(), labels); break;
        case 4: recheck3_kernel<4><<<152 * 4, 256, 0, s>>>(X4, dp / 4, C4, list3.get(), counts.get(), labels); break;
        case 8: recheck3_kernel<8><<<152 * 4, 256, 0, s>>>(X4, dp / 4, C4, list3.get(), counts.get(), labels); break;
        case 16: recheck3_kernel<16><<<152 * 4, 256, 0, s>>>(X4, dp / 4, C4, list3.get(), counts.get(), labels); break;
        default: recheck3_kernel<32><<<152 * 4, 256, 0, s>>>(X4, dp / 4, C4, list3.get(), counts.get(), labels); break;
        }
        MASK_LAUNCHED("recheck3");
        assign_recheck_rows(p.X, dp, C, k, listF.get(), counts.get() + 1, labels, s);
    }
}

void tc_assign_check(TcAssign &p, cudaStream_t s) {
    int e = 0;
    MASK_CUDA(cudaMemcpyAsync(&e, p.err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    MASK_CUDA(cudaStreamSynchronize(s));
    if (e) fail(MASK_ETIMEOUT, "assignment kernel: a bounded pipeline wait ran out");
}

}  // namespace mask
