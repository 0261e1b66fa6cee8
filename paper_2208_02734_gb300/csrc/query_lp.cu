// query_lp.cu -- the BF16 and FP8 e4m3 query modes (not in the paper, which
// states no precision): the leaf scan's distances on the tensor cores in low
// precision, re-ranked by exact FP32 distances.
//
// The leaf scan of the k-NN descent (§3.3, Algorithm 2) ranks the points of
// the kept leaf clusters.  In these modes the index also holds the points in
// BF16, or in FP8 e4m3 with a per-row scale s = max|x| / 448, with the squared
// norm of each quantised row.  Queries are grouped by cluster as in the FP32
// cluster-major scan; the distances of a group are
//     ||x~||^2 + ||q~||^2 - 2 x~.q~    (x~, q~ the quantised vectors)
// with x~.q~ from warp-level tensor-core MMAs (FP32 accumulation).  Those are
// a filter with a proven bound: with element errors |x~_t - x_t| <= eta |x_t|,
//     ||x~ - q~|| <= ||x - q|| + eta (||x|| + ||q||),
// so a row whose low-precision distance exceeds (sqrt(L) + eta (||x~|| +
// ||q~||))^2 (plus the FP32 rounding of the expanded form) is farther than L,
// where L is the smaller of the (query, cluster) pair's current k-th exact
// distance and T_q (the k-th exact distance within the query's nearest kept
// cluster, from an FP32 seed pass).  Every other row -- the shortlist -- is
// re-ranked with its exact FP32 distance sum_t (x_t - q_t)^2 (t ascending, FMA
// per term: the arithmetic of the FP32 scans), and the pair keeps its k best
// exact keys.  So these modes return exactly the FP32 answer; the low
// precision only decides which rows are worth the exact evaluation.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <climits>

#include "common.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int LP_THREADS = 256;
constexpr int LP_QB = 16;   // queries per work item (two n8 MMA tiles)
constexpr int LP_R = 128;   // rows per chunk (eight m16 MMA tiles, one per warp)
constexpr int LP_KMAX = 64; // per-pair list length limit (two keys per lane)

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
template <bool FP8>
__global__ __launch_bounds__(LP_THREADS) void lp_scan_kernel(
    const uint8_t *__restrict__ Xl, int dpl, const float *__restrict__ xn2,
    const float *__restrict__ xscale, const float4 *__restrict__ Xs, int dp4,
    const int32_t *__restrict__ xids, const int64_t *__restrict__ leaf_off,
    const uint8_t *__restrict__ Ql, const float *__restrict__ qn2, const float *__restrict__ qscale,
    const float4 *__restrict__ Qp, const float *__restrict__ seed_d, float eta, float rslack,
    float ulim, int P, const int64_t *__restrict__ poff, const int32_t *__restrict__ pairs,
    const int64_t *__restrict__ item_off, int k0, int K, unsigned long long *__restrict__ pair_out) {
    constexpr int ES = FP8 ? 1 : 2;                   // bytes per element
    constexpr int KSTEP = FP8 ? 32 : 16;              // elements per MMA k-step
    extern __shared__ __align__(16) unsigned char smem[];
    const int rowb = dpl * ES + 16;                   // padded row stride in bytes
    unsigned char *rows = smem;                       // [LP_R][rowb]
    unsigned char *qs = rows + (size_t)LP_R * rowb;   // [LP_QB][rowb]
    float *D = reinterpret_cast<float *>(qs + (size_t)LP_QB * rowb);  // [LP_QB][LP_R]
    float4 *qf = reinterpret_cast<float4 *>(D + LP_QB * LP_R);        // [LP_QB][dp4] FP32 queries
    float *rn = reinterpret_cast<float *>(qf + LP_QB * dp4);          // [LP_R] row norms
    float *rs = rn + LP_R;                            // [LP_R] row scales
    int32_t *rid = reinterpret_cast<int32_t *>(rs + LP_R);            // [LP_R] original ids
    float *qn = reinterpret_cast<float *>(rid + LP_R);                // [LP_QB]
    float *qsc = qn + LP_QB;                                          // [LP_QB]
    unsigned long long *top = reinterpret_cast<unsigned long long *>(qsc + LP_QB);  // [LP_QB][K]
    __shared__ int s_c;
    __shared__ int64_t s_pb, s_pe;
    __shared__ float s_tq[LP_QB];  // T_q: the seed's k-th exact distance

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const int c16 = dpl * ES / 16;                    // 16-byte chunks per row
    const int64_t n_items = item_off[k0];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        if (tid == 0) {
            int lo = 0, hi = k0 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (item_off[mid] <= item) lo = mid; else hi = mid - 1;
            }
            s_c = lo;
            s_pb = poff[lo] + (item - item_off[lo]) * LP_QB;
            s_pe = min(poff[lo + 1], s_pb + LP_QB);
        }
        __syncthreads();
        const int c = s_c;
        const int64_t pb = s_pb;
        const int nqb = (int)(s_pe - pb);
        for (int i = tid; i < LP_QB * c16; i += LP_THREADS) {
            const int qb = i / c16, cc = i % c16;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (qb < nqb) {
                const int64_t q = pairs[pb + qb] / P;
                v = reinterpret_cast<const uint4 *>(Ql + q * dpl * ES)[cc];
            }
            *reinterpret_cast<uint4 *>(qs + qb * rowb + cc * 16) = v;
        }
        for (int i = tid; i < LP_QB * dp4; i += LP_THREADS) {
            const int qb = i / dp4, cc = i % dp4;
            qf[i] = qb < nqb ? Qp[(pairs[pb + qb] / P) * dp4 + cc] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (tid < LP_QB) {
            const bool ok = tid < nqb;
            const int64_t q = ok ? pairs[pb + tid] / P : 0;
            qn[tid] = ok ? qn2[q] : 0.f;
            qsc[tid] = (ok && FP8) ? qscale[q] : 1.f;
            s_tq[tid] = ok ? seed_d[q * K + K - 1] : 0.f;  // +inf when the seed cluster is short
        }
        for (int i = tid; i < LP_QB * K; i += LP_THREADS) top[i] = kNoKey;
        const int64_t rb = leaf_off[c], re = leaf_off[c + 1];
        for (int64_t r0 = rb; r0 < re; r0 += LP_R) {
            const int nr = (int)((re - r0) < (int64_t)LP_R ? (re - r0) : (int64_t)LP_R);
            __syncthreads();
            for (int i = tid; i < LP_R * c16; i += LP_THREADS) {
                const int rr = i / c16, cc = i % c16;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (rr < nr) v = reinterpret_cast<const uint4 *>(Xl + (r0 + rr) * dpl * ES)[cc];
                *reinterpret_cast<uint4 *>(rows + rr * rowb + cc * 16) = v;
            }
            for (int i = tid; i < LP_R; i += LP_THREADS) {
                const bool ok = i < nr;
                rn[i] = ok ? xn2[r0 + i] : 0.f;
                rs[i] = (ok && FP8) ? xscale[r0 + i] : 1.f;
                rid[i] = ok ? xids[r0 + i] : -1;
            }
            __syncthreads();
            // warp w: rows 16w .. 16w+15 against the 16 queries (two n8 tiles)
            {
                float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
                const unsigned char *ra = rows + (16 * warp + g) * rowb;
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
                        const unsigned char *qb = qs + (nt * 8 + g) * rowb;
                        uint32_t b[2];
                        b[0] = *reinterpret_cast<const uint32_t *>(qb + e0 * ES);
                        b[1] = *reinterpret_cast<const uint32_t *>(qb + e1 * ES);
                        if (FP8) mma_e4m3_16832(acc[nt], a, b);
                        else mma_bf16_16816(acc[nt], a, b);
                    }
                }
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int rr = 16 * warp + g + (h >= 2 ? 8 : 0);
                        const int qb = nt * 8 + tig * 2 + (h & 1);
                        const float dot = acc[nt][h] * rs[rr] * qsc[qb];
                        D[qb * LP_R + rr] = fmaxf(rn[rr] + qn[qb] - 2.f * dot, 0.f);
                    }
            }
            __syncthreads();
            // filter, exact keys, merge: warp w owns queries 2w, 2w+1
            for (int qi = 0; qi < 2; ++qi) {
                const int qb = warp * 2 + qi;
                if (qb >= nqb) break;
                unsigned long long *tq = top + qb * K;
                const unsigned long long th = tq[K - 1];
                const float lim = fminf(s_tq[qb], th == kNoKey ? __int_as_float(0x7f800000)
                                                               : __uint_as_float((unsigned)(th >> 32)));
                const float rt = sqrtf(lim * ulim), qlen = sqrtf(qn[qb]);
                const float4 *qv = qf + qb * dp4;
                unsigned long long cand[LP_R / 32];
                bool any = false;
#pragma unroll
                for (int i = 0; i < LP_R / 32; ++i) {
                    const int rr = lane + 32 * i;
                    cand[i] = kNoKey;
                    if (rr >= nr) continue;
                    const float bound = rt + eta * (sqrtf(rn[rr]) + qlen);
                    if (!(D[qb * LP_R + rr] <= fmaf(bound, bound, rslack * (rn[rr] + qn[qb]))))
                        continue;
                    // exact FP32 key, the arithmetic of the FP32 scans
                    const float4 *xr = Xs + (r0 + rr) * dp4;
                    float e2 = 0.f;
                    for (int cc = 0; cc < dp4; ++cc) {
                        const float4 v = __ldg(xr + cc), w = qv[cc];
                        float e = v.x - w.x;
                        e2 = fmaf(e, e, e2);
                        e = v.y - w.y;
                        e2 = fmaf(e, e, e2);
                        e = v.z - w.z;
                        e2 = fmaf(e, e, e2);
                        e = v.w - w.w;
                        e2 = fmaf(e, e, e2);
                    }
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(e2) << 32) | (unsigned)rid[rr];
                    if (key < th) { cand[i] = key; any = true; }
                }
                if (!__any_sync(kFull, any)) continue;
                unsigned long long old0 = lane < K ? tq[lane] : kNoKey;
                unsigned long long old1 = lane + 32 < K ? tq[lane + 32] : kNoKey;
                unsigned long long out0 = kNoKey, out1 = kNoKey;
                for (int r = 0; r < K; ++r) {
                    unsigned long long mine = umin64(old0, old1);
#pragma unroll
                    for (int i = 0; i < LP_R / 32; ++i) mine = umin64(mine, cand[i]);
                    const unsigned long long w = warp_min64(mine);
                    if (w == kNoKey) break;
                    if (lane == (r & 31)) { if (r < 32) out0 = w; else out1 = w; }
                    if (old0 == w) old0 = kNoKey;
                    if (old1 == w) old1 = kNoKey;
#pragma unroll
                    for (int i = 0; i < LP_R / 32; ++i)
                        if (cand[i] == w) cand[i] = kNoKey;
                }
                __syncwarp();
                if (lane < K) tq[lane] = out0;
                if (lane + 32 < K) tq[lane + 32] = out1;
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = tid; i < nqb * K; i += LP_THREADS) {
            const int qb = i / K, j = i % K;
            pair_out[(int64_t)pairs[pb + qb] * K + j] = top[qb * K + j];
        }
        __syncthreads();
    }
}

}  // namespace

int lp_padded_dim(int dp) { return (dp + 31) / 32 * 32; }

bool lp_supported(int dp, int k) { return k >= 1 && k <= LP_KMAX && lp_padded_dim(dp) <= 256; }

void lp_quantize(const float *src, int64_t rows, int dp, bool fp8, void *dst, float *scale,
                 float *norm2, cudaStream_t s) {
    if (rows == 0) return;
    const int dpl = lp_padded_dim(dp);
    const int blocks = (int)std::min<int64_t>((rows + 7) / 8, 152 * 32);
    if (fp8) {
        quant_fp8_kernel<<<blocks, 256, 0, s>>>(src, rows, dp, dpl,
                                                static_cast<__nv_fp8_e4m3 *>(dst), scale, norm2);
        MASK_LAUNCHED("quant_fp8");
    } else {
        quant_bf16_kernel<<<blocks, 256, 0, s>>>(src, rows, dp, dpl,
                                                 static_cast<__nv_bfloat16 *>(dst), norm2);
        MASK_LAUNCHED("quant_bf16");
    }
}

void lp_leaf_scan(bool fp8, const void *Xl, const float *xn2, const float *xscale, const float *Xs,
                  int64_t leaf_rows, int dp, const int32_t *xids, const int64_t *leaf_off, int k0,
                  const float *Qp, int64_t nq, const int32_t *sel, int P, int k, int64_t *ids,
                  float *dists, cudaStream_t s) {
    (void)leaf_rows;
    if (nq == 0) return;
    MASK_REQUIRE(lp_supported(dp, k), "low-precision scan: k or dimension too large");
    const int dpl = lp_padded_dim(dp);
    Scratch<unsigned char> Ql((size_t)nq * dpl * (fp8 ? 1 : 2), s);
    Scratch<float> qn2(nq, s), qsc(fp8 ? nq : 1, s), seed_d((size_t)nq * k, s);
    lp_quantize(Qp, nq, dp, fp8, Ql.get(), qsc.get(), qn2.get(), s);
    // the FP32 seed: each query's k-th exact distance within its nearest kept
    // cluster bounds the distance of its k nearest from above
    leaf_seed(Xs, xids, leaf_off, dp, Qp, nq, sel, P, k, seed_d.get(), s);
    Scratch<int32_t> pairs;
    Scratch<int64_t> poff, item_off;
    cm_group_pairs(sel, nq, P, k0, pairs, poff, item_off, s);
    const int64_t npairs = nq * P;
    Scratch<unsigned long long> pair_out((size_t)npairs * k, s);
    // pairs of an absent parent (sel = -1, fewer children than probes) are in
    // no work item: their lists stay empty
    MASK_CUDA(cudaMemsetAsync(pair_out.get(), 0xFF, sizeof(unsigned long long) * npairs * k, s));
    // eta: element error relative to the element: BF16 keeps 8 significant
    // bits (2^-8; 2x margin), e4m3 4 (2^-4, and |x| <= |x~| / (1 - 2^-4):
    // 2^-4 x 1.125; subnormals of the per-row scaled range add at most
    // 2^-10 x max|x| / 448 per element).  rslack: rounding of the FP32
    // expanded form per unit of the squared norms (dot over dpl terms x 2,
    // norms, final roundings), x 2.  ulim: the exact FP32 key may undershoot
    // the distance by (dp + 2) 2^-24 of it.
    const float eta = fp8 ? 0x1.2p-4f : 0x1.0p-7f;
    const float rslack = (float)((4.0 * dpl + 16.0) * 0x1.0p-24);
    const float ulim = (float)(1.0 + (dp + 4.0) * 0x1.0p-24);
    {
        ProfRegion pr(fp8 ? "scan_leaf_fp8" : "scan_leaf_bf16", s, 0.0);
        const int rowb = dpl * (fp8 ? 1 : 2) + 16;
        const size_t smem = (size_t)(LP_R + LP_QB) * rowb + (size_t)LP_QB * LP_R * 4 +
                            (size_t)LP_QB * dp * 4 + (size_t)LP_R * 12 + LP_QB * 8 +
                            (size_t)LP_QB * k * 8 + 16;
        const float4 *X4 = reinterpret_cast<const float4 *>(Xs);
        const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
        if (fp8) {
            MASK_CUDA(cudaFuncSetAttribute(lp_scan_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            lp_scan_kernel<true><<<152 * 4, LP_THREADS, smem, s>>>(
                static_cast<const uint8_t *>(Xl), dpl, xn2, xscale, X4, dp / 4, xids, leaf_off,
                Ql.get(), qn2.get(), qsc.get(), Q4, seed_d.get(), eta, rslack, ulim, P, poff.get(),
                pairs.get(), item_off.get(), k0, k, pair_out.get());
        } else {
            MASK_CUDA(cudaFuncSetAttribute(lp_scan_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            lp_scan_kernel<false><<<152 * 4, LP_THREADS, smem, s>>>(
                static_cast<const uint8_t *>(Xl), dpl, xn2, nullptr, X4, dp / 4, xids, leaf_off,
                Ql.get(), qn2.get(), nullptr, Q4, seed_d.get(), eta, rslack, ulim, P, poff.get(),
                pairs.get(), item_off.get(), k0, k, pair_out.get());
        }
        MASK_LAUNCHED("lp_scan");
    }
    cm_merge(pair_out.get(), nq, P, k, ids, dists, s);
}

}  // namespace mask
