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
constexpr int LP_QB = 16;   // queries per work item (two n8 MMA tiles)
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
template <bool FP8>
__global__ __launch_bounds__(LP_THREADS) void lp_scan_kernel(
    const uint8_t *__restrict__ Xl, int dpl, const float *__restrict__ xn2,
    const float *__restrict__ xscale, const int64_t *__restrict__ leaf_off,
    const uint8_t *__restrict__ Ql, const float *__restrict__ qn2, const float *__restrict__ qscale,
    const float *__restrict__ seed_d, int kseed, float eta, float rslack, int P,
    const int64_t *__restrict__ poff, const int32_t *__restrict__ pairs,
    const int64_t *__restrict__ item_off, int k0, int K, unsigned long long *__restrict__ pair_out) {
    constexpr int ES = FP8 ? 1 : 2;                   // bytes per element
    constexpr int KSTEP = FP8 ? 32 : 16;              // elements per MMA k-step
    extern __shared__ __align__(16) unsigned char smem[];
    const int rowb = dpl * ES + 16;                   // padded row stride in bytes
    unsigned char *rows = smem;                       // [LP_R][rowb]
    unsigned char *qs = rows + (size_t)LP_R * rowb;   // [LP_QB][rowb]
    float *D = reinterpret_cast<float *>(qs + (size_t)LP_QB * rowb);  // [LP_QB][LP_R]
    float *rn = D + LP_QB * LP_R;                     // [LP_R] row norms
    float *rs = rn + LP_R;                            // [LP_R] row scales
    int32_t *pos = reinterpret_cast<int32_t *>(rs + LP_R);            // [LP_R] row positions
    float *qn = reinterpret_cast<float *>(pos + LP_R);                // [LP_QB]
    float *qsc = qn + LP_QB;                                          // [LP_QB]
    unsigned long long *top = reinterpret_cast<unsigned long long *>(qsc + LP_QB);  // [LP_QB][K]
    __shared__ int s_c;
    __shared__ int64_t s_pb, s_pe;
    __shared__ float s_rt[LP_QB];  // sqrt(T_q): the seed's k-th exact distance, as a length

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
        if (tid < LP_QB) {
            const bool ok = tid < nqb;
            const int64_t q = ok ? pairs[pb + tid] / P : 0;
            qn[tid] = ok ? qn2[q] : 0.f;
            qsc[tid] = (ok && FP8) ? qscale[q] : 1.f;
            s_rt[tid] = ok ? sqrtf(seed_d[q * kseed + kseed - 1]) : 0.f;
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
                pos[i] = ok ? (int32_t)(r0 + i) : -1;
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
            // merge the chunk into each query's shortlist: warp w owns queries 2w, 2w+1
            for (int qi = 0; qi < 2; ++qi) {
                const int qb = warp * 2 + qi;
                if (qb >= nqb) break;
                unsigned long long *tq = top + qb * K;
                const unsigned long long th = tq[K - 1];
                // a row whose quantised distance exceeds sqrt(T_q) + eta (|x| + |q|)
                // is farther than T_q exactly: it cannot be among the k nearest
                const float rt = s_rt[qb], qlen = sqrtf(qn[qb]);
                unsigned long long cand[LP_R / 32];
                bool any = false;
#pragma unroll
                for (int i = 0; i < LP_R / 32; ++i) {
                    const int rr = lane + 32 * i;
                    cand[i] = kNoKey;
                    if (rr < nr) {
                        const float dq = D[qb * LP_R + rr];
                        const float lim = rt + eta * (sqrtf(rn[rr]) + qlen);
                        // plus the rounding of the FP32 expanded form dq itself
                        const float slack = rslack * (rn[rr] + qn[qb]);
                        const unsigned long long key =
                            ((unsigned long long)__float_as_uint(dq) << 32) | (unsigned)pos[rr];
                        if (key < th && dq <= fmaf(lim, lim, slack)) { cand[i] = key; any = true; }
                    }
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
    {
        ProfRegion pr(fp8 ? "scan_leaf_fp8" : "scan_leaf_bf16", s, 0.0);
        const int rowb = dpl * (fp8 ? 1 : 2) + 16;
        const size_t smem = (size_t)(LP_R + LP_QB) * rowb + (size_t)LP_QB * LP_R * 4 +
                            (size_t)LP_R * 12 + LP_QB * 8 + (size_t)LP_QB * Kpair * 8 + 16;
        if (fp8) {
            MASK_CUDA(cudaFuncSetAttribute(lp_scan_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            lp_scan_kernel<true><<<152 * 4, LP_THREADS, smem, s>>>(
                static_cast<const uint8_t *>(Xl), dpl, xn2, xscale, leaf_off, Ql.get(), qn2.get(),
                qsc.get(), seed_d.get(), k, eta, rslack, P, poff.get(), pairs.get(), item_off.get(), k0,
                Kpair, pair_out.get());
        } else {
            MASK_CUDA(cudaFuncSetAttribute(lp_scan_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            lp_scan_kernel<false><<<152 * 4, LP_THREADS, smem, s>>>(
                static_cast<const uint8_t *>(Xl), dpl, xn2, nullptr, leaf_off, Ql.get(), qn2.get(),
                nullptr, seed_d.get(), k, eta, rslack, P, poff.get(), pairs.get(), item_off.get(), k0,
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
