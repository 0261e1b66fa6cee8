// kmeans.cu -- k-means building blocks of the MASK build (§2.4, §3.1, §3.2):
// row padding and norms, k-means++ seeding steps, the label counting sort that
// turns a labelling into membership lists, and the per-cluster mean update.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------ elementwise kernels

__global__ void pad_rows_kernel(const float *__restrict__ src, int64_t n, int d,
                                float *__restrict__ dst, int dp) {
    const int64_t total = n * dp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / dp;
        const int t = (int)(e - i * dp);
        dst[e] = t < d ? src[i * d + t] : 0.f;
    }
}

__global__ void unpad_rows_kernel(const float *__restrict__ src, int64_t n, int dp,
                                  float *__restrict__ dst, int d) {
    const int64_t total = n * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int t = (int)(e - i * d);
        dst[e] = src[i * dp + t];
    }
}

template <class I>
__global__ void gather_rows_kernel(const float4 *__restrict__ src, int dp4,
                                   const I *__restrict__ idx, int64_t m,
                                   float4 *__restrict__ dst) {
    const int64_t total = m * dp4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / dp4;
        const int c = (int)(e - r * dp4);
        dst[e] = src[(int64_t)idx[r] * dp4 + c];
    }
}

__global__ void iota_kernel(int32_t *p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

// Squared norm of each row, one group of LPR lanes per row.
template <int LPR>
__global__ void row_sqnorm_kernel(const float4 *__restrict__ X, int64_t n, int dp4,
                                  float *__restrict__ out) {
    const int gl = threadIdx.x % LPR;
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / LPR);
    int64_t row = (int64_t)blockIdx.x * (blockDim.x / LPR) + threadIdx.x / LPR;
    // every lane of a warp runs the same number of iterations (shuffles below)
    const int64_t n_round = (n + groups - 1) / groups * groups;
    for (; row < n_round; row += groups) {
        float acc = 0.f;
        if (row < n) {
            const float4 *xr = X + row * dp4;
            for (int c = gl; c < dp4; c += LPR) {
                float4 v = xr[c];
                acc = fmaf(v.x, v.x, acc);
                acc = fmaf(v.y, v.y, acc);
                acc = fmaf(v.z, v.z, acc);
                acc = fmaf(v.w, v.w, acc);
            }
        }
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (gl == 0 && row < n) out[row] = acc;
    }
}

// dist[i] = sum_t (x_it - c_{labels[i],t})^2
template <int LPR>
__global__ void label_dist_kernel(const float4 *__restrict__ X, int64_t n, int dp4,
                                  const float4 *__restrict__ C,
                                  const int32_t *__restrict__ labels, float *__restrict__ dist) {
    const int gl = threadIdx.x % LPR;
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / LPR);
    int64_t row = (int64_t)blockIdx.x * (blockDim.x / LPR) + threadIdx.x / LPR;
    const int64_t n_round = (n + groups - 1) / groups * groups;
    for (; row < n_round; row += groups) {
        float acc = 0.f;
        if (row < n) {
            const float4 *xr = X + row * dp4;
            const float4 *cr = C + (int64_t)labels[row] * dp4;
            for (int c = gl; c < dp4; c += LPR) {
                float4 a = xr[c], b = cr[c];
                float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
                acc = fmaf(e0, e0, acc);
                acc = fmaf(e1, e1, acc);
                acc = fmaf(e2, e2, acc);
                acc = fmaf(e3, e3, acc);
            }
        }
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (gl == 0 && row < n) dist[row] = acc;
    }
}

__global__ void max_reduce_kernel(const float *__restrict__ v, int64_t n, float *out) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    // values are >= 0, so their bit patterns order like unsigned integers
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned *>(out), __float_as_uint(m));
}

// --------------------------------------------------------------- k-means++

constexpr int kKppThreads = 512;
constexpr int kKppRows = 1024;   // rows per block; one D^2 block sum each
constexpr int kKppRpt = kKppRows / kKppThreads;  // rows per thread

// One k-means++ step (§3.2).  The step number t >= 1 is read from *t_dev.
// Fold the centre picked at step t-1 into D^2, then the last block to finish
// draws centre t: the smallest row whose inclusive prefix of D^2 exceeds
// u_t * sum(D^2); if that sum is 0, the lowest-index row not chosen yet.
// The last block then advances *t_dev, so identical launches can be replayed
// step after step.  Three kernels fold D^2 (dense rows one per thread with
// triangle-inequality pruning, wide dense rows one per warp, CSR rows one per
// lane group); they share the draw.
//
// The sums are exact integers: every D^2 (FP32) becomes the 64-bit integer
// q_i = round(D^2_i * 2^sh), with one power of two 2^sh per seeding run that
// keeps sum_i q_i below 2^62 (from the first step's total, which bounds every
// later one: D^2 only decreases).  Integer sums do not depend on their
// order, and u_t = a_t * 2^-53 (a_t the generator's 53-bit integer), so the
// pick rule "prefix_i > u_t * S" is decided exactly as the 128-bit
// comparison prefix_i * 2^53 > a_t * S.  q_i resolves 2^-61 of the first
// total, far below the FP32 rounding of D^2 itself.
//
// cc2[j] = ||c_{t-1} - c_j||^2 for the centres j < t-1 chosen so far (FP32
// difference form): the distances the narrow dense D^2 update prunes with.
__global__ void kpp_centre_dist_kernel(const float *__restrict__ X, int64_t m, int dp,
                                       const int *__restrict__ t_dev,
                                       const int64_t *__restrict__ chosen,
                                       float *__restrict__ cc2) {
    const int t = *t_dev;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < 2 || j >= t - 1) return;
    int64_t a = chosen[t - 1], b = chosen[j];
    if (a < 0 || a >= m) a = 0;
    if (b < 0 || b >= m) b = 0;
    const float4 *ca = reinterpret_cast<const float4 *>(X + a * dp);
    const float4 *cb = reinterpret_cast<const float4 *>(X + b * dp);
    float acc = 0.f;
    for (int c = 0; c < dp / 4; ++c) {
        const float4 x = __ldg(ca + c), y = __ldg(cb + c);
        float e = x.x - y.x;
        acc = fmaf(e, e, acc);
        e = x.y - y.y;
        acc = fmaf(e, e, acc);
        e = x.z - y.z;
        acc = fmaf(e, e, acc);
        e = x.w - y.w;
        acc = fmaf(e, e, acc);
    }
    cc2[j] = acc;
}

// 64 x 64 -> 128-bit unsigned products and comparisons for the draw.
struct U128 {
    unsigned long long hi, lo;
};
__device__ __forceinline__ U128 mul_u128(unsigned long long a, unsigned long long b) {
    return U128{__umul64hi(a, b), a * b};
}
// v * 2^53 for v < 2^64
__device__ __forceinline__ U128 shl53(unsigned long long v) { return U128{v >> 11, v << 53}; }
__device__ __forceinline__ bool gt_u128(U128 x, U128 y) {
    return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo);
}

// q = round(d2 * qs), qs = 2^sh (exact scaling, then one rounding).
__device__ __forceinline__ unsigned long long kpp_q(float d2, float qs) {
    return __float2ull_rn(d2 * qs);
}

// 2^sh with sum(D^2) * 2^sh < 2^61, from a bound s1 >= sum(D^2) (FP32 bits
// of s1 in *s1_bits; 0 gives 1).
__device__ __forceinline__ float kpp_scale(const unsigned *s1_bits) {
    const unsigned b = *s1_bits;
    if (b == 0u) return 1.f;
    const int e = (int)((b >> 23) & 0xffu) - 127;   // 2^e <= s1 < 2^(e+1)
    int sh = 60 - e;
    sh = sh < -126 ? -126 : (sh > 126 ? 126 : sh);
    return __uint_as_float((uint32_t)(sh + 127) << 23);
}

// Shared memory of the draw (all kKppThreads threads of the last block).
struct KppDrawSmem {
    unsigned long long wsum[kKppThreads / 32];   // per-warp totals of a block scan
    unsigned long long excl;
    long long fb, pick;
    int first;
};

// Inclusive prefix sum of v over the kKppThreads threads of the block (a
// warp scan then a scan of the warp totals); *total = the block's sum.
__device__ unsigned long long kpp_block_scan(unsigned long long v, unsigned long long *wsum,
                                             unsigned long long *total) {
    constexpr int W = kKppThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < W ? wsum[lane] : 0ull;
        for (int o = 1; o < W; o <<= 1) {
            const unsigned long long n = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += n;
        }
        if (lane < W) wsum[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += wsum[warp - 1];
    *total = wsum[W - 1];
    __syncthreads();  // wsum may be reused by the next scan
    return v;
}

// Smallest thread index of the block for which `flag` holds (INT_MAX if none).
__device__ int kpp_block_first(bool flag, int *slot) {
    if (threadIdx.x == 0) *slot = INT_MAX;
    __syncthreads();
    const unsigned bal = __ballot_sync(kFull, flag);
    if ((threadIdx.x & 31) == 0 && bal) atomicMin(slot, (int)(threadIdx.x + __ffs(bal) - 1));
    __syncthreads();
    const int r = *slot;
    __syncthreads();
    return r;
}

// Block total of the quantised D^2 -> bsum[blockIdx.x]; true in the last
// block to finish (which then draws).
__device__ bool kpp_block_done(unsigned long long local, unsigned long long *red,
                               unsigned long long *__restrict__ bsum,
                               unsigned *__restrict__ counter, int *s_last) {
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long bs = 0;
        for (int i = 0; i < kKppThreads / 32; ++i) bs += red[i];
        bsum[blockIdx.x] = bs;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    const bool last = *s_last != 0;
    if (last) __threadfence();
    return last;
}

// The measuring launch (before the first step): each block adds its FP32 sum
// of the first step's D^2 to *s1 (bits of a float, atomically as a float
// add); twice that bounds every step's sum.
__device__ void kpp_measure(float local, float *red, unsigned *__restrict__ s1_bits) {
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(kFull, local, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bs = 0.f;
        for (int i = 0; i < kKppThreads / 32; ++i) bs += red[i];
        atomicAdd(reinterpret_cast<float *>(s1_bits), 2.f * bs);
    }
}

// The draw of centre t by all threads of the last block (blocks of ROWS
// rows): the smallest row i with (sum_{j<=i} q_j) * 2^53 > a_t * Q, Q the
// total.  Thread i owns a contiguous run of block sums, then of the selected
// block's rows; block scans give each run's prefix, and the first run that
// crosses the target is walked by its owner.  The crossing always exists
// when Q > 0 (the full prefix Q times 2^53 exceeds a_t * Q as a_t < 2^53).
template <int ROWS>
__device__ void kpp_draw(int t, int64_t m, const unsigned long long *__restrict__ a53,
                         const float *__restrict__ D2, float qs,
                         const unsigned long long *__restrict__ bsum,
                         unsigned *__restrict__ counter, int *__restrict__ t_dev,
                         int64_t *__restrict__ chosen, unsigned char *__restrict__ taken,
                         KppDrawSmem &sm) {
    constexpr int RPT = ROWS >= kKppThreads ? ROWS / kKppThreads : 1;  // rows per thread
    static_assert(ROWS % kKppThreads == 0 || ROWS < kKppThreads, "rows per block");
    const int tid = threadIdx.x;
    const int nb = gridDim.x;
    if (t == 1 && tid == 0) taken[chosen[0]] = 1;
    if (tid == 0) sm.pick = -1;
    const unsigned long long at = a53[t];
    // block sums: thread tid owns [tid * per, (tid + 1) * per)
    const int per = (nb + kKppThreads - 1) / kKppThreads;
    const int b0 = tid * per;
    unsigned long long ls = 0;
    for (int q = 0; q < per; ++q)
        if (b0 + q < nb) ls += __ldcg(bsum + b0 + q);
    unsigned long long Q;
    const unsigned long long inc = kpp_block_scan(ls, sm.wsum, &Q);
    if (Q > 0) {
        const U128 target = mul_u128(at, Q);
        const int src = kpp_block_first(ls > 0 && gt_u128(shl53(inc), target), &sm.first);
        if (tid == src) {
            unsigned long long run = inc - ls;
            long long f = -1;
            for (int q = 0; q < per && b0 + q < nb; ++q) {
                const unsigned long long v = __ldcg(bsum + b0 + q);
                if (v > 0 && gt_u128(shl53(run + v), target)) {
                    f = b0 + q;
                    break;
                }
                run += v;
            }
            sm.fb = f;
            sm.excl = run;
        }
        if (tid == 0 && src == INT_MAX) sm.fb = -1;
        __syncthreads();
        const long long fb = sm.fb;
        if (fb >= 0) {
            // the block's rows: thread tid owns rows [tid * RPT, (tid + 1) * RPT)
            const int64_t r0 = fb * ROWS + (int64_t)tid * RPT;
            unsigned long long v[RPT];
            unsigned long long rs = 0;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int64_t i = r0 + q;
                v[q] = (tid * RPT + q < ROWS && i < m) ? kpp_q(__ldcg(D2 + i), qs) : 0ull;
                rs += v[q];
            }
            unsigned long long tot;
            const unsigned long long rinc = kpp_block_scan(rs, sm.wsum, &tot) + sm.excl;
            const int src2 = kpp_block_first(rs > 0 && gt_u128(shl53(rinc), target), &sm.first);
            if (tid == src2) {
                unsigned long long run = rinc - rs;
                long long p = -1;
#pragma unroll
                for (int q = 0; q < RPT; ++q) {
                    if (p < 0 && v[q] > 0 && gt_u128(shl53(run + v[q]), target)) p = r0 + q;
                    run += v[q];
                }
                sm.pick = p;
            }
            __syncthreads();
        }
    } else {
        // all remaining points coincide with chosen centres: lowest unchosen index
        for (int64_t c0 = 0; c0 < m; c0 += kKppThreads) {
            const int64_t i = c0 + tid;
            const int f = kpp_block_first(i < m && !taken[i], &sm.first);
            if (f != INT_MAX) {
                if (tid == 0) sm.pick = c0 + f;
                break;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const long long pick = sm.pick;
        chosen[t] = pick;
        if (pick >= 0 && pick < m) taken[pick] = 1;
        *counter = 0u;
        *t_dev = t + 1;
    }
}

// Narrow dense rows: one thread per row, FP32 difference form.
__global__ __launch_bounds__(kKppThreads, 2) void kpp_step_kernel(
    const float *__restrict__ X, int64_t m, int dp, int *__restrict__ t_dev,
    const unsigned long long *__restrict__ a53, float *__restrict__ D2,
    int32_t *__restrict__ asg, const float *__restrict__ cc2, unsigned long long *__restrict__ bsum,
    unsigned *__restrict__ counter, int64_t *__restrict__ chosen,
    unsigned char *__restrict__ taken, unsigned *__restrict__ s1_bits, int measure) {
    __shared__ unsigned long long red[kKppThreads / 32];
    __shared__ float fred[kKppThreads / 32];
    __shared__ int s_last;
    __shared__ KppDrawSmem sm;

    const int t = *t_dev;
    const int tid = threadIdx.x;
    const int dp4 = dp / 4;
    const float qs = measure ? 0.f : kpp_scale(s1_bits);
    int64_t c = chosen[t - 1];
    if (c < 0 || c >= m) c = 0;  // never out of bounds (a valid pick is always in [0, m))
    const float4 *crow = reinterpret_cast<const float4 *>(X + c * dp);
    const int64_t r0 = (int64_t)blockIdx.x * kKppRows;

    // D^2 update: thread owns rows r0 + tid + q * kKppThreads.  A row whose
    // nearest centre a lies at least 2 sqrt(D^2) (with a 1e-3 margin for
    // rounding) from the new centre cannot get closer to it (triangle
    // inequality), so its distance is not evaluated: the result is the same
    // as evaluating it and keeping min(D^2, distance).
    unsigned long long local = 0;
    float flocal = 0.f;
#pragma unroll
    for (int q = 0; q < kKppRpt; ++q) {
        const int64_t i = r0 + tid + q * kKppThreads;
        if (i >= m) continue;
        float d2 = FLT_MAX;
        int a = 0;
        bool eval = true;
        if (t > 1) {
            d2 = D2[i];
            a = asg[i];
            eval = !(cc2[a] >= 4.004f * d2);
        }
        if (eval) {
            const float4 *xr = reinterpret_cast<const float4 *>(X + i * dp);
            float acc = 0.f;
#pragma unroll 4
            for (int ch = 0; ch < dp4; ++ch) {
                const float4 xa = xr[ch], b = __ldg(crow + ch);
                const float e0 = xa.x - b.x, e1 = xa.y - b.y, e2 = xa.z - b.z, e3 = xa.w - b.w;
                acc = fmaf(e0, e0, acc);
                acc = fmaf(e1, e1, acc);
                acc = fmaf(e2, e2, acc);
                acc = fmaf(e3, e3, acc);
            }
            if (acc < d2) {
                d2 = acc;
                a = t - 1;
            }
            D2[i] = d2;
            asg[i] = a;
        }
        local += kpp_q(d2, qs);
        flocal += d2;
    }
    if (measure) {
        kpp_measure(flocal, fred, s1_bits);
        return;
    }
    if (!kpp_block_done(local, red, bsum, counter, &s_last)) return;
    kpp_draw<kKppRows>(t, m, a53, D2, qs, bsum, counter, t_dev, chosen, taken, sm);
}

// Wide dense rows (dp > kKppWideDim): one warp per row with coalesced float4
// loads, kKppWideRows rows per block so a few thousand rows still fill the
// GPU.  In many dimensions the pruning test above almost never holds, so it
// is not used here.
constexpr int kKppWideDim = 256;
constexpr int kKppWideRows = 64;
__global__ __launch_bounds__(kKppThreads) void kpp_step_wide_kernel(
    const float *__restrict__ X, int64_t m, int dp, int *__restrict__ t_dev,
    const unsigned long long *__restrict__ a53, float *__restrict__ D2,
    unsigned long long *__restrict__ bsum, unsigned *__restrict__ counter,
    int64_t *__restrict__ chosen, unsigned char *__restrict__ taken,
    unsigned *__restrict__ s1_bits, int measure) {
    __shared__ unsigned long long red[kKppThreads / 32];
    __shared__ float fred[kKppThreads / 32];
    __shared__ int s_last;
    __shared__ KppDrawSmem sm;
    constexpr int W = kKppThreads / 32;       // warps
    constexpr int RPW = kKppWideRows / W;     // rows per warp, all in flight

    const int t = *t_dev;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int dp4 = dp / 4;
    const float qs = measure ? 0.f : kpp_scale(s1_bits);
    int64_t c = chosen[t - 1];
    if (c < 0 || c >= m) c = 0;
    const float4 *crow = reinterpret_cast<const float4 *>(X + c * dp);
    const int64_t r0 = (int64_t)blockIdx.x * kKppWideRows + (int64_t)w * RPW;
    float acc[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) acc[q] = 0.f;
    for (int ch = lane; ch < dp4; ch += 32) {
        const float4 b = __ldg(crow + ch);
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int64_t i = r0 + q;
            if (i < m) {
                const float4 xa = reinterpret_cast<const float4 *>(X + i * dp)[ch];
                const float e0 = xa.x - b.x, e1 = xa.y - b.y, e2 = xa.z - b.z, e3 = xa.w - b.w;
                acc[q] = fmaf(e0, e0, acc[q]);
                acc[q] = fmaf(e1, e1, acc[q]);
                acc[q] = fmaf(e2, e2, acc[q]);
                acc[q] = fmaf(e3, e3, acc[q]);
            }
        }
    }
    unsigned long long local = 0;
    float flocal = 0.f;
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        float v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        const int64_t i = r0 + q;
        if (lane == 0 && i < m) {
            const float d2 = t > 1 ? fminf(D2[i], v) : v;
            D2[i] = d2;
            local += kpp_q(d2, qs);
            flocal += d2;
        }
    }
    if (measure) {
        kpp_measure(flocal, fred, s1_bits);
        return;
    }
    if (!kpp_block_done(local, red, bsum, counter, &s_last)) return;
    kpp_draw<kKppWideRows>(t, m, a53, D2, qs, bsum, counter, t_dev, chosen, taken, sm);
}

// CSR rows (§4.3 TF-IDF shape): the new centre (a CSR row) is scattered into a
// dense row in shared memory, and kKppGroup lanes take each row's nonzeros.
// With A = sum_{t in x} (x_t - c_t)^2 and B = sum_{t in x} c_t^2,
//   ||x - c||^2 = A + (||c||^2 - B),
// where ||c||^2 is summed by the same lane-group procedure over the centre's
// own nonzeros, so a row equal to the centre gets exactly 0.
constexpr int kKppGroup = 8;
__device__ __forceinline__ void csr_row_ab(const int64_t b, const int64_t e,
                                           const int32_t *__restrict__ col,
                                           const float *__restrict__ val, const float *cden,
                                           int gl, float &A, float &B) {
    A = 0.f;
    B = 0.f;
    for (int64_t j = b + gl; j < e; j += kKppGroup) {
        const float cv = cden[__ldg(col + j)];
        const float e0 = __ldg(val + j) - cv;
        A = fmaf(e0, e0, A);
        B = fmaf(cv, cv, B);
    }
#pragma unroll
    for (int o = kKppGroup / 2; o > 0; o >>= 1) {
        A += __shfl_xor_sync(kFull, A, o, kKppGroup);
        B += __shfl_xor_sync(kFull, B, o, kKppGroup);
    }
}

__global__ __launch_bounds__(kKppThreads, 2) void kpp_step_csr_kernel(
    const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
    const float *__restrict__ val, int64_t m, int dp, int *__restrict__ t_dev,
    const unsigned long long *__restrict__ a53, float *__restrict__ D2,
    unsigned long long *__restrict__ bsum, unsigned *__restrict__ counter,
    int64_t *__restrict__ chosen, unsigned char *__restrict__ taken,
    unsigned *__restrict__ s1_bits, int measure) {
    extern __shared__ __align__(16) float cden[];  // [dp] the new centre, dense
    __shared__ unsigned long long red[kKppThreads / 32];
    __shared__ float fred[kKppThreads / 32];
    __shared__ int s_last;
    __shared__ float s_cn;
    __shared__ KppDrawSmem sm;
    constexpr int G = kKppThreads / kKppGroup;  // lane groups (rows in flight per block)

    const int t = *t_dev;
    const int tid = threadIdx.x;
    const int g = tid / kKppGroup, gl = tid % kKppGroup;
    const float qs = measure ? 0.f : kpp_scale(s1_bits);
    int64_t c = chosen[t - 1];
    if (c < 0 || c >= m) c = 0;
    const int64_t cb = rp[c], ce = rp[c + 1];
    for (int i = tid; i < dp; i += kKppThreads) cden[i] = 0.f;
    __syncthreads();
    for (int64_t j = cb + tid; j < ce; j += kKppThreads) cden[col[j]] = val[j];
    __syncthreads();
    if (tid < 32) {
        // ||c||^2 by the row procedure: sum_{t in c} c_t^2 is B of the centre
        // itself (every group of warp 0 computes it; the shuffles need the warp)
        float A, B;
        csr_row_ab(cb, ce, col, val, cden, gl, A, B);
        if (tid == 0) s_cn = B;
    }
    __syncthreads();
    const float cn = s_cn;
    const int64_t r0 = (int64_t)blockIdx.x * kKppRows;
    unsigned long long local = 0;
    float flocal = 0.f;
#pragma unroll 2
    for (int q = 0; q < kKppRows / G; ++q) {
        const int64_t i = r0 + g + (int64_t)q * G;
        const bool ok = i < m;  // every lane reaches the shuffles; a row past the end is empty
        float A, B;
        csr_row_ab(ok ? rp[i] : 0, ok ? rp[i + 1] : 0, col, val, cden, gl, A, B);
        if (ok && gl == 0) {
            const float v = A + fmaxf(cn - B, 0.f);
            const float d2 = t > 1 ? fminf(D2[i], v) : v;
            D2[i] = d2;
            local += kpp_q(d2, qs);
            flocal += d2;
        }
    }
    if (measure) {
        kpp_measure(flocal, fred, s1_bits);
        return;
    }
    if (!kpp_block_done(local, red, bsum, counter, &s_last)) return;
    kpp_draw<kKppRows>(t, m, a53, D2, qs, bsum, counter, t_dev, chosen, taken, sm);
}

// ------------------------------------------------------------ label sort

__global__ void label_hist_kernel(const int32_t *__restrict__ labels, int64_t n,
                                  int32_t *__restrict__ counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + labels[i], 1);
}

// Exclusive scan of k counts into off[0..k] (one block of 1024 threads).
__global__ void __launch_bounds__(1024) count_scan_kernel(const int32_t *__restrict__ counts,
                                                          int k, int64_t *__restrict__ off) {
    __shared__ long long part[1024];
    const int tid = threadIdx.x;
    const int per = (k + 1023) / 1024;
    const int b = tid * per, e = min(k, b + per);
    long long s = 0;
    for (int j = b; j < e; ++j) s += counts[j];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    long long run = part[tid] - s;
    for (int j = b; j < e; ++j) {
        off[j] = run;
        run += counts[j];
    }
    if (tid == 1023) off[k] = part[1023];
}

__global__ void label_scatter_kernel(const int32_t *__restrict__ labels, int64_t n,
                                     const int64_t *__restrict__ off, int32_t *__restrict__ fill,
                                     int32_t *__restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = labels[i];
        const int32_t pos = atomicAdd(fill + l, 1);
        perm[off[l] + pos] = (int32_t)i;
    }
}

// Put each membership list in ascending item order (bitonic sort in shared
// memory; longer lists below), so sums over a cluster run in the same order
// on every build.
constexpr int kSegSortMax = 4096;
__global__ void __launch_bounds__(512) segment_sort_kernel(const int64_t *__restrict__ off,
                                                           int32_t *__restrict__ perm) {
    __shared__ int32_t s[kSegSortMax];
    const int64_t b = off[blockIdx.x], e = off[blockIdx.x + 1];
    const int m = (int)(e - b);
    if (m <= 1 || m > kSegSortMax) return;
    int S = 1;
    while (S < m) S <<= 1;
    for (int i = threadIdx.x; i < S; i += blockDim.x) s[i] = i < m ? perm[b + i] : INT_MAX;
    __syncthreads();
    for (int kk = 2; kk <= S; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < S; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    const int32_t a = s[i], c = s[ixj];
                    if ((a > c) == up) { s[i] = c; s[ixj] = a; }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < m; i += blockDim.x) perm[b + i] = s[i];
}

// Bitonic sort of perm[b, b + m) (block-wide) through tmp[2 b, 2 b + S).
__device__ void sort_long_list(int32_t *__restrict__ perm, int32_t *__restrict__ tmp, int64_t b,
                               int64_t m) {
    int64_t S = 1;
    while (S < m) S <<= 1;
    int32_t *t = tmp + 2 * b;
    for (int64_t i = threadIdx.x; i < S; i += blockDim.x) t[i] = i < m ? perm[b + i] : INT_MAX;
    __syncthreads();
    for (int64_t kk = 2; kk <= S; kk <<= 1)
        for (int64_t j = kk >> 1; j > 0; j >>= 1) {
            for (int64_t i = threadIdx.x; i < S; i += blockDim.x) {
                const int64_t ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    const int32_t a = t[i], c = t[ixj];
                    if ((a > c) == up) { t[i] = c; t[ixj] = a; }
                }
            }
            __syncthreads();
        }
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) perm[b + i] = t[i];
    __syncthreads();
}

// Lists longer than kSegSortMax: blocks stride over the lists and sort each
// long one by a bitonic sort in global memory over a padded copy (tmp holds
// 2 x n ints: list j uses [2 b, 2 b + S) with S < 2 m, so the regions of
// different lists never overlap).
__global__ void __launch_bounds__(1024) segment_sort_big_kernel(const int64_t *__restrict__ off,
                                                                int k,
                                                                int32_t *__restrict__ perm,
                                                                int32_t *__restrict__ tmp) {
    for (int j = blockIdx.x; j < k; j += gridDim.x) {
        const int64_t b = off[j], e = off[j + 1];
        const int64_t m = e - b;
        if (m > kSegSortMax) sort_long_list(perm, tmp, b, m);
    }
}

// --------------------------------------------------------- centroid update

// One block per (cluster j, column slice): sum the members' rows (gathered
// through the label-sorted membership list) and their squared distances to the
// previous centroid; C_new[j] = sum / count, or C_prev[j] for an empty cluster.
template <int LPR, int CPL, class Acc>
__device__ void update_body(const float4 *__restrict__ X, int dp4, const int32_t *__restrict__ perm,
                            int64_t b, int64_t m, const float4 *cp, float4 *__restrict__ Cn,
                            float *__restrict__ sse, int j, int ch0, bool write, float *fred) {
    extern __shared__ __align__(16) unsigned char dyn[];
    Acc *accs = reinterpret_cast<Acc *>(dyn);  // [G][LPR*CPL][4] partial sums
    const int tid = threadIdx.x;
    constexpr int G = 256 / LPR;
    const int g = tid / LPR, gl = tid % LPR;
    Acc ax[CPL], ay[CPL], az[CPL], aw[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) ax[q] = ay[q] = az[q] = aw[q] = Acc(0);
    float sl = 0.f;
#pragma unroll 1
    for (int64_t r = g; r < m; r += G) {
        const int64_t row = perm[b + r];
        const float4 *xr = X + row * dp4;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int ch = ch0 + gl + q * LPR;
            if (ch < dp4) {
                const float4 v = xr[ch];
                ax[q] += v.x; ay[q] += v.y; az[q] += v.z; aw[q] += v.w;
                const float e0 = v.x - cp[q].x, e1 = v.y - cp[q].y, e2 = v.z - cp[q].z,
                            e3 = v.w - cp[q].w;
                sl = fmaf(e0, e0, sl); sl = fmaf(e1, e1, sl);
                sl = fmaf(e2, e2, sl); sl = fmaf(e3, e3, sl);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        Acc *p = accs + ((size_t)g * LPR * CPL + gl * CPL + q) * 4;
        p[0] = ax[q]; p[1] = ay[q]; p[2] = az[q]; p[3] = aw[q];
    }
    for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(kFull, sl, o);
    if ((tid & 31) == 0) fred[tid >> 5] = sl;
    __syncthreads();
    // column sums over the G groups, in group order; then the mean
    if (write && tid < LPR * CPL) {
        const int lane_in = tid / CPL, q = tid % CPL;
        const int ch = ch0 + lane_in + q * LPR;
        Acc s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll 1
        for (int gg = 0; gg < G; ++gg) {
            const Acc *p = accs + ((size_t)gg * LPR * CPL + lane_in * CPL + q) * 4;
            s0 += p[0]; s1 += p[1]; s2 += p[2]; s3 += p[3];
        }
        if (ch < dp4) {
            const Acc cnt = Acc(m);
            Cn[(int64_t)j * dp4 + ch] = make_float4((float)(s0 / cnt), (float)(s1 / cnt),
                                                    (float)(s2 / cnt), (float)(s3 / cnt));
        }
    }
    if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += fred[w];
        atomicAdd(sse + j, t);
    }
}

template <int LPR, int CPL>
__global__ __launch_bounds__(256) void centroid_update_kernel(
    const float4 *__restrict__ X, int dp4, const int32_t *__restrict__ perm,
    const int64_t *__restrict__ off, const float4 *__restrict__ Cp, float4 *__restrict__ Cn,
    float *__restrict__ sse, int write) {
    __shared__ float fred[8];
    const int j = blockIdx.x;
    const int ch0 = blockIdx.y * LPR * CPL;
    const int gl = threadIdx.x % LPR;
    const int64_t b = off[j], m = off[j + 1] - b;
    float4 cp[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int ch = ch0 + gl + q * LPR;
        cp[q] = ch < dp4 ? Cp[(int64_t)j * dp4 + ch] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (m == 0) {
        // empty cluster: keep the previous centroid
        if (write && threadIdx.x < LPR * CPL) {
            const int ch = ch0 + threadIdx.x;
            if (ch < dp4) Cn[(int64_t)j * dp4 + ch] = Cp[(int64_t)j * dp4 + ch];
        }
        return;
    }
    if (m > (1 << 20))
        update_body<LPR, CPL, double>(X, dp4, perm, b, m, cp, Cn, sse, j, ch0, write != 0, fred);
    else
        update_body<LPR, CPL, float>(X, dp4, perm, b, m, cp, Cn, sse, j, ch0, write != 0, fred);
}

__global__ void off_to_counts_kernel(const int64_t *__restrict__ off, int k,
                                     int64_t *__restrict__ counts) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x)
        counts[j] = off[j + 1] - off[j];
}

__global__ void count_bad_labels_kernel(const int32_t *__restrict__ labels, int64_t n, int k,
                                        int *__restrict__ bad) {
    int b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b += (labels[i] < 0 || labels[i] >= k) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(kFull, b, o);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(bad, b);
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

// ================================================================ launchers

void pad_rows(const float *src, int64_t n, int d, float *dst, int dp, cudaStream_t s) {
    if (n == 0) return;
    pad_rows_kernel<<<grid_for(n * dp, 256), 256, 0, s>>>(src, n, d, dst, dp);
    MASK_LAUNCHED("pad_rows");
}

void unpad_rows(const float *src, int64_t n, int dp, float *dst, int d, cudaStream_t s) {
    if (n == 0) return;
    unpad_rows_kernel<<<grid_for(n * d, 256), 256, 0, s>>>(src, n, dp, dst, d);
    MASK_LAUNCHED("unpad_rows");
}

template <class I>
void gather_rows(const float *src, int dp, const I *idx, int64_t m, float *dst, cudaStream_t s) {
    if (m == 0) return;
    gather_rows_kernel<I><<<grid_for(m * (dp / 4), 256), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(src), dp / 4, idx, m, reinterpret_cast<float4 *>(dst));
    MASK_LAUNCHED("gather_rows");
}
template void gather_rows<int32_t>(const float *, int, const int32_t *, int64_t, float *,
                                   cudaStream_t);
template void gather_rows<int64_t>(const float *, int, const int64_t *, int64_t, float *,
                                   cudaStream_t);

void iota_i32(int32_t *p, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n);
    MASK_LAUNCHED("iota");
}

#define MASK_LPR_DISPATCH(lpr, KERNEL_CALL)      \
    switch (lpr) {                               \
    case 1: { constexpr int L = 1; KERNEL_CALL; } break;   \
    case 2: { constexpr int L = 2; KERNEL_CALL; } break;   \
    case 4: { constexpr int L = 4; KERNEL_CALL; } break;   \
    case 8: { constexpr int L = 8; KERNEL_CALL; } break;   \
    case 16: { constexpr int L = 16; KERNEL_CALL; } break; \
    default: { constexpr int L = 32; KERNEL_CALL; } break; \
    }

void row_sqnorm(const float *X, int64_t n, int dp, float *out, cudaStream_t s) {
    if (n == 0) return;
    const int lpr = lanes_per_row(dp);
    const int grid = grid_for(n * lpr, 256);
    MASK_LPR_DISPATCH(lpr, (row_sqnorm_kernel<L><<<grid, 256, 0, s>>>(
                               reinterpret_cast<const float4 *>(X), n, dp / 4, out)));
    MASK_LAUNCHED("row_sqnorm");
}

void label_dist(const float *X, int64_t n, int dp, const float *C, const int32_t *labels,
                float *dist, cudaStream_t s) {
    if (n == 0) return;
    const int lpr = lanes_per_row(dp);
    const int grid = grid_for(n * lpr, 256);
    MASK_LPR_DISPATCH(lpr, (label_dist_kernel<L><<<grid, 256, 0, s>>>(
                               reinterpret_cast<const float4 *>(X), n, dp / 4,
                               reinterpret_cast<const float4 *>(C), labels, dist)));
    MASK_LAUNCHED("label_dist");
}

void max_reduce(const float *v, int64_t n, float *out, cudaStream_t s) {
    MASK_CUDA(cudaMemsetAsync(out, 0, sizeof(float), s));
    if (n == 0) return;
    max_reduce_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, n, out);
    MASK_LAUNCHED("max_reduce");
}

// Run `steps` identical k-means++ step launches (the step number lives on the
// device): a captured graph of kBatch steps is replayed, the rest run directly.
template <class F>
void replay_steps(int steps, int kernels_per_step, F &&launch, cudaStream_t s) {
    constexpr int kBatch = 64;
    int done = 0;
    if (steps >= 2 * kBatch) {
        cudaStream_t cs;
        MASK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int i = 0; i < kBatch; ++i) launch(cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) {
            for (; done + kBatch <= steps && e == cudaSuccess; done += kBatch) {
                e = cudaGraphLaunch(exec, s);
                for (int i = 0; i < kernels_per_step * kBatch; ++i) count_launch();
            }
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) fail(MASK_ECUDA, std::string("kmeans++ graph: ") + cudaGetErrorString(e));
    }
    for (; done < steps; ++done) {
        launch(s);
        for (int i = 0; i < kernels_per_step; ++i) count_launch();
        MASK_LAUNCHED("kpp_step");
    }
}

struct KppState {
    Scratch<float> D2;
    Scratch<unsigned long long> bsum;
    Scratch<unsigned> counter, s1;   // s1: bound of the first step's sum (FP32 bits)
    Scratch<int> t_dev;
    Scratch<unsigned char> taken;
    KppState(int64_t m, int nb, cudaStream_t s)
        : D2(m, s), bsum(nb, s), counter(1, s), s1(1, s), t_dev(1, s), taken(m, s) {
        const int one = 1;
        MASK_CUDA(cudaMemsetAsync(counter.get(), 0, sizeof(unsigned), s));
        MASK_CUDA(cudaMemsetAsync(s1.get(), 0, sizeof(unsigned), s));
        MASK_CUDA(cudaMemsetAsync(taken.get(), 0, m, s));
        MASK_CUDA(cudaMemcpyAsync(t_dev.get(), &one, sizeof(int), cudaMemcpyHostToDevice, s));
    }
};

// Each seeding run starts with one measuring launch of its step kernel (the
// first step's D^2 and the bound of its sum that fixes the integer scale),
// then replays the steps.
void kmeanspp_steps(const float *Xs, int64_t m, int dp, int k, const unsigned long long *a53,
                    int64_t *chosen, cudaStream_t s) {
    if (k <= 1) return;
    ProfRegion pr("kmeanspp", s, (double)(k - 1) * (double)m * dp * 4.0);
    if (dp > kKppWideDim) {
        const int nb = (int)((m + kKppWideRows - 1) / kKppWideRows);
        KppState st(m, nb, s);
        auto launch = [&](cudaStream_t cs, int measure) {
            kpp_step_wide_kernel<<<nb, kKppThreads, 0, cs>>>(Xs, m, dp, st.t_dev.get(), a53,
                                                             st.D2.get(), st.bsum.get(),
                                                             st.counter.get(), chosen,
                                                             st.taken.get(), st.s1.get(), measure);
        };
        launch(s, 1);
        MASK_LAUNCHED("kpp_measure");
        replay_steps(k - 1, 1, [&](cudaStream_t cs) { launch(cs, 0); }, s);
        return;
    }
    const int nb = (int)((m + kKppRows - 1) / kKppRows);
    KppState st(m, nb, s);
    Scratch<float> cc2(k, s);
    Scratch<int32_t> asg(m, s);
    const int ccb = (k + 255) / 256;
    auto step = [&](cudaStream_t cs, int measure) {
        kpp_step_kernel<<<nb, kKppThreads, 0, cs>>>(Xs, m, dp, st.t_dev.get(), a53, st.D2.get(),
                                                    asg.get(), cc2.get(), st.bsum.get(),
                                                    st.counter.get(), chosen, st.taken.get(),
                                                    st.s1.get(), measure);
    };
    step(s, 1);
    MASK_LAUNCHED("kpp_measure");
    replay_steps(k - 1, 2, [&](cudaStream_t cs) {
        kpp_centre_dist_kernel<<<ccb, 256, 0, cs>>>(Xs, m, dp, st.t_dev.get(), chosen, cc2.get());
        step(cs, 0);
    }, s);
}

void kmeanspp_steps_csr(const int64_t *rp, const int32_t *col, const float *val, int64_t m,
                        int64_t nnz, int dp, int k, const unsigned long long *a53,
                        int64_t *chosen, cudaStream_t s) {
    if (k <= 1) return;
    const size_t smem = (size_t)dp * sizeof(float);
    MASK_REQUIRE(smem <= (size_t)kCsrMaxDim * sizeof(float), "CSR dimension too large");
    // per step: every nonzero (column + value) and, per row, its pointer and D^2
    ProfRegion pr("kmeanspp", s, (double)(k - 1) * (8.0 * (double)nnz + 16.0 * (double)m));
    MASK_CUDA(cudaFuncSetAttribute(kpp_step_csr_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nb = (int)((m + kKppRows - 1) / kKppRows);
    KppState st(m, nb, s);
    auto launch = [&](cudaStream_t cs, int measure) {
        kpp_step_csr_kernel<<<nb, kKppThreads, smem, cs>>>(rp, col, val, m, dp, st.t_dev.get(),
                                                           a53, st.D2.get(), st.bsum.get(),
                                                           st.counter.get(), chosen,
                                                           st.taken.get(), st.s1.get(), measure);
    };
    launch(s, 1);
    MASK_LAUNCHED("kpp_measure");
    replay_steps(k - 1, 1, [&](cudaStream_t cs) { launch(cs, 0); }, s);
}

void label_sort(const int32_t *labels, int64_t n, int k, int64_t *off, int32_t *perm,
                cudaStream_t s) {
    ProfRegion pr("label_sort", s, 20.0 * (double)n + 16.0 * (double)k);
    Scratch<int32_t> counts(k, s), fill(k, s);
    MASK_CUDA(cudaMemsetAsync(counts.get(), 0, sizeof(int32_t) * k, s));
    MASK_CUDA(cudaMemsetAsync(fill.get(), 0, sizeof(int32_t) * k, s));
    if (n > 0) {
        label_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(labels, n, counts.get());
        MASK_LAUNCHED("label_hist");
    }
    count_scan_kernel<<<1, 1024, 0, s>>>(counts.get(), k, off);
    MASK_LAUNCHED("count_scan");
    if (n > 0) {
        label_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(labels, n, off, fill.get(), perm);
        MASK_LAUNCHED("label_scatter");
        segment_sort_kernel<<<k, 512, 0, s>>>(off, perm);
        MASK_LAUNCHED("segment_sort");
        if (n > kSegSortMax) {
            // only lists longer than kSegSortMax do work here
            Scratch<int32_t> tmp((size_t)2 * n, s);
            segment_sort_big_kernel<<<std::min(k, 152 * 2), 1024, 0, s>>>(off, k, perm, tmp.get());
            MASK_LAUNCHED("segment_sort_big");
        }
    }
}

template <int L, int CPL>
void launch_update(dim3 grid, size_t smem, const float *X, int dp4, const int32_t *perm,
                   const int64_t *off, int k, const float *C_prev, float *C_new, float *sse,
                   bool write, cudaStream_t s) {
    (void)k;
    auto kfn = centroid_update_kernel<L, CPL>;
    MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, 256, smem, s>>>(reinterpret_cast<const float4 *>(X), dp4, perm, off,
                                reinterpret_cast<const float4 *>(C_prev),
                                reinterpret_cast<float4 *>(C_new), sse, write ? 1 : 0);
}

void centroid_update(const float *X, int dp, const int32_t *perm, const int64_t *off, int k,
                     const float *C_prev, float *C_new, float *sse, bool write,
                     cudaStream_t s) {
    const int dp4 = dp / 4;
    const int lpr = lanes_per_row(dp);
    int cpl = (dp4 + lpr - 1) / lpr;
    cpl = cpl >= 4 ? 4 : (cpl >= 2 ? 2 : 1);
    const int slices = (dp4 + lpr * cpl - 1) / (lpr * cpl);
    MASK_CUDA(cudaMemsetAsync(sse, 0, sizeof(float) * k, s));
    ProfRegion pr("centroid_update", s, 0.0);
    dim3 grid(k, slices);
    // dynamic shared memory holds the per-group partial sums (FP64 worst case)
    const size_t smem = (size_t)(256 / lpr) * lpr * cpl * 4 * sizeof(double);
    if (cpl == 1) {
        MASK_LPR_DISPATCH(lpr, (launch_update<L, 1>(grid, smem, X, dp4, perm, off, k, C_prev, C_new, sse, write, s)));
    } else if (cpl == 2) {
        MASK_LPR_DISPATCH(lpr, (launch_update<L, 2>(grid, smem, X, dp4, perm, off, k, C_prev, C_new, sse, write, s)));
    } else {
        MASK_LPR_DISPATCH(lpr, (launch_update<L, 4>(grid, smem, X, dp4, perm, off, k, C_prev, C_new, sse, write, s)));
    }
    MASK_LAUNCHED("centroid_update");
}

void off_to_counts(const int64_t *off, int k, int64_t *counts, cudaStream_t s) {
    if (k == 0) return;
    off_to_counts_kernel<<<grid_for(k, 256), 256, 0, s>>>(off, k, counts);
    MASK_LAUNCHED("off_to_counts");
}

void count_bad_labels(const int32_t *labels, int64_t n, int k, int *bad, cudaStream_t s) {
    MASK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (n == 0) return;
    count_bad_labels_kernel<<<grid_for(n, 256), 256, 0, s>>>(labels, n, k, bad);
    MASK_LAUNCHED("count_bad_labels");
}

}  // namespace mask
