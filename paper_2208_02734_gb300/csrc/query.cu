// query.cu -- one kernel for every step of the top-down k-NN search (§3.3,
// Algorithm 2, generalised to p kept centroids per level):
//
//   keep the K nearest rows among the children of each query's kept parents.
//
// The index stores every level parent-major: the children of a parent occupy
// one contiguous row range (off[parent] .. off[parent+1]) of the level below,
// and the points of a leaf cluster one contiguous range of the cluster-major
// point array.  So the top level (root range), each intermediate level and
// the final leaf scan are the same operation: stream a few row ranges, take
// exact FP32 distances sum_t (q_t - r_t)^2, keep the K smallest keys
// (distance bits << 32 | id) -- a total order, so the result does not depend
// on the order rows are visited in or on the other queries in the launch.
//
// One block per query; each thread owns whole rows and sums (r_t - q_t)^2 in
// increasing t with FMAs -- the same arithmetic as the cluster-major leaf scan
// (query_cm.cu), so a distance does not depend on which kernel computed it.
// Candidates below the current K-th key are appended to a shared-memory
// buffer, which is bitonic-sorted together with the current top list whenever
// it could overflow.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace mask {

// Bytes the scan kernels stream (rows x (row + id)), [0] levels, [1] leaf.
__device__ unsigned long long g_scan_bytes[2];

// Device address of a byte counter while profiling is on; null otherwise, so
// the kernels skip the count (one uniform test, no atomic) in normal runs.
unsigned long long *scan_bytes_counter(int which) {
    if (!profiling_enabled()) return nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scan_bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned long long *>(p) + which;
}

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kUnroll = 2;  // rows per thread per round

__device__ __forceinline__ void bitonic_sort_keys(unsigned long long *buf, int S) {
    for (int kk = 2; kk <= S; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < S; i += kThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    const unsigned long long a = buf[i], b = buf[ixj];
                    if ((a > b) == up) { buf[i] = b; buf[ixj] = a; }
                }
            }
            __syncthreads();
        }
}

// The key of 0-based rank `rank` among keys[0..n) (distinct keys), by a
// most-significant-digit-first radix select over 8-bit digits: each pass
// histograms the digit of the keys that share the digits fixed so far, and
// the select stops as soon as the rank falls on a digit held by one key.
__device__ unsigned long long radix_kth(const unsigned long long *keys, int n, int rank) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix, s_mask, s_kth;
    __shared__ int s_rank, s_done;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        s_prefix = 0;
        s_mask = 0;
        s_rank = rank;
        s_done = 0;
    }
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += kThreads) hist[i] = 0;
        __syncthreads();
        const unsigned long long pre = s_prefix, msk = s_mask;
        for (int i = tid; i < n; i += kThreads) {
            const unsigned long long k = keys[i];
            if ((k & msk) == pre) atomicAdd(&hist[(unsigned)(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid < 32) {
            unsigned c[8], ls = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                c[j] = hist[lane * 8 + j];
                ls += c[j];
            }
            unsigned inc = ls;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += v;
            }
            const unsigned r = (unsigned)s_rank;
            unsigned run = inc - ls;
            if (run <= r && r < inc) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (r < run + c[j]) {
                        s_prefix = pre | ((unsigned long long)(lane * 8 + j) << shift);
                        s_mask = msk | (255ull << shift);
                        s_rank = (int)(r - run);
                        s_done = c[j] == 1;
                        break;
                    }
                    run += c[j];
                }
            }
        }
        __syncthreads();
        if (s_done) break;
    }
    if (s_done) {
        const unsigned long long pre = s_prefix, msk = s_mask;
        for (int i = tid; i < n; i += kThreads)
            if ((keys[i] & msk) == pre) s_kth = keys[i];
    } else if (tid == 0) {
        s_kth = s_prefix;
    }
    __syncthreads();
    const unsigned long long r = s_kth;
    __syncthreads();
    return r;
}

// Squared distance of one row to the query, t ascending (FMA per term).
__device__ __forceinline__ float row_sqdist(const float4 *__restrict__ row, const float4 *qs,
                                            int dp4) {
    float acc = 0.f;
#pragma unroll 4
    for (int c = 0; c < dp4; ++c) {
        const float4 v = row[c], q = qs[c];
        float e = v.x - q.x;
        acc = fmaf(e, e, acc);
        e = v.y - q.y;
        acc = fmaf(e, e, acc);
        e = v.z - q.z;
        acc = fmaf(e, e, acc);
        e = v.w - q.w;
        acc = fmaf(e, e, acc);
    }
    return acc;
}

// ROWWISE: one thread per row, t ascending (the leaf arithmetic shared with
// the cluster-major scan).  Otherwise groups of LPR lanes read a row with
// coalesced float4 loads and reduce by shuffles (the centroid levels, whose
// results only ever come from this kernel).
template <bool ROWWISE, int LPR>
__global__ __launch_bounds__(kThreads) void scan_topk_kernel(
    const float4 *__restrict__ R, int dp4, const int32_t *__restrict__ rid,
    const int64_t *__restrict__ off, const int32_t *__restrict__ sel, int P, int64_t root_end,
    const float4 *__restrict__ Q, int K, int KP, int S, int32_t *__restrict__ out32,
    int64_t *__restrict__ out64, float *__restrict__ out_d,
    unsigned long long *__restrict__ bytes_ctr, int sorted) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *buf = reinterpret_cast<unsigned long long *>(smem);  // S keys
    // KP keys, padded to an even count so the float4 query chunks below stay
    // 16-byte aligned (S is even; rb and cum together hold an even count)
    unsigned long long *pick = buf + S;
    int64_t *rb = reinterpret_cast<int64_t *>(pick + (KP + (KP & 1)));       // P range begins
    int64_t *cum = rb + P;                                                   // P+1 prefix sizes
    float4 *qs = reinterpret_cast<float4 *>(cum + P + 2);                    // dp4 query chunks
    __shared__ int cnt;
    __shared__ unsigned long long thresh;

    // rows per round: rowwise, kUnroll per thread; lane groups, 4 per group
    constexpr int ROUND = ROWWISE ? kThreads * kUnroll : (kThreads / LPR) * 4;
    const int tid = threadIdx.x;
    const int64_t q = blockIdx.x;

    for (int c = tid; c < dp4; c += kThreads) qs[c] = Q[q * dp4 + c];
    for (int i = tid; i < S; i += kThreads) buf[i] = kNoKey;
    if (tid == 0) {
        cnt = 0;
        thresh = kNoKey;
        cum[0] = 0;
        if (sel == nullptr) {
            rb[0] = 0;
            cum[1] = root_end;
        }
    }
    if (sel != nullptr) {
        // the kept parents' row ranges, one thread each (loads in parallel);
        // cum[s + 1] holds range s's length until warp 0 turns it into a prefix
        for (int s = tid; s < P; s += kThreads) {
            const int32_t p = sel[q * P + s];
            int64_t b = 0, e = 0;
            if (p >= 0) { b = off[p]; e = off[p + 1]; }
            rb[s] = b;
            cum[s + 1] = e - b;
        }
        __syncthreads();
        if (tid < 32) {
            long long carry = 0;
            for (int c0 = 0; c0 < P; c0 += 32) {
                const int s = c0 + tid;
                long long v = s < P ? cum[s + 1] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    const long long n = __shfl_up_sync(kFull, v, o);
                    if (tid >= o) v += n;
                }
                if (s < P) cum[s + 1] = carry + v;
                carry += __shfl_sync(kFull, v, 31);
            }
        }
    }
    __syncthreads();
    const int nr = sel == nullptr ? 1 : P;
    const int64_t T = cum[nr];
    const int lim = S - KP - ROUND;
    // centroid levels whose candidates all fit: every key is kept (candidate
    // t at buf[t]) and the K smallest are selected once at the end
    const bool direct = !ROWWISE && T <= S;
    if (bytes_ctr != nullptr && tid == 0)
        atomicAdd(bytes_ctr, (unsigned long long)T * (dp4 * 16ull + 4ull));

    for (int64_t base = 0; base < T; base += ROUND) {
        const unsigned long long th = thresh;
        if (ROWWISE) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t t = base + tid + (int64_t)u * kThreads;
                if (t < T) {
                    // the range holding t: the last s with cum[s] <= t
                    int lo = 0, hi = nr - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (cum[mid] <= t) lo = mid; else hi = mid - 1;
                    }
                    const int64_t row = rb[lo] + (t - cum[lo]);
                    const float dist = row_sqdist(R + row * dp4, qs, dp4);
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)rid[row];
                    if (key < th) buf[KP + atomicAdd(&cnt, 1)] = key;
                }
            }
        } else {
            // lane groups: ROUND rows = (kThreads / LPR) groups x (kUnroll * LPR) rows
            // each, four rows in flight per group
            constexpr int G = kThreads / LPR;
            constexpr int PER = 4;
            const int g = tid / LPR, gl = tid % LPR;
#pragma unroll 1
            for (int u0 = 0; u0 < PER; u0 += 4) {
                int64_t row[4], tt[4];
                float acc[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int64_t t = base + g + (int64_t)(u0 + i) * G;
                    tt[i] = t;
                    row[i] = -1;
                    acc[i] = 0.f;
                    if (u0 + i < PER && t < T) {
                        int lo = 0, hi = nr - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (cum[mid] <= t) lo = mid; else hi = mid - 1;
                        }
                        row[i] = rb[lo] + (t - cum[lo]);
                    }
                }
                for (int c = gl; c < dp4; c += LPR) {
                    const float4 qv = qs[c];
                    float4 v[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[i] = row[i] >= 0 ? R[row[i] * dp4 + c] : qv;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float e0 = v[i].x - qv.x, e1 = v[i].y - qv.y, e2 = v[i].z - qv.z,
                                    e3 = v[i].w - qv.w;
                        acc[i] = fmaf(e0, e0, acc[i]);
                        acc[i] = fmaf(e1, e1, acc[i]);
                        acc[i] = fmaf(e2, e2, acc[i]);
                        acc[i] = fmaf(e3, e3, acc[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    for (int o = LPR / 2; o > 0; o >>= 1)
                        acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
                if (gl == 0) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (row[i] < 0) continue;
                        const unsigned long long key =
                            ((unsigned long long)__float_as_uint(acc[i]) << 32) |
                            (unsigned)rid[row[i]];
                        if (direct) buf[tt[i]] = key;
                        else if (key < th) buf[KP + atomicAdd(&cnt, 1)] = key;
                    }
                }
            }
        }
        if (direct) continue;
        __syncthreads();
        const int c_now = cnt;
        __syncthreads();
        if (c_now > lim || base + ROUND >= T) {
            // sort only the filled prefix (the list and this round's candidates,
            // rounded up to a power of two; the rest are empty keys)
            int L = KP;
            while (L < KP + c_now) L <<= 1;
            for (int i = KP + c_now + tid; i < L; i += kThreads) buf[i] = kNoKey;
            __syncthreads();
            bitonic_sort_keys(buf, L);
            for (int i = K + tid; i < KP; i += kThreads) buf[i] = kNoKey;
            if (tid == 0) {
                thresh = buf[K - 1];
                cnt = 0;
            }
            __syncthreads();
        }
    }
    if (direct) {
        // the K smallest of the T keys: radix-select the K-th, gather the keys
        // up to it (distinct keys: exactly K), sort only those
        __syncthreads();
        const int Ti = (int)T;
        int nsel = Ti;
        if (Ti <= K) {
            for (int i = tid; i < Ti; i += kThreads) pick[i] = buf[i];
        } else {
            const unsigned long long kth = radix_kth(buf, Ti, K - 1);
            if (tid == 0) cnt = 0;
            __syncthreads();
            for (int i = tid; i < Ti; i += kThreads) {
                const unsigned long long k = buf[i];
                if (k <= kth) {
                    const int slot = atomicAdd(&cnt, 1);
                    if (slot < KP) pick[slot] = k;
                }
            }
            __syncthreads();
            nsel = min(cnt, K);
        }
        if (sorted) {
            int L = 1;
            while (L < nsel) L <<= 1;
            for (int i = nsel + tid; i < L; i += kThreads) pick[i] = kNoKey;
            __syncthreads();
            bitonic_sort_keys(pick, L);
        } else {
            // the caller reads the keys as a set, except that the smallest
            // comes first: find it (block reduction) and swap it to the front
            __shared__ unsigned long long s_min[kThreads / 32];
            __shared__ int s_at[kThreads / 32];
            unsigned long long mn = kNoKey;
            int at = 0;
            for (int i = tid; i < nsel; i += kThreads)
                if (pick[i] < mn) { mn = pick[i]; at = i; }
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long v = __shfl_xor_sync(kFull, mn, o);
                const int ai = __shfl_xor_sync(kFull, at, o);
                if (v < mn) { mn = v; at = ai; }
            }
            if ((tid & 31) == 0) { s_min[tid >> 5] = mn; s_at[tid >> 5] = at; }
            __syncthreads();
            if (tid == 0 && nsel > 0) {
                int a0 = s_at[0];
                unsigned long long m0 = s_min[0];
                for (int w = 1; w < kThreads / 32; ++w)
                    if (s_min[w] < m0) { m0 = s_min[w]; a0 = s_at[w]; }
                pick[a0] = pick[0];
                pick[0] = m0;
            }
            __syncthreads();
        }
        for (int i = tid; i < K; i += kThreads) buf[i] = i < nsel ? pick[i] : kNoKey;
        __syncthreads();
    }
    for (int r = tid; r < K; r += kThreads) {
        const unsigned long long key = buf[r];
        const bool ok = key != kNoKey;
        const int32_t id = ok ? (int32_t)(key & 0xffffffffu) : -1;
        const float dist = ok ? __uint_as_float((unsigned)(key >> 32)) : __int_as_float(0x7f800000);
        if (out32) out32[q * K + r] = id;
        if (out64) out64[q * K + r] = id;
        if (out_d) out_d[q * K + r] = dist;
    }
}

// Lanes per row of the centroid-level distances (scan_topk_kernel's lane
// groups and the greedy descent, which must agree): at most 4, so a row of
// up to 64 floats takes at most two shuffle steps to reduce.
int level_lanes_per_row(int dp) { return std::min(lanes_per_row(dp), 4); }

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}


// The greedy descent of the paper's point query (§3.3: one kept centroid per
// level, then the nearest point of the reached leaf cluster), one warp per
// query through all levels in one launch.  Level rows are evaluated by groups
// of LPR lanes and leaf rows one per lane, with exactly the arithmetic of the
// level and leaf scans above, and every choice is the smallest (distance, id)
// key, so the results are those of the general descent with all probes 1.
template <int LPR>
__global__ __launch_bounds__(kThreads) void greedy_descent_kernel(GreedyLevels lv, int L,
                                                                  const float4 *__restrict__ Xs,
                                                                  const int32_t *__restrict__ xids,
                                                                  const float4 *__restrict__ Q,
                                                                  int64_t nq, int dp4,
                                                                  int32_t *__restrict__ leaf_out,
                                                                  int64_t *__restrict__ id_out,
                                                                  float *__restrict__ d_out) {
    constexpr int G = 32 / LPR;   // rows per warp step
    const int lane = threadIdx.x & 31, g = lane / LPR, gl = lane % LPR;
    const int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;   // whole warps leave together
    const float4 *qv = Q + q * dp4;
    int64_t b = 0, e = lv.k_top;
    int32_t c = -1;
    for (int l = L - 1; l >= 0; --l) {
        const float4 *R = lv.Cs[l];
        const int32_t *rid = lv.ids[l];
        unsigned long long best = kNoKey;
        for (int64_t r0 = b; r0 < e; r0 += G) {
            const int64_t row = r0 + g;
            float acc = 0.f;
            if (row < e) {
                for (int ch = gl; ch < dp4; ch += LPR) {
                    const float4 v = R[row * dp4 + ch], x = qv[ch];
                    const float e0 = v.x - x.x, e1 = v.y - x.y, e2 = v.z - x.z, e3 = v.w - x.w;
                    acc = fmaf(e0, e0, acc);
                    acc = fmaf(e1, e1, acc);
                    acc = fmaf(e2, e2, acc);
                    acc = fmaf(e3, e3, acc);
                }
            }
            for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if (row < e && gl == 0)
                best = min(best, ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)rid[row]);
        }
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
        if (best == kNoKey) { c = -1; break; }   // a kept centroid with no children
        c = (int32_t)(best & 0xffffffffull);
        b = lv.off[l][c];
        e = lv.off[l][c + 1];
    }
    if (leaf_out && lane == 0) leaf_out[q] = c;
    if (!id_out) return;
    unsigned long long best = kNoKey;
    if (c >= 0) {
        __shared__ __align__(16) float4 qsh[kThreads / 32][32];
        const int w = threadIdx.x >> 5;
        for (int ch = lane; ch < dp4 && ch < 32; ch += 32) qsh[w][ch] = qv[ch];
        __syncwarp();
        const float4 *qs = dp4 <= 32 ? qsh[w] : qv;
        for (int64_t row = b + lane; row < e; row += 32) {
            const float dist = row_sqdist(Xs + row * dp4, qs, dp4);
            best = min(best, ((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)xids[row]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
    if (lane == 0) {
        id_out[q] = best == kNoKey ? -1 : (int64_t)(best & 0xffffffffull);
        if (d_out) d_out[q] = best == kNoKey ? __int_as_float(0x7f800000)
                                             : __uint_as_float((unsigned)(best >> 32));
    }
}
}  // namespace

void scan_topk(const ScanArgs &a, cudaStream_t s) {
    if (a.nq == 0) return;
    MASK_REQUIRE(a.K >= 1 && a.K <= 4096, "scan_topk: K out of range");
    const int round =
        a.out_ids64 ? kThreads * kUnroll : (kThreads / level_lanes_per_row(a.dp)) * 4;
    const int KP = next_pow2(a.K);
    int S = next_pow2(KP + 2 * round > 4 * KP ? KP + 2 * round : 4 * KP);
    if (!a.out_ids64 && S < 2048) S = 2048;  // centroid levels: room to keep every candidate
    const int P = a.sel ? a.P : 1;
    const size_t smem = (size_t)(S + KP + (KP & 1)) * 8 + (size_t)(2 * P + 2) * 8 + (size_t)a.dp * 4;
    MASK_REQUIRE(smem <= 220 * 1024, "scan_topk: K, probes or dimension too large");
    ProfRegion pr(a.out_ids64 ? "scan_topk_leaf" : "scan_topk_level", s, 0.0);
    const float4 *R = reinterpret_cast<const float4 *>(a.R);
    const float4 *Qv = reinterpret_cast<const float4 *>(a.Q);
#define MASK_SCAN(ROWW, LPRV)                                                                \
    do {                                                                                     \
        auto kfn = scan_topk_kernel<ROWW, LPRV>;                                             \
        MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                       (int)smem));                                          \
        kfn<<<(unsigned)a.nq, kThreads, smem, s>>>(R, a.dp / 4, a.rid, a.off, a.sel, P,      \
                                                   a.root_end, Qv, a.K, KP, S, a.out_ids32,  \
                                                   a.out_ids64, a.out_d,                     \
                                                   scan_bytes_counter(a.out_ids64 ? 1 : 0),  \
                                                   a.sorted ? 1 : 0);                        \
    } while (0)
    if (a.out_ids64) {
        MASK_SCAN(true, 1);  // the leaf: per-row arithmetic shared with the cluster-major scan
    } else {
        switch (level_lanes_per_row(a.dp)) {
        case 1: MASK_SCAN(false, 1); break;
        case 2: MASK_SCAN(false, 2); break;
        case 4: MASK_SCAN(false, 4); break;
        case 8: MASK_SCAN(false, 8); break;
        case 16: MASK_SCAN(false, 16); break;
        default: MASK_SCAN(false, 32); break;
        }
    }
#undef MASK_SCAN
    MASK_LAUNCHED("scan_topk");
}

void greedy_descent(const GreedyLevels &lv, int L, const float *Xs, const int32_t *xids, int dp,
                    const float *Qp, int64_t nq, int32_t *leaf, int64_t *ids, float *dists,
                    cudaStream_t s) {
    if (nq == 0) return;
    ProfRegion pr("greedy_descent", s, 0.0);
    const unsigned blocks = (unsigned)((nq * 32 + kThreads - 1) / kThreads);
    const float4 *X4 = reinterpret_cast<const float4 *>(Xs);
    const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
#define MASK_GREEDY(LPRV)                                                                    \
    greedy_descent_kernel<LPRV><<<blocks, kThreads, 0, s>>>(lv, L, X4, xids, Q4, nq, dp / 4, \
                                                           leaf, ids, dists)
    switch (level_lanes_per_row(dp)) {
    case 1: MASK_GREEDY(1); break;
    case 2: MASK_GREEDY(2); break;
    case 4: MASK_GREEDY(4); break;
    case 8: MASK_GREEDY(8); break;
    case 16: MASK_GREEDY(16); break;
    default: MASK_GREEDY(32); break;
    }
#undef MASK_GREEDY
    MASK_LAUNCHED("greedy_descent");
}

double scan_bytes(int which) {
    unsigned long long v[2] = {0, 0};
    if (cudaMemcpyFromSymbol(v, g_scan_bytes, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return (double)v[which];
}

void scan_bytes_reset() {
    const unsigned long long z[2] = {0, 0};
    if (cudaMemcpyToSymbol(g_scan_bytes, z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}

}  // namespace mask
