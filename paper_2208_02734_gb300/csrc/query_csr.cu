// query_csr.cu -- the top-down k-NN search (§3.3, Algorithm 2 with p kept
// centroids per level) for CSR queries over an index built from CSR points.
//
// Two scans, both one block per query, keeping the K smallest keys
// (distance bits << 32 | id) in shared memory exactly like the dense scans:
//
//  * level scan: the query's nonzeros are staged in shared memory and each
//    centroid row (dense) is read only at those coordinates:
//      ||q - c||^2 = sum_{t in q} (q_t - c_t)^2 + (||c||^2 - sum_{t in q} c_t^2),
//    the second term being c's mass off the query's support (FP64 norm of c,
//    rounded once; clamped at 0);
//  * leaf scan: the query's nonzeros go into a small open-addressing table in
//    shared memory (column -> value, at most a quarter full) and each point (a
//    CSR row of the cluster-major point matrix) looks the query up at its own
//    nonzeros (q_t, or 0 where the query has no entry):
//      ||x - q||^2 = sum_{t in x} (x_t - q_t)^2 + (||q||^2 - sum_{t in x} q_t^2),
//    where ||q||^2 is summed by the same lane-group procedure over q's own
//    nonzeros, so a point equal to the query gets exactly 0.
//
// Groups of kGroup lanes take one row each, four rows in flight per group.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace mask {

// Bytes the CSR scans read ([0] levels: gathered centroid values, 4 per
// query nonzero per row; [1] leaf: 8 per nonzero + row pointer and id, 12
// per row), counted per block.
__device__ unsigned long long g_csr_scan_bytes[2];

// Device address of a byte counter while profiling is on; null otherwise, so
// the kernels skip the count (one uniform test, no atomic) in normal runs.
unsigned long long *csr_scan_bytes_counter(int which) {
    if (!profiling_enabled()) return nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_csr_scan_bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<unsigned long long *>(p) + which;
}

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kGroup = 8;                       // lanes per row
constexpr int kGroups = kThreads / kGroup;      // rows in flight per block / 4
constexpr int kInFlight = 4;                    // rows per group per round
constexpr int kRound = kGroups * kInFlight;     // rows per round

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

__device__ __forceinline__ void group_reduce2(float &A, float &B) {
#pragma unroll
    for (int o = kGroup / 2; o > 0; o >>= 1) {
        A += __shfl_xor_sync(kFull, A, o, kGroup);
        B += __shfl_xor_sync(kFull, B, o, kGroup);
    }
}

// Shared state of one query's scan.
struct ScanSmem {
    unsigned long long *buf;  // [S] keys: [0, KP) the current list, then candidates
    int64_t *rb;              // [P] range begins
    int64_t *cum;             // [P+1] prefix sizes
};

// Row ranges of query q: the root range, or the children of its kept parents.
__device__ void setup_ranges(const ScanSmem &sm, const int64_t *__restrict__ off,
                             const int32_t *__restrict__ sel, int P, int64_t root_end,
                             int64_t q) {
    if (threadIdx.x != 0) return;
    if (sel == nullptr) {
        sm.rb[0] = 0;
        sm.cum[0] = 0;
        sm.cum[1] = root_end;
        return;
    }
    int64_t tot = 0;
    sm.cum[0] = 0;
    for (int s = 0; s < P; ++s) {
        const int32_t p = sel[q * P + s];
        int64_t b = 0, e = 0;
        if (p >= 0) { b = off[p]; e = off[p + 1]; }
        sm.rb[s] = b;
        tot += e - b;
        sm.cum[s + 1] = tot;
    }
}

__device__ __forceinline__ int64_t row_of(const ScanSmem &sm, int nr, int64_t t) {
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sm.cum[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return sm.rb[lo] + (t - sm.cum[lo]);
}

// After a round: merge the candidates into the list when the buffer could
// overflow in the next round, or at the end.
__device__ __forceinline__ void maybe_merge(const ScanSmem &sm, int S, int K, int KP, int lim,
                                           bool last, int *cnt, unsigned long long *thresh) {
    __syncthreads();
    const int c_now = *cnt;
    __syncthreads();
    if (c_now > lim || last) {
        // sort only the filled prefix (rounded up to a power of two)
        int L = KP;
        while (L < KP + c_now) L <<= 1;
        for (int i = KP + c_now + threadIdx.x; i < L; i += kThreads) sm.buf[i] = kNoKey;
        __syncthreads();
        bitonic_sort_keys(sm.buf, L);
        for (int i = K + threadIdx.x; i < KP; i += kThreads) sm.buf[i] = kNoKey;
        if (threadIdx.x == 0) {
            *thresh = sm.buf[K - 1];
            *cnt = 0;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ level scan

__global__ __launch_bounds__(kThreads) void csr_level_scan_kernel(
    const float *__restrict__ R, int dp, const float *__restrict__ rcn,
    const int32_t *__restrict__ rid, const int64_t *__restrict__ off,
    const int32_t *__restrict__ sel, int P, int64_t root_end, const int64_t *__restrict__ qrp,
    const int32_t *__restrict__ qcol, const float *__restrict__ qval, int qcap, int K, int KP,
    int S, int32_t *__restrict__ out32, unsigned long long *__restrict__ bytes_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    ScanSmem sm;
    sm.buf = reinterpret_cast<unsigned long long *>(smem);
    sm.rb = reinterpret_cast<int64_t *>(sm.buf + S);
    sm.cum = sm.rb + P;
    int32_t *qc = reinterpret_cast<int32_t *>(sm.cum + P + 2);
    float *qv = reinterpret_cast<float *>(qc + qcap);
    __shared__ int cnt;
    __shared__ unsigned long long thresh;

    const int tid = threadIdx.x;
    const int64_t q = blockIdx.x;
    const int64_t qb = qrp[q];
    const int64_t qlen = qrp[q + 1] - qb;
    const int qn = (int)(qlen < (int64_t)qcap ? qlen : (int64_t)qcap);
    for (int j = tid; j < qn; j += kThreads) {
        qc[j] = qcol[qb + j];
        qv[j] = qval[qb + j];
    }
    for (int i = tid; i < S; i += kThreads) sm.buf[i] = kNoKey;
    if (tid == 0) {
        cnt = 0;
        thresh = kNoKey;
    }
    setup_ranges(sm, off, sel, P, root_end, q);
    __syncthreads();
    const int nr = sel == nullptr ? 1 : P;
    const int64_t T = sm.cum[nr];
    const int lim = S - KP - kRound;
    const int g = tid / kGroup, gl = tid % kGroup;
    if (bytes_ctr != nullptr && tid == 0)
        atomicAdd(bytes_ctr, (unsigned long long)T * (4ull * qn + 8ull));

    for (int64_t base = 0; base < T; base += kRound) {
        const unsigned long long th = thresh;
        int64_t row[kInFlight];
        float A[kInFlight], B[kInFlight];
#pragma unroll
        for (int i = 0; i < kInFlight; ++i) {
            const int64_t t = base + g + (int64_t)i * kGroups;
            row[i] = t < T ? row_of(sm, nr, t) : -1;
            A[i] = 0.f;
            B[i] = 0.f;
        }
        for (int j = gl; j < qn; j += kGroup) {
            const int c = qc[j];
            const float x = qv[j];
#pragma unroll
            for (int i = 0; i < kInFlight; ++i) {
                if (row[i] < 0) continue;
                const float r = __ldg(R + row[i] * dp + c);
                const float e = x - r;
                A[i] = fmaf(e, e, A[i]);
                B[i] = fmaf(r, r, B[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < kInFlight; ++i) {
            group_reduce2(A[i], B[i]);
            if (gl == 0 && row[i] >= 0) {
                const float dist = A[i] + fmaxf(rcn[row[i]] - B[i], 0.f);
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)rid[row[i]];
                if (key < th) sm.buf[KP + atomicAdd(&cnt, 1)] = key;
            }
        }
        maybe_merge(sm, S, K, KP, lim, base + kRound >= T, &cnt, &thresh);
    }
    for (int r = tid; r < K; r += kThreads) {
        const unsigned long long key = sm.buf[r];
        out32[q * K + r] = key != kNoKey ? (int32_t)(key & 0xffffffffu) : -1;
    }
}

// ------------------------------------------------------------- leaf scan

// Open-addressing table of a query's nonzeros: H slots (a power of two),
// linear probing from a multiplicative hash; key -1 = empty.
__device__ __forceinline__ unsigned qhash(int32_t col, unsigned mask) {
    return ((unsigned)col * 0x9E3779B1u) & mask;
}

__device__ __forceinline__ float qlookup(const int32_t *keys, const float *vals, unsigned mask,
                                         int32_t col) {
    unsigned h = qhash(col, mask);
    for (;;) {
        const int32_t k = keys[h];
        if (k == col) return vals[h];
        if (k < 0) return 0.f;
        h = (h + 1) & mask;
    }
}

__global__ __launch_bounds__(kThreads) void csr_leaf_scan_kernel(
    const int64_t *__restrict__ xrp, const int32_t *__restrict__ xcol,
    const float *__restrict__ xval, const int32_t *__restrict__ xids,
    const int64_t *__restrict__ off, const int32_t *__restrict__ sel, int P,
    const int64_t *__restrict__ qrp, const int32_t *__restrict__ qcol,
    const float *__restrict__ qval, int hslots, int64_t min_nnz, int K, int KP, int S,
    int64_t *__restrict__ out64, float *__restrict__ out_d,
    unsigned long long *__restrict__ bytes_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    ScanSmem sm;
    sm.buf = reinterpret_cast<unsigned long long *>(smem);
    sm.rb = reinterpret_cast<int64_t *>(sm.buf + S);
    sm.cum = sm.rb + P;
    int32_t *hkey = reinterpret_cast<int32_t *>(sm.cum + P + 2);  // [hslots] query table
    float *hval = reinterpret_cast<float *>(hkey + hslots);
    __shared__ int cnt;
    __shared__ unsigned long long thresh;
    __shared__ float s_qn;
    __shared__ unsigned long long s_nnz;

    const int tid = threadIdx.x;
    const int64_t q = blockIdx.x;
    const int64_t qb = qrp[q], qe = qrp[q + 1];
    if (qe - qb <= min_nnz) return;  // served by another scan (block-uniform exit)
    // this query's table: the smallest power of two >= 4 x its nonzeros (>= 32)
    unsigned hsize = 32;
    while ((int64_t)hsize < 4 * (qe - qb) && (int)hsize < hslots) hsize <<= 1;
    const unsigned hmask = hsize - 1;
    for (int i = tid; i < (int)hsize; i += kThreads) hkey[i] = -1;
    for (int i = tid; i < S; i += kThreads) sm.buf[i] = kNoKey;
    if (tid == 0) {
        cnt = 0;
        thresh = kNoKey;
        s_nnz = 0;
    }
    setup_ranges(sm, off, sel, P, 0, q);
    __syncthreads();
    for (int64_t j = qb + tid; j < qe; j += kThreads) {
        // column ids of a row are distinct, so every insert claims its own slot
        const int32_t c = qcol[j];
        unsigned h = qhash(c, hmask);
        while (atomicCAS(hkey + h, -1, c) != -1) h = (h + 1) & hmask;
        hval[h] = qval[j];
    }
    __syncthreads();
    const int g = tid / kGroup, gl = tid % kGroup;
    if (tid < 32) {
        // ||q||^2 as B of the query itself (every group of warp 0; shuffles need the warp)
        float A = 0.f, B = 0.f;
        for (int64_t j = qb + gl; j < qe; j += kGroup) {
            const float c = qlookup(hkey, hval, hmask, qcol[j]);
            const float e = qval[j] - c;
            A = fmaf(e, e, A);
            B = fmaf(c, c, B);
        }
        group_reduce2(A, B);
        if (tid == 0) s_qn = B;
    }
    __syncthreads();
    const float qn = s_qn;
    const int nr = P;
    const int64_t T = sm.cum[nr];
    const int lim = S - KP - kRound;

    for (int64_t base = 0; base < T; base += kRound) {
        const unsigned long long th = thresh;
        int64_t row[kInFlight], rb[kInFlight];
        int len[kInFlight];
        int maxlen = 0;
        float A[kInFlight], B[kInFlight];
#pragma unroll
        for (int i = 0; i < kInFlight; ++i) {
            const int64_t t = base + g + (int64_t)i * kGroups;
            row[i] = t < T ? row_of(sm, nr, t) : -1;
            rb[i] = row[i] >= 0 ? xrp[row[i]] : 0;
            len[i] = row[i] >= 0 ? (int)(xrp[row[i] + 1] - rb[i]) : 0;
            maxlen = max(maxlen, len[i]);
            A[i] = 0.f;
            B[i] = 0.f;
        }
        if (gl == 0) {
            int tot = 0;
#pragma unroll
            for (int i = 0; i < kInFlight; ++i) tot += len[i];
            if (tot) atomicAdd(&s_nnz, (unsigned long long)tot);
        }
        for (int j = gl; j < maxlen; j += kGroup) {
#pragma unroll
            for (int i = 0; i < kInFlight; ++i) {
                if (j >= len[i]) continue;
                const float x = __ldg(xval + rb[i] + j);
                const float c = qlookup(hkey, hval, hmask, __ldg(xcol + rb[i] + j));
                const float e = x - c;
                A[i] = fmaf(e, e, A[i]);
                B[i] = fmaf(c, c, B[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < kInFlight; ++i) {
            group_reduce2(A[i], B[i]);
            if (gl == 0 && row[i] >= 0) {
                const float dist = A[i] + fmaxf(qn - B[i], 0.f);
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)xids[row[i]];
                if (key < th) sm.buf[KP + atomicAdd(&cnt, 1)] = key;
            }
        }
        maybe_merge(sm, S, K, KP, lim, base + kRound >= T, &cnt, &thresh);
    }
    if (bytes_ctr != nullptr && tid == 0)
        atomicAdd(bytes_ctr, 8ull * s_nnz + 12ull * (unsigned long long)T);
    for (int r = tid; r < K; r += kThreads) {
        const unsigned long long key = sm.buf[r];
        const bool ok = key != kNoKey;
        out64[q * K + r] = ok ? (int64_t)(int32_t)(key & 0xffffffffu) : -1;
        if (out_d)
            out_d[q * K + r] = ok ? __uint_as_float((unsigned)(key >> 32))
                                  : __int_as_float(0x7f800000);
    }
}

// ------------------------------------------------- cluster-major leaf scan
//
// For large batches the (query, kept leaf cluster) pairs are grouped by
// cluster (cm_group_pairs, kCmQB pairs per work item) and a cluster's CSR rows
// are read once per item.  The item's queries share one table in shared
// memory: column -> the kCmQB query values at that column (0 where a query
// has no entry).  A lane group takes a row; for each nonzero every lane looks
// the column up once and updates, for each query, the same partial sums as the
// per-query scan (c = the query's value or 0), reduced by the same shuffle
// tree: the keys are bit-identical to the per-query scan's.  Each pair keeps
// its K smallest keys (cm_merge then takes each query's K over its pairs).

constexpr int kCmQB = 16;            // pairs per work item (the grouping's item size)
constexpr int kCmEntries = 1024;     // distinct columns one pass holds
constexpr int kCmSlots = 2 * kCmEntries;  // hash slots (at most half full)
constexpr int kCmLongestQuery = kCmEntries;  // one query always fits a pass

// ||q||^2 of every CSR query by the per-query scan's procedure (lanes gl of a
// group of 8 over nonzeros gl, gl+8, ..., then the xor tree), one warp each.
__global__ void csr_query_norm_kernel(const int64_t *__restrict__ qrp,
                                      const float *__restrict__ qval, int64_t nq,
                                      float *__restrict__ qn) {
    const int lane = threadIdx.x & 31, gl = lane % kGroup;
    for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nq;
         q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float A = 0.f, B = 0.f;
        for (int64_t j = qrp[q] + gl; j < qrp[q + 1]; j += kGroup) {
            const float c = qval[j];
            B = fmaf(c, c, B);
        }
        group_reduce2(A, B);
        if (lane == 0) qn[q] = B;
    }
}

// slot of column col in the union table (or -1 if absent)
__device__ __forceinline__ int union_find(const int32_t *keys, int32_t col) {
    unsigned h = qhash(col, kCmSlots - 1);
    for (;;) {
        const int32_t k = keys[h];
        if (k == col) return (int)h;
        if (k < 0) return -1;
        h = (h + 1) & (kCmSlots - 1);
    }
}

__global__ __launch_bounds__(kThreads) void csr_cm_scan_kernel(
    const int64_t *__restrict__ xrp, const int32_t *__restrict__ xcol,
    const float *__restrict__ xval, const int32_t *__restrict__ xids,
    const int64_t *__restrict__ leaf_off, int P, const int64_t *__restrict__ poff,
    const int32_t *__restrict__ pairs, const int64_t *__restrict__ item_off, int k0,
    const int64_t *__restrict__ qrp, const int32_t *__restrict__ qcol,
    const float *__restrict__ qval, const float *__restrict__ qn_all, int K,
    unsigned long long *__restrict__ pair_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    float4 *uval = reinterpret_cast<float4 *>(smem);                          // [kCmEntries][4]
    int32_t *ukey = reinterpret_cast<int32_t *>(uval + kCmEntries * 4);       // [kCmSlots]
    int32_t *uidx = ukey + kCmSlots;                                          // [kCmSlots]
    unsigned long long *cand = reinterpret_cast<unsigned long long *>(uidx + kCmSlots);
    unsigned long long *top = cand + kCmQB * kGroups;                         // [kCmQB][K]
    __shared__ int s_c, s_hi, s_nent;
    __shared__ int64_t s_pb, s_pe;
    __shared__ float s_qn[kCmQB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = tid / kGroup, gl = tid % kGroup;
    float *uv = reinterpret_cast<float *>(uval);
    const int64_t n_items = item_off[k0];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        if (tid == 0) {
            int lo = 0, hi = k0 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (item_off[mid] <= item) lo = mid; else hi = mid - 1;
            }
            s_c = lo;
            s_pb = poff[lo] + (item - item_off[lo]) * kCmQB;
            s_pe = min(poff[lo + 1], s_pb + kCmQB);
        }
        __syncthreads();
        const int c = s_c;
        const int64_t pb = s_pb;
        const int nqb = (int)(s_pe - pb);
        for (int i = tid; i < kCmQB * K; i += kThreads) top[i] = kNoKey;
        const int64_t rb = leaf_off[c], re = leaf_off[c + 1];
        for (int lo = 0; lo < nqb;) {
            // the queries of this pass: as many as fit kCmEntries columns
            if (tid == 0) {
                int64_t used = 0;
                int hi = lo;
                while (hi < nqb) {
                    const int64_t q = pairs[pb + hi] / P;
                    const int64_t m = qrp[q + 1] - qrp[q];
                    if (hi > lo && used + m > kCmEntries) break;
                    s_qn[hi - lo] = qn_all[q];
                    used += m;
                    ++hi;
                }
                s_hi = hi;
                s_nent = 0;
            }
            for (int i = tid; i < kCmSlots; i += kThreads) ukey[i] = -1;
            __syncthreads();
            const int hi = s_hi, np = hi - lo;
            // keys of the union (distinct columns claim distinct slots)
            for (int j = 0; j < np; ++j) {
                const int64_t q = pairs[pb + lo + j] / P;
                for (int64_t e = qrp[q] + tid; e < qrp[q + 1]; e += kThreads) {
                    const int32_t cc = qcol[e];
                    unsigned h = qhash(cc, kCmSlots - 1);
                    for (;;) {
                        const int32_t old = atomicCAS(ukey + h, -1, cc);
                        if (old == -1 || old == cc) break;
                        h = (h + 1) & (kCmSlots - 1);
                    }
                }
            }
            __syncthreads();
            // an entry (row of kCmQB values, zeroed) per occupied slot
            for (int i = tid; i < kCmSlots; i += kThreads)
                if (ukey[i] >= 0) {
                    const int e = atomicAdd(&s_nent, 1);
                    uidx[i] = e;
#pragma unroll
                    for (int v4 = 0; v4 < 4; ++v4) uval[e * 4 + v4] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            __syncthreads();
            for (int j = 0; j < np; ++j) {
                const int64_t q = pairs[pb + lo + j] / P;
                for (int64_t e = qrp[q] + tid; e < qrp[q + 1]; e += kThreads)
                    uv[uidx[union_find(ukey, qcol[e])] * kCmQB + j] = qval[e];
            }
            __syncthreads();
            for (int64_t r0 = rb; r0 < re; r0 += kGroups) {
                const int64_t row = r0 + g;
                const bool ok = row < re;
                float A[kCmQB], B[kCmQB];
#pragma unroll
                for (int j = 0; j < kCmQB; ++j) {
                    A[j] = 0.f;
                    B[j] = 0.f;
                }
                if (ok) {
                    for (int64_t e = xrp[row] + gl; e < xrp[row + 1]; e += kGroup) {
                        const float v = __ldg(xval + e);
                        const int slot = union_find(ukey, __ldg(xcol + e));
                        if (slot >= 0) {
                            const float4 *qv = uval + uidx[slot] * 4;
#pragma unroll
                            for (int v4 = 0; v4 < 4; ++v4) {
                                const float4 w = qv[v4];
                                const float cv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                for (int t = 0; t < 4; ++t) {
                                    const float d = v - cv[t];
                                    A[v4 * 4 + t] = fmaf(d, d, A[v4 * 4 + t]);
                                    B[v4 * 4 + t] = fmaf(cv[t], cv[t], B[v4 * 4 + t]);
                                }
                            }
                        } else {
                            // no query has this column: c = 0 for every query
#pragma unroll
                            for (int j = 0; j < kCmQB; ++j) {
                                A[j] = fmaf(v, v, A[j]);
                                B[j] = fmaf(0.f, 0.f, B[j]);
                            }
                        }
                    }
                }
                const int32_t xid = ok ? xids[row] : -1;
#pragma unroll
                for (int j = 0; j < kCmQB; ++j) {
                    if (j < np) {  // np is the same for the whole block: every lane shuffles
                        group_reduce2(A[j], B[j]);
                        if (gl == 0) {
                            const float dist = A[j] + fmaxf(s_qn[j] - B[j], 0.f);
                            cand[j * kGroups + g] =
                                ok ? (((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)xid)
                                   : kNoKey;
                        }
                    }
                }
                __syncthreads();
                // merge: warp w owns the pass's queries 2w, 2w+1 (one candidate per lane)
                for (int qi = 0; qi < 2; ++qi) {
                    const int j = warp * 2 + qi;
                    if (j >= np) break;
                    unsigned long long *tq = top + (lo + j) * K;
                    const unsigned long long th = tq[K - 1];
                    unsigned long long mine = cand[j * kGroups + lane];
                    if (!(mine < th)) mine = kNoKey;
                    if (!__any_sync(kFull, mine != kNoKey)) continue;
                    unsigned long long old0 = lane < K ? tq[lane] : kNoKey;
                    unsigned long long old1 = lane + 32 < K ? tq[lane + 32] : kNoKey;
                    unsigned long long out0 = kNoKey, out1 = kNoKey;
                    for (int r = 0; r < K; ++r) {
                        unsigned long long m = old0 < old1 ? old0 : old1;
                        m = m < mine ? m : mine;
                        for (int o = 16; o > 0; o >>= 1) {
                            const unsigned long long t = __shfl_xor_sync(kFull, m, o);
                            m = t < m ? t : m;
                        }
                        if (m == kNoKey) break;
                        if (lane == (r & 31)) { if (r < 32) out0 = m; else out1 = m; }
                        // keys are distinct (ids differ): exactly one holder drops it
                        if (old0 == m) old0 = kNoKey;
                        if (old1 == m) old1 = kNoKey;
                        if (mine == m) mine = kNoKey;
                    }
                    __syncwarp();
                    if (lane < K) tq[lane] = out0;
                    if (lane + 32 < K) tq[lane + 32] = out1;
                    __syncwarp();
                }
                __syncthreads();
            }
            lo = hi;
        }
        for (int i = tid; i < nqb * K; i += kThreads) {
            const int j = i / K, r = i % K;
            pair_out[(int64_t)pairs[pb + j] * K + r] = top[j * K + r];
        }
        __syncthreads();
    }
}

int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

int list_size(int K) {
    const int KP = next_pow2(K);
    return next_pow2(KP + 2 * kRound > 4 * KP ? KP + 2 * kRound : 4 * KP);
}

}  // namespace

double csr_scan_bytes(int which) {
    unsigned long long v[2] = {0, 0};
    if (cudaMemcpyFromSymbol(v, g_csr_scan_bytes, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return (double)v[which];
}

void csr_scan_bytes_reset() {
    const unsigned long long z[2] = {0, 0};
    if (cudaMemcpyToSymbol(g_csr_scan_bytes, z, sizeof(z)) != cudaSuccess) cudaGetLastError();
}

size_t csr_level_scan_smem(int K, int P, int qcap) {
    return (size_t)list_size(K) * 8 + (size_t)(2 * P + 2) * 8 + (size_t)qcap * 8;
}

int csr_leaf_table_slots(int longest) {
    int h = 32;
    while (h < 4 * longest) h <<= 1;
    return h;
}

size_t csr_leaf_scan_smem(int K, int P, int longest) {
    return (size_t)list_size(K) * 8 + (size_t)(2 * P + 2) * 8 +
           (size_t)csr_leaf_table_slots(longest) * 8;
}

void csr_level_scan(const float *R, int dp, const float *rcn, const int32_t *rid,
                    const int64_t *off, const int32_t *sel, int P, int64_t root_end,
                    const int64_t *qrp, const int32_t *qcol, const float *qval, int qcap,
                    int64_t nq, int K, int32_t *out32, cudaStream_t s) {
    if (nq == 0) return;
    MASK_REQUIRE(K >= 1 && K <= 4096, "csr_level_scan: K out of range");
    const int Pn = sel ? P : 1;
    const size_t smem = csr_level_scan_smem(K, Pn, qcap);
    MASK_REQUIRE(smem <= 220 * 1024, "csr_level_scan: probes or query length too large");
    ProfRegion pr("csr_scan_level", s, 0.0);
    MASK_CUDA(cudaFuncSetAttribute(csr_level_scan_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    csr_level_scan_kernel<<<(unsigned)nq, kThreads, smem, s>>>(
        R, dp, rcn, rid, off, sel, Pn, root_end, qrp, qcol, qval, qcap, K, next_pow2(K),
        list_size(K), out32, csr_scan_bytes_counter(0));
    MASK_LAUNCHED("csr_level_scan");
}

bool csr_cm_supported(int K) { return K >= 1 && K <= 64; }

int csr_cm_longest_query() { return kCmLongestQuery; }

// sel_cm = sel with the slots of queries longer than kCmLongestQuery blanked
__global__ void blank_long_kernel(const int32_t *__restrict__ sel, const int64_t *__restrict__ qrp,
                                  int64_t nq, int P, int32_t *__restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nq * P;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / P;
        out[e] = qrp[q + 1] - qrp[q] > kCmLongestQuery ? -1 : sel[e];
    }
}

void csr_cm_leaf_scan(const int64_t *xrp, const int32_t *xcol, const float *xval,
                      const int32_t *xids, const int64_t *leaf_off, int k0, const int32_t *sel,
                      int P, const int64_t *qrp, const int32_t *qcol, const float *qval,
                      int64_t nq, int K, int64_t *out64, float *out_d, cudaStream_t s) {
    if (nq == 0) return;
    Scratch<float> qn(nq, s);
    csr_query_norm_kernel<<<(unsigned)std::min<int64_t>((nq + 7) / 8, 152 * 32), 256, 0, s>>>(
        qrp, qval, nq, qn.get());
    MASK_LAUNCHED("csr_query_norm");
    // queries longer than one pass holds are served by the per-query scan:
    // their slots are blanked here (their rows come out empty and are rewritten)
    Scratch<int32_t> sel_cm((size_t)nq * P, s);
    blank_long_kernel<<<(unsigned)std::min<int64_t>((nq * P + 255) / 256, 152 * 32), 256, 0, s>>>(
        sel, qrp, nq, P, sel_cm.get());
    MASK_LAUNCHED("blank_long");
    Scratch<int32_t> pairs;
    Scratch<int64_t> poff, item_off;
    cm_group_pairs(sel_cm.get(), nq, P, k0, pairs, poff, item_off, s);
    const int64_t npairs = nq * P;
    Scratch<unsigned long long> pair_out((size_t)npairs * K, s);
    // pairs of an absent parent (sel = -1) are in no work item: empty lists
    MASK_CUDA(cudaMemsetAsync(pair_out.get(), 0xFF, sizeof(unsigned long long) * npairs * K, s));
    {
        ProfRegion pr("csr_scan_leaf_cm", s, 0.0);
        const size_t smem = (size_t)kCmEntries * kCmQB * 4 + (size_t)kCmSlots * 8 +
                            (size_t)kCmQB * kGroups * 8 + (size_t)kCmQB * K * 8;
        MASK_CUDA(cudaFuncSetAttribute(csr_cm_scan_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        csr_cm_scan_kernel<<<152 * 2, kThreads, smem, s>>>(xrp, xcol, xval, xids, leaf_off, P,
                                                           poff.get(), pairs.get(), item_off.get(),
                                                           k0, qrp, qcol, qval, qn.get(), K,
                                                           pair_out.get());
        MASK_LAUNCHED("csr_cm_scan");
    }
    cm_merge(pair_out.get(), nq, P, K, out64, out_d, s);
}

void csr_leaf_scan(const int64_t *xrp, const int32_t *xcol, const float *xval,
                   const int32_t *xids, const int64_t *off, const int32_t *sel, int P,
                   const int64_t *qrp, const int32_t *qcol, const float *qval, int longest,
                   int64_t nq, int K, int64_t *out64, float *out_d, cudaStream_t s,
                   int64_t min_nnz) {
    if (nq == 0) return;
    MASK_REQUIRE(K >= 1 && K <= 4096, "csr_leaf_scan: K out of range");
    const size_t smem = csr_leaf_scan_smem(K, P, longest);
    MASK_REQUIRE(smem <= 220 * 1024, "csr_leaf_scan: k, probes or query length too large");
    ProfRegion pr("csr_scan_leaf", s, 0.0);
    MASK_CUDA(cudaFuncSetAttribute(csr_leaf_scan_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    csr_leaf_scan_kernel<<<(unsigned)nq, kThreads, smem, s>>>(xrp, xcol, xval, xids, off, sel, P,
                                                              qrp, qcol, qval,
                                                              csr_leaf_table_slots(longest), min_nnz, K,
                                                              next_pow2(K), list_size(K), out64,
                                                              out_d, csr_scan_bytes_counter(1));
    MASK_LAUNCHED("csr_leaf_scan");
}

}  // namespace mask
