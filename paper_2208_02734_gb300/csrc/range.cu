// range.cu -- range search down the index (§3.3, Algorithm 3): from the top
// level down, keep the candidate centroids that lie within the ball of the
// query's radius and descend into their children; at the data layer return
// the points of the kept leaf clusters that lie within the ball, ascending by
// (distance, id).
//
// Every level is two passes of one block per query over the children of the
// query's kept centroids (contiguous rows of the parent-major arrays): a count
// pass sizes the next kept lists, a fill pass writes them in row order (block
// ballots give each kept row its slot).  The results of each query are then
// sorted in place by a bitonic network whose compare-exchanges all put the
// smaller key first, so a segment of any length sorts as if padded with +inf.
// Distances are the FP32 difference form sum_t (q_t - x_t)^2.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "index.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRgThreads = 256;

__device__ __forceinline__ float row_dist(const float4 *__restrict__ r, const float4 *q, int dp4) {
    float acc = 0.f;
    for (int c = 0; c < dp4; ++c) {
        const float4 a = r[c], b = q[c];
        const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
        acc = fmaf(e0, e0, acc);
        acc = fmaf(e1, e1, acc);
        acc = fmaf(e2, e2, acc);
        acc = fmaf(e3, e3, acc);
    }
    return acc;
}

// Exclusive prefix of `flag` over the block (row order) and the block total.
__device__ __forceinline__ int block_rank(bool flag, int *warp_tot, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(kFull, flag);
    if (lane == 0) warp_tot[w] = __popc(bal);
    __syncthreads();
    int before = 0, all = 0;
    for (int i = 0; i < kRgThreads / 32; ++i) {
        if (i < w) before += warp_tot[i];
        all += warp_tot[i];
    }
    __syncthreads();
    *total = all;
    return before + __popc(bal & ((1u << lane) - 1u));
}

// One level for query q (block q): parents kept[koff[q] .. koff[q+1]) (or the
// root range [0, root_end) when koff is null), their children rows
// [off[p], off[p+1]) of R with ids rid.  count mode (out == null): cnt[q] =
// children within the ball; fill mode: the kept children's ids (levels) or
// keys dist << 32 | id (leaf) from slot noff[q].
__global__ __launch_bounds__(kRgThreads) void range_level_kernel(
    const float4 *__restrict__ R, int dp4, const int32_t *__restrict__ rid,
    const int64_t *__restrict__ off, const int64_t *__restrict__ koff,
    const int32_t *__restrict__ kept, int64_t root_end, const float4 *__restrict__ Q, float r2,
    int64_t *__restrict__ cnt, const int64_t *__restrict__ noff, int32_t *__restrict__ out_ids,
    unsigned long long *__restrict__ out_keys) {
    extern __shared__ __align__(16) float4 qs[];
    __shared__ int warp_tot[kRgThreads / 32];
    const int64_t q = blockIdx.x;
    const int tid = threadIdx.x;
    for (int c = tid; c < dp4; c += kRgThreads) qs[c] = Q[q * dp4 + c];
    __syncthreads();
    const bool fill = out_ids != nullptr || out_keys != nullptr;
    const int64_t np = koff ? koff[q + 1] - koff[q] : 1;
    int64_t pos = fill ? noff[q] : 0, count = 0;
    for (int64_t pi = 0; pi < np; ++pi) {
        int64_t b = 0, e = root_end;
        if (koff) {
            const int32_t p = kept[koff[q] + pi];
            b = off[p];
            e = off[p + 1];
        }
        for (int64_t base = b; base < e; base += kRgThreads) {
            const int64_t row = base + tid;
            float dd = 0.f;
            bool in = false;
            if (row < e) {
                dd = row_dist(R + row * dp4, qs, dp4);
                in = dd <= r2;
            }
            int tot;
            const int rank = block_rank(in, warp_tot, &tot);
            if (fill && in) {
                if (out_keys)
                    out_keys[pos + rank] = ((unsigned long long)__float_as_uint(dd) << 32) |
                                           (unsigned)rid[row];
                else
                    out_ids[pos + rank] = rid[row];
            }
            pos += tot;
            count += tot;
        }
    }
    if (!fill && tid == 0) cnt[q] = count;
}

// Sorts each query's keys [noff[q], noff[q+1]) ascending in place.  The
// network: for block size 2^(k+1), first compare i with its mirror in the
// block (i xor (2^(k+1) - 1)), then the half-cleaners i xor 2^j; every
// exchange puts the smaller key at the lower index, so slots past the
// segment's end behave as +inf and are never touched.  Small segments are
// sorted in shared memory, longer ones in place in global memory.
constexpr int kRgSortSmem = 4096;   // keys (32 KB of static shared memory)
__device__ __forceinline__ void cmpx(unsigned long long *a, int64_t i, int64_t j, int64_t n) {
    if (j < n && a[j] < a[i]) {
        const unsigned long long t = a[i];
        a[i] = a[j];
        a[j] = t;
    }
}

__device__ void bitonic_any(unsigned long long *a, int64_t n) {
    int64_t P = 1;
    while (P < n) P <<= 1;
    for (int64_t blk = 2; blk <= P; blk <<= 1) {
        // mirror step within each block of size blk
        for (int64_t t = threadIdx.x; t < P / 2; t += kRgThreads) {
            const int64_t half = blk >> 1;
            const int64_t i = (t / half) * blk + (t % half);
            const int64_t j = i ^ (blk - 1);
            if (i < n) cmpx(a, i, j, n);
        }
        __syncthreads();
        for (int64_t h = blk >> 2; h >= 1; h >>= 1) {
            for (int64_t t = threadIdx.x; t < P / 2; t += kRgThreads) {
                const int64_t i = (t / h) * (2 * h) + (t % h);
                const int64_t j = i + h;
                if (i < n) cmpx(a, i, j, n);
            }
            __syncthreads();
        }
    }
}

__global__ __launch_bounds__(kRgThreads) void range_sort_kernel(unsigned long long *__restrict__ keys,
                                                                const int64_t *__restrict__ noff) {
    __shared__ unsigned long long sk[kRgSortSmem];
    const int64_t b = noff[blockIdx.x], n = noff[blockIdx.x + 1] - b;
    if (n <= 1) return;
    if (n <= kRgSortSmem) {
        for (int64_t i = threadIdx.x; i < n; i += kRgThreads) sk[i] = keys[b + i];
        __syncthreads();
        bitonic_any(sk, n);
        for (int64_t i = threadIdx.x; i < n; i += kRgThreads) keys[b + i] = sk[i];
    } else {
        bitonic_any(keys + b, n);
    }
}

__global__ void range_unpack_kernel(const unsigned long long *__restrict__ keys, int64_t total,
                                    int64_t *__restrict__ ids, float *__restrict__ dists) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        ids[i] = (int64_t)(k & 0xffffffffull);
        if (dists) dists[i] = __uint_as_float((unsigned)(k >> 32));
    }
}

int grid_for_rows(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

}  // namespace

// The per-query kept lists of one level: koff [nq+1] and ids.
struct KeptList {
    Scratch<int64_t> off;
    Scratch<int32_t> ids;
};

int64_t range_search(const mask_index &idx, const float *Qp, int64_t nq, float radius,
                     int64_t *counts_out, int64_t capacity, int64_t *ids_out, float *dists_out,
                     cudaStream_t s) {
    const int dp = idx.dp, dp4 = dp / 4;
    const float r2 = radius * radius;
    const size_t qsm = (size_t)dp * sizeof(float);
    const float4 *Q4 = reinterpret_cast<const float4 *>(Qp);
    ProfRegion pr("range_query", s, 0.0);
    Scratch<int64_t> cnt((size_t)nq, s);
    // sizes a level's output lists: counts, then their offsets (noff[0] = 0)
    auto offsets = [&](Scratch<int64_t> &noff) -> int64_t {
        noff.alloc((size_t)nq + 1, s);
        MASK_CUDA(cudaMemsetAsync(noff.get(), 0, sizeof(int64_t), s));
        MASK_CUDA(cudaMemcpyAsync(noff.get() + 1, cnt.get(), sizeof(int64_t) * nq,
                                  cudaMemcpyDeviceToDevice, s));
        inclusive_scan_i64(noff.get() + 1, nq, s);
        int64_t total = 0;
        MASK_CUDA(cudaMemcpyAsync(&total, noff.get() + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        MASK_CUDA(cudaStreamSynchronize(s));
        return total;
    };
    KeptList cur;   // empty: the root range
    bool root = true;
    for (int lv = idx.L - 1; lv >= 0; --lv) {
        // rows of this step: level lv's centroids under the kept level-lv+1
        // parents (the root range at the top), or the points at the end
        const auto &Lv = idx.lv[(size_t)lv];
        const float4 *R = reinterpret_cast<const float4 *>(Lv.Cs.get());
        const int32_t *rid = Lv.ids.get();
        const int64_t *off = root ? nullptr : idx.lv[(size_t)lv + 1].off.get();
        range_level_kernel<<<(unsigned)nq, kRgThreads, qsm, s>>>(
            R, dp4, rid, off, root ? nullptr : cur.off.get(), root ? nullptr : cur.ids.get(),
            Lv.k, Q4, r2, cnt.get(), nullptr, nullptr, nullptr);
        MASK_LAUNCHED("range_level (count)");
        KeptList nxt;
        const int64_t total = offsets(nxt.off);
        nxt.ids.alloc((size_t)std::max<int64_t>(1, total), s);
        range_level_kernel<<<(unsigned)nq, kRgThreads, qsm, s>>>(
            R, dp4, rid, off, root ? nullptr : cur.off.get(), root ? nullptr : cur.ids.get(),
            Lv.k, Q4, r2, cnt.get(), nxt.off.get(), nxt.ids.get(), nullptr);
        MASK_LAUNCHED("range_level (fill)");
        cur = std::move(nxt);
        root = false;
    }
    // the data layer: points of the kept leaf clusters
    const float4 *X4 = reinterpret_cast<const float4 *>(idx.Xs.get());
    range_level_kernel<<<(unsigned)nq, kRgThreads, qsm, s>>>(
        X4, dp4, idx.xids.get(), idx.lv[0].off.get(), cur.off.get(), cur.ids.get(), 0, Q4, r2,
        cnt.get(), nullptr, nullptr, nullptr);
    MASK_LAUNCHED("range_leaf (count)");
    Scratch<int64_t> roff;
    const int64_t total = offsets(roff);
    MASK_CUDA(cudaMemcpyAsync(counts_out, cnt.get(), sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, s));
    MASK_CUDA(cudaStreamSynchronize(s));
    if (ids_out == nullptr || total == 0) return total;
    if (total > capacity) return total;
    Scratch<unsigned long long> keys((size_t)total, s);
    range_level_kernel<<<(unsigned)nq, kRgThreads, qsm, s>>>(
        X4, dp4, idx.xids.get(), idx.lv[0].off.get(), cur.off.get(), cur.ids.get(), 0, Q4, r2,
        cnt.get(), roff.get(), nullptr, keys.get());
    MASK_LAUNCHED("range_leaf (fill)");
    range_sort_kernel<<<(unsigned)nq, kRgThreads, 0, s>>>(keys.get(), roff.get());
    MASK_LAUNCHED("range_sort");
    range_unpack_kernel<<<grid_for_rows(total), 256, 0, s>>>(keys.get(), total, ids_out, dists_out);
    MASK_LAUNCHED("range_unpack");
    return total;
}

}  // namespace mask
