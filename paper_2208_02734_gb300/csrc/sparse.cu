// sparse.cu -- the build steps on CSR points (the TF-IDF shape of §4.3):
// row norms, row gathers, and the two halves of a Lloyd iteration (§2.4) with
// sparse points and dense centroids.
//
// Assignment.  labels[i] = argmin_j ||x_i||^2 - 2 x_i.c_j + ||c_j||^2 is a
// CSR-times-dense product with the argmin fused: the centroids are held
// transposed (CT[t][j], centroid j of coordinate t contiguous in j), a block
// takes kSpBM rows and one chunk of kSpBN centroids, each nonzero x_it pulls
// the chunk's slice CT[t][chunk] (float4 per thread) and FMAs it into the
// rows' accumulators.  Consecutive blocks share a chunk, so the slice table of
// the chunk in flight (d x kSpBN x 4 bytes) stays in L2.  Each (row, chunk)
// keeps its best and second-best; a combine pass merges the chunks and lists
// every row whose gap is within the rounding bound of the FP32 arithmetic,
// and those rows are decided again exactly (FP64 difference form over the
// candidates the FP32 pass cannot separate).
//
// Mean update.  One block per cluster (and column window) sums its members'
// rows into a dense shared-memory row, member by member in membership-list
// order, each warp owning a slice of the columns -- so every coordinate is
// summed in the same order on every run, with no atomics.
#include <cfloat>
#include <climits>

#include "common.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, unit roundoff of FP32

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// -------------------------------------------------------------- validation

// bad[0] += rows whose row_ptr decreases or whose column ids do not strictly
// increase (warp per row); bad[1] += column ids outside [0, d); bad[2] = the
// longest row (clamped to INT_MAX)
__global__ void csr_check_rows_kernel(const int64_t *__restrict__ rp,
                                      const int32_t *__restrict__ col, int64_t n,
                                      int *__restrict__ bad) {
    const int lane = threadIdx.x & 31;
    int b = 0;
    int64_t longest = 0;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t rb = rp[i], re = rp[i + 1];
        int bad_row = re < rb ? 1 : 0;
        for (int64_t t = rb + 1 + lane; t < re; t += 32) bad_row |= col[t] <= col[t - 1] ? 1 : 0;
        bad_row = __any_sync(kFull, bad_row) ? 1 : 0;
        b += lane == 0 ? bad_row : 0;
        longest = max(longest, re - rb);
    }
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(kFull, b, o);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(bad, b);
    if (lane == 0 && longest > 0) atomicMax(bad + 2, (int)(longest < (int64_t)INT_MAX ? longest : (int64_t)INT_MAX));
}

__global__ void csr_check_cols_kernel(const int32_t *__restrict__ col, int64_t nnz, int d,
                                      int *__restrict__ bad) {
    int b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        b += (col[i] < 0 || col[i] >= d) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(kFull, b, o);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(bad + 1, b);
}

// ------------------------------------------------- float-float arithmetic
//
// Long sums of squares (rows and centroids of up to tens of thousands of
// coordinates) and the exact re-decision of near-tie rows are carried in
// float-float form: a value is hi + lo with |lo| <= ulp(hi) / 2, kept by the
// error-free transformations TwoSum (Knuth) and TwoProduct (one fma), which
// give about 48 significant bits with FP32 instructions only.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
    const FF s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
// x + a * a
__device__ __forceinline__ FF ff_add_sq(FF x, float a) {
    const float p = a * a;
    return ff_add(x, FF{p, fmaf(a, a, -p)});
}
// x + (a - b)^2 with a - b kept exactly as a float-float pair
__device__ __forceinline__ FF ff_add_sq_diff(FF x, float a, float b) {
    const FF d = two_sum(a, -b);
    const float p = d.hi * d.hi, q = 2.f * d.hi * d.lo;
    x = ff_add(x, FF{p, fmaf(d.hi, d.hi, -p)});
    x = ff_add(x, FF{q, fmaf(2.f * d.hi, d.lo, -q)});
    return ff_add(x, FF{d.lo * d.lo, 0.f});
}
__device__ __forceinline__ FF ff_shfl_xor(FF x, int o) {
    return FF{__shfl_xor_sync(kFull, x.hi, o), __shfl_xor_sync(kFull, x.lo, o)};
}
// strict order of normalised float-float values
__device__ __forceinline__ bool ff_lt(FF x, FF y) {
    return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}

// ------------------------------------------------------------ row helpers

// ||x_i||^2 (float-float sum over the row, rounded once), one warp per row.
__global__ void csr_sqnorm_kernel(const int64_t *__restrict__ rp, const float *__restrict__ val,
                                  int64_t n, float *__restrict__ xn) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        FF s{0.f, 0.f};
        for (int64_t j = rp[i] + lane; j < rp[i + 1]; j += 32) s = ff_add_sq(s, val[j]);
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_xor(s, o));
        if (lane == 0) xn[i] = s.hi + s.lo;
    }
}

// len[i+1] = length of source row idx[i] (len[0] = 0), for the scan below.
template <class I>
__global__ void csr_gather_len_kernel(const int64_t *__restrict__ rp, const I *__restrict__ idx,
                                      int64_t m, int64_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = (int64_t)idx[i];
        out[i + 1] = rp[r + 1] - rp[r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

// In-place inclusive scan of v[0..n) (int64), three passes over blocks of
// kScanTile elements.
constexpr int kScanThreads = 512, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__device__ int64_t block_incl_scan_i64(int64_t v, int64_t *wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    int64_t base = 0;
    for (int i = 0; i < w; ++i) base += wsum[i];
    __syncthreads();
    return v + base;
}

__global__ __launch_bounds__(kScanThreads) void scan_tiles_kernel(int64_t *__restrict__ v,
                                                                 int64_t n,
                                                                 int64_t *__restrict__ tsum) {
    __shared__ int64_t wsum[kScanThreads / 32];
    const int64_t b = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t loc[kScanPer], s = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        loc[q] = b + q < n ? v[b + q] : 0;
        s += loc[q];
    }
    const int64_t inc = block_incl_scan_i64(s, wsum);
    int64_t run = inc - s;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        run += loc[q];
        if (b + q < n) v[b + q] = run;
    }
    if (threadIdx.x == kScanThreads - 1) tsum[blockIdx.x] = inc;
}

// Exclusive scan of the tile sums (one block, sequential over chunks).
__global__ __launch_bounds__(kScanThreads) void scan_tile_sums_kernel(int64_t *__restrict__ tsum,
                                                                     int64_t nt) {
    __shared__ int64_t wsum[kScanThreads / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nt; c0 += kScanThreads) {
        const int64_t i = c0 + threadIdx.x;
        const int64_t x = i < nt ? tsum[i] : 0;
        const int64_t inc = block_incl_scan_i64(x, wsum);
        const int64_t base = carry;
        if (i < nt) tsum[i] = base + inc - x;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = base + inc;
        __syncthreads();
    }
}

__global__ void scan_add_kernel(int64_t *__restrict__ v, int64_t n,
                                const int64_t *__restrict__ tsum) {
    const int64_t b = (int64_t)blockIdx.x * kScanTile;
    const int64_t add = tsum[blockIdx.x];
    for (int q = threadIdx.x; q < kScanTile; q += blockDim.x)
        if (b + q < n) v[b + q] += add;
}

// Copy source rows idx[i] into destination rows i (warp per row).
template <class I>
__global__ void csr_gather_copy_kernel(const int64_t *__restrict__ rp,
                                       const int32_t *__restrict__ col,
                                       const float *__restrict__ val, const I *__restrict__ idx,
                                       int64_t m, const int64_t *__restrict__ orp,
                                       int32_t *__restrict__ ocol, float *__restrict__ oval) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t r = (int64_t)idx[i];
        const int64_t sb = rp[r], len = rp[r + 1] - sb, db = orp[i];
        for (int64_t j = lane; j < len; j += 32) {
            ocol[db + j] = col[sb + j];
            oval[db + j] = val[sb + j];
        }
    }
}

// out[i][:] = dense copy of source row rows[i] (out zeroed beforehand).
__global__ void csr_densify_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                   const float *__restrict__ val,
                                   const int64_t *__restrict__ rows, int64_t m, int dp,
                                   float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t r = rows ? rows[i] : i;
        for (int64_t j = rp[r] + lane; j < rp[r + 1]; j += 32)
            out[i * dp + col[j]] = val[j];
    }
}

// ------------------------------------------------------ centroid tables

// cn[j] = ||c_j||^2 (float-float sum, rounded once), cn_lo[j] its
// remainder (cn + cn_lo is the float-float value); the padding entries j in
// [k, kp) get +inf so they never win.
__global__ void centroid_norms_kernel(const float *__restrict__ C, int k, int dp, int kp,
                                      float *__restrict__ cn, float *__restrict__ cn_lo) {
    const int lane = threadIdx.x & 31;
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < kp;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        if (j >= k) {
            if (lane == 0) cn[j] = __int_as_float(0x7f800000);
            continue;
        }
        FF s{0.f, 0.f};
        for (int t = lane; t < dp; t += 32) s = ff_add_sq(s, C[j * dp + t]);
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_xor(s, o));
        if (lane == 0) {
            cn[j] = s.hi;
            cn_lo[j] = s.lo;
        }
    }
}

// CT[t][j] = C[j][t] for j < k, 0 for j in [k, kp); 32 x 32 tiles.
__global__ void transpose_ct_kernel(const float *__restrict__ C, int k, int dp, int kp,
                                    float *__restrict__ CT) {
    __shared__ float tile[32][33];
    const int t0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r, t = t0 + tx;
        tile[r][tx] = (j < k && t < dp) ? C[(int64_t)j * dp + t] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int t = t0 + r, j = j0 + tx;
        if (t < dp && j < kp) CT[(int64_t)t * kp + j] = tile[tx][r];
    }
}

// ----------------------------------------------------------- assignment

constexpr int kSpBM = 16;                  // rows per block
constexpr int kSpThreads = 128;            // 4 centroids (one float4) per thread
constexpr int kSpBN = 4 * kSpThreads;      // centroids per chunk
constexpr int kSpWin = 1024;               // staged nonzeros per window

struct Top2 {
    float b1, b2;
    int i1;
};

__device__ __forceinline__ void top2_push(Top2 &t, float d, int j) {
    if (d < t.b1 || (d == t.b1 && j < t.i1)) {
        t.b2 = t.b1;
        t.b1 = d;
        t.i1 = j;
    } else if (d < t.b2) {
        t.b2 = d;
    }
}

__device__ __forceinline__ void top2_merge(Top2 &a, float ob1, int oi1, float ob2) {
    if (ob1 < a.b1 || (ob1 == a.b1 && oi1 < a.i1)) {
        a.b2 = fminf(a.b1, ob2);
        a.b1 = ob1;
        a.i1 = oi1;
    } else {
        a.b2 = fminf(a.b2, ob1);
    }
}

// Partial best / second-best of rows [blockIdx.x*kSpBM, +kSpBM) over centroid
// chunk blockIdx.y: distance ||c_j||^2 - 2 x.c_j (the row's ||x||^2 is common
// to all j and left out).  Nonzeros are FMA'd in row order.
__global__ __launch_bounds__(kSpThreads) void spmm_assign_kernel(
    const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
    const float *__restrict__ val, int64_t n, const float4 *__restrict__ CT, int kp4,
    const float *__restrict__ cn, float *__restrict__ pb1, int32_t *__restrict__ pi1,
    float *__restrict__ pb2) {
    __shared__ int64_t s_rp[kSpBM + 1];
    __shared__ int32_t s_col[kSpWin];
    __shared__ float s_val[kSpWin];
    __shared__ float w_b1[kSpThreads / 32][kSpBM], w_b2[kSpThreads / 32][kSpBM];
    __shared__ int32_t w_i1[kSpThreads / 32][kSpBM];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kSpBM;
    const int j4 = blockIdx.y * kSpThreads + tid;  // this thread's float4 of CT rows
    if (tid <= kSpBM) s_rp[tid] = rp[min(r0 + tid, n)];
    __syncthreads();

    float acc[kSpBM][4];
#pragma unroll
    for (int p = 0; p < kSpBM; ++p) acc[p][0] = acc[p][1] = acc[p][2] = acc[p][3] = 0.f;
    const int64_t a = s_rp[0], z = s_rp[kSpBM];
    for (int64_t w0 = a; w0 < z; w0 += kSpWin) {
        const int64_t w1 = min(z, w0 + (int64_t)kSpWin);
        __syncthreads();
        for (int64_t e = w0 + tid; e < w1; e += kSpThreads) {
            s_col[e - w0] = col[e];
            s_val[e - w0] = val[e];
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < kSpBM; ++p) {
            const int lo = (int)(max(s_rp[p], w0) - w0);
            const int hi = (int)(min(s_rp[p + 1], w1) - w0);
#pragma unroll 4
            for (int e = lo; e < hi; ++e) {
                const float v = s_val[e];
                const float4 c = __ldg(CT + (int64_t)s_col[e] * kp4 + j4);
                acc[p][0] = fmaf(v, c.x, acc[p][0]);
                acc[p][1] = fmaf(v, c.y, acc[p][1]);
                acc[p][2] = fmaf(v, c.z, acc[p][2]);
                acc[p][3] = fmaf(v, c.w, acc[p][3]);
            }
        }
    }

    const int jb = 4 * j4;
    const float4 cv = reinterpret_cast<const float4 *>(cn)[j4];
    const float cq[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
    for (int p = 0; p < kSpBM; ++p) {
        Top2 t{FLT_MAX, FLT_MAX, INT_MAX};
#pragma unroll
        for (int q = 0; q < 4; ++q) top2_push(t, fmaf(-2.f, acc[p][q], cq[q]), jb + q);
        for (int o = 16; o > 0; o >>= 1) {
            const float ob1 = __shfl_xor_sync(kFull, t.b1, o);
            const float ob2 = __shfl_xor_sync(kFull, t.b2, o);
            const int oi1 = __shfl_xor_sync(kFull, t.i1, o);
            top2_merge(t, ob1, oi1, ob2);
        }
        if (lane == 0) {
            w_b1[w][p] = t.b1;
            w_b2[w][p] = t.b2;
            w_i1[w][p] = t.i1;
        }
    }
    __syncthreads();
    if (tid < kSpBM && r0 + tid < n) {
        Top2 t{w_b1[0][tid], w_b2[0][tid], w_i1[0][tid]};
#pragma unroll
        for (int v = 1; v < kSpThreads / 32; ++v) top2_merge(t, w_b1[v][tid], w_i1[v][tid], w_b2[v][tid]);
        const int64_t o = (int64_t)blockIdx.y * n + r0 + tid;
        pb1[o] = t.b1;
        pb2[o] = t.b2;
        pi1[o] = t.i1;
    }
}

// Rounding bound of the FP32 distances above for a row of m nonzeros: each is
// within (m + 4) u (||x||^2 + ||c||^2) of the exact value (m FMAs of products
// bounded by Cauchy-Schwarz, the rounded FP64 norm, the final FMA), so two of
// them can swap order only if they differ by less than twice that.
__device__ __forceinline__ float sp_margin(int64_t m, float xn, float cn_max) {
    return 2.02f * ((float)m + 4.f) * kU * (xn + cn_max);
}

__global__ void sp_combine_kernel(const float *__restrict__ pb1, const int32_t *__restrict__ pi1,
                                  const float *__restrict__ pb2, int nch, int64_t n, int k,
                                  const int64_t *__restrict__ rp, const float *__restrict__ xn,
                                  const float *__restrict__ cn_max, int32_t *__restrict__ labels,
                                  int32_t *__restrict__ flagged, int *__restrict__ n_flagged) {
    const float cmax = *cn_max;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Top2 t{pb1[i], pb2[i], pi1[i]};
        for (int c = 1; c < nch; ++c) {
            const int64_t o = (int64_t)c * n + i;
            top2_merge(t, pb1[o], pi1[o], pb2[o]);
        }
        // (a row with no finite distance -- NaN input -- gets label 0 and is listed)
        const bool ok = t.i1 >= 0 && t.i1 < k;
        labels[i] = ok ? t.i1 : 0;
        if (!ok || !(t.b2 - t.b1 > sp_margin(rp[i + 1] - rp[i], xn[i], cmax)))
            flagged[atomicAdd(n_flagged, 1)] = (int32_t)i;
    }
}

// Listed rows, decided exactly: an FP32 pass over all k finds the smallest
// distance; every centroid within the rounding bound of it is then evaluated
// in float-float as sum_{t in x} (x_t - c_t)^2 + (||c||^2 - sum_{t in x}
// c_t^2) (the difference form over the row's support plus the centroid's
// mass outside it), and the smallest (distance, j) wins.
constexpr int kRcThreads = 256;
__global__ __launch_bounds__(kRcThreads) void sp_recheck_kernel(
    const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ CT, int kp,
    const float *__restrict__ cn, const float *__restrict__ cn_lo, int k,
    const int32_t *__restrict__ flagged, const int *__restrict__ n_flagged,
    const float *__restrict__ xn, const float *__restrict__ cn_max,
    int32_t *__restrict__ labels) {
    __shared__ float red_f[kRcThreads / 32];
    __shared__ FF red_d[kRcThreads / 32];
    __shared__ int red_i[kRcThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int nf = *n_flagged;
    const float cmax = *cn_max;
    for (int f = blockIdx.x; f < nf; f += gridDim.x) {
        const int64_t i = flagged[f];
        const int64_t b = rp[i], e = rp[i + 1];
        auto d32 = [&](int j) {
            float acc = 0.f;
            for (int64_t t = b; t < e; ++t) acc = fmaf(val[t], CT[(int64_t)col[t] * kp + j], acc);
            return fmaf(-2.f, acc, cn[j]);
        };
        float mn = FLT_MAX;
        for (int j = tid; j < k; j += kRcThreads) mn = fminf(mn, d32(j));
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(kFull, mn, o));
        if (lane == 0) red_f[w] = mn;
        __syncthreads();
        mn = red_f[0];
        for (int v = 1; v < kRcThreads / 32; ++v) mn = fminf(mn, red_f[v]);
        const float thr = mn + sp_margin(e - b, xn[i], cmax);
        FF best{FLT_MAX, 0.f};
        int bj = INT_MAX;
        for (int j = tid; j < k; j += kRcThreads) {
            if (!(d32(j) <= thr)) continue;
            FF A{0.f, 0.f}, B{0.f, 0.f};
            for (int64_t t = b; t < e; ++t) {
                const float c = CT[(int64_t)col[t] * kp + j];
                A = ff_add_sq_diff(A, val[t], c);
                B = ff_add_sq(B, c);
            }
            const FF D = ff_add(A, ff_add(FF{cn[j], cn_lo[j]}, ff_neg(B)));
            if (ff_lt(D, best) || (D.hi == best.hi && D.lo == best.lo && j < bj)) {
                best = D;
                bj = j;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const FF ob = ff_shfl_xor(best, o);
            const int oj = __shfl_xor_sync(kFull, bj, o);
            if (ff_lt(ob, best) || (ob.hi == best.hi && ob.lo == best.lo && oj < bj)) {
                best = ob;
                bj = oj;
            }
        }
        if (lane == 0) {
            red_d[w] = best;
            red_i[w] = bj;
        }
        __syncthreads();
        if (tid == 0) {
            for (int v = 1; v < kRcThreads / 32; ++v)
                if (ff_lt(red_d[v], best) ||
                    (red_d[v].hi == best.hi && red_d[v].lo == best.lo && red_i[v] < bj)) {
                    best = red_d[v];
                    bj = red_i[v];
                }
            if (bj >= 0 && bj < k) labels[i] = bj;
        }
        __syncthreads();
    }
}

// dist[i] = ||x_i - c_{labels[i]}||^2 as A + (||c||^2 - B), warp per row.
__global__ void csr_label_dist_kernel(const int64_t *__restrict__ rp,
                                      const int32_t *__restrict__ col,
                                      const float *__restrict__ val, int64_t n,
                                      const float *__restrict__ C, int dp,
                                      const float *__restrict__ cn,
                                      const int32_t *__restrict__ labels,
                                      float *__restrict__ dist) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t j = labels[i];
        const float *cj = C + (int64_t)j * dp;
        float A = 0.f, B = 0.f;
        for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) {
            const float c = cj[col[t]];
            const float x = val[t] - c;
            A = fmaf(x, x, A);
            B = fmaf(c, c, B);
        }
        for (int o = 16; o > 0; o >>= 1) {
            A += __shfl_xor_sync(kFull, A, o);
            B += __shfl_xor_sync(kFull, B, o);
        }
        if (lane == 0) dist[i] = A + fmaxf(cn[j] - B, 0.f);
    }
}

// ---------------------------------------------------------- mean update

constexpr int kUpThreads = 512;
constexpr int kUpWarps = kUpThreads / 32;
constexpr size_t kUpSmem = 96 * 1024;  // the dense accumulator row (window)

// Block (j, window): Cn[j][c0 .. c0+cw) = mean of the members' rows (member
// order; warp w owns columns [c0 + w*cw/16, ...)), or Cp[j] for an empty
// cluster.  Blocks of window 0 also add sum_i ||x_i - c_j||^2 over the
// members to sse[j] (distance to the previous centroid, A + (||c||^2 - B)).
// Acc = float for clusters of at most 2^20 members, double above; a launch
// with BIG handles only clusters above, one without only clusters up to it.
template <class Acc, bool BIG>
__global__ __launch_bounds__(kUpThreads) void csr_update_kernel(
    const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
    const float *__restrict__ val, const int32_t *__restrict__ perm,
    const int64_t *__restrict__ off, int dp, int cw, const float *__restrict__ Cp,
    const float *__restrict__ cnp, float *__restrict__ Cn, float *__restrict__ sse) {
    extern __shared__ __align__(16) unsigned char upd_smem[];
    Acc *acc = reinterpret_cast<Acc *>(upd_smem);
    __shared__ float wsse[kUpWarps];
    const int j = blockIdx.x;
    const int64_t b = off[j], m = off[j + 1] - b;
    if ((m > (1 << 20)) != BIG) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int c0 = blockIdx.y * cw;
    const int cwin = min(cw, dp - c0);
    if (m == 0) {
        if (Cn)
            for (int c = tid; c < cwin; c += kUpThreads)
                Cn[(int64_t)j * dp + c0 + c] = Cp[(int64_t)j * dp + c0 + c];
        return;
    }
    if (blockIdx.y == 0) {
        // squared distances of the members to the previous centroid (warp per member)
        const float *cj = Cp + (int64_t)j * dp;
        const float cnj = cnp[j];
        float s = 0.f;
        for (int64_t r = w; r < m; r += kUpWarps) {
            const int64_t row = perm[b + r];
            float A = 0.f, B = 0.f;
            for (int64_t t = rp[row] + lane; t < rp[row + 1]; t += 32) {
                const float c = cj[col[t]];
                const float x = val[t] - c;
                A = fmaf(x, x, A);
                B = fmaf(c, c, B);
            }
            for (int o = 16; o > 0; o >>= 1) {
                A += __shfl_xor_sync(kFull, A, o);
                B += __shfl_xor_sync(kFull, B, o);
            }
            s += A + fmaxf(cnj - B, 0.f);
        }
        if (lane == 0) wsse[w] = s;
    }
    if (Cn) {
        for (int c = tid; c < cwin; c += kUpThreads) acc[c] = Acc(0);
        __syncthreads();
        const int per = (cwin + kUpWarps - 1) / kUpWarps;
        const int lo = c0 + w * per, hi = min(c0 + cwin, lo + per);
        for (int64_t r = 0; r < m; ++r) {
            const int64_t row = perm[b + r];
            const int64_t rb = rp[row], re = rp[row + 1];
            for (int64_t t = rb + lane; t < re; t += 32) {
                const int c = col[t];
                if (c >= lo && c < hi) acc[c - c0] += (Acc)val[t];
            }
            __syncwarp();
        }
        __syncthreads();
        const Acc cnt = Acc(m);
        for (int c = tid; c < cwin; c += kUpThreads)
            Cn[(int64_t)j * dp + c0 + c] = (float)(acc[c] / cnt);
    }
    if (blockIdx.y == 0) {
        __syncthreads();
        if (tid == 0) {
            float t = 0.f;
            for (int v = 0; v < kUpWarps; ++v) t += wsse[v];
            sse[j] = t;
        }
    }
}

}  // namespace

// ================================================================ launchers

void csr_validate(const int64_t *rp, const int32_t *col, int64_t n, int64_t nnz, int d, int *bad,
                  cudaStream_t s) {
    MASK_CUDA(cudaMemsetAsync(bad, 0, 3 * sizeof(int), s));
    if (n > 0) {
        csr_check_rows_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(rp, col, n, bad);
        MASK_LAUNCHED("csr_check_rows");
    }
    if (nnz > 0) {
        csr_check_cols_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(col, nnz, d, bad);
        MASK_LAUNCHED("csr_check_cols");
    }
}

void csr_row_sqnorm(const int64_t *rp, const float *val, int64_t n, float *xn, cudaStream_t s) {
    if (n == 0) return;
    csr_sqnorm_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(rp, val, n, xn);
    MASK_LAUNCHED("csr_sqnorm");
}

void inclusive_scan_i64(int64_t *v, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    Scratch<int64_t> tsum(nt, s);
    scan_tiles_kernel<<<(unsigned)nt, kScanThreads, 0, s>>>(v, n, tsum.get());
    MASK_LAUNCHED("scan_tiles");
    if (nt > 1) {
        scan_tile_sums_kernel<<<1, kScanThreads, 0, s>>>(tsum.get(), nt);
        MASK_LAUNCHED("scan_tile_sums");
        scan_add_kernel<<<(unsigned)nt, 256, 0, s>>>(v, n, tsum.get());
        MASK_LAUNCHED("scan_add");
    }
}

template <class I>
void csr_gather_rows(const int64_t *rp, const int32_t *col, const float *val, const I *idx,
                     int64_t m, DevArray<int64_t> &orp, DevArray<int32_t> &ocol,
                     DevArray<float> &oval, cudaStream_t s) {
    orp.alloc((size_t)m + 1);
    csr_gather_len_kernel<I><<<grid_for(m, 256), 256, 0, s>>>(rp, idx, m, orp.get());
    MASK_LAUNCHED("csr_gather_len");
    inclusive_scan_i64(orp.get() + 1, m, s);
    int64_t nnz = 0;
    MASK_CUDA(cudaMemcpyAsync(&nnz, orp.get() + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MASK_CUDA(cudaStreamSynchronize(s));
    ocol.alloc((size_t)(nnz > 0 ? nnz : 1));
    oval.alloc((size_t)(nnz > 0 ? nnz : 1));
    if (m == 0) return;
    csr_gather_copy_kernel<I><<<grid_for(m * 32, 256), 256, 0, s>>>(rp, col, val, idx, m, orp.get(),
                                                                  ocol.get(), oval.get());
    MASK_LAUNCHED("csr_gather_copy");
}
template void csr_gather_rows<int32_t>(const int64_t *, const int32_t *, const float *,
                                       const int32_t *, int64_t, DevArray<int64_t> &,
                                       DevArray<int32_t> &, DevArray<float> &, cudaStream_t);
template void csr_gather_rows<int64_t>(const int64_t *, const int32_t *, const float *,
                                       const int64_t *, int64_t, DevArray<int64_t> &,
                                       DevArray<int32_t> &, DevArray<float> &, cudaStream_t);

void csr_densify_rows(const int64_t *rp, const int32_t *col, const float *val,
                      const int64_t *rows, int64_t m, int dp, float *out, cudaStream_t s) {
    if (m == 0) return;
    MASK_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)m * dp, s));
    csr_densify_kernel<<<grid_for(m * 32, 256), 256, 0, s>>>(rp, col, val, rows, m, dp, out);
    MASK_LAUNCHED("csr_densify");
}

void centroid_norms(const float *C, int k, int dp, int kp, float *cn, float *cn_lo,
                    cudaStream_t s) {
    centroid_norms_kernel<<<grid_for((int64_t)kp * 32, 256), 256, 0, s>>>(C, k, dp, kp, cn, cn_lo);
    MASK_LAUNCHED("centroid_norms");
}

int csr_assign_kp(int k) { return (k + kSpBN - 1) / kSpBN * kSpBN; }

void csr_assign(const int64_t *rp, const int32_t *col, const float *val, int64_t n,
                int64_t nnz, const float *xn, const float *C, int k, int dp, int32_t *labels, float *cn_out,
                cudaStream_t s) {
    if (n == 0) return;
    const int kp = csr_assign_kp(k);
    const int nch = kp / kSpBN;
    ProfRegion pr("csr_assign", s, 0.0);
    Scratch<float> CT((size_t)dp * kp, s), cn(kp, s), cmax(1, s);
    Scratch<float> cn_lo(k, s);
    centroid_norms(C, k, dp, kp, cn.get(), cn_lo.get(), s);
    max_reduce(cn.get(), k, cmax.get(), s);
    dim3 tg((dp + 31) / 32, kp / 32), tb(32, 8);
    transpose_ct_kernel<<<tg, tb, 0, s>>>(C, k, dp, kp, CT.get());
    MASK_LAUNCHED("transpose_ct");
    Scratch<float> pb1((size_t)nch * n, s), pb2((size_t)nch * n, s);
    Scratch<int32_t> pi1((size_t)nch * n, s), flagged(n, s);
    Scratch<int> nflag(1, s);
    MASK_CUDA(cudaMemsetAsync(nflag.get(), 0, sizeof(int), s));
    dim3 g((unsigned)((n + kSpBM - 1) / kSpBM), nch);
    {
        ProfRegion pk("csr_spmm_assign", s, 2.0 * (double)nnz * (double)k);
        spmm_assign_kernel<<<g, kSpThreads, 0, s>>>(rp, col, val, n,
                                                    reinterpret_cast<const float4 *>(CT.get()),
                                                    kp / 4, cn.get(), pb1.get(), pi1.get(),
                                                    pb2.get());
        MASK_LAUNCHED("spmm_assign");
    }
    sp_combine_kernel<<<grid_for(n, 256), 256, 0, s>>>(pb1.get(), pi1.get(), pb2.get(), nch, n, k,
                                                       rp, xn, cmax.get(), labels, flagged.get(),
                                                       nflag.get());
    MASK_LAUNCHED("sp_combine");
    sp_recheck_kernel<<<152 * 4, kRcThreads, 0, s>>>(rp, col, val, CT.get(), kp, cn.get(),
                                                     cn_lo.get(), k, flagged.get(), nflag.get(), xn,
                                                     cmax.get(), labels);
    MASK_LAUNCHED("sp_recheck");
    if (cn_out) MASK_CUDA(cudaMemcpyAsync(cn_out, cn.get(), sizeof(float) * k,
                                          cudaMemcpyDeviceToDevice, s));
}

void csr_label_dist(const int64_t *rp, const int32_t *col, const float *val, int64_t n,
                    const float *C, int dp, const float *cn, const int32_t *labels, float *dist,
                    cudaStream_t s) {
    if (n == 0) return;
    csr_label_dist_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(rp, col, val, n, C, dp, cn, labels,
                                                                dist);
    MASK_LAUNCHED("csr_label_dist");
}

void csr_centroid_update(const int64_t *rp, const int32_t *col, const float *val,
                         const int32_t *perm, const int64_t *off, int64_t n_rows, int k, int dp,
                         const float *C_prev, const float *cn_prev, float *C_new, float *sse,
                         cudaStream_t s) {
    ProfRegion pr("csr_centroid_update", s, 0.0);
    MASK_CUDA(cudaMemsetAsync(sse, 0, sizeof(float) * k, s));
    auto launch = [&](auto kfn, size_t elem) {
        int cw = (int)(kUpSmem / elem);
        if (cw > dp) cw = dp;
        const int windows = C_new ? (dp + cw - 1) / cw : 1;
        const size_t smem = C_new ? (size_t)cw * elem : 0;
        MASK_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kUpSmem));
        kfn<<<dim3(k, windows), kUpThreads, smem, s>>>(rp, col, val, perm, off, dp, cw, C_prev,
                                                       cn_prev, C_new, sse);
        MASK_LAUNCHED("csr_centroid_update");
    };
    launch(csr_update_kernel<float, false>, sizeof(float));
    if (n_rows > (1 << 20)) launch(csr_update_kernel<double, true>, sizeof(double));
}

}  // namespace mask
