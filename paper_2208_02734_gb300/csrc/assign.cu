// assign.cu -- Lloyd assignment half-step (§2.4, used by Algorithm 1):
// labels[i] = argmin_j ||x_i - c_j||^2, ties to the smallest j.
//
// Two stages:
//  1. A distance GEMM in the expanded form ||x||^2 - 2 x.c + ||c||^2 with the
//     running best / second-best fused into the epilogue (no distance matrix
//     is ever written).  FP32 FMA accumulation; its rounding error is bounded
//     by (2*dp + 4) * 2^-24 * (||x||^2 + ||c||^2) per distance, so a row whose
//     best and second-best differ by more than twice that bound has a certain
//     label.
//  2. Rows whose gap is within the bound are listed and re-decided exactly in
//     the difference form sum_t (x_t - c_t)^2 (relative error ~ dp * 2^-24 of
//     the distance itself) over all centroids.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>

#include "common.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

__device__ __forceinline__ void merge_best(float &b1, int &j1, float &b2, float ob1, int oj1,
                                           float ob2) {
    if (ob1 < b1 || (ob1 == b1 && oj1 < j1)) {
        b2 = fminf(b1, ob2);
        b1 = ob1;
        j1 = oj1;
    } else {
        b2 = fminf(b2, ob1);
    }
}

// Rows [blockIdx.x*BM, +BM) against all k centroids, tile by tile.
// Thread (ty, tx) owns rows {ty*4+i, 64+ty*4+i} and columns {tx*4+j, 64+tx*4+j}.
__global__ __launch_bounds__(NT, 2) void assign_gemm_kernel(
    const float *__restrict__ X, const float *__restrict__ xn, int64_t n, int dp,
    const float *__restrict__ C, const float *__restrict__ cn, int k,
    const float *__restrict__ cn_max, float margin_coef, int32_t *__restrict__ labels,
    int32_t *__restrict__ flagged, int *__restrict__ n_flagged) {
    __shared__ __align__(16) float As[BK][BM];
    __shared__ __align__(16) float Bs[BK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * BM;

    // tile loaders: one float4 of A and one of B per thread per K step
    const int lr = tid >> 1, lk = (tid & 1) * 4;
    const int64_t arow = row0 + lr;

    float xr[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        xr[i] = r < n ? xn[r] : 0.f;
    }
    float b1[8], b2[8];
    int j1[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { b1[i] = FLT_MAX; b2[i] = FLT_MAX; j1[i] = INT_MAX; }

    for (int c0 = 0; c0 < k; c0 += BN) {
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        const int bcol = c0 + lr;
        for (int k0 = 0; k0 < dp; k0 += BK) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (arow < n) a = *reinterpret_cast<const float4 *>(X + arow * dp + k0 + lk);
            if (bcol < k) b = *reinterpret_cast<const float4 *>(C + (int64_t)bcol * dp + k0 + lk);
            As[lk + 0][lr] = a.x; As[lk + 1][lr] = a.y; As[lk + 2][lr] = a.z; As[lk + 3][lr] = a.w;
            Bs[lk + 0][lr] = b.x; Bs[lk + 1][lr] = b.y; Bs[lk + 2][lr] = b.z; Bs[lk + 3][lr] = b.w;
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
                const float4 q0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                const float4 q1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
        // epilogue: fold this tile's distances into the running best/second
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (c < k) {
                const float cc = cn[c];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float dd = xr[i] - 2.f * acc[i][j] + cc;
                    if (dd < b1[i]) { b2[i] = b1[i]; b1[i] = dd; j1[i] = c; }
                    else if (dd < b2[i]) b2[i] = dd;
                }
            }
        }
    }
    // merge across the 16 threads (tx) that share each row
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        for (int o = 1; o < 16; o <<= 1) {
            const float ob1 = __shfl_xor_sync(kFull, b1[i], o);
            const int oj1 = __shfl_xor_sync(kFull, j1[i], o);
            const float ob2 = __shfl_xor_sync(kFull, b2[i], o);
            merge_best(b1[i], j1[i], b2[i], ob1, oj1, ob2);
        }
    }
    if (tx == 0) {
        const float cmax = *cn_max;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (r >= n) continue;
            labels[r] = j1[i];
            const float margin = margin_coef * (xr[i] + cmax);
            if (k > 1 && !(b2[i] - b1[i] > margin)) {
                const int slot = atomicAdd(n_flagged, 1);
                flagged[slot] = (int32_t)r;
            }
        }
    }
}

// Exact re-decision of the listed rows: one block per row, one group of LPR
// lanes per centroid, difference form, minimum of (distance, index) keys.
template <int LPR>
__global__ __launch_bounds__(256) void assign_recheck_kernel(
    const float4 *__restrict__ X, int dp4, const float4 *__restrict__ C, int k,
    const int32_t *__restrict__ flagged, const int *__restrict__ n_flagged,
    int32_t *__restrict__ labels) {
    __shared__ unsigned long long red[8];
    constexpr int G = 256 / LPR;
    const int g = threadIdx.x / LPR, gl = threadIdx.x % LPR;
    const int cnt = *n_flagged;
    for (int f = blockIdx.x; f < cnt; f += gridDim.x) {
        const int64_t r = flagged[f];
        const float4 *xr = X + r * dp4;
        unsigned long long best = kNoKey;
        const int k_round = (k + G - 1) / G * G;
        for (int j = g; j < k_round; j += G) {
            float acc = 0.f;
            if (j < k) {
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
            if (j < k) {
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(acc) << 32) | (unsigned)j;
                best = min(best, key);
            }
        }
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(kFull, best, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = red[0];
            for (int w = 1; w < 8; ++w) b = min(b, red[w]);
            labels[r] = (int32_t)(b & 0xffffffffu);
        }
        __syncthreads();
    }
}

}  // namespace

void assign_labels(const float *X, const float *xn, int64_t n, int dp, const float *C, int k,
                   int32_t *labels, cudaStream_t s) {
    if (n == 0) return;
    Scratch<float> cn(k, s), cmax(1, s);
    Scratch<int32_t> flagged(n, s);
    Scratch<int> nflag(1, s);
    row_sqnorm(C, k, dp, cn.get(), s);
    max_reduce(cn.get(), k, cmax.get(), s);
    MASK_CUDA(cudaMemsetAsync(nflag.get(), 0, sizeof(int), s));
    // per-distance bound (2dp+4) u (||x||^2+||c||^2); a certain label needs a
    // gap above twice the bound
    const float coef = (float)(2.0 * (2.0 * dp + 4.0) * 0x1.0p-24);
    const int64_t blocks = (n + BM - 1) / BM;
    {
        ProfRegion pr("assign_gemm", s, 2.0 * (double)n * (double)k * (double)dp);
        assign_gemm_kernel<<<(unsigned)blocks, NT, 0, s>>>(X, xn, n, dp, C, cn.get(), k,
                                                          cmax.get(), coef, labels,
                                                          flagged.get(), nflag.get());
        MASK_LAUNCHED("assign_gemm");
    }
    const int lpr = lanes_per_row(dp);
    const int grid = 152 * 8;
    ProfRegion pr("assign_recheck", s, 0.0);
    switch (lpr) {
    case 1: assign_recheck_kernel<1><<<grid, 256, 0, s>>>((const float4 *)X, dp / 4, (const float4 *)C, k, flagged.get(), nflag.get(), labels); break;
    case 2: assign_recheck_kernel<2><<<grid, 256, 0, s>>>((const float4 *)X, dp / 4, (const float4 *)C, k, flagged.get(), nflag.get(), labels); break;
    case 4: assign_recheck_kernel<4><<<grid, 256, 0, s>>>((const float4 *)X, dp / 4, (const float4 *)C, k, flagged.get(), nflag.get(), labels); break;
    case 8: assign_recheck_kernel<8><<<grid, 256, 0, s>>>((const float4 *)X, dp / 4, (const float4 *)C, k, flagged.get(), nflag.get(), labels); break;
    case 16: assign_recheck_kernel<16><<<grid, 256, 0, s>>>((const float4 *)X, dp / 4, (const float4 *)C, k, flagged.get(), nflag.get(), labels); break;
    default: assign_recheck_kernel<32><<<grid, 256, 0, s>>>((const float4 *)X, dp / 4, (const float4 *)C, k, flagged.get(), nflag.get(), labels); break;
    }
    MASK_LAUNCHED("assign_recheck");
}

}  // namespace mask

namespace mask {

void assign_recheck_rows(const float *X, int dp, const float *C, int k, const int32_t *rows,
                         const int *count, int32_t *labels, cudaStream_t s) {
    const int lpr = lanes_per_row(dp);
    const int grid = 152 * 8;
    const float4 *X4 = reinterpret_cast<const float4 *>(X);
    const float4 *C4 = reinterpret_cast<const float4 *>(C);
    switch (lpr) {
    case 1: assign_recheck_kernel<1><<<grid, 256, 0, s>>>(X4, dp / 4, C4, k, rows, count, labels); break;
    case 2: assign_recheck_kernel<2><<<grid, 256, 0, s>>>(X4, dp / 4, C4, k, rows, count, labels); break;
    case 4: assign_recheck_kernel<4><<<grid, 256, 0, s>>>(X4, dp / 4, C4, k, rows, count, labels); break;
    case 8: assign_recheck_kernel<8><<<grid, 256, 0, s>>>(X4, dp / 4, C4, k, rows, count, labels); break;
    case 16: assign_recheck_kernel<16><<<grid, 256, 0, s>>>(X4, dp / 4, C4, k, rows, count, labels); break;
    default: assign_recheck_kernel<32><<<grid, 256, 0, s>>>(X4, dp / 4, C4, k, rows, count, labels); break;
    }
    MASK_LAUNCHED("assign_recheck_rows");
}

}  // namespace mask

// ------------------------------------------------- allocation-free variant
//
// mask_kmeans_assign_noalloc runs the same two kernels as mask_kmeans_assign,
// but every temporary lives in one file-scope device array instead of memory
// obtained from cudaMalloc/cudaMallocAsync.  The array is sized for at most
// kNoAllocMaxK centroids; rows are processed kNoAllocChunk at a time, so the
// number of rows is unbounded.  Layout in 4-byte words, each section starting
// on a 256-byte boundary:
//   [centroid norms: kNoAllocMaxK][max norm: 64][flag count: 64]
//   [row norms: kNoAllocChunk][flagged rows: kNoAllocChunk]
namespace mask {
namespace {

constexpr int kNoAllocMaxK = 65536;
constexpr int64_t kNoAllocChunk = 1 << 18;
constexpr size_t kOffCn = 0;
constexpr size_t kOffCmax = kOffCn + kNoAllocMaxK;
constexpr size_t kOffNflag = kOffCmax + 64;
constexpr size_t kOffXn = kOffNflag + 64;
constexpr size_t kOffFlagged = kOffXn + kNoAllocChunk;
constexpr size_t kNoAllocWords = kOffFlagged + kNoAllocChunk;  // 2.36 MB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up once per device (with that device current) and cached.
uint32_t *noalloc_scratch() {
    int dev = 0;
    MASK_CUDA(cudaGetDevice(&dev));
    MASK_REQUIRE(dev >= 0 && dev < kNoAllocMaxDevices, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            fail(MASK_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    return static_cast<uint32_t *>(g_noalloc_ptr[dev]);
}

// True for device (or managed) memory of device `dev`: the scratch array
// used with it is the one of the current device.
bool is_device_memory(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

void assign_noalloc(const float *X, int64_t n, int d, const float *C, int k, int32_t *labels,
                    float *dist, cudaStream_t s) {
    uint32_t *base = noalloc_scratch();
    float *cn = reinterpret_cast<float *>(base + kOffCn);
    float *cmax = reinterpret_cast<float *>(base + kOffCmax);
    int *nflag = reinterpret_cast<int *>(base + kOffNflag);
    float *xn = reinterpret_cast<float *>(base + kOffXn);
    int32_t *flagged = reinterpret_cast<int32_t *>(base + kOffFlagged);

    row_sqnorm(C, k, d, cn, s);
    max_reduce(cn, k, cmax, s);  // clears cmax first
    const float coef = (float)(2.0 * (2.0 * d + 4.0) * 0x1.0p-24);
    const int lpr = lanes_per_row(d);
    for (int64_t c0 = 0; c0 < n; c0 += kNoAllocChunk) {
        const int64_t m = std::min<int64_t>(kNoAllocChunk, n - c0);
        const float *Xc = X + c0 * d;
        row_sqnorm(Xc, m, d, xn, s);
        MASK_CUDA(cudaMemsetAsync(nflag, 0, sizeof(int), s));
        assign_gemm_kernel<<<(unsigned)((m + BM - 1) / BM), NT, 0, s>>>(
            Xc, xn, m, d, C, cn, k, cmax, coef, labels + c0, flagged, nflag);
        MASK_LAUNCHED("assign_gemm (no-alloc)");
        const float4 *X4 = reinterpret_cast<const float4 *>(Xc);
        const float4 *C4 = reinterpret_cast<const float4 *>(C);
        const int grid = 152 * 8;
        switch (lpr) {
        case 1: assign_recheck_kernel<1><<<grid, 256, 0, s>>>(X4, d / 4, C4, k, flagged, nflag, labels + c0); break;
        case 2: assign_recheck_kernel<2><<<grid, 256, 0, s>>>(X4, d / 4, C4, k, flagged, nflag, labels + c0); break;
        case 4: assign_recheck_kernel<4><<<grid, 256, 0, s>>>(X4, d / 4, C4, k, flagged, nflag, labels + c0); break;
        case 8: assign_recheck_kernel<8><<<grid, 256, 0, s>>>(X4, d / 4, C4, k, flagged, nflag, labels + c0); break;
        case 16: assign_recheck_kernel<16><<<grid, 256, 0, s>>>(X4, d / 4, C4, k, flagged, nflag, labels + c0); break;
        default: assign_recheck_kernel<32><<<grid, 256, 0, s>>>(X4, d / 4, C4, k, flagged, nflag, labels + c0); break;
        }
        MASK_LAUNCHED("assign_recheck (no-alloc)");
        if (dist) label_dist(Xc, m, d, C, labels + c0, dist + c0, s);
    }
}

}  // namespace
}  // namespace mask

extern "C" mask_status mask_kmeans_assign_noalloc(const float *X, int64_t n, int32_t d,
                                                  const float *C, int32_t k, int32_t *labels_out,
                                                  float *dist_out, mask_stream stream) {
    using namespace mask;
    try {
        MASK_REQUIRE(X && C && labels_out, "NULL argument");
        MASK_REQUIRE(n >= 0 && n <= INT32_MAX, "n must be in [0, 2^31)");
        MASK_REQUIRE(d >= 8 && d % 8 == 0, "d must be a positive multiple of 8 (rows are used in place)");
        MASK_REQUIRE(k >= 1 && k <= kNoAllocMaxK,
                     "k must be in [1, 65536]: the no-alloc scratch holds at most 65536 centroid norms");
        MASK_REQUIRE((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(C)) % 16 == 0,
                     "X and C must be 16-byte aligned");
        int dev = 0;
        MASK_CUDA(cudaGetDevice(&dev));
        MASK_REQUIRE(is_device_memory(X, dev) && is_device_memory(C, dev) &&
                         is_device_memory(labels_out, dev) &&
                         (dist_out == nullptr || is_device_memory(dist_out, dev)),
                     "all arrays must be device memory of the current device (host staging "
                     "would allocate; another device's arrays cannot use this device's scratch)");
        if (n == 0) return MASK_OK;
        assign_noalloc(X, n, d, C, k, labels_out, dist_out, (cudaStream_t)stream);
        return MASK_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return MASK_ECUDA;
    }
}
