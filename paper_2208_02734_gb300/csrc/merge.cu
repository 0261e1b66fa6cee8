// merge.cu -- the one exchange step of the distributed design (§3.4): every
// node answers a query batch on its own partition with its own index, the
// nodes' k-NN lists are gathered, and each query keeps the k smallest
// (distance, global id) over all of them.  One block per query sorts its
// G x k candidates in shared memory (a bitonic network on (distance, id)
// pairs) and writes the first k.
#include <cfloat>

#include "common.cuh"

namespace mask {
namespace {

constexpr int kMgThreads = 256;

__device__ __forceinline__ bool pair_less(float da, int64_t ia, float db, int64_t ib) {
    return da < db || (da == db && ia < ib);
}

// ids/dists [G x nq x k] (partition-major, as gathered); id_offset[g] (may be
// null) is added to partition g's non-negative ids; P = next power of two of
// G * k.
__global__ __launch_bounds__(kMgThreads) void merge_topk_kernel(
    const int64_t *__restrict__ ids, const float *__restrict__ dists, int G, int64_t nq, int k,
    const int64_t *__restrict__ id_offset, int P, int64_t *__restrict__ ids_out,
    float *__restrict__ dists_out) {
    extern __shared__ __align__(16) unsigned char sm[];
    int64_t *sid = reinterpret_cast<int64_t *>(sm);
    float *sd = reinterpret_cast<float *>(sid + P);
    const int64_t q = blockIdx.x;
    const int n = G * k;
    for (int i = threadIdx.x; i < P; i += kMgThreads) {
        if (i < n) {
            const int g = i / k, r = i - g * k;
            const int64_t src = ((int64_t)g * nq + q) * k + r;
            const int64_t id = ids[src];
            const bool valid = id >= 0;
            sid[i] = valid ? id + (id_offset ? id_offset[g] : 0) : -1;
            sd[i] = valid ? dists[src] : __int_as_float(0x7f800000);
        } else {
            sid[i] = INT64_MAX;
            sd[i] = __int_as_float(0x7f800000);
        }
    }
    __syncthreads();
    // padding (-1 ids) must follow every real entry: order by (dist, id) with
    // invalid entries at +inf and ids INT64_MAX past the end
    for (int i = threadIdx.x; i < P; i += kMgThreads)
        if (sid[i] == -1) sid[i] = INT64_MAX - 1;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += kMgThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & kk) == 0;
                    const bool gt = pair_less(sd[ixj], sid[ixj], sd[i], sid[i]);
                    if (gt == up) {
                        const float td = sd[i];
                        sd[i] = sd[ixj];
                        sd[ixj] = td;
                        const int64_t ti = sid[i];
                        sid[i] = sid[ixj];
                        sid[ixj] = ti;
                    }
                }
            }
            __syncthreads();
        }
    for (int r = threadIdx.x; r < k; r += kMgThreads) {
        const bool valid = sid[r] < INT64_MAX - 1;
        ids_out[q * k + r] = valid ? sid[r] : -1;
        dists_out[q * k + r] = valid ? sd[r] : __int_as_float(0x7f800000);
    }
}

}  // namespace

size_t merge_topk_smem(int G, int k) {
    int P = 1;
    while (P < G * k) P <<= 1;
    return (size_t)P * (sizeof(int64_t) + sizeof(float));
}

void merge_topk(const int64_t *ids, const float *dists, int G, int64_t nq, int k,
                const int64_t *id_offset, int64_t *ids_out, float *dists_out, cudaStream_t s) {
    if (nq == 0) return;
    int P = 1;
    while (P < G * k) P <<= 1;
    const size_t smem = merge_topk_smem(G, k);
    MASK_CUDA(cudaFuncSetAttribute(merge_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
    ProfRegion pr("merge_topk", s, 0.0);
    merge_topk_kernel<<<(unsigned)nq, kMgThreads, smem, s>>>(ids, dists, G, nq, k, id_offset, P,
                                                             ids_out, dists_out);
    MASK_LAUNCHED("merge_topk");
}

}  // namespace mask
