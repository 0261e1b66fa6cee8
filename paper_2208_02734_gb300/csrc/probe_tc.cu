// probe_tc.cu -- a timing probe of the 5th-generation tensor-core MMA
// (tcgen05.mma.cta_group::1.kind::f16, M = 128, K = 16): one CTA, one issuing
// thread, `rounds` rounds of the assignment kernel's 12-MMA pattern (4
// K-steps x 3 products) into n_acc accumulators used round-robin, A from
// shared or tensor memory, B from shared memory, timed with clock64 from the
// first issue to the commit's arrival.  It measures how an MMA's time
// depends on N (the tile width choice of the tensor-core assignment); the
// operands are zeros, the results unused.
#include <cuda.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace mask {
namespace {

using namespace tc;

__device__ __forceinline__ void probe_mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void probe_mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc,
                                             uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

constexpr int kProbeSmem = 96 * 1024;   // A hi/lo (2 x 16 KB), B hi/lo (2 x 32 KB)

// out[0] = cycles spent issuing, out[1] = cycles until the last MMA completed,
// out[2] = 1 if the completion arrived within the wait limit.
__global__ void __launch_bounds__(128, 1)
    probe_mma_kernel(int n, int a_tmem, int n_acc, int rounds, long long *out, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const uint32_t raw = smem_u32(smem_raw), base = (raw + 1023u) & ~1023u;
    unsigned char *bp = smem_raw + (base - raw);
    for (int i = threadIdx.x; i < kProbeSmem / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(bp)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();   // the zeros, seen by the tensor core's operand reads
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tslot;
    if (threadIdx.x == 0) {
        // D = F32, A = B = F16, both K-major, N = n, M = 128
        const uint32_t idesc = (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        const uint64_t dA = sw128_desc(base), dAl = sw128_desc(base + 16384);
        const uint64_t dB = sw128_desc(base + 32768), dBl = sw128_desc(base + 65536);
        const uint32_t tA = tmem + 448u, tAl = tmem + 480u;   // A parts in columns 448..511
        const long long t0 = clock64();
        for (int r = 0; r < rounds; ++r) {
            const uint32_t d = tmem + (uint32_t)((r % n_acc) * n);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t off = (uint64_t)(kk * 2);
                if (a_tmem) {
                    probe_mma_ts(d, tA + kk * 8, dB + off, idesc, kk > 0 ? 1u : 0u);
                    probe_mma_ts(d, tA + kk * 8, dBl + off, idesc, 1u);
                    probe_mma_ts(d, tAl + kk * 8, dB + off, idesc, 1u);
                } else {
                    probe_mma_ss(d, dA + off, dB + off, idesc, kk > 0 ? 1u : 0u);
                    probe_mma_ss(d, dA + off, dBl + off, idesc, 1u);
                    probe_mma_ss(d, dAl + off, dB + off, idesc, 1u);
                }
            }
        }
        const long long t1 = clock64();
        mma_commit(smem_u32(&bar));
        const bool ok = mbar_wait(smem_u32(&bar), 0, err, true);
        out[0] = t1 - t0;
        out[1] = clock64() - t0;
        out[2] = ok ? 1 : 0;
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem)
                     : "memory");
    }
}

}  // namespace

void probe_tc_mma(int n, int a_in_tmem, int n_acc, int rounds, int64_t *cycles_out) {
    MASK_REQUIRE(cycles_out != nullptr, "cycles_out is NULL");
    MASK_REQUIRE(n >= 16 && n <= 256 && n % 16 == 0, "n must be a multiple of 16 in [16, 256]");
    MASK_REQUIRE(n_acc >= 1 && rounds >= 1 && rounds <= (1 << 16), "n_acc or rounds out of range");
    MASK_REQUIRE(n_acc * n <= (a_in_tmem ? 448 : 512), "accumulators exceed tensor memory");
    MASK_REQUIRE(encode_fn() != nullptr, "no tensor-core support on this device");
    const int smem = kProbeSmem + 1024;
    MASK_CUDA(cudaFuncSetAttribute(probe_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem));
    Scratch<long long> out(3, nullptr);
    Scratch<int> err(1, nullptr);
    MASK_CUDA(cudaMemset(err.get(), 0, sizeof(int)));
    probe_mma_kernel<<<1, 128, smem>>>(n, a_in_tmem ? 1 : 0, n_acc, rounds, out.get(), err.get());
    MASK_LAUNCHED("probe_mma");
    long long h[3] = {0, 0, 0};
    MASK_CUDA(cudaMemcpy(h, out.get(), sizeof(h), cudaMemcpyDeviceToHost));
    if (h[2] != 1) fail(MASK_ETIMEOUT, "tensor-core probe: the MMAs did not complete in time");
    cycles_out[0] = h[0];
    cycles_out[1] = h[1];
}

}  // namespace mask
