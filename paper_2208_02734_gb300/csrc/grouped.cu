// grouped.cu -- the grouped multilevel build of §3.1 (Algorithm 1 as printed):
// the items of a level are split at random into floor(items / lengthGroup)
// groups, every group is clustered into nCentroids centroids by its own
// k-means (k-means++ seeding, §3.2, then Lloyd iterations, §2.4), and the
// centroids of all groups are the items of the next level, until fewer than
// lengthGroup items remain.
//
// On the GPU this is a batch of many small, independent k-means problems:
// one block per group, its items staged in shared memory, k-means++ picks
// decided by one thread in exact integers, assignment and mean update by the
// whole block.  The random split (a Fisher-Yates shuffle) and the seeding
// draws are taken on the host from the published SplitMix64 generator, like
// every draw of the library; the groups' member lists come from the same
// counting sort as the cluster membership lists.
#include <cfloat>
#include <climits>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace mask {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGkThreads = 128;

// x + y with the rounding error kept (Knuth's TwoSum), for member sums that
// stay exact far beyond FP32 over the longest groups.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    const float t = s + v;
    const float bb = t - s;
    c += (s - (t - bb)) + (v - bb);
    s = t;
}

__device__ __forceinline__ float sqdist_f32(const float *a, const float *b, int dp) {
    float acc = 0.f;
    for (int t = 0; t < dp; ++t) {
        const float e = a[t] - b[t];
        acc = fmaf(e, e, acc);
    }
    return acc;
}

// One group per block.  X: the level's items [m x dp]; gperm/goff: the
// items of each group in ascending index; a53[g * nc + t]: the group's t-th
// draw as the generator's 53-bit integer; first[g]: its first pick (index
// into the group, floor(u_0 * m_g) taken on the host).  Writes the group's
// centroids C[(g * nc + j) x dp] and the global label g * nc + j of every
// item.  Shared memory: items (m_g x dp), centres (nc x dp), D^2, labels.
__global__ __launch_bounds__(kGkThreads) void group_kmeans_kernel(
    const float *__restrict__ X, int dp, const int32_t *__restrict__ gperm,
    const int64_t *__restrict__ goff, const unsigned long long *__restrict__ a53,
    const int32_t *__restrict__ first, int nc, int iters, float *__restrict__ C,
    int32_t *__restrict__ labels) {
    extern __shared__ __align__(16) float sm[];
    const int g = blockIdx.x, tid = threadIdx.x;
    const int64_t b = goff[g];
    const int mg = (int)(goff[g + 1] - b);
    float *xs = sm;                          // [mg x dp]
    float *cs = xs + (size_t)mg * dp;        // [nc x dp]
    float *d2 = cs + (size_t)nc * dp;        // [mg]
    int *lab = reinterpret_cast<int *>(d2 + mg);       // [mg] (-2 marks a chosen item while seeding)
    __shared__ int s_pick;
    __shared__ float s_qs;

    for (int e = tid; e < mg * dp; e += kGkThreads) {
        const int q = e / dp, t = e - q * dp;
        xs[e] = X[(int64_t)gperm[b + q] * dp + t];
    }
    for (int q = tid; q < mg; q += kGkThreads) {
        d2[q] = FLT_MAX;
        lab[q] = 0;
    }
    __syncthreads();

    // ---- k-means++ (§3.2, R2): the draw rule decided in exact integers
    // (each D^2 as a 64-bit fixed-point value, scale from the first total,
    // pick = smallest q with prefix_q * 2^53 > a_t * Q).
    for (int t = 0; t < nc; ++t) {
        if (tid == 0) {
            int pick = -1;
            if (t == 0) {
                pick = first[g];
            } else {
                const float qs = s_qs;
                unsigned long long Q = 0;
                for (int q = 0; q < mg; ++q) Q += __float2ull_rn(d2[q] * qs);
                if (Q > 0) {
                    const unsigned long long at = a53[(int64_t)g * nc + t];
                    const unsigned long long thi = __umul64hi(at, Q), tlo = at * Q;
                    unsigned long long run = 0;
                    for (int q = 0; q < mg; ++q) {
                        run += __float2ull_rn(d2[q] * qs);
                        const unsigned long long hi = run >> 11, lo = run << 53;
                        if (hi > thi || (hi == thi && lo > tlo)) { pick = q; break; }
                    }
                } else {
                    // every item coincides with a chosen centre: the lowest
                    // index not chosen yet (chosen items have D^2 = 0 and are
                    // marked in lab[] below)
                    for (int q = 0; q < mg; ++q)
                        if (lab[q] != -2) { pick = q; break; }
                }
                if (pick < 0) pick = 0;
            }
            s_pick = pick;
            lab[pick] = -2;   // chosen
        }
        __syncthreads();
        const int pick = s_pick;
        for (int e = tid; e < dp; e += kGkThreads) cs[(size_t)t * dp + e] = xs[(size_t)pick * dp + e];
        __syncthreads();
        if (t + 1 < nc) {
            float part = 0.f;
            for (int q = tid; q < mg; q += kGkThreads) {
                const float v = sqdist_f32(xs + (size_t)q * dp, cs + (size_t)t * dp, dp);
                if (v < d2[q]) d2[q] = v;
                part += d2[q];
            }
            if (t == 0) {
                // the integer scale: 2^sh with 2 * (first total) * 2^sh < 2^61
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
                __shared__ float s_part[kGkThreads / 32];
                if ((tid & 31) == 0) s_part[tid >> 5] = part;
                __syncthreads();
                if (tid == 0) {
                    float tot = 0.f;
                    for (int w = 0; w < kGkThreads / 32; ++w) tot += s_part[w];
                    tot *= 2.f;
                    int sh = 0;
                    if (tot > 0.f) {
                        const int e = (int)((__float_as_uint(tot) >> 23) & 0xffu) - 127;
                        sh = 60 - e;
                        sh = sh < -126 ? -126 : (sh > 126 ? 126 : sh);
                    }
                    s_qs = __uint_as_float((uint32_t)(sh + 127) << 23);
                }
            }
            __syncthreads();
        }
    }

    // ---- Lloyd (§2.4, R4): iters assignment + update rounds, then a final
    // assignment; ties to the smallest centroid, member sums in ascending
    // item order, an empty cluster keeps its centroid.
    for (int it = 0; it <= iters; ++it) {
        for (int q = tid; q < mg; q += kGkThreads) {
            float best = FLT_MAX;
            int bj = 0;
            for (int j = 0; j < nc; ++j) {
                const float v = sqdist_f32(xs + (size_t)q * dp, cs + (size_t)j * dp, dp);
                if (v < best) { best = v; bj = j; }
            }
            lab[q] = bj;
        }
        __syncthreads();
        if (it == iters) break;
        for (int e = tid; e < nc * dp; e += kGkThreads) {
            const int j = e / dp, t = e - j * dp;
            float s = 0.f, c = 0.f;
            int n_j = 0;
            for (int q = 0; q < mg; ++q)
                if (lab[q] == j) {
                    kahan_add(s, c, xs[(size_t)q * dp + t]);
                    ++n_j;
                }
            if (n_j > 0) cs[e] = (s + c) / (float)n_j;
        }
        __syncthreads();
    }
    for (int e = tid; e < nc * dp; e += kGkThreads) C[((int64_t)g * nc) * dp + e] = cs[e];
    for (int q = tid; q < mg; q += kGkThreads) labels[gperm[b + q]] = g * nc + lab[q];
}

}  // namespace

// SplitMix64 state of group g's seeding at level lv (R17).
uint64_t group_state(uint64_t seed, int lv, int64_t g) {
    return level_state(seed, lv) ^ (0xD1B54A32D192ED03ull * (uint64_t)(g + 1));
}

std::vector<int64_t> grouped_sizes(int64_t n, int lg, int nc) {
    std::vector<int64_t> sizes;
    int64_t items = n, groups = n / lg;
    while (groups >= 1) {
        sizes.push_back(groups * nc);
        items = groups * nc;
        groups = items / lg;
    }
    return sizes;
}

// R16: group_of[item] for m items split at random into G groups (a full
// Fisher-Yates shuffle, then consecutive parts of sizes differing by at most
// one, the first m mod G parts one larger).
std::vector<int32_t> split_groups(int64_t m, int64_t G, SplitMix64 &rng) {
    std::vector<int64_t> perm((size_t)m);
    for (int64_t i = 0; i < m; ++i) perm[(size_t)i] = i;
    for (int64_t j = 0; j + 1 < m; ++j) {
        int64_t r = j + (int64_t)std::floor(rng.uniform() * (double)(m - j));
        if (r > m - 1) r = m - 1;
        std::swap(perm[(size_t)j], perm[(size_t)r]);
    }
    std::vector<int32_t> group_of((size_t)m);
    const int64_t base = m / G, extra = m % G;
    int64_t pos = 0;
    for (int64_t g = 0; g < G; ++g) {
        const int64_t len = base + (g < extra ? 1 : 0);
        for (int64_t q = 0; q < len; ++q) group_of[(size_t)perm[(size_t)(pos + q)]] = (int32_t)g;
        pos += len;
    }
    return group_of;
}

size_t group_kmeans_smem(int64_t max_group, int dp, int nc) {
    return ((size_t)max_group * dp + (size_t)nc * dp + (size_t)max_group) * sizeof(float) +
           (size_t)max_group * sizeof(int);
}

// One level of the grouped build on the m padded rows X: group_of (host) gives
// each item's group; writes C [G*nc x dp] and labels [m] (global ids).
void grouped_level(const float *X, int64_t m, int dp, const std::vector<int32_t> &group_of,
                   int64_t G, int nc, int iters, uint64_t seed, int lv, float *C,
                   int32_t *labels, cudaStream_t s) {
    std::vector<int64_t> count((size_t)G, 0);
    for (int32_t v : group_of) count[(size_t)v] += 1;
    int64_t max_group = 0;
    for (int64_t c : count) {
        MASK_REQUIRE(c >= nc, "a group holds fewer items than nCentroids");
        max_group = std::max(max_group, c);
    }
    const size_t smem = group_kmeans_smem(max_group, dp, nc);
    MASK_REQUIRE(smem <= 200 * 1024, "group too large for shared memory (items x dimension)");
    // the groups' seeding draws (R17) and first picks (floor(u_0 m_g))
    std::vector<unsigned long long> a((size_t)G * nc);
    std::vector<int32_t> first((size_t)G);
    for (int64_t g = 0; g < G; ++g) {
        SplitMix64 rng{group_state(seed, lv, g)};
        for (int t = 0; t < nc; ++t) a[(size_t)(g * nc + t)] = rng.next() >> 11;
        int64_t f = (int64_t)std::floor((double)a[(size_t)(g * nc)] * 0x1.0p-53 * (double)count[(size_t)g]);
        if (f > count[(size_t)g] - 1) f = count[(size_t)g] - 1;
        first[(size_t)g] = (int32_t)f;
    }
    Scratch<int32_t> gof((size_t)m, s), gperm((size_t)m, s), dfirst((size_t)G, s);
    Scratch<int64_t> goff((size_t)G + 1, s);
    Scratch<unsigned long long> da((size_t)G * nc, s);
    MASK_CUDA(cudaMemcpyAsync(gof.get(), group_of.data(), sizeof(int32_t) * m,
                              cudaMemcpyHostToDevice, s));
    MASK_CUDA(cudaMemcpyAsync(da.get(), a.data(), sizeof(unsigned long long) * G * nc,
                              cudaMemcpyHostToDevice, s));
    MASK_CUDA(cudaMemcpyAsync(dfirst.get(), first.data(), sizeof(int32_t) * G,
                              cudaMemcpyHostToDevice, s));
    label_sort(gof.get(), m, (int)G, goff.get(), gperm.get(), s);
    MASK_CUDA(cudaFuncSetAttribute(group_kmeans_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        ProfRegion pr("group_kmeans", s, 0.0);
        group_kmeans_kernel<<<(unsigned)G, kGkThreads, smem, s>>>(
            X, dp, gperm.get(), goff.get(), da.get(), dfirst.get(), nc, iters, C, labels);
        MASK_LAUNCHED("group_kmeans");
    }
    MASK_CUDA(cudaStreamSynchronize(s));  // host vectors above are released on return
}

}  // namespace mask
