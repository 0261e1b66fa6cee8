// profile.cu -- launch counter and per-region device timing (CUDA events on
// the launching stream).  The paper reports only wall-clock build ("tree")
// and search times (§4.2); these counters split the device time by kernel so
// each can be set against its roofline.
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace mask {
namespace {

std::atomic<long long> g_launches{0};
std::atomic<long long> g_allocs{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;

struct Rec {
    cudaEvent_t a, b;
    double work;
};
struct Total {
    long long launches = 0;
    double ms = 0.0, work = 0.0;
};
std::map<std::string, std::vector<Rec>> g_pending;
std::map<std::string, Total> g_totals;

void drain_locked(const std::string &name) {
    auto it = g_pending.find(name);
    if (it == g_pending.end()) return;
    Total &t = g_totals[name];
    for (auto &r : it->second) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            t.launches += 1;
            t.ms += ms;
            t.work += r.work;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    cudaGetLastError();
    g_pending.erase(it);
}

}  // namespace

bool profiling_enabled() { return g_enabled.load(std::memory_order_relaxed); }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void count_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
}  // namespace

void *scratch_alloc(size_t bytes, cudaStream_t s) {
    void *p = nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cudaGetLastError();
    if (cs != cudaStreamCaptureStatusNone) {
        MASK_CUDA(cudaMallocAsync(&p, bytes, s));
        return p;
    }
    int dev = 0;
    MASK_CUDA(cudaGetDevice(&dev));
    MASK_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (g_pools[dev] == nullptr) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t created = nullptr;
            MASK_CUDA(cudaMemPoolCreate(&created, &props));
            unsigned long long keep = kScratchKeepBytes;
            MASK_CUDA(cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep));
            g_pools[dev] = created;
        }
        pool = g_pools[dev];
    }
    MASK_CUDA(cudaMallocFromPoolAsync(&p, bytes, pool, s));
    return p;
}

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

ProfRegion::ProfRegion(const char *name, cudaStream_t s, double work)
    : name_(name), s_(s), work_(work) {
    if (!g_enabled.load(std::memory_order_relaxed)) return;
    // regions inside a stream capture (a graph being built) are not timed
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    if (cudaEventCreate(&a_) != cudaSuccess) return;
    if (cudaEventCreate(&b_) != cudaSuccess) {
        cudaEventDestroy(a_);
        return;
    }
    cudaEventRecord(a_, s_);
    active_ = true;
}

ProfRegion::~ProfRegion() {
    if (!active_) return;
    cudaEventRecord(b_, s_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending[name_].push_back({a_, b_, work_});
}

}  // namespace mask

extern "C" {

void mask_profile_enable(int32_t on) { mask::g_enabled.store(on != 0); }

void mask_profile_reset(void) {
    std::lock_guard<std::mutex> lk(mask::g_mu);
    std::vector<std::string> names;
    for (auto &kv : mask::g_pending) names.push_back(kv.first);
    for (auto &n : names) mask::drain_locked(n);
    mask::g_totals.clear();
    mask::scan_bytes_reset();
    mask::cm_bytes_reset();
    mask::csr_scan_bytes_reset();
}

int32_t mask_profile_read(const char *name, int64_t *launches, double *total_ms, double *work) {
    if (name == nullptr) return 0;
    std::lock_guard<std::mutex> lk(mask::g_mu);
    mask::drain_locked(name);
    auto it = mask::g_totals.find(name);
    if (it == mask::g_totals.end()) return 0;
    if (launches) *launches = it->second.launches;
    if (total_ms) *total_ms = it->second.ms;
    double w = it->second.work;
    if (it->first == "scan_topk_level") w = mask::scan_bytes(0);
    if (it->first == "scan_topk_leaf") w = mask::scan_bytes(1);
    if (it->first == "scan_leaf_cm") w = mask::cm_bytes();
    if (it->first == "csr_scan_level") w = mask::csr_scan_bytes(0);
    if (it->first == "csr_scan_leaf") w = mask::csr_scan_bytes(1);
    if (work) *work = w;
    return 1;
}

int64_t mask_launch_count(void) { return mask::g_launches.load(); }

int64_t mask_test_alloc_count(void) { return mask::g_allocs.load(); }

}  // extern "C"
