// server.cu -- continuous-batching k-NN service over a resident dense index
// (the query of §3.3, Algorithm 2, answered for a stream of requests).
//
// Callers submit requests (a batch of queries, k, per-level probes,
// precision) from any thread and poll or wait on a ticket.  One worker
// thread runs the loop:
//
//   retire  -- batches whose completion event fired: copy each request's rows
//              out (first k of the batch's K columns), finish requests,
//              release their memory;
//   admit   -- while a slot (stream) is free: take the oldest pending request
//              and every pending request with the same batch key (equal
//              probes and precision; low precision also equal k), up to
//              max_batch queries and as many as the memory budget left
//              allows (a request may be split across batches); stage the
//              queries, replay the batch shape's captured CUDA graph on the
//              slot's stream, queue the copy back and an event.
//
// So requests that arrive while others are on the GPU join the next batch as
// slots and memory free up, and batches on different slots overlap on the
// device.  A query's result depends only on the query (every scan orders
// candidates by the total order (distance, id), and the K-th list of an FP32
// batch whose K exceeds a request's k starts with that request's k nearest),
// so a request gets the same answer alone and in any mix.
//
// Graphs: one per (batch key, batch size bucket, K, leaf scan), captured on
// first use with the batch padded to the bucket (copies of the last query).
// Autotuning: for an FP32 shape where both leaf scans apply, the first batch
// of that shape times both captured graphs and keeps the faster (their
// results are bit-identical).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "index.cuh"

namespace mask {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    std::vector<float> q;  // [nq x d], the caller's queries (copied at submit)
    int64_t nq = 0;
    int k = 0;
    std::vector<int> probes;
    mask_precision prec = MASK_FP32;
    int64_t *ids_out = nullptr;
    float *dists_out = nullptr;
    int64_t left = 0;       // queries not yet retired
    bool failed = false;
    mask_status status = MASK_PENDING;
    std::string err;
    Clock::time_point t_submit, t_done;
};

struct Piece {
    std::shared_ptr<Request> r;
    int64_t q0, q1;
};

// Requests with equal keys share a launch.
struct Key {
    std::vector<int> probes;
    int prec = 0;
    int kkey = 0;  // 0 for FP32 (K = max k of the batch), k for low precision
    bool operator<(const Key &o) const {
        return std::tie(probes, prec, kkey) < std::tie(o.probes, o.prec, o.kkey);
    }
    bool operator==(const Key &o) const {
        return probes == o.probes && prec == o.prec && kkey == o.kkey;
    }
};

// The leaf-scan configurations the autotuner times for an FP32 shape: the
// query-major scan, and the cluster-major scan at each (queries per work
// item, blocks per SM) pair (0 queries: the kernel's widest item, 32 on the
// tensor-core scan for K <= 16, else 16; 0 blocks per SM: as many as fit;
// the tensor-core scan runs one block per SM).  All give bit-identical
// results.
struct LeafConfig {
    LeafMode mode;
    CmTile tile;
};
const LeafConfig kLeafConfigs[] = {
    {LeafMode::Query, CmTile{0, 0}},    {LeafMode::Cluster, CmTile{0, 0}},
    {LeafMode::Cluster, CmTile{16, 1}}, {LeafMode::Cluster, CmTile{8, 0}},
    {LeafMode::Cluster, CmTile{8, 1}},
};
constexpr int kNumLeafConfigs = (int)(sizeof(kLeafConfigs) / sizeof(kLeafConfigs[0]));

struct Shape {
    Key key;
    int64_t bucket = 0;
    int K = 0;
    int mode = 0;  // index into kLeafConfigs
    bool operator<(const Shape &o) const {
        return std::tie(key, bucket, K, mode) < std::tie(o.key, o.bucket, o.K, o.mode);
    }
};

struct Instance {
    Shape shape;
    DevArray<float> Qp;
    DevArray<int64_t> ids;
    DevArray<float> dists;
    float *hQ = nullptr;
    int64_t *hids = nullptr;
    float *hd = nullptr;
    int *herr = nullptr;      // pinned copy of the tensor-core scan's error word
    bool check_tc = false;    // the graph holds the tensor-core leaf scan
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    bool busy = false;
    Instance() = default;
    Instance(const Instance &) = delete;
    ~Instance() {
        if (exec) cudaGraphExecDestroy(exec);
        if (hQ) cudaFreeHost(hQ);
        if (hids) cudaFreeHost(hids);
        if (hd) cudaFreeHost(hd);
        if (herr) cudaFreeHost(herr);
    }
};

struct Batch {
    Instance *inst = nullptr;
    std::vector<Piece> pieces;
    int64_t nq = 0;
    size_t bytes = 0;
};

int64_t next_pow2_64(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace
}  // namespace mask

using namespace mask;

struct mask_server {
    const mask_index *idx = nullptr;
    int device = 0;
    int64_t budget = 0;
    int max_slots = 0;
    int64_t max_batch = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<Batch> slots;  // slots[i].inst != null while slot i is busy
    cudaStream_t cap_stream = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Piece> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread worker;

    // worker-owned
    std::multimap<Shape, std::unique_ptr<Instance>> cache;
    std::map<std::tuple<Key, int64_t, int>, int> tuned;  // (key, bucket, K) -> leaf config
    size_t inflight_bytes = 0;

    // statistics (under mu)
    std::vector<double> lat_ms;
    int64_t req_done = 0, req_failed = 0, q_done = 0, batches = 0, batch_queries = 0;
    int64_t graph_launches = 0, captures = 0, autotuned = 0;
    size_t peak_inflight = 0;
    bool any = false;
    Clock::time_point t_first, t_last;
};

namespace mask {
namespace {

Key key_of(const Request &r) {
    Key k;
    k.probes = r.probes;
    k.prec = (int)r.prec;
    k.kkey = r.prec == MASK_FP32 ? 0 : r.k;
    return k;
}

// Device bytes a batch of B queries holds while it runs: the graph's
// input/output buffers and the scratch its kernels allocate.
size_t batch_bytes(const mask_index &idx, const Key &key, int64_t B, int K) {
    const size_t dp = (size_t)idx.dp;
    const size_t p0 = (size_t)key.probes[0];
    size_t sp = 0;
    for (int p : key.probes) sp += (size_t)p;
    size_t per = dp * 4 + (size_t)K * 12 + sp * 4;
    if (key.prec == MASK_FP32) {
        // cluster-major pairs, and per-pair lists (mma.sync scan) or the
        // candidate list (tensor-core scan), whichever is larger
        size_t lists = p0 * (size_t)K * 8;
        if (cm_tc_supported(idx.dp, K))
            lists = std::max(lists, (size_t)cm_tc_cand_cap(B) * 4 + 4);
        per += p0 * 12 + lists;
    } else {
        const size_t dpl = (size_t)lp_padded_dim(idx.dp);
        const size_t Kp = (size_t)lp_shortlist(K);
        const size_t Kpair = std::min(Kp, (size_t)std::max(K, 4));
        per += dpl * 2 + 8 + p0 * (12 + Kpair * 8) + Kp * 4;
    }
    const size_t fixed = (size_t)(idx.lv[0].k + 2) * 32 + (256u << 10);
    return fixed + per * (size_t)B;
}

int fp32_kbucket(int k) { return (int)next_pow2_64(k); }

int64_t bucket_of(int64_t nq) { return std::max<int64_t>(8, next_pow2_64(nq)); }

void finish_locked(mask_server *S, Request &r) {
    r.t_done = Clock::now();
    r.status = r.failed ? (r.status == MASK_PENDING ? MASK_ECUDA : r.status) : MASK_OK;
    if (r.failed) {
        S->req_failed += 1;
    } else {
        S->req_done += 1;
        S->q_done += r.nq;
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
    }
    S->t_last = r.t_done;
    S->cv_done.notify_all();
}

// Marks a request failed and drops its pending pieces (in-flight pieces
// still retire; the request is final when none is left).
void fail_locked(mask_server *S, const std::shared_ptr<Request> &r, mask_status st,
                 const std::string &msg) {
    if (!r->failed) {
        r->failed = true;
        r->status = st;
        r->err = msg;
    }
    for (auto it = S->pending.begin(); it != S->pending.end();) {
        if (it->r == r) {
            r->left -= it->q1 - it->q0;
            it = S->pending.erase(it);
        } else {
            ++it;
        }
    }
    if (r->left == 0) finish_locked(S, *r);
}

// Captures the graph of one shape into a new instance.
std::unique_ptr<Instance> make_instance(mask_server *S, const Shape &sh) {
    const mask_index &idx = *S->idx;
    auto inst = std::make_unique<Instance>();
    inst->shape = sh;
    const size_t B = (size_t)sh.bucket, dp = (size_t)idx.dp, K = (size_t)sh.K;
    inst->Qp.alloc(B * dp);
    inst->ids.alloc(B * K);
    inst->dists.alloc(B * K);
    count_alloc();
    MASK_CUDA(cudaMallocHost((void **)&inst->hQ, B * dp * sizeof(float)));
    count_alloc();
    MASK_CUDA(cudaMallocHost((void **)&inst->hids, B * K * sizeof(int64_t)));
    count_alloc();
    MASK_CUDA(cudaMallocHost((void **)&inst->hd, B * K * sizeof(float)));
    count_alloc();
    MASK_CUDA(cudaMallocHost((void **)&inst->herr, sizeof(int)));
    *inst->herr = 0;
    std::memset(inst->hQ, 0, B * dp * sizeof(float));
    MASK_CUDA(cudaMemsetAsync(inst->Qp.get(), 0, B * dp * sizeof(float), S->cap_stream));
    if (sh.key.prec != MASK_FP32) ensure_lowp(idx, sh.key.prec == MASK_FP8E4M3, S->cap_stream);
    MASK_CUDA(cudaStreamSynchronize(S->cap_stream));
    cudaGraph_t g = nullptr;
    cm_tc_take_launched();
    MASK_CUDA(cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
        const LeafConfig &lc = kLeafConfigs[sh.mode];
        query_dense(idx, inst->Qp.get(), sh.bucket, sh.K, sh.key.probes,
                    (mask_precision)sh.key.prec, lc.mode, inst->ids.get(), inst->dists.get(),
                    S->cap_stream, lc.tile);
    } catch (...) {
        cudaStreamEndCapture(S->cap_stream, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    MASK_CUDA(cudaStreamEndCapture(S->cap_stream, &g));
    inst->check_tc = cm_tc_take_launched();
    cudaError_t e = cudaGraphInstantiate(&inst->exec, g, 0);
    size_t nn = 0;
    if (e == cudaSuccess) e = cudaGraphGetNodes(g, nullptr, &nn);
    if (e == cudaSuccess && nn) {
        std::vector<cudaGraphNode_t> nodes(nn);
        e = cudaGraphGetNodes(g, nodes.data(), &nn);
        for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                inst->kernels += 1;
        }
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) fail(MASK_ECUDA, std::string("query graph: ") + cudaGetErrorString(e));
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->captures += 1;
    }
    return inst;
}

Instance *get_instance(mask_server *S, const Shape &sh) {
    auto range = S->cache.equal_range(sh);
    for (auto it = range.first; it != range.second; ++it)
        if (!it->second->busy) return it->second.get();
    auto inst = make_instance(S, sh);
    Instance *p = inst.get();
    S->cache.emplace(sh, std::move(inst));
    return p;
}

// Queries of the batch into the instance's pinned buffer (padding rows repeat
// the last query; padding columns stay zero).
void stage(mask_server *S, Batch &b) {
    const int d = S->idx->d, dp = S->idx->dp;
    float *h = b.inst->hQ;
    int64_t row = 0;
    const float *last = nullptr;
    for (const Piece &p : b.pieces)
        for (int64_t q = p.q0; q < p.q1; ++q, ++row) {
            last = p.r->q.data() + (size_t)q * d;
            std::memcpy(h + (size_t)row * dp, last, sizeof(float) * d);
        }
    for (; row < b.inst->shape.bucket; ++row) std::memcpy(h + (size_t)row * dp, last, sizeof(float) * d);
}

void launch(mask_server *S, int slot, Batch &b) {
    Instance *in = b.inst;
    cudaStream_t st = S->streams[(size_t)slot];
    const size_t B = (size_t)in->shape.bucket, K = (size_t)in->shape.K, dp = (size_t)S->idx->dp;
    MASK_CUDA(cudaMemcpyAsync(in->Qp.get(), in->hQ, B * dp * sizeof(float), cudaMemcpyHostToDevice, st));
    MASK_CUDA(cudaGraphLaunch(in->exec, st));
    count_launches(in->kernels);
    MASK_CUDA(cudaMemcpyAsync(in->hids, in->ids.get(), (size_t)b.nq * K * sizeof(int64_t),
                              cudaMemcpyDeviceToHost, st));
    MASK_CUDA(cudaMemcpyAsync(in->hd, in->dists.get(), (size_t)b.nq * K * sizeof(float),
                              cudaMemcpyDeviceToHost, st));
    if (in->check_tc)
        MASK_CUDA(cudaMemcpyAsync(in->herr, cm_tc_error_word(), sizeof(int),
                                  cudaMemcpyDeviceToHost, st));
    MASK_CUDA(cudaEventRecord(S->events[(size_t)slot], st));
}

// Leaf scan for an FP32 shape: the fastest of the configurations' captured
// graphs, each timed once on the batch at hand; other shapes take the
// query-major scan (configuration 0).
int tune_mode(mask_server *S, int slot, Batch &b, const Key &key, int64_t bucket, int K) {
    if (key.prec != MASK_FP32 || !cm_leaf_supported(S->idx->dp, K)) return 0;
    const auto tk = std::make_tuple(key, bucket, K);
    auto it = S->tuned.find(tk);
    if (it != S->tuned.end()) return it->second;
    cudaStream_t st = S->streams[(size_t)slot];
    float best_ms = 0.f;
    int best = 0;
    // the events are released on every exit, including a failed CUDA call
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    MASK_CUDA(cudaEventCreate(&ev.a));
    MASK_CUDA(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    for (int mode = 0; mode < kNumLeafConfigs; ++mode) {
        Shape sh{key, bucket, K, mode};
        b.inst = get_instance(S, sh);
        stage(S, b);
        MASK_CUDA(cudaMemcpyAsync(b.inst->Qp.get(), b.inst->hQ,
                                  (size_t)bucket * S->idx->dp * sizeof(float),
                                  cudaMemcpyHostToDevice, st));
        MASK_CUDA(cudaGraphLaunch(b.inst->exec, st));  // warm
        MASK_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < 3; ++r) MASK_CUDA(cudaGraphLaunch(b.inst->exec, st));
        MASK_CUDA(cudaEventRecord(e1, st));
        MASK_CUDA(cudaEventSynchronize(e1));
        count_launches(4 * b.inst->kernels);
        float ms = 0.f;
        MASK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (mode == 0 || ms < best_ms) {
            best_ms = ms;
            best = mode;
        }
    }
    S->tuned[tk] = best;
    // the losing configurations' graphs and buffers are not needed again
    for (int mode = 0; mode < kNumLeafConfigs; ++mode)
        if (mode != best) S->cache.erase(Shape{key, bucket, K, mode});
    b.inst = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    S->autotuned += 1;
    return best;
}

// Takes the next batch off the queue (under the lock); false if nothing fits.
bool form_batch(mask_server *S, Batch &b, Key &key, int &K, int64_t &bucket) {
    if (S->pending.empty()) return false;
    const Piece &head = S->pending.front();
    key = key_of(*head.r);
    int kmax = 0;
    for (const Piece &p : S->pending)
        if (key_of(*p.r) == key) kmax = std::max(kmax, p.r->k);
    K = key.prec == MASK_FP32 ? std::min(1024, fp32_kbucket(kmax)) : kmax;
    // the largest bucket the memory left admits
    const size_t left = S->budget > (int64_t)S->inflight_bytes ? (size_t)S->budget - S->inflight_bytes : 0;
    int64_t cap = S->max_batch;
    while (cap > 8 && batch_bytes(*S->idx, key, cap, K) > left) cap >>= 1;
    if (batch_bytes(*S->idx, key, cap, K) > left) {
        if (S->inflight_bytes > 0) return false;  // wait for memory to free up
        // nothing runs and even the smallest batch does not fit: fail the head request
        auto r = head.r;
        fail_locked(S, r, MASK_ENOMEM, "a batch of this request exceeds the server's memory budget");
        return false;
    }
    b.pieces.clear();
    b.nq = 0;
    for (auto it = S->pending.begin(); it != S->pending.end() && b.nq < cap;) {
        if (!(key_of(*it->r) == key)) {
            ++it;
            continue;
        }
        const int64_t take = std::min(it->q1 - it->q0, cap - b.nq);
        b.pieces.push_back({it->r, it->q0, it->q0 + take});
        b.nq += take;
        if (take < it->q1 - it->q0) {
            it->q0 += take;
            ++it;
        } else {
            it = S->pending.erase(it);
        }
    }
    bucket = bucket_of(b.nq);
    b.bytes = batch_bytes(*S->idx, key, bucket, K);
    return true;
}

// Copies finished batches' rows out and completes requests.
bool retire(mask_server *S) {
    bool progressed = false;
    for (size_t s = 0; s < S->slots.size(); ++s) {
        Batch &b = S->slots[s];
        if (b.inst == nullptr) continue;
        const cudaError_t e = cudaEventQuery(S->events[s]);
        if (e == cudaErrorNotReady) continue;
        const size_t K = (size_t)b.inst->shape.K;
        // a leaf scan whose bounded wait ran out fails the batch's requests
        const bool stalled = e == cudaSuccess && b.inst->check_tc && *b.inst->herr != 0;
        if (stalled) {
            *b.inst->herr = 0;
            MASK_CUDA(cudaMemsetAsync(cm_tc_error_word(), 0, sizeof(int), S->streams[s]));
        }
        if (e == cudaSuccess && !stalled) {
            int64_t row = 0;
            for (const Piece &p : b.pieces) {
                Request &r = *p.r;
                if (!r.failed)
                    for (int64_t q = p.q0; q < p.q1; ++q) {
                        const size_t src = (size_t)(row + q - p.q0) * K;
                        std::memcpy(r.ids_out + (size_t)q * r.k, b.inst->hids + src,
                                    sizeof(int64_t) * r.k);
                        if (r.dists_out)
                            std::memcpy(r.dists_out + (size_t)q * r.k, b.inst->hd + src,
                                        sizeof(float) * r.k);
                    }
                row += p.q1 - p.q0;
            }
        } else {
            cudaGetLastError();
        }
        std::lock_guard<std::mutex> lk(S->mu);
        for (const Piece &p : b.pieces) {
            if (e != cudaSuccess && !p.r->failed) {
                p.r->failed = true;
                p.r->status = MASK_ECUDA;
                p.r->err = std::string("query batch: ") + cudaGetErrorString(e);
            } else if (stalled && !p.r->failed) {
                p.r->failed = true;
                p.r->status = MASK_ETIMEOUT;
                p.r->err = "query batch: a bounded pipeline wait of the leaf scan ran out";
            }
            p.r->left -= p.q1 - p.q0;
            if (p.r->left == 0) finish_locked(S, *p.r);
        }
        S->inflight_bytes -= b.bytes;
        b.inst->busy = false;
        b.inst = nullptr;
        b.pieces.clear();
        progressed = true;
    }
    return progressed;
}

void worker_main(mask_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool progressed = retire(S);
        int free_slot = -1;
        for (size_t s = 0; s < S->slots.size(); ++s)
            if (S->slots[s].inst == nullptr) { free_slot = (int)s; break; }
        Batch b;
        Key key;
        int K = 0;
        int64_t bucket = 0;
        bool got = false, inflight = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            inflight = S->inflight_bytes > 0;
            for (const Batch &x : S->slots) inflight = inflight || x.inst != nullptr;
            if (free_slot >= 0) got = form_batch(S, b, key, K, bucket);
            if (!got && !progressed) {
                if (S->stopping && S->pending.empty() && !inflight) return;
                if (!inflight) {
                    S->cv_work.wait(lk, [&] { return S->stopping || !S->pending.empty(); });
                    continue;
                }
            }
            if (got) {
                S->inflight_bytes += b.bytes;
                S->peak_inflight = std::max(S->peak_inflight, S->inflight_bytes);
                S->batches += 1;
                S->batch_queries += b.nq;
            }
        }
        if (got) {
            try {
                const int mode = tune_mode(S, free_slot, b, key, bucket, K);
                b.inst = get_instance(S, Shape{key, bucket, K, mode});
                b.inst->busy = true;
                stage(S, b);
                launch(S, free_slot, b);
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->graph_launches += 1;
                }
                S->slots[(size_t)free_slot] = std::move(b);
            } catch (const std::exception &ex) {
                if (b.inst) b.inst->busy = false;
                std::lock_guard<std::mutex> lk(S->mu);
                S->inflight_bytes -= b.bytes;
                const mask_status st = dynamic_cast<const Error *>(&ex)
                                           ? static_cast<const Error &>(ex).status
                                           : MASK_ECUDA;
                for (const Piece &p : b.pieces) {
                    if (!p.r->failed) {
                        p.r->failed = true;
                        p.r->status = st;
                        p.r->err = ex.what();
                    }
                    p.r->left -= p.q1 - p.q0;
                    if (p.r->left == 0) finish_locked(S, *p.r);
                }
            }
            continue;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace mask

extern "C" {

mask_status mask_server_open(const mask_index *index, int64_t mem_budget, int32_t max_slots,
                             int32_t max_batch, mask_server **out) {
    mask_server *S = nullptr;
    const mask_status st = [&]() -> mask_status {
        try {
            MASK_REQUIRE(index && out, "NULL argument");
            MASK_REQUIRE(!index->sparse, "the server answers dense queries (index built by mask_build)");
            MASK_REQUIRE(max_slots >= 1 && max_slots <= 64, "max_slots must be in [1, 64]");
            MASK_REQUIRE(max_batch >= 8 && max_batch <= (1 << 20), "max_batch must be in [8, 2^20]");
            MASK_REQUIRE(mem_budget > 0, "mem_budget must be > 0");
            int dev = 0;
            MASK_CUDA(cudaGetDevice(&dev));
            MASK_REQUIRE(dev == index->device, "index lives on another device");
            auto srv = std::make_unique<mask_server>();
            srv->idx = index;
            srv->device = dev;
            srv->budget = mem_budget;
            srv->max_slots = max_slots;
            srv->max_batch = next_pow2_64(max_batch);
            srv->streams.resize((size_t)max_slots);
            srv->events.resize((size_t)max_slots);
            srv->slots.resize((size_t)max_slots);
            for (int i = 0; i < max_slots; ++i) {
                MASK_CUDA(cudaStreamCreateWithFlags(&srv->streams[(size_t)i], cudaStreamNonBlocking));
                MASK_CUDA(cudaEventCreateWithFlags(&srv->events[(size_t)i], cudaEventDisableTiming));
            }
            MASK_CUDA(cudaStreamCreateWithFlags(&srv->cap_stream, cudaStreamNonBlocking));
            S = srv.release();
            S->worker = std::thread(worker_main, S);
            *out = S;
            return MASK_OK;
        } catch (const Error &e) {
            set_last_error(e.what());
            return e.status;
        } catch (const std::exception &e) {
            set_last_error(e.what());
            return MASK_ECUDA;
        }
    }();
    return st;
}

mask_status mask_server_submit(mask_server *S, const float *queries, int64_t nq, int32_t k,
                               const int32_t *probes, mask_precision precision, int64_t *ids_out,
                               float *dists_out, uint64_t *ticket_out) {
    try {
        MASK_REQUIRE(S && ticket_out, "NULL argument");
        const mask_index &idx = *S->idx;
        MASK_REQUIRE(nq >= 0, "nq must be >= 0");
        MASK_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
        MASK_REQUIRE(probes != nullptr, "probes is NULL");
        MASK_REQUIRE(precision == MASK_FP32 || precision == MASK_BF16 ||
                         precision == MASK_FP8E4M3, "unknown precision");
        if (precision != MASK_FP32 && !lp_supported(idx.dp, k))
            fail(MASK_EUNSUPPORTED, "BF16/FP8 modes keep a 4k shortlist: k <= 16 and d <= 256");
        MASK_REQUIRE(nq == 0 || (queries && ids_out), "NULL queries or ids_out");
        auto r = std::make_shared<Request>();
        r->probes.resize((size_t)idx.L);
        for (int l = 0; l < idx.L; ++l) {
            MASK_REQUIRE(probes[l] >= 1, "probes must be >= 1");
            r->probes[(size_t)l] = std::min<int>(probes[l], idx.lv[(size_t)l].k);
        }
        if (nq > 0) {
            cudaPointerAttributes a;
            const bool dev_ptr = cudaPointerGetAttributes(&a, queries) == cudaSuccess &&
                                 (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            MASK_REQUIRE(!dev_ptr, "the server takes host queries and host outputs");
            r->q.assign(queries, queries + (size_t)nq * idx.d);
        }
        r->nq = nq;
        r->k = k;
        r->prec = precision;
        r->ids_out = ids_out;
        r->dists_out = dists_out;
        r->left = nq;
        r->t_submit = Clock::now();
        std::lock_guard<std::mutex> lk(S->mu);
        r->ticket = S->next_ticket++;
        if (!S->any) {
            S->any = true;
            S->t_first = r->t_submit;
        }
        S->live[r->ticket] = r;
        if (nq == 0) {
            finish_locked(S, *r);
        } else {
            S->pending.push_back({r, 0, nq});
            S->cv_work.notify_one();
        }
        *ticket_out = r->ticket;
        return MASK_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return MASK_ECUDA;
    }
}

static mask_status take_result(mask_server *S, std::unique_lock<std::mutex> &lk, uint64_t ticket,
                               int32_t timeout_ms) {
    auto it = S->live.find(ticket);
    if (it == S->live.end()) {
        set_last_error("unknown ticket");
        return MASK_EINVAL;
    }
    auto r = it->second;
    if (timeout_ms != 0 && r->status == MASK_PENDING) {
        auto ready = [&] { return r->status != MASK_PENDING; };
        if (timeout_ms < 0) S->cv_done.wait(lk, ready);
        else S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    }
    if (r->status == MASK_PENDING) return MASK_PENDING;
    S->live.erase(ticket);
    if (r->status != MASK_OK) set_last_error(r->err);
    return r->status;
}

mask_status mask_server_poll(mask_server *S, uint64_t ticket) {
    if (!S) return MASK_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    return take_result(S, lk, ticket, 0);
}

mask_status mask_server_wait(mask_server *S, uint64_t ticket, int32_t timeout_ms) {
    if (!S) return MASK_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    return take_result(S, lk, ticket, timeout_ms);
}

mask_status mask_server_stats(mask_server *S, mask_server_info *out, int32_t reset) {
    if (!S || !out) return MASK_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->requests_done = S->req_done;
    out->requests_failed = S->req_failed;
    out->queries_done = S->q_done;
    out->batches = S->batches;
    out->graph_launches = S->graph_launches;
    out->graph_captures = S->captures;
    out->autotuned_shapes = S->autotuned;
    out->mean_batch_queries = S->batches ? (double)S->batch_queries / (double)S->batches : 0.0;
    out->peak_inflight_bytes = (int64_t)S->peak_inflight;
    out->mem_budget = S->budget;
    out->elapsed_s = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    if (!S->lat_ms.empty()) {
        std::vector<double> v = S->lat_ms;
        auto pct = [&](double f) {
            const size_t i = std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + (long)i, v.end());
            return v[i];
        };
        double sum = 0.0;
        for (double x : v) sum += x;
        out->latency_mean_ms = sum / (double)v.size();
        out->latency_p50_ms = pct(0.50);
        out->latency_p99_ms = pct(0.99);
        out->latency_max_ms = *std::max_element(v.begin(), v.end());
    }
    if (reset) {
        S->lat_ms.clear();
        S->req_done = S->req_failed = S->q_done = S->batches = S->batch_queries = 0;
        S->graph_launches = 0;
        S->peak_inflight = S->inflight_bytes;
        S->any = false;
    }
    return MASK_OK;
}

void mask_server_close(mask_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto s : S->streams) cudaStreamSynchronize(s);
    S->cache.clear();
    for (auto s : S->streams) cudaStreamDestroy(s);
    for (auto e : S->events) cudaEventDestroy(e);
    if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
    cudaSetDevice(prev);
    delete S;
}

}  // extern "C"
