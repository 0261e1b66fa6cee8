// index.cuh -- the index object behind the opaque mask_index handle, and the
// internal query entry the C ABI and the serving loop share (not part of the
// C ABI; see include/mask.h for that).
#pragma once

#include <mutex>
#include <vector>

#include "common.cuh"

struct mask_index {
    int device = 0;
    int64_t n = 0;
    int d = 0, dp = 0, L = 0, iters = 0;
    bool sparse = false;
    mask::DevArray<float> Xs;        // [n x dp] points, cluster-major (level-0 parent-major)
    mask::DevArray<int32_t> xids;    // [n] original id of each row of Xs (or of xrp)
    mask::DevArray<float> xn;        // [n] ||row of Xs||^2 (FP32), for the leaf-scan filter
    // CSR index: the points' rows cluster-major (row i is point xids[i])
    mask::DevArray<int64_t> xrp;     // [n+1]
    mask::DevArray<int32_t> xcol;    // [nnz]
    mask::DevArray<float> xval;      // [nnz]
    struct Level {
        int k = 0;
        mask::DevArray<float> C;       // [k x dp] centroids in k-means cluster order
        mask::DevArray<float> Cs;      // [k x dp] centroids parent-major (top: cluster order)
        mask::DevArray<int32_t> ids;   // [k] cluster id of each row of Cs
        mask::DevArray<int64_t> off;   // [k+1] children of centroid j: rows off[j]..off[j+1]
                                       //       of the level below's parent-major array
        mask::DevArray<int32_t> labels;// [n_below] centroid of every item one level below
        mask::DevArray<float> cns;     // [k] ||row of Cs||^2 (CSR index: level-scan norms)
        std::vector<int64_t> chosen;   // k-means++ picks (indices into the level's inputs)
        std::vector<double> objective; // k-means objective after each assignment
    };
    std::vector<Level> lv;
    // quantised copies of Xs for the BF16 / FP8 query modes, made on first use
    mutable std::mutex lp_mu;
    mutable mask::DevArray<unsigned char> Xlp[2];  // [0] BF16, [1] FP8 e4m3
    mutable mask::DevArray<float> xn_lp[2], xscale_fp8;
};

namespace mask {

// Leaf-scan variant of a dense FP32 query: chosen by the batch shape (Auto),
// or one of the two (their results are bit-identical).
enum class LeafMode { Auto = 0, Query = 1, Cluster = 2 };

// Makes the BF16 (fp8 = false) or FP8 copy of the points if it is missing
// (allocates; not for use under stream capture).
void ensure_lowp(const mask_index &idx, bool fp8, cudaStream_t s);

// The descent of nq padded dense queries (device [nq x dp]) through a dense
// index: per-level probes p (finest first, already clamped to k_l), results
// into device ids [nq x k] / dists [nq x k].  Stream-ordered, no host
// synchronisation (capturable once ensure_lowp has run for lowp modes).
void query_dense(const mask_index &idx, const float *Qp, int64_t nq, int k,
                 const std::vector<int> &p, mask_precision prec, LeafMode mode, int64_t *ids,
                 float *dists, cudaStream_t s,
                 CmTile tile = CmTile{});

}  // namespace mask
