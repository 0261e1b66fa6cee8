/*
 * mask_oracle.c -- plain, slow FP64 CPU oracle for the MASK hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it follows (Ortega et al., "Unconventional application of k-means for
 * distributed approximate similarity search"):
 *   - k-means: k centroids minimising the sum of squared distances of the
 *     points to their closest centroid (§2.4), computed by Lloyd iterations.
 *   - k-means++ seeding, which spreads the initial centroids (§3.2, citing
 *     Arthur & Vassilvitskii 2007: first centre uniform, then each next centre
 *     drawn with probability proportional to D^2, the squared distance to the
 *     nearest centre chosen so far).
 *   - multilevel index construction, bottom-up: the centroids of one level are
 *     the data of the next (§3.1, Algorithm 1), here with one group per level
 *     and a caller-given number of centroids per level.
 *   - k-NN search, top-down (§3.3, Algorithm 2): distances from the query to a
 *     level's candidate centroids, keep the nearest, descend into their
 *     children, and rank the points of the reached leaf clusters.  Generalised
 *     from one kept centroid per level to p_l kept centroids per level.
 *   - Euclidean metric (§4.2); squared distances are returned (same order).
 *
 * Readings where the paper is silent (each one is listed with its reason in
 * the design notes of the repository):
 *   R1 random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 *      pseudorandom number generators", OOPSLA 2014); the state of level lv
 *      (0-based) is seed ^ (0x9E3779B97F4A7C15 * (lv + 1)); a uniform draw is
 *      (next() >> 11) * 2^-53.
 *   R2 k-means++: first centre x[floor(u*n)]; next centre = smallest i whose
 *      inclusive left-to-right prefix sum of D^2 exceeds u*S, S = sum D^2;
 *      if S == 0, the lowest-index point not yet chosen.  One draw per centre.
 *   R3 seeding subsample: when n*k > 2^32 and 8k < n, k-means++ runs on 8k
 *      points drawn by a partial Fisher-Yates shuffle (draws taken from the
 *      same level stream, before the k-means++ draws).
 *   R4 Lloyd: fixed iteration count; assignment ties go to the smallest
 *      centroid index; the mean is summed in ascending point index; an empty
 *      cluster keeps its previous centroid; one final assignment after the
 *      last update (iters updates, iters+1 assignments).
 *   R5 descent: at each level the kept set is the global p_l smallest of the
 *      union of the children of the previous level's kept set, ordered by
 *      (distance, id); the result is the k smallest (distance, point id),
 *      padded with (-1, +inf).
 *
 * Every per-point and per-query result is computed by one thread in a fixed
 * order, so results do not depend on the OpenMP thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MO_OK 0
#define MO_EINVAL (-1)
#define MO_ENOMEM (-2)

/* ---------------------------------------------------------------- threads */

void mo_set_threads(int32_t t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int32_t mo_max_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* -------------------------------------------------------- R1: SplitMix64 */

/* One SplitMix64 step: advance the state by the golden gamma, then mix. */
uint64_t mo_splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform double in [0, 1) from the top 53 bits. */
double mo_uniform(uint64_t *state) {
    return (double)(mo_splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

uint64_t mo_level_state(uint64_t seed, int32_t level) {
    return seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(level + 1));
}

/* ------------------------------------------------------------- distance */

/* Squared Euclidean distance sum_t (a_t - b_t)^2, t ascending. */
static double sqdist(const double *a, const double *b, int32_t d) {
    double s = 0.0;
    for (int32_t t = 0; t < d; ++t) {
        double e = a[t] - b[t];
        s += e * e;
    }
    return s;
}

/* out[j] = ||q - X[ids[j]]||^2 for j < m. */
void mo_sqdist_rows(const double *X, int32_t d, const int64_t *ids, int64_t m,
                    const double *q, double *out) {
    for (int64_t j = 0; j < m; ++j) out[j] = sqdist(q, X + ids[j] * (int64_t)d, d);
}

/* ------------------------------------------------------- R2: k-means++ */

/*
 * k-means++ over the n rows of X.  Writes the chosen row indices to chosen[k]
 * and the centres (copies of those rows) to C[k][d].  Consumes k draws.
 */
int32_t mo_kmeanspp(const double *X, int64_t n, int32_t d, int32_t k,
                    uint64_t *state, int64_t *chosen, double *C) {
    if (n < 1 || d < 1 || k < 1 || (int64_t)k > n) return MO_EINVAL;
    double *D2 = (double *)malloc(sizeof(double) * (size_t)n);
    unsigned char *taken = (unsigned char *)calloc((size_t)n, 1);
    if (!D2 || !taken) { free(D2); free(taken); return MO_ENOMEM; }

    double u0 = mo_uniform(state);
    int64_t first = (int64_t)floor(u0 * (double)n);
    if (first > n - 1) first = n - 1;
    chosen[0] = first;
    taken[first] = 1;
    memcpy(C, X + first * (int64_t)d, sizeof(double) * (size_t)d);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) D2[i] = sqdist(X + i * (int64_t)d, C, d);

    for (int32_t t = 1; t < k; ++t) {
        double u = mo_uniform(state);
        double S = 0.0;
        for (int64_t i = 0; i < n; ++i) S += D2[i];
        int64_t pick = -1;
        if (S > 0.0) {
            double target = u * S, acc = 0.0;
            int64_t last_pos = -1;
            for (int64_t i = 0; i < n; ++i) {
                if (D2[i] > 0.0) last_pos = i;
                acc += D2[i];
                if (acc > target) { pick = i; break; }
            }
            if (pick < 0) pick = last_pos; /* rounding left the target past the end */
        } else {
            for (int64_t i = 0; i < n; ++i)
                if (!taken[i]) { pick = i; break; }
        }
        chosen[t] = pick;
        taken[pick] = 1;
        double *ct = C + (int64_t)t * d;
        memcpy(ct, X + pick * (int64_t)d, sizeof(double) * (size_t)d);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double e = sqdist(X + i * (int64_t)d, ct, d);
            if (e < D2[i]) D2[i] = e;
        }
    }
    free(D2);
    free(taken);
    return MO_OK;
}

/* ------------------------------------------- R3: Fisher-Yates subsample */

/* First m entries of a partial Fisher-Yates shuffle of 0..n-1 (m draws). */
int32_t mo_subsample(int64_t n, int64_t m, uint64_t *state, int64_t *out) {
    if (m < 0 || m > n) return MO_EINVAL;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!idx) return MO_ENOMEM;
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    for (int64_t j = 0; j < m; ++j) {
        double u = mo_uniform(state);
        int64_t r = j + (int64_t)floor(u * (double)(n - j));
        if (r > n - 1) r = n - 1;
        int64_t tmp = idx[j];
        idx[j] = idx[r];
        idx[r] = tmp;
    }
    memcpy(out, idx, sizeof(int64_t) * (size_t)m);
    free(idx);
    return MO_OK;
}

/* Does seeding level with n inputs and k centres run on a subsample? */
int64_t mo_seed_sample_size(int64_t n, int32_t k) {
    if ((double)n * (double)k > 4294967296.0 && 8 * (int64_t)k < n) return 8 * (int64_t)k;
    return n;
}

/*
 * Seeding of one level: k-means++ on X, or on a subsample when R3 applies.
 * chosen[] receives indices into X.
 */
int32_t mo_seed_level(const double *X, int64_t n, int32_t d, int32_t k,
                      uint64_t seed, int32_t level, int64_t *chosen, double *C) {
    uint64_t state = mo_level_state(seed, level);
    int64_t m = mo_seed_sample_size(n, k);
    if (m == n) return mo_kmeanspp(X, n, d, k, &state, chosen, C);
    int64_t *sample = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    double *Xs = (double *)malloc(sizeof(double) * (size_t)m * (size_t)d);
    if (!sample || !Xs) { free(sample); free(Xs); return MO_ENOMEM; }
    int32_t rc = mo_subsample(n, m, &state, sample);
    if (rc == MO_OK) {
        for (int64_t j = 0; j < m; ++j)
            memcpy(Xs + j * (int64_t)d, X + sample[j] * (int64_t)d, sizeof(double) * (size_t)d);
        rc = mo_kmeanspp(Xs, m, d, k, &state, chosen, C);
        if (rc == MO_OK)
            for (int32_t t = 0; t < k; ++t) chosen[t] = sample[chosen[t]];
    }
    free(sample);
    free(Xs);
    return rc;
}

/* ------------------------------------------------------------- R4: Lloyd */

/*
 * Assignment half-step: labels[i] = argmin_j ||x_i - c_j||^2 (ties to the
 * smallest j); dist[i] = that minimum.
 */
void mo_assign(const double *X, int64_t n, int32_t d, const double *C, int32_t k,
               int32_t *labels, double *dist) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double *x = X + i * (int64_t)d;
        double best = INFINITY;
        int32_t bj = 0;
        for (int32_t j = 0; j < k; ++j) {
            double e = sqdist(x, C + (int64_t)j * d, d);
            if (e < best) { best = e; bj = j; }
        }
        labels[i] = bj;
        if (dist) dist[i] = best;
    }
}

/*
 * Update half-step: c_j = mean of the points labelled j, summed in ascending
 * point index; an empty cluster keeps its previous centroid.  counts[j]
 * receives the cluster sizes (may be NULL).
 */
int32_t mo_update(const double *X, int64_t n, int32_t d, const int32_t *labels,
                  int32_t k, double *C, int64_t *counts) {
    double *sum = (double *)calloc((size_t)k * (size_t)d, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    if (!sum || !cnt) { free(sum); free(cnt); return MO_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        int32_t j = labels[i];
        if (j < 0 || j >= k) { free(sum); free(cnt); return MO_EINVAL; }
        cnt[j] += 1;
        const double *x = X + i * (int64_t)d;
        double *s = sum + (int64_t)j * d;
        for (int32_t t = 0; t < d; ++t) s[t] += x[t];
    }
    for (int32_t j = 0; j < k; ++j) {
        if (cnt[j] == 0) continue;
        for (int32_t t = 0; t < d; ++t)
            C[(int64_t)j * d + t] = sum[(int64_t)j * d + t] / (double)cnt[j];
    }
    if (counts) memcpy(counts, cnt, sizeof(int64_t) * (size_t)k);
    free(sum);
    free(cnt);
    return MO_OK;
}

/* k-means objective J = sum_i ||x_i - c_{labels[i]}||^2 (ascending i). */
double mo_objective(const double *X, int64_t n, int32_t d, const double *C,
                    const int32_t *labels) {
    double J = 0.0;
    for (int64_t i = 0; i < n; ++i)
        J += sqdist(X + i * (int64_t)d, C + (int64_t)labels[i] * d, d);
    return J;
}

/*
 * Lloyd's algorithm from the centres in C (updated in place): iters
 * assignment+update rounds, then one final assignment into labels.
 * J_trace (may be NULL) receives 2*iters+1 objective values: after each
 * assignment and after each update, the last one after the final assignment.
 */
int32_t mo_lloyd(const double *X, int64_t n, int32_t d, int32_t k, int32_t iters,
                 double *C, int32_t *labels, double *J_trace) {
    double *dist = (double *)malloc(sizeof(double) * (size_t)n);
    if (!dist) return MO_ENOMEM;
    for (int32_t it = 0; it < iters; ++it) {
        mo_assign(X, n, d, C, k, labels, dist);
        if (J_trace) J_trace[2 * it] = mo_objective(X, n, d, C, labels);
        int32_t rc = mo_update(X, n, d, labels, k, C, NULL);
        if (rc != MO_OK) { free(dist); return rc; }
        if (J_trace) J_trace[2 * it + 1] = mo_objective(X, n, d, C, labels);
    }
    mo_assign(X, n, d, C, k, labels, dist);
    if (J_trace) J_trace[2 * iters] = mo_objective(X, n, d, C, labels);
    free(dist);
    return MO_OK;
}

/* ------------------------------------------------ multilevel build (A1) */

/*
 * Global form of Algorithm 1: level lv (0-based, finest first) clusters the
 * n_{lv} inputs (the points for lv = 0, else the centroids of level lv-1)
 * into k_per_level[lv] centroids.  C_levels[lv] (k_lv x d) and
 * labels_levels[lv] (n_{lv}) are caller-allocated.  chosen_levels[lv] (k_lv,
 * may be NULL) receives the seeding picks.
 */
int32_t mo_build(const double *X, int64_t n, int32_t d, const int32_t *k_per_level,
                 int32_t L, int32_t iters, uint64_t seed, double *const *C_levels,
                 int32_t *const *labels_levels, int64_t *const *chosen_levels) {
    if (L < 1 || iters < 0) return MO_EINVAL;
    const double *in = X;
    int64_t n_in = n;
    for (int32_t lv = 0; lv < L; ++lv) {
        int32_t k = k_per_level[lv];
        if (k < 1 || (int64_t)k > n_in) return MO_EINVAL;
        int64_t *chosen = chosen_levels && chosen_levels[lv]
                              ? chosen_levels[lv]
                              : (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        if (!chosen) return MO_ENOMEM;
        int32_t rc = mo_seed_level(in, n_in, d, k, seed, lv, chosen, C_levels[lv]);
        if (!(chosen_levels && chosen_levels[lv])) free(chosen);
        if (rc != MO_OK) return rc;
        rc = mo_lloyd(in, n_in, d, k, iters, C_levels[lv], labels_levels[lv], NULL);
        if (rc != MO_OK) return rc;
        in = C_levels[lv];
        n_in = k;
    }
    return MO_OK;
}

/* ------------------------------------------------- R5: top-down k-NN */

typedef struct {
    double d;
    int64_t id;
} mo_pair;

static int pair_cmp(const void *a, const void *b) {
    const mo_pair *x = (const mo_pair *)a, *y = (const mo_pair *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Members of each cluster as lists in ascending item index (counting sort). */
static int32_t member_lists(const int32_t *labels, int64_t n, int32_t k, int64_t **off_out,
                            int64_t **items_out) {
    int64_t *off = (int64_t *)calloc((size_t)k + 1, sizeof(int64_t));
    int64_t *items = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!off || !items || !fill) { free(off); free(items); free(fill); return MO_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) off[labels[i] + 1] += 1;
    for (int32_t j = 0; j < k; ++j) off[j + 1] += off[j];
    for (int32_t j = 0; j < k; ++j) fill[j] = off[j];
    for (int64_t i = 0; i < n; ++i) items[fill[labels[i]]++] = i;
    free(fill);
    *off_out = off;
    *items_out = items;
    return MO_OK;
}

/*
 * k-NN search down a multilevel index.  Level lv has C_levels[lv]
 * (k_per_level[lv] x d) and labels_levels[lv] (the level-lv centroid of each
 * item one level below: points for lv = 0).  probes[lv] = p at level lv.
 * Writes ids_out/dists_out [nq x k] ascending by (distance, id), padded with
 * (-1, +inf).  sel_clear (may be NULL) gets 1 for a query when no kept set
 * was decided by a near-tie: at every level with more candidates than p,
 * d_(p+1) - d_(p) > tie_rtol * d_(p).
 */
int32_t mo_query(const double *X, int64_t n, int32_t d, int32_t L, const int32_t *k_per_level,
                 const double *const *C_levels, const int32_t *const *labels_levels,
                 const double *Q, int64_t nq, int32_t k, const int32_t *probes,
                 int64_t *ids_out, double *dists_out, double tie_rtol, uint8_t *sel_clear) {
    if (L < 1 || k < 1 || d < 1) return MO_EINVAL;
    int64_t **off = (int64_t **)calloc((size_t)L, sizeof(int64_t *));
    int64_t **items = (int64_t **)calloc((size_t)L, sizeof(int64_t *));
    if (!off || !items) { free(off); free(items); return MO_ENOMEM; }
    int32_t rc = MO_OK;
    for (int32_t lv = 0; lv < L && rc == MO_OK; ++lv) {
        int64_t n_below = lv == 0 ? n : (int64_t)k_per_level[lv - 1];
        rc = member_lists(labels_levels[lv], n_below, k_per_level[lv], &off[lv], &items[lv]);
    }
    int64_t max_n = n;
    for (int32_t lv = 0; lv < L; ++lv)
        if ((int64_t)k_per_level[lv] > max_n) max_n = k_per_level[lv];

    if (rc == MO_OK) {
#pragma omp parallel
        {
            mo_pair *cand = (mo_pair *)malloc(sizeof(mo_pair) * (size_t)max_n);
            int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)max_n);
#pragma omp for schedule(dynamic, 4)
            for (int64_t qi = 0; qi < nq; ++qi) {
                const double *q = Q + qi * (int64_t)d;
                uint8_t clear = 1;
                /* top level: every centroid is a candidate */
                int64_t nc = 0;
                int32_t top = L - 1;
                for (int64_t j = 0; j < k_per_level[top]; ++j) {
                    cand[nc].d = sqdist(q, C_levels[top] + j * (int64_t)d, d);
                    cand[nc].id = j;
                    ++nc;
                }
                for (int32_t lv = top; lv >= 0; --lv) {
                    qsort(cand, (size_t)nc, sizeof(mo_pair), pair_cmp);
                    int64_t p = probes[lv] < nc ? probes[lv] : nc;
                    if (nc > p && cand[p].d - cand[p - 1].d <= tie_rtol * cand[p - 1].d) clear = 0;
                    for (int64_t s = 0; s < p; ++s) kept[s] = cand[s].id;
                    /* children of the kept centroids become the candidates */
                    const double *below = lv == 0 ? X : C_levels[lv - 1];
                    nc = 0;
                    for (int64_t s = 0; s < p; ++s) {
                        int64_t c = kept[s];
                        for (int64_t m = off[lv][c]; m < off[lv][c + 1]; ++m) {
                            int64_t it = items[lv][m];
                            cand[nc].d = sqdist(q, below + it * (int64_t)d, d);
                            cand[nc].id = it;
                            ++nc;
                        }
                    }
                }
                /* data layer: rank the reached points, return the k lowest */
                qsort(cand, (size_t)nc, sizeof(mo_pair), pair_cmp);
                for (int32_t r = 0; r < k; ++r) {
                    ids_out[qi * k + r] = r < nc ? cand[r].id : -1;
                    dists_out[qi * k + r] = r < nc ? cand[r].d : INFINITY;
                }
                if (sel_clear) sel_clear[qi] = clear;
            }
            free(cand);
            free(kept);
        }
    }
    for (int32_t lv = 0; lv < L; ++lv) { free(off[lv]); free(items[lv]); }
    free(off);
    free(items);
    return rc;
}

/* ------------------------------------------- exact k-NN by full scan */

/* Exact k nearest points of each query, ascending by (distance, id). */
int32_t mo_bruteforce_knn(const double *X, int64_t n, int32_t d, const double *Q, int64_t nq,
                          int32_t k, int64_t *ids_out, double *dists_out) {
    if (k < 1) return MO_EINVAL;
#pragma omp parallel
    {
        mo_pair *best = (mo_pair *)malloc(sizeof(mo_pair) * (size_t)k);
#pragma omp for schedule(dynamic, 4)
        for (int64_t qi = 0; qi < nq; ++qi) {
            const double *q = Q + qi * (int64_t)d;
            int32_t have = 0;
            for (int64_t i = 0; i < n; ++i) {
                mo_pair c = {sqdist(q, X + i * (int64_t)d, d), i};
                if (have == k && pair_cmp(&c, &best[k - 1]) >= 0) continue;
                /* insert c into the sorted list best[0..have) */
                int32_t pos = have < k ? have : k - 1;
                while (pos > 0 && pair_cmp(&c, &best[pos - 1]) < 0) {
                    best[pos] = best[pos - 1];
                    --pos;
                }
                best[pos] = c;
                if (have < k) ++have;
            }
            for (int32_t r = 0; r < k; ++r) {
                ids_out[qi * k + r] = r < have ? best[r].id : -1;
                dists_out[qi * k + r] = r < have ? best[r].d : INFINITY;
            }
        }
        free(best);
    }
    return MO_OK;
}

/* ------------------------------------------ grouped build (Algorithm 1) */

/*
 * Algorithm 1 as printed (§3.1): the items of a level are split at random into
 * ngroups = floor(items / lengthGroup) groups, each group is clustered into
 * nCentroids centroids by its own k-means, and the centroids of all groups
 * are the items of the next level; the loop stops when ngroups < 1.
 *
 * Readings (where the paper is silent):
 *   R16 split: a full Fisher-Yates shuffle of the level's items with the
 *       level stream of R1 (draws j = 0..m-2: r = j + floor(u (m - j))), then
 *       consecutive parts of the shuffled order whose sizes differ by at
 *       most one, the first (m mod G) parts one larger.  Within a group the
 *       items are taken in ascending item index.
 *   R17 group g of level lv seeds its k-means++ from the state
 *       level_state(seed, lv) ^ (0xD1B54A32D192ED03 * (g + 1)); its k-means is
 *       R2 + R4 with nCentroids centres and `iters` Lloyd iterations.
 *   R18 centroid j of group g is item g * nCentroids + j of the next level;
 *       the labels of a level map each item to that global centroid id.
 * With those, the index is the same structure as the global form's, so the
 * top-down search (mo_query) applies unchanged.
 */

/* Level sizes of the grouped build: sizes[lv] = centroids at level lv
 * (finest first); returns the number of levels (0 if n < lengthGroup), or
 * MO_EINVAL for bad parameters.  Integer arithmetic only. */
int32_t mo_grouped_sizes(int64_t n, int32_t lg, int32_t nc, int64_t *sizes, int32_t max_levels) {
    if (lg < 1 || nc < 1 || nc > lg || n < 0) return MO_EINVAL;
    int32_t L = 0;
    int64_t items = n;
    int64_t groups = items / lg;
    while (groups >= 1) {
        if (L >= max_levels) return MO_EINVAL;
        sizes[L++] = groups * nc;
        items = groups * nc;
        groups = items / lg;
    }
    return L;
}

uint64_t mo_group_state(uint64_t seed, int32_t level, int64_t group) {
    return mo_level_state(seed, level) ^ (0xD1B54A32D192ED03ull * (uint64_t)(group + 1));
}

/* R16: group_of[item] for m items split into G groups with the stream state. */
int32_t mo_split_groups(int64_t m, int64_t G, uint64_t *state, int32_t *group_of) {
    if (G < 1 || m < G) return MO_EINVAL;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!perm) return MO_ENOMEM;
    for (int64_t i = 0; i < m; ++i) perm[i] = i;
    for (int64_t j = 0; j + 1 < m; ++j) {
        int64_t r = j + (int64_t)floor(mo_uniform(state) * (double)(m - j));
        if (r > m - 1) r = m - 1;
        int64_t t = perm[j];
        perm[j] = perm[r];
        perm[r] = t;
    }
    const int64_t base = m / G, extra = m % G;
    int64_t pos = 0;
    for (int64_t g = 0; g < G; ++g) {
        const int64_t len = base + (g < extra ? 1 : 0);
        for (int64_t q = 0; q < len; ++q) group_of[perm[pos + q]] = (int32_t)g;
        pos += len;
    }
    free(perm);
    return MO_OK;
}

/*
 * One level of the grouped build: items X (m x d), their groups group_of[m]
 * (each group with at least nc items), G groups.  C (G*nc x d) and labels
 * (m, global centroid ids) are written.
 */
static int32_t grouped_level(const double *X, int64_t m, int32_t d, const int32_t *group_of,
                             int64_t G, int32_t nc, int32_t iters, uint64_t seed, int32_t lv,
                             double *C, int32_t *labels) {
    int64_t *off = NULL, *items = NULL;
    int32_t rc = member_lists(group_of, m, (int32_t)G, &off, &items);
    if (rc != MO_OK) return rc;
    for (int64_t g = 0; g < G && rc == MO_OK; ++g) {
        const int64_t mg = off[g + 1] - off[g];
        if (mg < nc) { rc = MO_EINVAL; break; }
        double *Xg = (double *)malloc(sizeof(double) * (size_t)mg * (size_t)d);
        int32_t *lg_ = (int32_t *)malloc(sizeof(int32_t) * (size_t)mg);
        int64_t *chosen = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
        if (!Xg || !lg_ || !chosen) { free(Xg); free(lg_); free(chosen); rc = MO_ENOMEM; break; }
        for (int64_t q = 0; q < mg; ++q)   /* items in ascending index (member_lists order) */
            memcpy(Xg + q * d, X + items[off[g] + q] * (int64_t)d, sizeof(double) * (size_t)d);
        uint64_t st = mo_group_state(seed, lv, g);
        double *Cg = C + g * (int64_t)nc * d;
        rc = mo_kmeanspp(Xg, mg, d, nc, &st, chosen, Cg);
        if (rc == MO_OK) rc = mo_lloyd(Xg, mg, d, nc, iters, Cg, lg_, NULL);
        if (rc == MO_OK)
            for (int64_t q = 0; q < mg; ++q)
                labels[items[off[g] + q]] = (int32_t)(g * nc + lg_[q]);
        free(Xg);
        free(lg_);
        free(chosen);
    }
    free(off);
    free(items);
    return rc;
}

/*
 * Grouped multilevel build.  L = mo_grouped_sizes(n, lg, nc, ...) levels;
 * C_levels[lv] (sizes[lv] x d) and labels_levels[lv] (items of level lv: n
 * for lv = 0, else sizes[lv-1]) are caller-allocated.  group0 (may be NULL)
 * gives the level-0 groups of the points (values in [0, floor(n/lg)), each
 * group with at least nc points) instead of the random split; the levels
 * above are always split at random.
 */
int32_t mo_build_grouped(const double *X, int64_t n, int32_t d, int32_t lg, int32_t nc,
                         int32_t iters, uint64_t seed, const int32_t *group0, int32_t L,
                         double *const *C_levels, int32_t *const *labels_levels) {
    int64_t sizes[64];
    int32_t Lc = mo_grouped_sizes(n, lg, nc, sizes, 64);
    if (Lc < 0 || Lc != L || iters < 0) return MO_EINVAL;
    const double *in = X;
    int64_t m = n;
    for (int32_t lv = 0; lv < L; ++lv) {
        const int64_t G = m / lg;
        int32_t *grp = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
        if (!grp) return MO_ENOMEM;
        int32_t rc = MO_OK;
        if (lv == 0 && group0) {
            for (int64_t i = 0; i < m; ++i) {
                if (group0[i] < 0 || group0[i] >= G) { rc = MO_EINVAL; break; }
                grp[i] = group0[i];
            }
        } else {
            uint64_t st = mo_level_state(seed, lv);
            rc = mo_split_groups(m, G, &st, grp);
        }
        if (rc == MO_OK)
            rc = grouped_level(in, m, d, grp, G, nc, iters, seed, lv, C_levels[lv], labels_levels[lv]);
        free(grp);
        if (rc != MO_OK) return rc;
        in = C_levels[lv];
        m = G * nc;
    }
    return MO_OK;
}

/* -------------------------------------------- descent to the leaf clusters */

/*
 * The kept leaf clusters of the top-down search (the kept set of level 0
 * after the same descent as mo_query): leaf_out [nq x probes[0]], nearest
 * first, padded with -1.
 */
int32_t mo_descend(int64_t n, int32_t d, int32_t L, const int32_t *k_per_level,
                   const double *const *C_levels, const int32_t *const *labels_levels,
                   const double *Q, int64_t nq, const int32_t *probes, int32_t *leaf_out) {
    if (L < 1 || d < 1) return MO_EINVAL;
    int64_t **off = (int64_t **)calloc((size_t)L, sizeof(int64_t *));
    int64_t **items = (int64_t **)calloc((size_t)L, sizeof(int64_t *));
    if (!off || !items) { free(off); free(items); return MO_ENOMEM; }
    int32_t rc = MO_OK;
    for (int32_t lv = 1; lv < L && rc == MO_OK; ++lv)
        rc = member_lists(labels_levels[lv], (int64_t)k_per_level[lv - 1], k_per_level[lv],
                          &off[lv], &items[lv]);
    int64_t max_n = 1;
    for (int32_t lv = 0; lv < L; ++lv)
        if ((int64_t)k_per_level[lv] > max_n) max_n = k_per_level[lv];
    (void)n;
    if (rc == MO_OK) {
#pragma omp parallel
        {
            mo_pair *cand = (mo_pair *)malloc(sizeof(mo_pair) * (size_t)max_n);
#pragma omp for schedule(dynamic, 16)
            for (int64_t qi = 0; qi < nq; ++qi) {
                const double *q = Q + qi * (int64_t)d;
                int64_t ncand = 0;
                const int32_t top = L - 1;
                for (int64_t j = 0; j < k_per_level[top]; ++j) {
                    cand[ncand].d = sqdist(q, C_levels[top] + j * (int64_t)d, d);
                    cand[ncand].id = j;
                    ++ncand;
                }
                for (int32_t lv = top; lv >= 0; --lv) {
                    qsort(cand, (size_t)ncand, sizeof(mo_pair), pair_cmp);
                    int64_t p = probes[lv] < ncand ? probes[lv] : ncand;
                    if (lv == 0) {
                        for (int32_t s = 0; s < probes[0]; ++s)
                            leaf_out[qi * probes[0] + s] = s < p ? (int32_t)cand[s].id : -1;
                        break;
                    }
                    int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p > 0 ? p : 1));
                    for (int64_t s = 0; s < p; ++s) kept[s] = cand[s].id;
                    ncand = 0;
                    for (int64_t s = 0; s < p; ++s) {
                        const int64_t c = kept[s];
                        for (int64_t mm = off[lv][c]; mm < off[lv][c + 1]; ++mm) {
                            const int64_t it = items[lv][mm];
                            cand[ncand].d = sqdist(q, C_levels[lv - 1] + it * (int64_t)d, d);
                            cand[ncand].id = it;
                            ++ncand;
                        }
                    }
                    free(kept);
                }
            }
            free(cand);
        }
    }
    for (int32_t lv = 0; lv < L; ++lv) { free(off[lv]); free(items[lv]); }
    free(off);
    free(items);
    return rc;
}

/* --------------------------------------------------- range query (A3) */

/*
 * Range search (§3.3, Algorithm 3), reading R19: at every level, from the top
 * centroids down, keep the candidate centroids within the ball of squared
 * radius r2 around q (||q - c||^2 <= r2) and descend into their children;
 * return the points of the kept leaf clusters within the ball, ascending by
 * (distance, id).  counts_out[q] receives each query's result count; when
 * ids_out is not NULL the results are written query after query (the first
 * counts_out[0] entries for query 0, ...), at most cap entries in all
 * (MO_EINVAL if they do not fit; counts_out is filled either way).
 */
int32_t mo_range_query(const double *X, int64_t n, int32_t d, int32_t L,
                       const int32_t *k_per_level, const double *const *C_levels,
                       const int32_t *const *labels_levels, const double *Q, int64_t nq,
                       double r2, int64_t *counts_out, int64_t cap, int64_t *ids_out,
                       double *dists_out) {
    if (L < 1 || d < 1) return MO_EINVAL;
    int64_t **off = (int64_t **)calloc((size_t)L, sizeof(int64_t *));
    int64_t **items = (int64_t **)calloc((size_t)L, sizeof(int64_t *));
    mo_pair **res = (mo_pair **)calloc((size_t)(nq > 0 ? nq : 1), sizeof(mo_pair *));
    if (!off || !items || !res) { free(off); free(items); free(res); return MO_ENOMEM; }
    int32_t rc = MO_OK;
    for (int32_t lv = 0; lv < L && rc == MO_OK; ++lv) {
        int64_t n_below = lv == 0 ? n : (int64_t)k_per_level[lv - 1];
        rc = member_lists(labels_levels[lv], n_below, k_per_level[lv], &off[lv], &items[lv]);
    }
    int64_t max_n = n;
    for (int32_t lv = 0; lv < L; ++lv)
        if ((int64_t)k_per_level[lv] > max_n) max_n = k_per_level[lv];
    if (rc == MO_OK) {
#pragma omp parallel
        {
            int64_t *kept = (int64_t *)malloc(sizeof(int64_t) * (size_t)max_n);
            int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)max_n);
            mo_pair *pts = (mo_pair *)malloc(sizeof(mo_pair) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 8)
            for (int64_t qi = 0; qi < nq; ++qi) {
                const double *q = Q + qi * (int64_t)d;
                const int32_t top = L - 1;
                int64_t nk = 0;
                for (int64_t j = 0; j < k_per_level[top]; ++j)
                    if (sqdist(q, C_levels[top] + j * (int64_t)d, d) <= r2) kept[nk++] = j;
                for (int32_t lv = top; lv >= 1; --lv) {
                    int64_t nn = 0;
                    for (int64_t s = 0; s < nk; ++s)
                        for (int64_t mm = off[lv][kept[s]]; mm < off[lv][kept[s] + 1]; ++mm) {
                            const int64_t it = items[lv][mm];
                            if (sqdist(q, C_levels[lv - 1] + it * (int64_t)d, d) <= r2)
                                next[nn++] = it;
                        }
                    for (int64_t s = 0; s < nn; ++s) kept[s] = next[s];
                    nk = nn;
                }
                int64_t np = 0;
                for (int64_t s = 0; s < nk; ++s)
                    for (int64_t mm = off[0][kept[s]]; mm < off[0][kept[s] + 1]; ++mm) {
                        const int64_t it = items[0][mm];
                        const double e = sqdist(q, X + it * (int64_t)d, d);
                        if (e <= r2) { pts[np].d = e; pts[np].id = it; ++np; }
                    }
                qsort(pts, (size_t)np, sizeof(mo_pair), pair_cmp);
                counts_out[qi] = np;
                res[qi] = (mo_pair *)malloc(sizeof(mo_pair) * (size_t)(np > 0 ? np : 1));
                if (res[qi]) memcpy(res[qi], pts, sizeof(mo_pair) * (size_t)np);
            }
            free(kept);
            free(next);
            free(pts);
        }
        int64_t total = 0;
        for (int64_t qi = 0; qi < nq; ++qi) {
            if (!res[qi]) rc = MO_ENOMEM;
            total += counts_out[qi];
        }
        if (rc == MO_OK && ids_out) {
            if (total > cap) rc = MO_EINVAL;
            else {
                int64_t pos = 0;
                for (int64_t qi = 0; qi < nq; ++qi)
                    for (int64_t s = 0; s < counts_out[qi]; ++s, ++pos) {
                        ids_out[pos] = res[qi][s].id;
                        dists_out[pos] = res[qi][s].d;
                    }
            }
        }
    }
    for (int64_t qi = 0; qi < nq; ++qi) free(res[qi]);
    free(res);
    for (int32_t lv = 0; lv < L; ++lv) { free(off[lv]); free(items[lv]); }
    free(off);
    free(items);
    return rc;
}

/* ------------------------------------------ relocation (§4.1), reading R20 */

/*
 * One relocation pass of the grouped build (§4.1): every point is searched
 * for by the greedy descent (one kept centroid per level, as the point query
 * of §3.3); a point is missed when the reached leaf cluster is not its own.
 * A missed point moves to the level-0 group of the reached leaf cluster
 * (leaf / nc), in ascending point order, unless its own group would drop
 * below nc points.  group0 [n] is updated in place; *moved receives the
 * number of moves.  Returns the number of missed points (< 0 on error).
 */
int64_t mo_relocate(const double *X, int64_t n, int32_t d, int32_t L, const int32_t *k_per_level,
                    const double *const *C_levels, const int32_t *const *labels_levels,
                    int32_t nc, int32_t *group0, int64_t *moved) {
    int32_t *leaf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *probes = (int32_t *)malloc(sizeof(int32_t) * (size_t)L);
    if (!leaf || !probes) { free(leaf); free(probes); return MO_ENOMEM; }
    for (int32_t lv = 0; lv < L; ++lv) probes[lv] = 1;
    int32_t rc = mo_descend(n, d, L, k_per_level, C_levels, labels_levels, X, n, probes, leaf);
    free(probes);
    if (rc != MO_OK) { free(leaf); return rc; }
    int64_t G = 0;
    for (int64_t i = 0; i < n; ++i) if (group0[i] + 1 > G) G = group0[i] + 1;
    int64_t *size = (int64_t *)calloc((size_t)(G > 0 ? G : 1), sizeof(int64_t));
    if (!size) { free(leaf); return MO_ENOMEM; }
    for (int64_t i = 0; i < n; ++i) size[group0[i]] += 1;
    int64_t missed = 0, mv = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (leaf[i] == labels_levels[0][i]) continue;
        ++missed;
        const int32_t tgt = leaf[i] / nc, src = group0[i];
        if (leaf[i] < 0 || tgt == src || size[src] <= nc) continue;
        size[src] -= 1;
        size[tgt] += 1;
        group0[i] = tgt;
        ++mv;
    }
    if (moved) *moved = mv;
    free(size);
    free(leaf);
    return missed;
}
