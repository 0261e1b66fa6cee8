"""Seeded synthetic inputs for the MASK hot path.

This module only draws random inputs; it holds none of the method's arithmetic
(no distances, no k-means, no search), so both the CUDA path and the FP64
oracle can be fed from it without sharing any computation.

The paper evaluates on Gaussian clouds (§4.2) and on the Reuters-21578 TF-IDF
matrix (§4.3).  Neither dataset ships with the paper; these generators stand in
for them with the shapes and distributions the workloads below state:

* ``IsotropicMixture``   - isotropic Gaussian blobs, centres uniform in a box,
  equal weights (the small dense workload: 20,000 x 16, 10 blobs, sigma 1).
* ``AnisotropicMixture`` - blobs with random covariance Q diag(lambda) Q^T,
  lambda log-uniform, Zipf-distributed blob weights (the 10^7 x 64 dense
  workload with 1,000 blobs).
* ``sparse_tfidf_like``  - CSR rows with lognormal row lengths, Zipf column
  ids and L2-normalised |N(0,1)| values (the 10^6 x 20,000 sparse workload, a
  stand-in for the shape of a TF-IDF term-document matrix, §4.3).
* ``gaussian_clouds_2d`` - 8 Gaussian clouds in R^2 (the synthetic datasets of
  §4.2: centres evenly on a circle, the radius setting how much adjacent
  clouds overlap).

Every generator is a pure function of its seed (numpy PCG64).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "IsotropicMixture",
    "AnisotropicMixture",
    "sparse_tfidf_like",
    "CSR",
    "gaussian_clouds_2d",
    "CLOUD_RADIUS",
]

# Circle radius of the cloud centres for the three datasets of §4.2 (sigma 1):
# adjacent centres are 2 R sin(pi/8) = 0.765 R apart, i.e. 7.7, 3.6 and 2.1
# standard deviations: clearly separated (GNO), moderate overlap (GMO),
# strong overlap (GRO).  The paper does not state its cloud parameters; GMO
# and GRO are set so that, at 200 points per cloud, the share of points whose
# point query lands on another cloud is near the first values the paper
# reports for them (about 12% and 40%).
CLOUD_RADIUS = {"GNO": 10.0, "GMO": 4.75, "GRO": 2.8}


class IsotropicMixture:
    """Mixture of ``n_blobs`` isotropic Gaussians N(mu_b, sigma^2 I) in R^d.

    Centres are uniform in [-box, box]^d, drawn from ``seed``; blob weights are
    equal.  ``sample(n, seed)`` draws points from the same mixture with an
    independent stream, so data and queries share centres but not samples.
    """

    def __init__(self, d: int, n_blobs: int, sigma: float = 1.0,
                 box: float = 10.0, seed: int = 0):
        rng = np.random.default_rng([seed, 0x5EED])
        self.d = int(d)
        self.n_blobs = int(n_blobs)
        self.sigma = float(sigma)
        self.centres = rng.uniform(-box, box, size=(n_blobs, d))

    def sample(self, n: int, seed: int, return_blob: bool = False):
        rng = np.random.default_rng([seed, 0xDA7A])
        blob = rng.integers(0, self.n_blobs, size=n)
        z = rng.standard_normal(size=(n, self.d))
        x = (self.centres[blob] + self.sigma * z).astype(np.float32)
        return (x, blob) if return_blob else x


class AnisotropicMixture:
    """Mixture of ``n_blobs`` Gaussians with random covariance in R^d.

    Blob b has centre mu_b ~ U[-box, box]^d and covariance
    Q_b diag(lambda_b) Q_b^T, where Q_b is the sign-fixed Q factor of a
    Gaussian matrix and lambda_b is log-uniform in [eig_lo, eig_hi].  Blob
    weights follow Zipf: w_b proportional to b^-zipf_s for b = 1..n_blobs.
    """

    def __init__(self, d: int, n_blobs: int, eig_lo: float = 0.1,
                 eig_hi: float = 10.0, zipf_s: float = 1.1, box: float = 10.0,
                 seed: int = 0):
        rng = np.random.default_rng([seed, 0xA150])
        self.d = int(d)
        self.n_blobs = int(n_blobs)
        self.centres = rng.uniform(-box, box, size=(n_blobs, d))
        self.eig = np.exp(rng.uniform(np.log(eig_lo), np.log(eig_hi),
                                      size=(n_blobs, d)))
        self.rot = np.empty((n_blobs, d, d))
        for b in range(n_blobs):
            g = rng.standard_normal(size=(d, d))
            q, r = np.linalg.qr(g)
            self.rot[b] = q * np.sign(np.diag(r))[None, :]
        w = np.arange(1, n_blobs + 1, dtype=np.float64) ** (-zipf_s)
        self.weights = w / w.sum()
        # x = mu + Q (sqrt(lambda) * z)  <=>  x = mu + z @ (Q * sqrt(lambda))^T
        self._maps = (self.rot * np.sqrt(self.eig)[:, None, :]).transpose(0, 2, 1)

    def sample(self, n: int, seed: int, chunk: int = 1 << 20,
               return_blob: bool = False):
        out = np.empty((n, self.d), dtype=np.float32)
        blobs = np.empty(n, dtype=np.int32) if return_blob else None
        cdf = np.cumsum(self.weights)
        cdf[-1] = 1.0
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            rng = np.random.default_rng([seed, 0xB10B, c0 // chunk])
            blob = np.searchsorted(cdf, rng.random(c1 - c0), side="right")
            blob = np.minimum(blob, self.n_blobs - 1)
            z = rng.standard_normal(size=(c1 - c0, self.d))
            order = np.argsort(blob, kind="stable")
            bs = blob[order]
            starts = np.flatnonzero(np.r_[True, bs[1:] != bs[:-1]])
            ends = np.r_[starts[1:], len(bs)]
            x = np.empty((c1 - c0, self.d))
            for s, e in zip(starts, ends):
                b = bs[s]
                rows = order[s:e]
                x[rows] = self.centres[b] + z[rows] @ self._maps[b]
            out[c0:c1] = x
            if return_blob:
                blobs[c0:c1] = blob
        return (out, blobs) if return_blob else out


class CSR:
    """Compressed sparse rows: ``row_ptr`` int64 [n+1], ``col`` int32 [nnz],
    ``val`` float32 [nnz]; columns sorted ascending within each row."""

    def __init__(self, row_ptr, col, val, n_cols):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float32)
        self.n_rows = len(self.row_ptr) - 1
        self.n_cols = int(n_cols)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self, sel) -> "CSR":
        sel = np.asarray(sel, dtype=np.int64)
        lens = self.row_ptr[sel + 1] - self.row_ptr[sel]
        rp = np.zeros(len(sel) + 1, dtype=np.int64)
        np.cumsum(lens, out=rp[1:])
        idx = np.concatenate([np.arange(self.row_ptr[s], self.row_ptr[s + 1])
                              for s in sel]) if len(sel) else np.zeros(0, np.int64)
        return CSR(rp, self.col[idx], self.val[idx], self.n_cols)

    def to_dense(self, dtype=np.float64) -> np.ndarray:
        out = np.zeros((self.n_rows, self.n_cols), dtype=dtype)
        r = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        out[r, self.col] = self.val
        return out


def _first_distinct(rng, m, d, cdf, vocab):
    """Column ids of len(m) rows: row r keeps the first m[r] distinct values of
    an iid sequence of Zipf draws (mapped through ``vocab``).  Returns the
    (row, column) pairs sorted by row, then column."""
    n = len(m)
    kr = np.zeros(0, np.int64)   # kept rows / columns / sequence numbers
    kc = np.zeros(0, np.int64)
    ks = np.zeros(0, np.int64)
    seq_base = np.zeros(n, np.int64)
    need = m.copy()
    active = np.arange(n, dtype=np.int64)
    while len(active):
        b = (need[active] * 13) // 10 + 8          # draws per active row this round
        r = np.repeat(active, b)
        starts = np.cumsum(b) - b
        seq = seq_base[r] + (np.arange(len(r), dtype=np.int64) - np.repeat(starts, b))
        seq_base[active] += b
        rank = np.minimum(np.searchsorted(cdf, rng.random(len(r)), side="right"), d - 1)
        c = vocab[rank].astype(np.int64)
        # candidates of the active rows: what they kept so far (earlier in
        # their sequences) and the new draws
        ka = np.isin(kr, active)
        R = np.concatenate([kr[ka], r])
        Cc = np.concatenate([kc[ka], c])
        S = np.concatenate([ks[ka], seq])
        kr, kc, ks = kr[~ka], kc[~ka], ks[~ka]
        # first occurrence of each (row, column) in sequence order
        key = (R * d + Cc) * (1 << 24) + S
        key.sort()
        rc = key >> 24
        first = np.ones(len(key), bool)
        first[1:] = rc[1:] != rc[:-1]
        rc, s1 = rc[first], key[first] & ((1 << 24) - 1)
        rr = rc // d
        cc = rc - rr * d
        # per row in sequence order, keep the first m[row]
        o = np.argsort(rr * (1 << 24) + s1, kind="stable")
        rr, cc, s1 = rr[o], cc[o], s1[o]
        bnd = np.flatnonzero(np.r_[True, rr[1:] != rr[:-1]])
        pos = np.arange(len(rr)) - np.repeat(bnd, np.diff(np.r_[bnd, len(rr)]))
        keep = pos < m[rr]
        kr = np.concatenate([kr, rr[keep]])
        kc = np.concatenate([kc, cc[keep]])
        ks = np.concatenate([ks, s1[keep]])
        need = m - np.bincount(kr, minlength=n)
        active = np.flatnonzero(need > 0)
    key = np.sort(kr * d + kc)
    rows = key // d
    return rows, key - rows * d


def sparse_tfidf_like(n: int, d: int, nnz_mean: float = 60.0,
                      nnz_sigma: float = 0.8, zipf_s: float = 1.0,
                      seed: int = 0, vocab_seed: int = 0, chunk: int = 1 << 16) -> CSR:
    """Sparse rows shaped like an L2-normalised TF-IDF matrix.

    Row length m_r ~ round(LogNormal(mu, nnz_sigma)) clipped to [1, d], with mu
    chosen so the arithmetic mean is ``nnz_mean`` (mu = ln(mean) - sigma^2/2).
    Column ids follow Zipf(``zipf_s``) over a fixed permutation of the d ids
    (drawn from ``vocab_seed``, so data and queries share the vocabulary), drawn
    without replacement within a row: the first m_r distinct values of an iid
    sequence of draws (the same as draw, drop repeats, redraw the deficit).
    Values are |N(0,1)|, then each row is scaled to unit L2 norm.  Rows are
    generated in chunks of ``chunk`` rows.
    """
    rng = np.random.default_rng([seed, 0x5BA5])
    vocab = np.random.default_rng([vocab_seed, 0x70CA]).permutation(d)
    mu = np.log(nnz_mean) - 0.5 * nnz_sigma ** 2
    m = np.clip(np.rint(rng.lognormal(mu, nnz_sigma, size=n)), 1, d).astype(np.int64)
    w = np.arange(1, d + 1, dtype=np.float64) ** (-zipf_s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    cols = []
    for c0 in range(0, n, chunk):
        _, c = _first_distinct(rng, m[c0:c0 + chunk], d, cdf, vocab)
        cols.append(c.astype(np.int32))
    col = np.concatenate(cols) if cols else np.zeros(0, np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(m, out=row_ptr[1:])
    val = np.abs(rng.standard_normal(len(col)))
    sq = np.add.reduceat(val * val, row_ptr[:-1]) if len(val) else np.zeros(n)
    val = val / np.sqrt(np.repeat(sq, m))
    return CSR(row_ptr, col, val.astype(np.float32), d)


def gaussian_clouds_2d(npc: int, radius: float, sigma: float = 1.0, seed: int = 0,
                       return_cloud: bool = False):
    """8 isotropic Gaussian clouds in R^2 with ``npc`` points each, centres at
    angles 2 pi c / 8 on a circle of the given radius, cloud c's points
    contiguous (rows c * npc ...).  Returns float32 points (and the cloud of
    every point)."""
    rng = np.random.default_rng([seed, 0xC10D])
    ang = np.arange(8) * 2.0 * np.pi / 8.0
    centres = np.stack([np.cos(ang), np.sin(ang)], 1) * radius
    cloud = np.repeat(np.arange(8), npc)
    x = (centres[cloud] + sigma * rng.standard_normal(size=(8 * npc, 2))).astype(np.float32)
    return (x, cloud) if return_cloud else x
