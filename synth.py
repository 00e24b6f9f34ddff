"""Seeded synthetic inputs for the exterior NMF workloads.

This module only draws random inputs.  It holds none of the factorisation's
arithmetic, so the CPU oracle, the tests and the benchmark can all take the
same bytes from it without sharing method code.

Every generator uses NumPy's ``default_rng(seed)`` (PCG64) and draws in a
fixed order so that a seed always gives the same matrix.  Shapes follow the
convention X (m x n) ~ U V^T with U (m x r) and V (n x r).

Workloads (sizes, distributions):

* ``planted``     -- X = U0 V0^T + E with U0, V0 entries Uniform[0,1] or
  Exponential(1), a fraction of entries set to zero, and E a clamped Gaussian.
  This is the exact-factorisation recipe of Sec. 5.1 (noise-free when
  ``noise == 0``) with an optional noise term.
* ``image_stack`` -- columns are 92x112 images made from a nonnegative mixture
  of r smooth 2D Gaussian bumps (stands in for the Face data of Sec. 5.1).
* ``spectrogram`` -- Gamma(0.5, 1) magnitudes modulating r harmonic spectral
  templates times sparse activations (stands in for the Audio data of
  Sec. 5.1).
* ``request_stream`` -- a Poisson stream of mixed-size planted problems.
* ``sparse_docs`` -- a document-term matrix in compressed-row form: lognormal
  document lengths, Zipf term frequencies, tf-idf weights with unit rows
  (stands in for the Reuters matrix, 804,414 x 47,236 at 99.84 % sparsity, and
  at 282 x 1,528 / 97.3 % for the Verb data of Sec. 5).
* ``ratings`` -- a user-item rating matrix with a known-entry pattern
  (power-law user activity and item popularity, ratings 1..5 from a planted
  low-rank score); stands in for MovieLens 1M (App. C).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def planted(m, n, r, seed=0, dist="uniform", zero_frac=0.3, noise=0.01,
            noise_relative=False, dtype=np.float64):
    """Planted nonnegative factors plus clamped Gaussian noise.

    Draw order: U0, mask(U0), V0, mask(V0), noise.  ``noise`` is the Gaussian
    standard deviation; with ``noise_relative`` it is multiplied by the RMS of
    U0 V0^T.  The noise is clamped at zero before it is added (so X >= 0).
    Returns (X, U0, V0).
    """
    rng = np.random.default_rng(seed)

    def factor(rows):
        if dist == "uniform":
            F = rng.random((rows, r))
        elif dist == "exponential":
            F = rng.exponential(1.0, (rows, r))
        else:
            raise ValueError(dist)
        keep = rng.random((rows, r)) >= zero_frac
        return F * keep

    U0 = factor(m)
    V0 = factor(n)
    X = U0 @ V0.T
    if noise > 0:
        sigma = noise * (math.sqrt(float(np.mean(X * X))) if noise_relative else 1.0)
        E = np.maximum(rng.normal(0.0, sigma, (m, n)), 0.0)
        X = X + E
    return X.astype(dtype, copy=False), U0, V0


def config_small(seed=0):
    """200 x 150, r = 5, Uniform[0,1] factors with 30% zeros, noise 0.01."""
    X, _, _ = planted(200, 150, 5, seed=seed, dist="uniform", zero_frac=0.3, noise=0.01)
    return X, 5


def config_dense(seed=0, dtype=np.float64):
    """8192 x 6144, r = 32, Exponential(1) factors with 50% zeros, 1% noise."""
    X, _, _ = planted(8192, 6144, 32, seed=seed, dist="exponential", zero_frac=0.5,
                      noise=0.01, noise_relative=True, dtype=dtype)
    return X, 32


def image_stack(m_rows=92, m_cols=112, n=4096, r=49, seed=0, dtype=np.float64):
    """Image-stack matrix: m = m_rows*m_cols pixels, n images, r bumps.

    Bump k is exp(-|p - c_k|^2 / (2 s_k^2)) with the centre c_k uniform on the
    pixel grid and s_k ~ Uniform[3, 12] pixels.  Image weights ~ Exponential(1).
    Each column is scaled to a maximum of 1, then Uniform[0, 0.02] noise is
    added.  Returns (X, r).
    """
    rng = np.random.default_rng(seed)
    cy = rng.uniform(0, m_rows - 1, r)
    cx = rng.uniform(0, m_cols - 1, r)
    s = rng.uniform(3.0, 12.0, r)
    yy, xx = np.meshgrid(np.arange(m_rows), np.arange(m_cols), indexing="ij")
    yy = yy.reshape(-1, 1)
    xx = xx.reshape(-1, 1)
    B = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * s ** 2))   # (m, r)
    Wt = rng.exponential(1.0, (n, r))
    X = B @ Wt.T
    X /= np.maximum(X.max(axis=0, keepdims=True), 1e-300)
    X += rng.uniform(0.0, 0.02, X.shape)
    return X.astype(dtype, copy=False), r


def spectrogram(m=1025, n=131072, r=64, seed=0, dtype=np.float64):
    """Spectrogram-shaped matrix (frequency bins x frames).

    Templates: harmonic combs with fundamental bin f0 log-uniform on [5, 200],
    partial h at bin h*f0 with amplitude 1/h, smoothed by a Gaussian of width
    2 bins.  Activations: Exponential(1) with 80% zeros.  X = (W0 H0^T) * G with
    G ~ Gamma(0.5, 1) elementwise.  Returns (X, r).
    """
    rng = np.random.default_rng(seed)
    f0 = np.exp(rng.uniform(math.log(5.0), math.log(200.0), r))
    bins = np.arange(m, dtype=np.float64).reshape(-1, 1)
    W0 = np.zeros((m, r))
    for k in range(r):
        h = 1
        while h * f0[k] < m:
            W0[:, k] += (1.0 / h) * np.exp(-(bins[:, 0] - h * f0[k]) ** 2 / (2.0 * 2.0 ** 2))
            h += 1
    H0 = rng.exponential(1.0, (n, r)) * (rng.random((n, r)) >= 0.8)
    X = (W0 @ H0.T).astype(dtype)
    X *= rng.gamma(0.5, 1.0, (m, n)).astype(dtype)
    return X, r


@dataclass
class Request:
    rid: int
    arrival_s: float
    m: int
    n: int
    r: int
    seed: int


def request_stream(count=4096, seed=0, rate_per_s=None, m_lo=64, m_hi=4096,
                   ranks=(4, 8, 16, 32, 64)):
    """Poisson stream of planted-factor NMF requests.

    m and n are round(exp(Uniform[ln m_lo, ln m_hi])) and r is uniform over
    ``ranks`` (capped at min(m, n)).  With ``rate_per_s`` None every request
    arrives at t = 0 (saturation).  Request i's matrix comes from
    ``request_matrix(req)`` with seed i.
    """
    rng = np.random.default_rng(seed)
    lo, hi = math.log(m_lo), math.log(m_hi)
    ms = np.rint(np.exp(rng.uniform(lo, hi, count))).astype(int)
    ns = np.rint(np.exp(rng.uniform(lo, hi, count))).astype(int)
    rs = rng.choice(np.asarray(ranks), count)
    if rate_per_s:
        t = np.cumsum(rng.exponential(1.0 / rate_per_s, count))
    else:
        t = np.zeros(count)
    out = []
    for i in range(count):
        r = int(min(rs[i], ms[i], ns[i]))
        out.append(Request(i, float(t[i]), int(ms[i]), int(ns[i]), r, i))
    return out


def request_matrix(req, dtype=np.float64):
    """The planted matrix of one request (Uniform factors, 30% zeros, noise 0.01)."""
    X, _, _ = planted(req.m, req.n, req.r, seed=req.seed, dist="uniform",
                      zero_frac=0.3, noise=0.01, dtype=dtype)
    return X


def sparse_docs(m, n, density, seed=0, dtype=np.float32, zipf_s=1.05, len_sigma=0.9):
    """Document-term matrix in compressed-row form (row_ptr int64 (m + 1),
    col int32 (nnz), val (nnz)); columns strictly increasing within a row.

    Draw order: document lengths (lognormal, sigma ``len_sigma``), a random
    permutation of the terms, then every document's term draws (Zipf
    exponent ``zipf_s`` over the permuted terms, with replacement).  Repeated
    terms of a document merge into one entry with count tf; the weight is
    (1 + ln tf) * idf, idf = ln((1 + m) / (1 + df)) + 1, and every row is
    scaled to unit norm.  Lengths are rescaled twice so that the stored entries
    after merging come to about density * m * n.
    """
    rng = np.random.default_rng(seed)
    L0 = rng.lognormal(0.0, len_sigma, m)
    perm = rng.permutation(n)
    p = np.arange(1, n + 1, dtype=np.float64) ** -zipf_s
    cdf = np.cumsum(p / p.sum())
    target = density * m * n
    u_state = rng.bit_generator.state

    def draw(scale):
        rng.bit_generator.state = u_state
        L = np.maximum(1, np.rint(L0 * scale)).astype(np.int64)
        L = np.minimum(L, n)
        u = rng.random(int(L.sum()))
        terms = perm[np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)]
        rows = np.repeat(np.arange(m, dtype=np.int64), L)
        key, tf = np.unique(rows * n + terms, return_counts=True)
        return key, tf

    scale = target / L0.sum()
    key, tf = draw(scale)
    for _ in range(2):
        scale *= target / max(1, key.size)
        key, tf = draw(scale)
    r_i = key // n
    c_j = (key % n).astype(np.int32)
    df = np.bincount(c_j, minlength=n)
    idf = np.log((1.0 + m) / (1.0 + df)) + 1.0
    w = (1.0 + np.log(tf)) * idf[c_j]
    nrm = np.sqrt(np.bincount(r_i, weights=w * w, minlength=m))
    w = w / nrm[r_i]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(r_i, minlength=m))
    return row_ptr, c_j, w.astype(dtype)


def ratings(m=6040, n=3706, known=0.045, r0=8, seed=0, dtype=np.float32):
    """User-item ratings with a known-entry pattern, in compressed-row form
    (row_ptr, col, val); the known entries are the mask M_E of App. C.

    Draw order: user activity (Pareto 1.2, scaled), item popularity (Pareto
    1.0), user and item factors (Exponential(1), rank r0), per-entry noise.
    User i rates about known * n * activity_i items (rescaled once so that
    the total is about known * m * n) drawn without replacement
    in proportion to popularity (at least 5); the rating of (i, j) is the
    planted score u_i . v_j mapped to 1..5 by quantiles of all scores plus
    Gaussian noise (sigma 0.5), rounded and clipped to 1..5.
    """
    rng = np.random.default_rng(seed)
    act = rng.pareto(1.2, m) + 1.0
    pop = rng.pareto(1.0, n) + 1.0
    Uf = rng.exponential(1.0, (m, r0))
    Vf = rng.exponential(1.0, (n, r0))
    base = act / act.mean() * known * n
    cnt = np.clip(np.rint(base), 5, n)
    cnt = np.clip(np.rint(base * (known * m * n / cnt.sum())), 5, n).astype(np.int64)
    w = pop / pop.sum()
    rows, cols = [], []
    for i in range(m):
        # Gumbel top-k: k items without replacement, in proportion to w
        g = np.log(w) - np.log(-np.log(rng.random(n)))
        sel = np.sort(np.argpartition(-g, cnt[i] - 1)[:cnt[i]])
        rows.append(np.full(sel.size, i, dtype=np.int64))
        cols.append(sel)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols).astype(np.int32)
    score = np.einsum("ij,ij->i", Uf[rows], Vf[cols])
    q = np.quantile(score, [0.06, 0.17, 0.43, 0.78])
    val = 1.0 + np.searchsorted(q, score) + rng.normal(0.0, 0.5, score.size)
    val = np.clip(np.rint(val), 1.0, 5.0)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(rows, minlength=m))
    return row_ptr, cols, val.astype(dtype)
