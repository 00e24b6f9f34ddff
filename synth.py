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
