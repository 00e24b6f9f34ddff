"""Pins of the oracle's sparse-X helpers (Sec. 5, Reuters) and its matrix
completion path (App. C, Algorithm eNMC).

Sparse X: the compressed-row helpers against SciPy's own sparse matrix (an
independent library, not an oracle routine), on the document-term generator's
output; the generator's format invariants.

eNMC:
* with every entry known (M_E = 1) the masked objective is Eq. 1's and the
  masked PBCD is Algorithm 2's (the pinned unmasked oracle), step for step;
* the masked gradient of App. C against central differences of f^;
* the masked row step is the exact minimiser of f^ along -g_i (a dense scan
  refined by golden-section search, rows where the projection does not clip);
* the rows of U are independent (Sec. 4.2): row-at-a-time in any order equals
  the parallel sweep;
* the masked-ALS start is a fixed point of its row ridge systems (the App. C
  gradient plus the ridge term vanishes row by row) and, without a ridge,
  with every entry known and X of exact rank r, reaches f^ ~ 0;
* Algorithm eNMC ends nonnegative and far below its first round's f^.
"""
import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O

sp = pytest.importorskip("scipy.sparse")


def _docs(m=200, n=300, density=0.05, seed=3):
    return synth.sparse_docs(m, n, density, seed=seed, dtype=np.float64)


def test_csr_dense_matches_scipy():
    rp, c, v = _docs()
    X = O.csr_dense(200, 300, rp, c, v)
    ref = sp.csr_matrix((v, c, rp), shape=(200, 300)).toarray()
    assert np.array_equal(X, ref)


def test_csr_products_match_scipy():
    rp, c, v = _docs()
    S = sp.csr_matrix((v, c, rp), shape=(200, 300))
    rng = np.random.default_rng(0)
    B = rng.standard_normal((300, 7))
    C = rng.standard_normal((200, 7))
    rows = np.arange(200)
    np.testing.assert_allclose(O.csr_rows_times(rp, c, v, rows, B), S @ B, rtol=1e-13, atol=1e-13)
    cols = np.arange(0, 300, 7)
    np.testing.assert_allclose(O.csr_cols_times(rp, c, v, cols, C), (S.T @ C)[cols], rtol=1e-13,
                               atol=1e-13)
    assert O.csr_sumsq(v) == pytest.approx(float(S.multiply(S).sum()), rel=1e-14)


def test_generators_give_canonical_compressed_rows():
    for rp, c, v, m, n in ((*_docs(), 200, 300), (*synth.ratings(300, 200, 0.1, seed=1), 300, 200)):
        assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == c.size == v.size
        assert c.min() >= 0 and c.max() < n
        for i in range(m):
            seg = c[rp[i]:rp[i + 1]]
            assert np.all(np.diff(seg) > 0)
        assert np.all(v > 0)
    rp, c, v = _docs()
    norms = np.sqrt(np.bincount(np.repeat(np.arange(200), np.diff(rp)), weights=v * v, minlength=200))
    np.testing.assert_allclose(norms[np.diff(rp) > 0], 1.0, rtol=1e-12)
    _, _, val = synth.ratings(300, 200, 0.1, seed=1)
    assert set(np.unique(val)) <= {1.0, 2.0, 3.0, 4.0, 5.0}


def _masked_problem(m=40, n=30, r=4, known=0.6, seed=5):
    rng = np.random.default_rng(seed)
    U0 = rng.random((m, r))
    V0 = rng.random((n, r))
    X = U0 @ V0.T + 0.01 * rng.random((m, n))
    M = (rng.random((m, n)) < known).astype(np.float64)
    U = rng.random((m, r))
    V = rng.random((n, r))
    return X, M, U, V


def test_all_known_reduces_to_the_unmasked_method():
    X, _, U, V = _masked_problem()
    M = np.ones_like(X)
    assert O.objective_masked(X, M, U, V) == pytest.approx(O.objective(X, U, V), rel=1e-14)
    Um = U - 0.3
    mask = Um >= 0
    a, ia = O.pbcd_masked(X, M, Um, V, mask.astype(np.float64))
    b, ib = O.pbcd(X, Um, V, mask)
    assert ia.iters == ib.iters
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_masked_gradient_is_the_derivative():
    X, M, U, V = _masked_problem()
    G = O.grad_masked(X, M, U, V)
    h = 1e-6
    for (i, j) in ((0, 0), (7, 2), (39, 3)):
        E = np.zeros_like(U)
        E[i, j] = h
        fd = (O.objective_masked(X, M, U + E, V) - O.objective_masked(X, M, U - E, V)) / (2 * h)
        assert G[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    GV = O.grad_masked(X.T, M.T, V, U)
    E = np.zeros_like(V)
    E[5, 1] = h
    fd = (O.objective_masked(X, M, U, V + E) - O.objective_masked(X, M, U, V - E)) / (2 * h)
    assert GV[5, 1] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def _golden(f, a, b, it=200):
    g = (np.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(it):
        if f(c) < f(d):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    return 0.5 * (a + b)


def test_masked_step_is_the_exact_line_minimiser():
    X, M, U, V = _masked_problem()
    U = U + 1.0
    g = O.grad_masked(X, M, U, V)
    num = np.sum(g * g, axis=1)
    den = np.sum(M * (g @ V.T) ** 2, axis=1)
    d = num / den
    for i in (0, 11, 23):
        def phi(t):
            W = U.copy()
            W[i] -= t * g[i]
            return O.objective_masked(X, M, W, V)
        ts = np.linspace(0, 4 * d[i], 4001)
        k = int(np.argmin([phi(t) for t in ts]))
        t_star = _golden(phi, ts[max(k - 1, 0)], ts[min(k + 1, 4000)])
        assert d[i] == pytest.approx(t_star, rel=1e-6)
    U1, _ = O.pbcd_masked(X, M, U, V, np.ones_like(U), max_iter=1)
    np.testing.assert_allclose(U1, np.maximum(U - d[:, None] * g, 0.0), rtol=1e-13)


def test_masked_rows_are_independent():
    """Sec. 4.2: with V fixed the rows of U do not interact, so updating the
    rows one at a time in any order (the paper's row loop) gives the parallel
    sweep's result."""
    X, M, U, V = _masked_problem(seed=8)
    mask = np.ones_like(U)
    Upar, _ = O.pbcd_masked(X, M, U, V, mask, eps=0.0, max_iter=1)
    Useq = U.copy()
    for i in np.random.default_rng(1).permutation(U.shape[0]):
        g = O.grad_masked(X, M, Useq, V)[i]
        num = g @ g
        den = np.sum(M[i] * (V @ g) ** 2)
        Useq[i] = np.maximum(Useq[i] - (num / den) * g, 0.0)
    np.testing.assert_allclose(Upar, Useq, rtol=1e-12, atol=1e-15)


def test_masked_als_reaches_a_stationary_point():
    """At the ALS fixed point every row solves its ridge system: the masked
    gradient of App. C plus the ridge term lam c_i u_i vanishes, row by row
    (c_i from the final other factor); without a ridge, with every entry
    known and X of exact rank r, ALS reaches f^ ~ 0."""
    X, M, _, _ = _masked_problem(m=50, n=40, r=3, known=0.7, seed=9)
    lam = 1e-3
    U, V, sw = O.masked_als(X, M, 3, sweeps=2000, lam=lam, tol=1e-15)
    for F, G, Xs, Ms in ((U, V, X, M), (V, U, X.T, M.T)):
        g = O.grad_masked(Xs, Ms, F, G)
        for i in range(F.shape[0]):
            sel = Ms[i] > 0
            Gi = G[sel].T @ G[sel]
            c = float(np.trace(Gi)) / 3
            res = g[i] + lam * (c if c > 0 else 1.0) * F[i]
            assert np.linalg.norm(res) <= 1e-9 * (np.linalg.norm(g[i]) + c * np.linalg.norm(F[i])), i
    rng = np.random.default_rng(4)
    A, B = rng.random((30, 3)), rng.random((20, 3))
    Xe = A @ B.T
    U, V, _ = O.masked_als(Xe, np.ones_like(Xe), 3, sweeps=100, lam=0.0)
    assert O.objective_masked(Xe, np.ones_like(Xe), U, V) < 1e-18 * np.sum(Xe * Xe)


def test_enmc_ends_nonnegative_and_makes_progress():
    X, M, _, _ = _masked_problem(m=60, n=45, r=4, known=0.5, seed=2)
    res = O.enmc(X, M, 4, 60)
    assert res.U.min() >= 0.0 and res.V.min() >= 0.0
    tr = np.asarray(res.trace)
    assert tr[-1] < 0.2 * tr[0]
    assert tr[-1] < 0.05 * O.objective_masked(X, M, np.zeros((60, 4)), np.zeros((45, 4)))
