"""Pins of the oracle's generalized rotation (Eq. 5, Algorithm 4, App. A.2).

* level set: U V^T = U* V*^T for the output, whatever R1, Lambda, R2 are
  (R2 R2^T = I and Lambda Lambda^-1 = I, App. A.1);
* R1, R2 orthogonal and Lambda > 0 after every run;
* the W1 and W2 closed forms are the minimisers of their ADMM subproblems
  (checked against a least-squares solve of the same quadratic);
* the Lambda update is the minimiser of its one-dimensional objective over
  lambda > 0 (checked against a dense logarithmic grid refined by
  golden-section search);
* scale invariance: scaling (U*, V*) by c leaves R1, Lambda, R2 unchanged
  (rho = gamma = t scale with 1 / RMS(W));
* on a small exact-NMF input (the paper's 50 x 40, r = 10, sparsity 0.1
  example) the negative mass drops by more than two orders of magnitude.
"""
import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O


def _start(m=50, n=40, r=10, seed=0, noise=0.0, zero_frac=0.1):
    X, _, _ = synth.planted(m, n, r, seed=seed, zero_frac=zero_frac, noise=noise)
    Us, Vs, _ = O.truncated_svd(X, r)
    return X, Us, Vs


def test_level_set_orthogonality_and_positive_scales():
    X, Us, Vs = _start(60, 45, 6, seed=1, noise=0.01)
    U, V, R1, lam, R2, info = O.rotate_general(Us, Vs, max_iter=80)
    np.testing.assert_allclose(U @ V.T, Us @ Vs.T, atol=1e-12 * np.abs(Us @ Vs.T).max())
    for R in (R1, R2):
        np.testing.assert_allclose(R.T @ R, np.eye(6), atol=1e-13)
    assert np.all(lam > 0)
    np.testing.assert_allclose(U, Us @ R1 @ np.diag(lam) @ R2, rtol=0, atol=1e-13 * np.abs(U).max())


def test_w1_closed_form_minimises_its_subproblem():
    rng = np.random.default_rng(2)
    m, n, r = 7, 5, 3
    Ws = rng.standard_normal((m + n, r))
    R1, _ = np.linalg.qr(rng.standard_normal((r, r)))
    M, W2, N = (rng.standard_normal((m + n, r)) for _ in range(3))
    lam = rng.uniform(0.3, 2.0, r)
    rho, gamma = 1.7, 0.6
    W1 = O.general_w1_update(Ws, m, R1, M, W2, N, lam, rho, gamma)
    # rho/2 |W1 - Ws R1 + M|^2 + gamma/2 |W2 - [W11 L; W12 L^-1] + N|^2, column by column,
    # as a stacked least-squares problem in each entry's column block
    for blk, sl, sc in ((0, slice(0, m), lam), (1, slice(m, m + n), 1.0 / lam)):
        for j in range(r):
            A = np.vstack([np.sqrt(rho) * np.eye(sl.stop - sl.start),
                           np.sqrt(gamma) * sc[j] * np.eye(sl.stop - sl.start)])
            rhs = np.concatenate([np.sqrt(rho) * (Ws[sl] @ R1 - M[sl])[:, j],
                                  np.sqrt(gamma) * (W2[sl] + N[sl])[:, j]])
            sol = np.linalg.lstsq(A, rhs, rcond=None)[0]
            np.testing.assert_allclose(W1[sl, j], sol, rtol=1e-12, atol=1e-13)


def test_w2_closed_form_minimises_its_subproblem():
    rng = np.random.default_rng(3)
    m, n, r = 6, 4, 3
    W1, N, W3, P = (rng.standard_normal((m + n, r)) for _ in range(4))
    R2, _ = np.linalg.qr(rng.standard_normal((r, r)))
    lam = rng.uniform(0.3, 2.0, r)
    gamma, t = 0.8, 1.9
    W2 = O.general_w2_update(W1, m, N, W3, P, R2, lam, gamma, t)
    # gamma/2 |W2 - [W11 L; W12 L^-1] + N|^2 + t/2 |W3 - W2 R2 + P|^2 over the
    # rows of W2 (vec form, W2 R2 = (R2^T kron I) vec W2, row-major rows)
    for blk, sl, sc in ((0, slice(0, m), lam), (1, slice(m, m + n), 1.0 / lam)):
        for i in range(sl.start, sl.stop):
            A = np.vstack([np.sqrt(gamma) * np.eye(r), np.sqrt(t) * R2.T])
            rhs = np.concatenate([np.sqrt(gamma) * (W1[i] * sc - N[i]),
                                  np.sqrt(t) * (W3[i] + P[i])])
            sol = np.linalg.lstsq(A, rhs, rcond=None)[0]
            np.testing.assert_allclose(W2[i], sol, rtol=1e-12, atol=1e-13)


def _g(lv, w11, w21n, w12, w22n):
    return float(np.sum((w21n - lv * w11) ** 2) + np.sum((w22n - w12 / lv) ** 2))


@pytest.mark.parametrize("seed", range(6))
def test_lambda_is_the_one_dimensional_minimiser(seed):
    rng = np.random.default_rng(10 + seed)
    w11, w21n = rng.standard_normal(9), rng.standard_normal(9)
    w12, w22n = rng.standard_normal(7), rng.standard_normal(7)
    if seed % 2:
        w21n = 2.5 * w11 + 0.1 * w21n   # a clear interior minimum
    lam = O.quartic_lambda(w11, w21n, w12, w22n, 1.0)
    grid = np.exp(np.linspace(np.log(1e-4), np.log(1e4), 200001))
    vals = np.array([_g(x, w11, w21n, w12, w22n) for x in grid[::50]])
    k = int(np.argmin(vals)) * 50
    lo, hi = grid[max(k - 50, 0)], grid[min(k + 50, len(grid) - 1)]
    phi = (np.sqrt(5) - 1) / 2
    a, b = lo, hi
    for _ in range(200):
        c, d = b - phi * (b - a), a + phi * (b - a)
        if _g(c, w11, w21n, w12, w22n) < _g(d, w11, w21n, w12, w22n):
            b = d
        else:
            a = c
    best = 0.5 * (a + b)
    assert _g(lam, w11, w21n, w12, w22n) <= _g(best, w11, w21n, w12, w22n) + 1e-12
    assert lam == pytest.approx(best, rel=1e-6)


def test_scale_invariance():
    X, Us, Vs = _start(40, 30, 5, seed=4, noise=0.02)
    a = O.rotate_general(Us, Vs, max_iter=40)
    b = O.rotate_general(3.0 * Us, 3.0 * Vs, max_iter=40)
    for x, y in zip(a[2:5], b[2:5]):
        np.testing.assert_allclose(x, y, atol=1e-9)


def test_exact_nmf_input_gets_close_to_the_orthant():
    X, Us, Vs = _start()
    U, V, R1, lam, R2, info = O.rotate_general(Us, Vs, max_iter=300)
    before = O.neg_mass(np.vstack([Us, Vs]))
    after = O.neg_mass(np.vstack([U, V]))
    assert after < 1e-2 * before, (before, after)
