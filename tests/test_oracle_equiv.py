"""Pins of the oracle's equivalence tools (Sec. 5, App. F and App. H).

* generalized_transform (App. F): a pair built as (U_e A, V_e A^-T) for an
  invertible A is recovered exactly (R1 Lambda R2^T = A, zero residuals); a
  component orthogonal to range(U_e) shows up as exactly its norm in delta_u;
  a scaled permutation has Lambda = its sorted scales; R1 and R2 orthogonal.
* permutation_check (App. H): a scaled column permutation is found whole, with
  the inverse permutation; columns replaced by unrelated ones are dropped; the
  1 - eps threshold is applied as stated; the cross-similarity pruning drops a
  candidate whose relations to the other columns changed.
"""
import itertools

import numpy as np
import pytest

from oracle import enmf_oracle as O


def _factors(m, n, r, seed):
    rng = np.random.default_rng(seed)
    U = rng.random((m, r)) * (rng.random((m, r)) > 0.3)
    V = rng.random((n, r)) * (rng.random((n, r)) > 0.3)
    return U, V, rng


def test_transform_recovers_an_invertible_map():
    U, V, rng = _factors(60, 45, 7, 0)
    A = rng.standard_normal((7, 7)) + 3 * np.eye(7)
    g = O.generalized_transform(U, V, U @ A, V @ np.linalg.inv(A).T)
    np.testing.assert_allclose(g.R1 @ np.diag(g.lam) @ g.R2.T, A, atol=1e-11 * np.abs(A).max())
    assert g.delta_u <= 1e-11 * np.linalg.norm(U @ A)
    assert g.delta_v <= 1e-10 * np.linalg.norm(V @ np.linalg.inv(A).T)
    for R in (g.R1, g.R2):
        np.testing.assert_allclose(R.T @ R, np.eye(7), atol=1e-13)
    assert np.all(g.lam > 0) and np.all(np.diff(g.lam) <= 0)


def test_transform_residual_is_the_orthogonal_component():
    U, V, rng = _factors(80, 50, 5, 1)
    A = rng.standard_normal((5, 5)) + 2 * np.eye(5)
    E = rng.standard_normal((80, 5))
    Qb, _ = np.linalg.qr(U)
    E = E - Qb @ (Qb.T @ E)                 # orthogonal to range(U)
    g = O.generalized_transform(U, V, U @ A + E, V @ np.linalg.inv(A).T)
    assert g.delta_u == pytest.approx(float(np.linalg.norm(E)), rel=1e-10)
    assert g.delta_v <= 1e-10 * np.linalg.norm(V)


def test_transform_of_a_scaled_permutation():
    U, V, rng = _factors(40, 30, 4, 2)
    perm = np.array([2, 0, 3, 1])
    s = np.array([0.5, 3.0, 1.5, 0.25])
    A = np.eye(4)[:, perm] * s                # column j of U A = s_j U_(perm_j)
    g = O.generalized_transform(U, V, U @ A, V @ np.linalg.inv(A).T)
    np.testing.assert_allclose(g.lam, np.sort(s)[::-1], rtol=1e-12)
    assert g.delta_u <= 1e-12 * np.linalg.norm(U)


def test_permutation_found_whole():
    U, _, rng = _factors(100, 10, 8, 3)
    perm = rng.permutation(8)
    UB = U[:, perm] * rng.uniform(0.2, 5.0, 8)
    a, b = O.permutation_check(U, UB)
    np.testing.assert_array_equal(a, np.arange(8))
    np.testing.assert_array_equal(b, np.argsort(perm))


def test_unrelated_columns_are_dropped():
    U, _, rng = _factors(200, 10, 10, 4)
    U[0:10, :] = 0.0                         # rows no column of U uses
    perm = rng.permutation(10)
    UB = U[:, perm].copy()
    # two columns of U_B replaced by columns living on those rows only
    UB[:, 3] = 0.0
    UB[:, 7] = 0.0
    UB[0:5, 3] = 1.0
    UB[5:10, 7] = 1.0
    a, b = O.permutation_check(U, UB)
    inv = np.argsort(perm)
    expect = [i for i in range(10) if inv[i] not in (3, 7)]
    np.testing.assert_array_equal(a, expect)
    np.testing.assert_array_equal(b, inv[expect])


def test_threshold_is_one_minus_eps():
    rng = np.random.default_rng(5)
    u = rng.random(500)
    w = rng.random(500)
    w = w - (w @ u) / (u @ u) * u          # orthogonal to u
    w /= np.linalg.norm(w)
    un = u / np.linalg.norm(u)
    for c, found in ((0.951, True), (0.949, False)):
        v = c * un + np.sqrt(1 - c * c) * w   # cos(u, v) = c exactly
        a, _ = O.permutation_check(u[:, None], v[:, None], eps=0.05, keep_frac=0.0)
        assert (len(a) == 1) == found, c


def test_pruning_drops_changed_cross_similarity():
    """Column 0 of U_B is within the cosine threshold of U_A's column 0 but
    leans toward U_A's column 1, so its cosines with the other columns differ
    after rounding: the pruning step drops it (with r = 4, one changed entry
    is already 25 % of a column, so the columns it touches go too)."""
    rng = np.random.default_rng(6)
    r = 4
    Q, _ = np.linalg.qr(rng.standard_normal((300, r)))
    UA = np.abs(Q) + 0.0
    UA /= np.linalg.norm(UA, axis=0)
    UB = UA.copy()
    UB[:, 0] = UA[:, 0] + 0.3 * UA[:, 1]
    c = O._cosines(UA, UB)
    assert c[0, 0] >= 0.95
    a_full, b_full = O.permutation_check(UA, UB, keep_frac=0.0)     # no pruning
    assert 0 in a_full
    a, b = O.permutation_check(UA, UB)
    assert 0 not in a and len(a) < len(a_full)


def test_round1_is_half_up_to_one_decimal():
    np.testing.assert_array_equal(O.round1([0.04, 0.05, 0.96, 1.0, -0.05]), [0, 1, 10, 10, 0])


def test_candidates_are_one_to_one_brute_force():
    """The greedy pairing equals the exhaustive choice of the one-to-one pairs
    above the threshold that takes higher cosines first (r = 4, duplicates in
    U_B compete for one column of U_A)."""
    U, _, rng = _factors(50, 5, 4, 7)
    UB = np.stack([U[:, 1], U[:, 1] * 2.0, U[:, 0], U[:, 3]], axis=1)
    a, b = O.permutation_check(U, UB, keep_frac=0.0)
    c = O._cosines(U, UB)
    best = None
    for perm in itertools.permutations(range(4)):
        sel = sorted((c[i, perm[i]], i, perm[i]) for i in range(4) if c[i, perm[i]] >= 0.95)
        key = sorted([-x[0] for x in sel])
        if best is None or (len(sel), [-k for k in key]) > (len(best[0]), best[1]):
            best = (sel, [-k for k in key])
    assert len(a) == len(best[0])
    for i, j in zip(a, b):
        assert c[i, j] >= 0.95
