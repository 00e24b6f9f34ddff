"""Pins for the FP64 oracle: what the paper and the mathematics fix.

Each test checks the oracle against something other than itself -- a closed
form, an invariant of the method, brute force on a tiny case, or a textbook
special case -- so that a dropped term, a wrong sign or a transposed operand
anywhere in the oracle fails at least one of them (tests/test_oracle_mutants.py
plants such mistakes and checks that they are caught).
"""
import math

import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- SVD start
def test_svd_start_eckart_young_tail():
    """Sec. 4: U* V*^T is the best rank-r approximation; its squared error is
    the sum of the discarded squared singular values (Eckart-Young)."""
    X, r = synth.config_small(0)
    Us, Vs, s = O.truncated_svd(X, r)
    err = np.sum((X - Us @ Vs.T) ** 2)
    assert err == pytest.approx(np.sum(s[r:] ** 2), rel=1e-10)
    # Eq. 1's objective is half the squared error; the relative error of App. D
    # is the error's norm over ||X||_F
    assert O.objective(X, Us, Vs) == pytest.approx(0.5 * np.sum(s[r:] ** 2), rel=1e-10)
    assert O.rel_err(X, Us, Vs) == pytest.approx(
        math.sqrt(np.sum(s[r:] ** 2)) / math.sqrt(np.sum(s ** 2)), rel=1e-10)


def test_svd_start_balanced_factors():
    """U* = U_r S^(1/2), V* = V_r S^(1/2): both Grams equal diag(sigma_1..r)."""
    X, r = synth.config_small(1)
    Us, Vs, s = O.truncated_svd(X, r)
    np.testing.assert_allclose(Us.T @ Us, np.diag(s[:r]), atol=1e-10 * s[0])
    np.testing.assert_allclose(Vs.T @ Vs, np.diag(s[:r]), atol=1e-10 * s[0])
    # the residual is orthogonal to both factor spans
    Rres = X - Us @ Vs.T
    assert np.abs(Rres.T @ Us).max() < 1e-10 * s[0]
    assert np.abs(Rres @ Vs).max() < 1e-10 * s[0]


def test_svd_start_rank_one_closed_form():
    """X = a b^T (a, b > 0): U* = a sqrt(|b|/|a|), V* = b sqrt(|a|/|b|), both >= 0
    after the sign rule (reading R2)."""
    rng = _rng(3)
    a = rng.random(17) + 0.1
    b = rng.random(11) + 0.1
    Us, Vs, s = O.truncated_svd(np.outer(a, b), 1)
    na, nb = np.linalg.norm(a), np.linalg.norm(b)
    np.testing.assert_allclose(Us[:, 0], a * math.sqrt(nb / na), rtol=1e-12)
    np.testing.assert_allclose(Vs[:, 0], b * math.sqrt(na / nb), rtol=1e-12)
    assert s[0] == pytest.approx(na * nb, rel=1e-13)


def test_svd_start_linear_map_to_planted_factors():
    """Sec. 3 / App. A.1: for noise-free X = U0 V0^T, U0 = U* A and
    V0 = V* A^{-T} with A = S^{-1/2} U_r^T U0 (Eq. gen_4)."""
    X, U0, V0 = synth.planted(60, 40, 4, seed=2, zero_frac=0.3, noise=0.0)
    Us, Vs, s = O.truncated_svd(X, 4)
    Ur = Us / np.sqrt(s[:4])
    A = np.diag(s[:4] ** -0.5) @ Ur.T @ U0
    np.testing.assert_allclose(Us @ A, U0, atol=1e-10)
    np.testing.assert_allclose(Vs @ np.linalg.inv(A).T, V0, atol=1e-10)


def test_svd_sign_rule():
    X, r = synth.config_small(0)
    Us, Vs, _ = O.truncated_svd(X, r)
    assert np.all(Us.sum(0) + Vs.sum(0) >= 0)
    # leading pair of a nonnegative matrix is nonnegative (Perron-Frobenius)
    assert Us[:, 0].min() >= -1e-12 and Vs[:, 0].min() >= -1e-12


# ---------------------------------------------------------------- rotation
def test_prox_matches_dense_1d_minimisation():
    """Eq. 7 is the minimiser of h(z) + rho/2 (z - b)^2: compare with a grid."""
    rho = 2.5
    z = np.linspace(-3, 3, 600001)
    for b in [-2.0, -0.7, -0.4, -0.2, 0.0, 0.3, 1.7]:
        obj = np.maximum(0.0, -z) + 0.5 * rho * (z - b) ** 2
        zstar = z[np.argmin(obj)]
        assert O.prox_h(np.array([b]), rho)[0] == pytest.approx(zstar, abs=2e-5)


def test_procrustes_matches_brute_force_r2():
    """R = C D^T minimises ||B - W R||_F over orthogonal R (Sec. 4.1.2):
    compare with a scan over all 2x2 rotations and reflections."""
    rng = _rng(4)
    W = rng.standard_normal((30, 2))
    B = rng.standard_normal((30, 2))
    R = O.procrustes(W.T @ B)
    best = np.inf
    for th in np.linspace(0, 2 * np.pi, 200001):
        c, s = math.cos(th), math.sin(th)
        for Q in (np.array([[c, -s], [s, c]]), np.array([[c, s], [s, -c]])):
            best = min(best, np.sum((B - W @ Q) ** 2))
    assert np.sum((B - W @ R) ** 2) <= best + 1e-8
    np.testing.assert_allclose(R.T @ R, np.eye(2), atol=1e-14)
    # B = W Q0 exactly, Q0 a proper rotation of r = 3: the minimiser is Q0
    # itself (zero residual; not its transpose)
    W3 = rng.standard_normal((30, 3))
    a, b = 0.7, -0.4
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    Q0 = Rz @ Rx
    np.testing.assert_allclose(O.procrustes(W3.T @ (W3 @ Q0)), Q0, atol=1e-12)


def test_rotation_keeps_level_set_and_orthogonality():
    """Eq. 4.4: f(U* R, V* R) = f(U*, V*) for orthogonal R; R^T R = I
    (the paper prints ||R^T R - I|| ~ 0 after the ADMM, App. J tables)."""
    X, r = synth.config_small(0)
    Us, Vs, _ = O.truncated_svd(X, r)
    U, V, R, info = O.rotate(Us, Vs)
    assert np.linalg.norm(R.T @ R - np.eye(r)) < 1e-13
    assert O.objective(X, U, V) == pytest.approx(O.objective(X, Us, Vs), rel=1e-12)
    # the rotation moves toward the orthant
    assert O.neg_mass(np.vstack([U, V])) < 0.05 * O.neg_mass(np.vstack([Us, Vs]))


def _negmass_rot(W, th, refl):
    c, s = math.cos(th), math.sin(th)
    Q = np.array([[c, s], [s, -c]]) if refl else np.array([[c, -s], [s, c]])
    return O.neg_mass(W @ Q)


def _scan_min(W):
    """Grid over theta (rotations and reflections), then golden-section refine."""
    from scipy.optimize import minimize_scalar
    grid = np.linspace(0, 2 * np.pi, 100001)
    step = grid[1] - grid[0]
    best = np.inf
    for f in (0, 1):
        vals = np.array([_negmass_rot(W, t, f) for t in grid])
        t0 = grid[int(np.argmin(vals))]
        res = minimize_scalar(lambda t: _negmass_rot(W, t, f), bounds=(t0 - step, t0 + step),
                              method="bounded", options={"xatol": 1e-14})
        best = min(best, vals.min(), res.fun)
    return best


def test_rotation_brute_force_r2():
    """r = 2: scan theta over rotations and reflections.  ADMM's R is
    orthogonal, so its negative mass cannot beat the scan; on an instance whose
    minimum is 0 (a rotated nonnegative W0) ADMM reaches the orthant."""
    rng = _rng(5)
    W0 = rng.random((80, 2)) * (rng.random((80, 2)) > 0.3)
    th0 = 0.9
    Q0 = np.array([[math.cos(th0), -math.sin(th0)], [math.sin(th0), math.cos(th0)]])
    W = W0 @ Q0.T
    # the minimum 0 is attained at the planted rotation only; the scan comes
    # within its grid spacing of it
    assert _scan_min(W) < 1e-6
    U, V, R, _ = O.rotate(W[:50], W[50:])
    assert O.neg_mass(np.vstack([U, V])) < 1e-9
    # a generic instance: ADMM can be no better than the true minimum
    W = rng.standard_normal((80, 2)) + 0.8
    scan = _scan_min(W)
    U, V, R, _ = O.rotate(W[:40], W[40:])
    nm = O.neg_mass(np.vstack([U, V]))
    assert nm >= scan - 1e-12
    assert nm <= 1.5 * scan + 1e-12


# ---------------------------------------------------------------- ascent
def test_row_step_matches_line_search():
    """Eq. 10 / App. B: one PBCD sweep moves each row to the exact minimiser of
    ||X_i - (U_i - d g_i) V^T||^2 over d (no projection active here)."""
    from scipy.optimize import minimize_scalar
    rng = _rng(6)
    V = rng.random((30, 3))
    Ut = rng.random((5, 3)) + 1.0
    X = Ut @ V.T + 0.01 * rng.random((5, 30))
    U = Ut + 0.05 * rng.standard_normal((5, 3))
    mask = np.ones_like(U, dtype=bool)
    U1, _ = O.pbcd(X, U, V, mask, max_iter=1)
    assert np.all(U1 > 0)          # the projection did not act
    g = (U @ V.T - X) @ V
    for i in range(5):
        res = minimize_scalar(lambda d: np.sum((X[i] - (U[i] - d * g[i]) @ V.T) ** 2),
                              bracket=(0.0, 1e-3), tol=1e-12)
        np.testing.assert_allclose(U1[i], U[i] - res.x * g[i], rtol=1e-9, atol=1e-12)


def test_pbcd_decreases_objective_and_keeps_mask():
    """Alg. 2: masked entries stay >= 0, unmasked (negative) entries are not
    touched, and each row step cannot increase the row objective."""
    rng = _rng(7)
    X = rng.random((40, 30))
    U = rng.standard_normal((40, 4))
    V = rng.random((30, 4))
    U = O.shift_negative(U, 0.1)
    mask = U >= 0
    U1, info = O.pbcd(X, U, V, mask, max_iter=1)
    assert np.all(U1[mask] >= 0)
    np.testing.assert_array_equal(U1[~mask], U[~mask])
    # with no projection active, one step is the exact line minimum per row
    rows_before = np.sum((X - U @ V.T) ** 2, axis=1)
    rows_after = np.sum((X - U1 @ V.T) ** 2, axis=1)
    assert np.all(rows_after <= rows_before * (1 + 1e-14) + 1e-14)


def test_shift_step_and_count():
    """Eq. 8 with reading R5: the worst entry needs exactly N_SHIFT shifts."""
    rng = _rng(8)
    U = rng.standard_normal((50, 5))
    U0 = U.copy()
    s = O.shift_step(U)
    k = 0
    while np.any(U < 0):
        U = O.shift_negative(U, s)
        k += 1
    assert k == O.N_SHIFT
    # Eq. 8 moves the negative entries only: entries that start >= 0 never move
    np.testing.assert_array_equal(U[U0 >= 0], U0[U0 >= 0])


# ---------------------------------------------------------------- HALS
def test_hals_half_steps_are_monotone():
    """Each HALS half-step is an exact block minimisation: f cannot grow."""
    X, r = synth.config_small(2)
    rng = _rng(9)
    U = rng.random((X.shape[0], r))
    V = rng.random((X.shape[1], r))
    f = O.objective(X, U, V)
    for _ in range(20):
        U = O.hals_update(X, U, V)
        f1 = O.objective(X, U, V)
        assert f1 <= f * (1 + 1e-14)
        V = O.hals_update(X.T, V, U)
        f2 = O.objective(X, U, V)
        assert f2 <= f1 * (1 + 1e-14)
        f = f2


def test_hals_column_is_exact_nnls_minimiser():
    """The HALS column update is the closed-form minimiser of f over U_:j >= 0
    with the other columns fixed: brute-force check on one entry."""
    rng = _rng(10)
    X = rng.random((6, 8))
    U = rng.random((6, 3))
    V = rng.random((8, 3))
    U1 = O.hals_update(X, U.copy(), V)
    # only column 0 changes first; check its entries against a 1D scan
    Ucol = U.copy()
    for i in range(6):
        best, bestv = np.inf, None
        for t in np.linspace(0, 3, 30001):
            Ucol[i, 0] = t
            val = np.sum((X[i] - Ucol[i] @ V.T) ** 2)
            if val < best:
                best, bestv = val, t
        assert U1[i, 0] == pytest.approx(bestv, abs=2e-4)


def test_kkt_measures_against_finite_difference_gradient():
    """App. G / Table 10 at a point that is not stationary: the gradient of
    f = 1/2 ||X - U V^T||^2 by central differences (exact up to rounding for a
    quadratic), then delta = max(grad o W) (signed), sigma = sum(grad o W),
    min grad, min W and the projected gradient of reading R11."""
    rng = _rng(12)
    U0 = rng.random((6, 2)) + 0.5
    V0 = rng.random((5, 2)) + 0.5
    X = U0 @ V0.T
    # column 0 of U overshoots and column 1 undershoots the planted factors,
    # so grad o W has both signs and its most negative entry is the largest
    U = U0 * np.array([1.1, 0.3])
    U[0, 0] = 0.0                                   # an entry at the bound
    V = V0.copy()
    h = 1e-3

    def grad(F, which):
        G = np.zeros_like(F)
        for idx in np.ndindex(F.shape):
            Fp, Fm = F.copy(), F.copy()
            Fp[idx] += h
            Fm[idx] -= h
            fp = 0.5 * np.sum((X - (Fp @ V.T if which == 0 else U @ Fp.T)) ** 2)
            fm = 0.5 * np.sum((X - (Fm @ V.T if which == 0 else U @ Fm.T)) ** 2)
            G[idx] = (fp - fm) / (2 * h)
        return G

    W = np.vstack([U, V])
    G = np.vstack([grad(U, 0), grad(V, 1)])
    prod = G * W
    assert prod.max() != np.abs(prod).max()        # the signed max is the one asked for
    P_ = np.where(W > 0, G, np.minimum(G, 0.0))
    rep = O.kkt(X, U, V)
    assert rep.delta == pytest.approx(prod.max(), rel=1e-8)
    assert rep.sigma == pytest.approx(prod.sum(), rel=1e-8)
    assert rep.min_grad == pytest.approx(G.min(), rel=1e-8)
    assert rep.min_w == W.min()
    assert rep.pg_norm == pytest.approx(np.linalg.norm(P_), rel=1e-8)


# ---------------------------------------------------------------- whole method
def test_enmf_starts_from_the_rotated_svd_and_alternates_u_then_v():
    """Algorithm 3: the iteration starts from Algorithm 1's output on the SVD
    start, and one alternation is the U-half (V fixed) then the V-half with
    the new U; in the HALS stage those are the HALS sweeps (Sec. 4.3)."""
    X, r = synth.config_small(0)
    res = O.enmf(X, r, 0)
    Us, Vs, _ = O.truncated_svd(X, r)
    U1, V1, R1, _ = O.rotate(Us, Vs)
    np.testing.assert_allclose(res.U, U1, rtol=0, atol=1e-13)
    np.testing.assert_allclose(res.V, V1, rtol=0, atol=1e-13)
    assert np.linalg.norm(res.R - np.eye(r)) > 1e-3
    rng = _rng(13)
    U = rng.random((X.shape[0], r))
    V = rng.random((X.shape[1], r))
    Ua, Va, tr, st = O.iterate(X, U, V, 1, state=O.IterState(stage="hals"))
    Ub = O.hals_update(X, U, V)
    Vb = O.hals_update(X.T, V, Ub)
    np.testing.assert_array_equal(Ua, Ub)
    np.testing.assert_array_equal(Va, Vb)
    assert tr[0] == O.objective(X, Ub, Vb)


def test_enmf_reaches_kkt_point():
    """App. G, Table 10: at the end of eNMF the KKT conditions hold."""
    X, r = synth.config_small(0)
    res = O.enmf(X, r, 600)
    rep = O.kkt(X, res.U, res.V)
    assert rep.min_w >= 0.0
    assert rep.pg_rel < 1e-6
    assert abs(rep.delta) < 1e-6 * np.linalg.norm(X) ** 2
    # the error is never below the unconstrained optimum (RE_svd >= 1, Fig. 2)
    assert O.objective(X, res.U, res.V) >= O.objective(X, res.Us, res.Vs) * (1 - 1e-12)


@pytest.mark.parametrize("sparsity", [0.3, 0.5])
def test_enmf_recovers_planted_factors(sparsity):
    """Fig. 1B / App. H: on noise-free exact-NMF data with sparsity 0.3-0.5
    eNMF reaches the global minimum and the planted factors up to
    permutation and scale."""
    from scipy.optimize import linear_sum_assignment
    X, U0, V0 = synth.planted(120, 90, 4, seed=0, zero_frac=sparsity, noise=0.0)
    res = O.enmf(X, 4, 1500)
    assert O.rel_err(X, res.U, res.V) < 1e-9
    un = res.U / np.linalg.norm(res.U, axis=0)
    u0 = U0 / np.linalg.norm(U0, axis=0)
    C = un.T @ u0
    ri, ci = linear_sum_assignment(-C)
    assert C[ri, ci].min() > 1 - 1e-9


def test_rank_one_is_perron_pair():
    """r = 1: the sign-fixed SVD start is already nonnegative, so no ascent step
    runs and HALS leaves the optimum in place."""
    X, _ = synth.config_small(3)
    res = O.enmf(X, 1, 5)
    assert res.state.asc_iters == 0
    np.testing.assert_allclose(res.U @ res.V.T, res.Us @ res.Vs.T, rtol=1e-10, atol=1e-12)


def test_ascent_stage_ends_in_n_shift_iterations():
    X, r = synth.config_small(0)
    res = O.enmf(X, r, 30)
    assert res.state.asc_iters == O.N_SHIFT
    assert res.state.hals_iters == 30 - O.N_SHIFT


def test_sharded_xtu_is_rank_ordered_sum():
    rng = _rng(11)
    X = rng.random((37, 23))
    U = rng.random((37, 4))
    for P in (1, 2, 3, 5):
        np.testing.assert_allclose(O.xtu_sharded(X, U, P), X.T @ U, rtol=1e-13)


def test_input_checks():
    with pytest.raises(ValueError):
        O.enmf(-np.ones((4, 4)), 2, 1)
    with pytest.raises(ValueError):
        O.enmf(np.ones((4, 4)), 5, 1)
    X = np.ones((4, 4))
    X[0, 0] = np.nan
    with pytest.raises(ValueError):
        O.enmf(X, 2, 1)


# ---------------------------------------------------------------- FP8 form
def _e4m3_grid():
    """Every nonnegative finite E4M3 value, by code, from the format's
    definition (bias 7, 3 mantissa bits, code 0x7F is NaN)."""
    vals = []
    for code in range(127):
        e, m = code >> 3, code & 7
        vals.append(m * 2.0 ** -9 if e == 0 else 2.0 ** (e - 7) * (1 + m / 8))
    return np.array(vals)


def test_e4m3_round_is_nearest_with_ties_to_even():
    """Brute force over the 127-value grid: the nearest value, ties to the
    even code (= even significand); the grid's ends and codes round-trip."""
    grid = _e4m3_grid()
    assert grid[0] == 0 and grid[1] == 2.0 ** -9 and grid[8] == 2.0 ** -6 and grid[-1] == 448
    assert np.all(np.diff(grid) > 0)
    np.testing.assert_array_equal(O.e4m3_round(grid), grid)
    np.testing.assert_array_equal(O.e4m3_code(grid), np.arange(127, dtype=np.uint8))
    mids = 0.5 * (grid[:-1] + grid[1:])
    even = np.where(np.arange(126) % 2 == 0, grid[:-1], grid[1:])
    np.testing.assert_array_equal(O.e4m3_round(mids), even)
    rng = np.random.default_rng(7)
    v = np.concatenate([rng.uniform(0, 448, 4000), 2.0 ** rng.uniform(-12, 8.8, 4000)])
    d = np.abs(v[:, None] - grid[None, :])
    best = grid[np.argmin(d, axis=1)]
    np.testing.assert_array_equal(O.e4m3_round(v), best)   # no exact ties in random data
    assert np.all(O.e4m3_round(np.array([460.0, 1e6])) == 448)


def test_e4m3_round_matches_torch_cast():
    """Library pin: torch's float8_e4m3fn cast (round to nearest even)."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn")
    rng = np.random.default_rng(8)
    v = np.concatenate([2.0 ** rng.uniform(-11, 8.8, 20000), 0.5 * (_e4m3_grid()[:-1] + _e4m3_grid()[1:])])
    v = v.astype(np.float32).astype(np.float64)
    t = torch.tensor(v, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.e4m3_round(v), t)


def test_bf16_round_is_nearest_with_ties_to_even():
    """Brute force between the two BF16 neighbours of each FP32 value, and
    the library cast of torch."""
    rng = np.random.default_rng(9)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32)
    b = x.view(np.uint32)
    lo = (b & 0xFFFF0000).view(np.float32).astype(np.float64)
    hi_bits = (b & 0xFFFF0000) + 0x10000
    hi = hi_bits.astype(np.uint32).view(np.float32).astype(np.float64)
    xd = x.astype(np.float64)
    dl, dh = np.abs(xd - lo), np.abs(hi - xd)
    lo_even = ((b >> 16) & 1) == 0
    want = np.where(dl < dh, lo, np.where(dh < dl, hi, np.where(lo_even, lo, hi)))
    np.testing.assert_array_equal(O.bf16_round(x), want)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], dtype=np.float32)   # exact midpoints
    np.testing.assert_array_equal(O.bf16_round(ties), [1.0, 1 + 2 ** -6])
    torch = pytest.importorskip("torch")
    t = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16_round(x), t)


def test_tile_exponent_is_least_power_covering_the_tile():
    rng = np.random.default_rng(10)
    for a in np.concatenate([2.0 ** rng.uniform(-60, 60, 300), [448.0, 449.0, 1.0, 0.875]]):
        k = O.tile_exponent(float(a))
        assert a <= 448 * 2.0 ** k and (a > 448 * 2.0 ** (k - 1) or k == O.TILE_K_MIN)
    assert O.tile_exponent(0.0) == O.TILE_K_MIN
    assert O.tile_exponent(448 * 2.0 ** -120) == O.TILE_K_MIN
    with pytest.raises(ValueError):
        O.tile_exponent(448 * 2.0 ** 101)


def test_fp8_tile_split_bounds_and_per_tile_scales():
    """Per tile the scaled maximum lies in (224, 448]; |X - X_hi| <=
    2^-4 max(X, 2^(k-6)) where the code is normal, X < 2^(k-6) where it was
    flushed; X_lo is X - X_hi
    to BF16 (relative 2^-9); tiles of very different magnitude on a ragged,
    non-square X get their own exponents (a transposed tile index fails)."""
    rng = np.random.default_rng(11)
    m, n = 300, 200
    X = rng.random((m, n)) ** 3
    X[:128, 128:] *= 2.0 ** 20          # tile (0, 1)
    X[256:, :128] *= 2.0 ** -30         # tile (2, 0)
    X[128:256, :] *= 0.0                # tile row 1 all zero
    X32 = X.astype(np.float32)
    codes, K, Xh, Xl = O.quantize_fp8_tiles(X32)
    assert K.shape == (3, 2) and codes.shape == (m, n)
    Xd = X32.astype(np.float64)
    for I in range(3):
        for J in range(2):
            blk = Xd[I * 128:(I + 1) * 128, J * 128:(J + 1) * 128]
            if blk.max() > 0:
                assert 224 < blk.max() * 2.0 ** -K[I, J] <= 448
    assert K[1, 0] == K[1, 1] == O.TILE_K_MIN
    assert K[0, 1] - K[0, 0] in (19, 20, 21) and K[0, 0] - K[2, 0] in (29, 30, 31)
    kk = np.repeat(np.repeat(K, 128, 0), 128, 1)[:m, :n].astype(float)
    err = np.abs(Xd - Xh)
    normal = codes >= 8
    # half a quantum: 2^-4 of the binade's start, which for values just
    # under 2^-6 (rounded up to the smallest normal) is 2^(k-6)
    assert np.all(err[normal] <= 2.0 ** -4 * np.maximum(Xd[normal], 2.0 ** (kk[normal] - 6)))
    assert np.all(codes[~normal] == 0) and np.all(Xh[~normal] == 0)
    assert np.all(Xd[~normal] < 2.0 ** (kk[~normal] - 6))
    assert np.all(np.abs(Xd - Xh - Xl) <= 2.0 ** -8 * err)   # BF16: 8 significant bits
    # X_lo is a BF16 number: an FP32 value whose low 16 bits are zero
    Xl32 = Xl.astype(np.float32)
    assert np.array_equal(Xl32.astype(np.float64), Xl)
    assert np.all((Xl32.view(np.uint32) & 0xFFFF) == 0)
    # decoding the codes gives X_hi
    np.testing.assert_array_equal(_e4m3_grid()[codes] * 2.0 ** kk, Xh)
