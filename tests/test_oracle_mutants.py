"""Planted mistakes in the oracle, each caught by a pin (CPU only).

Every case replaces one oracle function with a plausible wrong version: a
dropped term, a wrong sign or index, a transposed operand, an off-by-one, a
wrong rounding rule. It then runs the pins of tests/test_oracle_pins.py that
should notice, and requires at least one of them to fail. The mistakes live
only in this file and only for the duration of one case (monkeypatch); the
oracle itself is untouched.
"""
import math

import numpy as np
import pytest

import test_oracle_pins as P
from oracle import enmf_oracle as O

ORIG = {name: getattr(O, name) for name in (
    "truncated_svd", "prox_h", "procrustes", "rotate", "shift_step", "shift_negative",
    "pbcd", "hals_update", "kkt", "objective", "e4m3_round", "bf16_round", "tile_exponent",
    "quantize_fp8_tiles", "xtu_sharded", "rel_err", "h", "enmf", "e4m3_code", "iterate")}


# ------------------------------------------------------------------ mutants
def svd_unbalanced(X, r):
    """S given to U only (U* = U_r S, V* = V_r) instead of S^(1/2) to both."""
    Ur, s, Vt = np.linalg.svd(X, full_matrices=False)
    Us, Vs = Ur[:, :r] * s[:r], Vt[:r].T.copy()
    flip = (Us.sum(0) + Vs.sum(0)) < 0
    Us[:, flip] *= -1
    Vs[:, flip] *= -1
    return Us, Vs, s


def svd_sign_inverted(X, r):
    Us, Vs, s = ORIG["truncated_svd"](X, r)
    return -Us, -Vs, s


def svd_off_by_one(X, r):
    """Singular triplets 2..r+1 instead of 1..r."""
    Ur, s, Vt = np.linalg.svd(X, full_matrices=False)
    root = np.sqrt(s[1:r + 1])
    Us, Vs = Ur[:, 1:r + 1] * root, Vt[1:r + 1].T * root
    return Us, Vs, s


def prox_half_threshold(b, rho):
    return np.where(b > 0, b, np.where(b >= -0.5 / rho, 0.0, b + 0.5 / rho))


def prox_wrong_sign(b, rho):
    return np.where(b > 0, b, np.where(b >= -1.0 / rho, 0.0, b - 1.0 / rho))


def procrustes_transposed(M):
    return ORIG["procrustes"](M).T


def rotate_identity(Us, Vs, **kw):
    r = Us.shape[1]
    return Us.copy(), Vs.copy(), np.eye(r), O.RotateInfo(steps=0)


def rotate_y_sign(Us, Vs, rho=None, R0=None, Y0=None, max_iter=O.ADMM_MAX_ITER, tol=O.ADMM_TOL):
    """Algorithm 1 with the multiplier update's sign flipped."""
    W = np.vstack([Us, Vs])
    r = W.shape[1]
    rho = rho or O.RHO_SCALE / math.sqrt(float(np.mean(W * W)))
    R, Y = np.eye(r), np.zeros_like(W)
    for _ in range(max_iter):
        Z = O.prox_h(W @ R - Y / rho, rho)
        R = O.procrustes(W.T @ (Z + Y / rho))
        Y = Y - rho * (Z - W @ R)
    return Us @ R, Vs @ R, R, O.RotateInfo(steps=max_iter)


def shift_all_entries(F, s):
    return F + s


def shift_step_more(F, n_shift=O.N_SHIFT):
    return ORIG["shift_step"](F, n_shift + 1)


def pbcd_unsquared_numerator(X, U, V, mask, eps=O.PBCD_EPS, max_iter=O.PBCD_MAX_ITER):
    """d_i = ||g_i|| / ||g_i V^T||^2 (the square on the numerator dropped)."""
    U = np.array(U, dtype=np.float64)
    Mk = mask.astype(np.float64)
    for t in range(max_iter):
        g = Mk * ((U @ V.T - X) @ V)
        num = np.sqrt(np.sum(g * g, axis=1))
        den = np.sum((g @ V.T) ** 2, axis=1)
        d = np.where(den > 0, num / np.where(den > 0, den, 1), 0.0)
        U = np.where(mask, np.maximum(U - d[:, None] * g, 0.0), U)
    return U, O.PbcdInfo(iters=max_iter)


def pbcd_ignores_mask(X, U, V, mask, eps=O.PBCD_EPS, max_iter=O.PBCD_MAX_ITER):
    return ORIG["pbcd"](X, U, V, np.ones_like(mask, dtype=bool), eps, max_iter)


def pbcd_gradient_sign(X, U, V, mask, eps=O.PBCD_EPS, max_iter=O.PBCD_MAX_ITER):
    """Steps along +grad (the gradient of X - U V^T taken with the wrong sign)."""
    return ORIG["pbcd"](-X, -U, V, mask, eps, max_iter)


def hals_no_diagonal(X, U, V):
    """The column update without the division by B_jj."""
    U = np.array(U, dtype=np.float64)
    A, B = X @ V, V.T @ V
    for j in range(U.shape[1]):
        U[:, j] = np.maximum(0.0, U[:, j] + (A[:, j] - U @ B[:, j]))
    return U


def hals_no_floor(X, U, V):
    U = np.array(U, dtype=np.float64)
    A, B = X @ V, V.T @ V
    for j in range(U.shape[1]):
        U[:, j] = U[:, j] + (A[:, j] - U @ B[:, j]) / B[j, j]
    return U


def kkt_wrong_projection(X, U, V):
    """Projected gradient taking max(0, grad) where W = 0."""
    rep = ORIG["kkt"](X, U, V)
    E = U @ V.T - X
    W = np.vstack([U, V])
    G = np.vstack([E @ V, E.T @ U])
    P_ = np.where(W > 0, G, np.maximum(G, 0.0))
    rep.pg_norm = float(np.linalg.norm(P_))
    rep.pg_rel = rep.pg_norm / (np.linalg.norm(X @ V) + np.linalg.norm(X.T @ U))
    return rep


def objective_without_half(X, U, V):
    return 2.0 * ORIG["objective"](X, U, V)


def e4m3_ties_away(v):
    v = np.asarray(v, dtype=np.float64)
    sub = v < 2.0 ** -6
    e = np.floor(np.log2(np.where(sub, 1.0, v)))
    q = np.where(sub, 2.0 ** -9, 2.0 ** (e - 3))
    return np.minimum(np.floor(v / q + 0.5) * q, 448.0)


def e4m3_no_saturation(v):
    v = np.asarray(v, dtype=np.float64)
    out = ORIG["e4m3_round"](np.minimum(v, 448.0))
    return np.where(v > 464.0, v, out)


def bf16_truncate(x32):
    b = np.asarray(x32, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return b.view(np.float32).astype(np.float64)


def tile_exponent_plus_one(amax):
    k = ORIG["tile_exponent"](amax)
    return k + 1 if amax > 0 else k


def fp8_split_no_flush(X32, tile=128):
    """The split without flushing codes below the smallest normal."""
    X32 = np.asarray(X32, dtype=np.float32)
    m, n = X32.shape
    X = X32.astype(np.float64)
    ti, tj = -(-m // tile), -(-n // tile)
    K = np.zeros((ti, tj), dtype=np.int64)
    Q = np.zeros_like(X)
    for I in range(ti):
        for J in range(tj):
            blk = X[I * tile:(I + 1) * tile, J * tile:(J + 1) * tile]
            k = O.tile_exponent(float(blk.max()))
            K[I, J] = k
            Q[I * tile:(I + 1) * tile, J * tile:(J + 1) * tile] = O.e4m3_round(blk * 2.0 ** -k)
    Xh = Q * 2.0 ** np.repeat(np.repeat(K, tile, 0), tile, 1)[:m, :n]
    return O.e4m3_code(Q), K, Xh, O.bf16_round((X - Xh).astype(np.float32))


def fp8_split_unrounded_lo(X32, tile=128):
    """X_lo kept in full precision instead of BF16."""
    codes, K, Xh, _ = ORIG["quantize_fp8_tiles"](X32, tile)
    X = np.asarray(X32, dtype=np.float32).astype(np.float64)
    return codes, K, Xh, X - Xh


def fp8_split_transposed_tiles(X32, tile=128):
    """Tile exponents indexed (J, I) when applied."""
    codes, K, Xh, Xl = ORIG["quantize_fp8_tiles"](X32, tile)
    X = np.asarray(X32, dtype=np.float32).astype(np.float64)
    m, n = X.shape
    if K.shape[0] == K.shape[1]:
        Kt = K.T
    else:
        Kt = np.resize(K.T, K.shape)
    kk = np.repeat(np.repeat(Kt, tile, 0), tile, 1)[:m, :n].astype(float)
    Q = Xh / 2.0 ** np.repeat(np.repeat(K, tile, 0), tile, 1)[:m, :n]
    Xh2 = Q * 2.0 ** kk
    return codes, Kt, Xh2, O.bf16_round((X - Xh2).astype(np.float32))


def xtu_sharded_overlap(X, U, P):
    """Row panels that overlap by one row."""
    bounds = np.linspace(0, X.shape[0], P + 1).astype(int)
    out = np.zeros((X.shape[1], U.shape[1]))
    for p in range(P):
        a, b = max(bounds[p] - 1, 0), bounds[p + 1]
        out = out + X[a:b].T @ U[a:b]
    return out


def kkt_abs_delta(X, U, V):
    """delta as max |grad o W| instead of the signed max of Table 10."""
    rep = ORIG["kkt"](X, U, V)
    E = U @ V.T - X
    W = np.vstack([U, V])
    G = np.vstack([E @ V, E.T @ U])
    rep.delta = float(np.abs(G * W).max())
    return rep


def kkt_gradient_sign(X, U, V):
    """The gradient of X - U V^T instead of U V^T - X."""
    return ORIG["kkt"](-X, -U, V)


def rel_err_squared(X, U, V):
    return 2.0 * O.objective(X, U, V) / float(np.linalg.norm(X)) ** 2


def hals_jacobi(X, U, V):
    """All columns updated from the old U (no Gauss-Seidel sweep)."""
    U0 = np.array(U, dtype=np.float64)
    U = U0.copy()
    A, B = X @ V, V.T @ V
    for j in range(U.shape[1]):
        if B[j, j] > 0:
            U[:, j] = np.maximum(0.0, U0[:, j] + (A[:, j] - U0 @ B[:, j]) / B[j, j])
    return U


def negative_part_sign(q):
    return np.maximum(0.0, q)


def rotate_rho_times_rms(Us, Vs, rho=None, **kw):
    W = np.vstack([Us, Vs])
    rms = math.sqrt(float(np.mean(W * W)))
    return ORIG["rotate"](Us, Vs, rho=O.RHO_SCALE * rms if rho is None else rho, **kw)


def shift_step_from_max(F, n_shift=O.N_SHIFT):
    return float(max(0.0, F.max())) / (n_shift - 0.5)


def enmf_without_rotation(X, r, n_iter, **kw):
    X = O._check(X, r)
    Us, Vs, s = O.truncated_svd(X, r)
    U, V, tr, st = O.iterate(X, Us, Vs, n_iter)
    return O.EnmfResult(U, V, Us, Vs, s, np.eye(r), O.RotateInfo(), tr, st)


def e4m3_code_bias(q):
    c = ORIG["e4m3_code"](q).astype(np.int64)
    return np.where(c >= 8, c + 8, c).astype(np.uint8)


def iterate_v_first(X, U, V, n_iter, state=None, **kw):
    V2, U2, tr, st = ORIG["iterate"](np.asarray(X).T, V, U, n_iter, state, **kw)
    return U2, V2, tr, st


def iterate_hals_first(X, U, V, n_iter, state=None, **kw):
    st = state if state is not None else O.IterState()
    st.stage = "hals"
    return ORIG["iterate"](X, U, V, n_iter, st, **kw)


MUTANTS = [
    ("svd S on U only", "truncated_svd", svd_unbalanced,
     [P.test_svd_start_balanced_factors, P.test_svd_start_rank_one_closed_form]),
    ("svd signs inverted", "truncated_svd", svd_sign_inverted,
     [P.test_svd_sign_rule, P.test_svd_start_rank_one_closed_form]),
    ("svd triplets off by one", "truncated_svd", svd_off_by_one,
     [P.test_svd_start_eckart_young_tail]),
    ("prox threshold halved", "prox_h", prox_half_threshold,
     [P.test_prox_matches_dense_1d_minimisation]),
    ("prox shift sign", "prox_h", prox_wrong_sign, [P.test_prox_matches_dense_1d_minimisation]),
    ("procrustes transposed", "procrustes", procrustes_transposed,
     [P.test_procrustes_matches_brute_force_r2]),
    ("rotation skipped", "rotate", rotate_identity,
     [P.test_rotation_keeps_level_set_and_orthogonality, P.test_rotation_brute_force_r2]),
    ("ADMM multiplier sign", "rotate", rotate_y_sign,
     [P.test_rotation_keeps_level_set_and_orthogonality, P.test_rotation_brute_force_r2]),
    ("shift moves every entry", "shift_negative", shift_all_entries,
     [P.test_shift_step_and_count, P.test_pbcd_decreases_objective_and_keeps_mask,
      P.test_ascent_stage_ends_in_n_shift_iterations]),
    ("shift step one count too small", "shift_step", shift_step_more,
     [P.test_shift_step_and_count, P.test_ascent_stage_ends_in_n_shift_iterations]),
    ("PBCD step numerator unsquared", "pbcd", pbcd_unsquared_numerator,
     [P.test_row_step_matches_line_search]),
    ("PBCD ignores the mask", "pbcd", pbcd_ignores_mask,
     [P.test_pbcd_decreases_objective_and_keeps_mask]),
    ("PBCD gradient sign", "pbcd", pbcd_gradient_sign,
     [P.test_row_step_matches_line_search, P.test_pbcd_decreases_objective_and_keeps_mask]),
    ("HALS without 1/B_jj", "hals_update", hals_no_diagonal,
     [P.test_hals_half_steps_are_monotone, P.test_hals_column_is_exact_nnls_minimiser]),
    ("HALS without the floor", "hals_update", hals_no_floor,
     [P.test_hals_column_is_exact_nnls_minimiser, P.test_enmf_reaches_kkt_point]),
    ("KKT projection at W = 0", "kkt", kkt_wrong_projection, [P.test_enmf_reaches_kkt_point]),
    ("objective without 1/2", "objective", objective_without_half,
     [P.test_svd_start_eckart_young_tail]),
    ("E4M3 ties away from zero", "e4m3_round", e4m3_ties_away,
     [P.test_e4m3_round_is_nearest_with_ties_to_even]),
    ("E4M3 without saturation", "e4m3_round", e4m3_no_saturation,
     [P.test_e4m3_round_is_nearest_with_ties_to_even]),
    ("BF16 truncated", "bf16_round", bf16_truncate,
     [P.test_bf16_round_is_nearest_with_ties_to_even]),
    ("tile exponent one too large", "tile_exponent", tile_exponent_plus_one,
     [P.test_tile_exponent_is_least_power_covering_the_tile,
      P.test_fp8_tile_split_bounds_and_per_tile_scales]),
    ("FP8 split without the subnormal flush", "quantize_fp8_tiles", fp8_split_no_flush,
     [P.test_fp8_tile_split_bounds_and_per_tile_scales]),
    ("FP8 split with X_lo unrounded", "quantize_fp8_tiles", fp8_split_unrounded_lo,
     [P.test_fp8_tile_split_bounds_and_per_tile_scales]),
    ("FP8 split with tile exponents transposed", "quantize_fp8_tiles",
     fp8_split_transposed_tiles, [P.test_fp8_tile_split_bounds_and_per_tile_scales]),
    ("shard panels overlap", "xtu_sharded", xtu_sharded_overlap,
     [P.test_sharded_xtu_is_rank_ordered_sum]),
    ("KKT delta unsigned", "kkt", kkt_abs_delta,
     [P.test_kkt_measures_against_finite_difference_gradient]),
    ("KKT gradient sign", "kkt", kkt_gradient_sign,
     [P.test_kkt_measures_against_finite_difference_gradient]),
    ("relative error squared", "rel_err", rel_err_squared, [P.test_svd_start_eckart_young_tail]),
    ("HALS Jacobi instead of Gauss-Seidel", "hals_update", hals_jacobi,
     [P.test_hals_half_steps_are_monotone, P.test_enmf_reaches_kkt_point]),
    ("negative part sign", "h", negative_part_sign,
     [P.test_rotation_keeps_level_set_and_orthogonality, P.test_rotation_brute_force_r2]),
    ("rho times RMS", "rotate", rotate_rho_times_rms, [P.test_rotation_brute_force_r2]),
    ("shift step from the max", "shift_step", shift_step_from_max,
     [P.test_shift_step_and_count, P.test_ascent_stage_ends_in_n_shift_iterations]),
    ("enmf without the rotation", "enmf", enmf_without_rotation,
     [P.test_enmf_starts_from_the_rotated_svd_and_alternates_u_then_v]),
    ("E4M3 code exponent bias", "e4m3_code", e4m3_code_bias,
     [P.test_e4m3_round_is_nearest_with_ties_to_even]),
    ("V-half before U-half", "iterate", iterate_v_first,
     [P.test_enmf_starts_from_the_rotated_svd_and_alternates_u_then_v]),
    ("HALS before the ascent stage", "iterate", iterate_hals_first,
     [P.test_ascent_stage_ends_in_n_shift_iterations]),
]


@pytest.mark.parametrize("name,attr,fn,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(monkeypatch, name, attr, fn, pins):
    monkeypatch.setattr(O, attr, fn)
    failures = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError,
                IndexError) as e:
            failures.append((pin.__name__, type(e).__name__))
            break
    assert failures, f"planted mistake '{name}' passed every pin in {[p.__name__ for p in pins]}"


# ------------------------- equivalence tools (App. F, H) and Algorithm 4
import test_oracle_equiv as E  # noqa: E402
import test_oracle_general as GR  # noqa: E402

ORIG2 = {name: getattr(O, name) for name in (
    "general_w1_update", "general_w2_update", "quartic_lambda", "generalized_transform",
    "permutation_check", "_cosines", "round1")}


def w1_without_coupling(Ws, m, R1, M, W2, N, lam, rho, gamma):
    """The gamma term (the W2 coupling) dropped from the W1 update."""
    return ORIG2["general_w1_update"](Ws, m, R1, M, W2, N, lam, rho, 0.0)


def w2_scales_swapped(W1, m, N, W3, P, R2, lam, gamma, t):
    """Lambda and Lambda^-1 exchanged between the two blocks."""
    return ORIG2["general_w2_update"](W1, m, N, W3, P, R2, 1.0 / lam, gamma, t)


def w2_without_transpose(W1, m, N, W3, P, R2, lam, gamma, t):
    return ORIG2["general_w2_update"](W1, m, N, W3, P, R2.T, lam, gamma, t)


def quartic_c_sign(w11, w21n, w12, w22n, lam_prev):
    """The V-block cross term enters with the wrong sign."""
    return ORIG2["quartic_lambda"](w11, w21n, -w12, w22n, lam_prev)


def transform_r2_untransposed(Ue, Ve, Ualg, Valg):
    g = ORIG2["generalized_transform"](Ue, Ve, Ualg, Valg)
    return O.GeneralTransform(g.R1, g.lam, g.R2.T, g.delta_u, g.delta_v)


def transform_inverse_map(Ue, Ve, Ualg, Valg):
    """The map of U_alg onto U_e instead of U_e onto U_alg."""
    return ORIG2["generalized_transform"](Ualg, Valg, Ue, Ve)


def perm_without_pruning(UA, UB, eps=0.05, keep_frac=0.9):
    return ORIG2["permutation_check"](UA, UB, eps, 0.0)


def perm_threshold_halved(UA, UB, eps=0.05, keep_frac=0.9):
    return ORIG2["permutation_check"](UA, UB, eps / 2, keep_frac)


def cosines_unnormalised(A, B):
    return A.T @ B


def round1_truncates(x):
    return np.floor(10.0 * np.asarray(x, dtype=np.float64)).astype(np.int64)


MUTANTS2 = [
    ("Algorithm 4 W1 without the W2 coupling", "general_w1_update", w1_without_coupling,
     [GR.test_w1_closed_form_minimises_its_subproblem]),
    ("Algorithm 4 W2 scales swapped", "general_w2_update", w2_scales_swapped,
     [GR.test_w2_closed_form_minimises_its_subproblem]),
    ("Algorithm 4 W2 with R2 instead of R2^T", "general_w2_update", w2_without_transpose,
     [GR.test_w2_closed_form_minimises_its_subproblem]),
    ("Algorithm 4 quartic cross-term sign", "quartic_lambda", quartic_c_sign,
     [lambda: GR.test_lambda_is_the_one_dimensional_minimiser(0),
      lambda: GR.test_lambda_is_the_one_dimensional_minimiser(1)]),
    ("App. F R2 untransposed", "generalized_transform", transform_r2_untransposed,
     [E.test_transform_recovers_an_invertible_map]),
    ("App. F inverse map", "generalized_transform", transform_inverse_map,
     [E.test_transform_recovers_an_invertible_map, E.test_transform_of_a_scaled_permutation]),
    ("App. H without pruning", "permutation_check", perm_without_pruning,
     [E.test_pruning_drops_changed_cross_similarity]),
    ("App. H threshold halved", "permutation_check", perm_threshold_halved,
     [E.test_threshold_is_one_minus_eps]),
    ("App. H cosines unnormalised", "_cosines", cosines_unnormalised,
     [E.test_permutation_found_whole, E.test_threshold_is_one_minus_eps]),
    ("App. H rounding truncates", "round1", round1_truncates,
     [E.test_round1_is_half_up_to_one_decimal]),
]


@pytest.mark.parametrize("name,attr,fn,pins", MUTANTS2, ids=[m[0] for m in MUTANTS2])
def test_planted_mistake_in_the_equivalence_and_general_rotation_is_caught(monkeypatch, name,
                                                                           attr, fn, pins):
    monkeypatch.setattr(O, attr, fn)
    failures = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError,
                IndexError) as e:
            failures.append(type(e).__name__)
            break
    assert failures, f"planted mistake '{name}' passed its pins"


# ------------------------------------------- sparse X and matrix completion
import test_oracle_sparse as SP  # noqa: E402

ORIG3 = {name: getattr(O, name) for name in (
    "csr_dense", "csr_rows_times", "grad_masked", "pbcd_masked", "masked_als")}


def csr_dense_row_shift(m, n, row_ptr, col, val):
    """Entries of row i placed in row i + 1 (row_ptr read one off)."""
    X = ORIG3["csr_dense"](m, n, row_ptr, col, val)
    return np.roll(X, 1, axis=0)


def csr_rows_times_unweighted(row_ptr, col, val, rows, B):
    """Values dropped: the pattern's sum of B rows."""
    return ORIG3["csr_rows_times"](row_ptr, col, np.ones_like(np.asarray(val)), rows, B)


def grad_masked_unmasked(X, M, U, V):
    """The mask dropped from the gradient (unknown entries taken as zeros)."""
    return (U @ V.T - X) @ V


def pbcd_masked_full_denominator(X, M, U, V, mask, eps=O.PBCD_EPS, max_iter=O.PBCD_MAX_ITER):
    """Eq. 10's unmasked denominator g_i V^T V g_i^T kept under the mask."""
    U = np.array(U, dtype=np.float64)
    Mk = np.asarray(mask, dtype=np.float64)
    g = Mk * O.grad_masked(X, M, U, V)
    info = O.PbcdInfo(g0=float(np.linalg.norm(g)))
    for t in range(max_iter):
        num = np.sum(g * g, axis=1)
        den = np.sum((g @ V.T) ** 2, axis=1)
        d = np.where((num > 0) & (den > 0), num / np.where(den > 0, den, 1.0), 0.0)
        U = np.where(Mk > 0, np.maximum(U - d[:, None] * g, 0.0), U)
        g = Mk * O.grad_masked(X, M, U, V)
        info.pg = float(np.linalg.norm(g))
        info.iters = t + 1
        if info.pg < eps * info.g0 or info.pg == 0.0:
            break
    return U, info


def masked_als_unmasked_gram(X, M, r, sweeps=50, lam=1e-9, tol=1e-10):
    """Row least squares with the full Gram V^T V instead of the known
    entries' Gram."""
    U, V, _ = O.truncated_svd(M * X, r)
    k = 0
    for k in range(1, sweeps + 1):
        U = np.linalg.solve(V.T @ V + lam * np.eye(r), V.T @ (M * X).T).T
        V = np.linalg.solve(U.T @ U + lam * np.eye(r), U.T @ (M * X)).T
    return U, V, k


MUTANTS3 = [
    ("compressed rows placed one row down", "csr_dense", csr_dense_row_shift,
     [SP.test_csr_dense_matches_scipy]),
    ("compressed-row product without the values", "csr_rows_times", csr_rows_times_unweighted,
     [SP.test_csr_products_match_scipy]),
    ("App. C gradient without the mask", "grad_masked", grad_masked_unmasked,
     [SP.test_masked_gradient_is_the_derivative]),
    ("masked PBCD with the unmasked step denominator", "pbcd_masked",
     pbcd_masked_full_denominator, [SP.test_masked_step_is_the_exact_line_minimiser]),
    ("masked ALS with the full Gram", "masked_als", masked_als_unmasked_gram,
     [SP.test_masked_als_reaches_a_stationary_point]),
]


@pytest.mark.parametrize("name,attr,fn,pins", MUTANTS3, ids=[m[0] for m in MUTANTS3])
def test_planted_mistake_in_the_sparse_and_completion_oracle_is_caught(monkeypatch, name, attr,
                                                                       fn, pins):
    monkeypatch.setattr(O, attr, fn)
    failures = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError,
                IndexError) as e:
            failures.append(type(e).__name__)
            break
    assert failures, f"planted mistake '{name}' passed its pins"
