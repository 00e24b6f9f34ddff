"""Plain FP64 CPU oracle for the exterior NMF (eNMF) hot path.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
reference the CUDA path is checked against.  Only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and it shares no code with the CUDA kernels.

Convention (App. I): X is m x n and nonnegative, U is m x r, V is n x r and
X ~ U V^T.  All arithmetic is IEEE double.  Library primitives used as steps:
``numpy`` matrix products, ``numpy.linalg.svd`` (the LAPACK SVD),
``numpy.linalg.solve`` (the masked least-squares rows of App. C) and
``numpy.roots`` (the quartic of Algorithm 4).

Sections and equations cited are those of "An Exterior Method for Nonnegative
Matrix Factorization" (ICML 2026).  Where the paper leaves a value open, the
reading taken is named in the function's docstring (readings R1..R12; the
same list is kept with the design notes of the repository).

Parity status: every function below is pinned by a CPU test against a closed
form, an invariant, an independent library or brute force
(tests/test_oracle_pins.py, test_oracle_equiv.py, test_oracle_general.py,
test_oracle_sparse.py), except the
exact ADMM and PBCD trajectories, which the paper does not print; those are
pinned only through their invariants (orthogonality, level-set invariance,
brute force at r = 2, optimal step size by line search).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Defaults for the values the paper leaves open (readings R3..R7).
RHO_SCALE = 3.0         # R3: rho = RHO_SCALE / RMS(W)
ADMM_MAX_ITER = 200     # R4
ADMM_TOL = 1e-12        # R4: stop when ||R_{k+1} - R_k||_F <= ADMM_TOL * sqrt(r)
N_SHIFT = 3             # R5: shift step = max(-U) / (N_SHIFT - 1/2)
PBCD_EPS = 1e-4         # R6
PBCD_MAX_ITER = 5       # R6


def _check(X, r):
    """Input rules of Eq. 1: X finite and nonnegative, 1 <= r <= min(m, n)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim != 2:
        raise ValueError("X must be a matrix")
    if not np.all(np.isfinite(X)) or np.any(X < 0):
        raise ValueError("X must be finite and nonnegative")
    if not (1 <= r <= min(X.shape)):
        raise ValueError("need 1 <= r <= min(m, n)")
    return X


# --------------------------------------------------------------------------
# Eq. 1 and the error measures.
def objective(X, U, V):
    """f(U, V) = 1/2 ||X - U V^T||_F^2 (Eq. 1), with the error matrix formed."""
    E = X - U @ V.T
    return 0.5 * float(np.sum(E * E))


def rel_err(X, U, V):
    """||X - U V^T||_F / ||X||_F (relative error against the data, App. D)."""
    return math.sqrt(2.0 * objective(X, U, V)) / float(np.linalg.norm(X))


# --------------------------------------------------------------------------
# Sec. 4: start from the truncated SVD.
def truncated_svd(X, r):
    """Rank-r truncated SVD start: U* = U_r S_r^(1/2), V* = V_r S_r^(1/2) (Sec. 4).

    Reading R2 (the paper fixes no signs): column j of both factors is negated
    when sum_i U*_ij + sum_i V*_ij < 0, so the leading pair of a nonnegative X
    comes out nonnegative (Perron-Frobenius).
    Returns (U*, V*, sigma) with sigma all singular values, descending.
    """
    Ur, s, Vt = np.linalg.svd(X, full_matrices=False)
    root = np.sqrt(s[:r])
    Us = Ur[:, :r] * root
    Vs = Vt[:r, :].T * root
    flip = (Us.sum(axis=0) + Vs.sum(axis=0)) < 0
    Us[:, flip] *= -1.0
    Vs[:, flip] *= -1.0
    return Us, Vs, s


# --------------------------------------------------------------------------
# Sec. 4.1, Algorithm 1: ADMM rotation toward the orthant.
def h(q):
    """Negative part h(q) = max(0, -q) (Sec. 4.2)."""
    return np.maximum(0.0, -q)


def neg_mass(W):
    """sum_ij h(W_ij): the objective of the rotation problem (Sec. 4.1)."""
    return float(np.sum(h(W)))


def prox_h(b, rho):
    """Z update of Eq. 7: entrywise minimiser of h(z) + rho/2 (z - b)^2."""
    return np.where(b > 0, b, np.where(b >= -1.0 / rho, 0.0, b + 1.0 / rho))


def procrustes(M):
    """R update of Sec. 4.1.2: with M = W^T B = C S D^T, R = C D^T."""
    C, _, Dt = np.linalg.svd(M)
    return C @ Dt


@dataclass
class RotateInfo:
    steps: int = 0
    converged: bool = False
    rho: float = 0.0
    dR: float = 0.0


def rotate(Us, Vs, rho=None, R0=None, Y0=None, max_iter=ADMM_MAX_ITER, tol=ADMM_TOL):
    """Algorithm 1: ADMM for min sum h(Z) s.t. Z = W R, R^T R = I.

    W stacks U* over V* (Eq. w).  One step: Z from Eq. 7 with b = W R - Y/rho;
    R from the Procrustes problem with B = Z + Y/rho; Y <- Y + rho (Z - W R_new).
    The output is (U* R, V* R) with the last R (Algorithm 1 outputs UR, VR).

    Reading R3: R0 = I, Y0 = 0, rho = RHO_SCALE / RMS(W).
    Reading R4: stop when ||R_{k+1} - R_k||_F <= tol * sqrt(r), or after
    max_iter steps.
    """
    W = np.vstack([Us, Vs])
    r = W.shape[1]
    if rho is None:
        rms = math.sqrt(float(np.mean(W * W)))
        rho = RHO_SCALE / rms if rms > 0 else 1.0
    R = np.eye(r) if R0 is None else np.array(R0, dtype=np.float64)
    Y = np.zeros_like(W) if Y0 is None else np.array(Y0, dtype=np.float64)
    info = RotateInfo(rho=rho)
    for k in range(max_iter):
        b = W @ R - Y / rho
        Z = prox_h(b, rho)
        B = Z + Y / rho
        R_new = procrustes(W.T @ B)
        Y = Y + rho * (Z - W @ R_new)
        info.dR = float(np.linalg.norm(R_new - R))
        R = R_new
        info.steps = k + 1
        if info.dR <= tol * math.sqrt(r):
            info.converged = True
            break
    return Us @ R, Vs @ R, R, info


# --------------------------------------------------------------------------
# Sec. 4.2: exterior penalty / ascent stage.
def shift_step(F, n_shift=N_SHIFT):
    """Fixed step rho_u*delta_u of Eq. 8 (reading R5).

    The paper fixes no value.  The step is max(-F) / (n_shift - 1/2): the most
    negative entry turns nonnegative after n_shift shifts, with half a step of
    margin so that the count does not hinge on rounding.  Zero when F >= 0.
    """
    worst = float(max(0.0, -F.min()))
    return worst / (n_shift - 0.5)


def shift_negative(F, s):
    """Eq. 8 / Eq. 9 (negative-entry update): F_ij += s for F_ij < 0."""
    return np.where(F < 0, F + s, F)


@dataclass
class PbcdInfo:
    iters: int = 0
    g0: float = 0.0
    pg: float = 0.0


def pbcd(X, U, V, mask, eps=PBCD_EPS, max_iter=PBCD_MAX_ITER):
    """Algorithm 2 (PBCD) for U with V fixed, M_E = 1.

    Gradient (Sec. 4.2): grad_U f = (U V^T - X) V, masked by M_{U+}.  Each sweep
    updates every row i (rows are independent, so the row loop has no order):
    d_i = ||g_i||^2 / ||g_i V^T||^2 (Eq. 10), U_ij <- (U_ij - d_i g_ij)_+ on the
    mask (Eq. 9 pbcdu).  Stop when the masked gradient norm falls below
    eps * ||grad_init||_F, or after max_iter sweeps.

    Reading R6: d_i = 0 when g_i = 0 or ||g_i V^T|| = 0; the loop also stops
    once the masked gradient is exactly zero (nothing can move).
    """
    U = np.array(U, dtype=np.float64)
    Mk = mask.astype(np.float64)
    g = Mk * ((U @ V.T - X) @ V)
    info = PbcdInfo(g0=float(np.linalg.norm(g)))
    for t in range(max_iter):
        num = np.sum(g * g, axis=1)
        a = g @ V.T
        den = np.sum(a * a, axis=1)
        d = np.where((num > 0) & (den > 0), num / np.where(den > 0, den, 1.0), 0.0)
        step = np.maximum(U - d[:, None] * g, 0.0)
        U = np.where(mask, step, U)
        g = Mk * ((U @ V.T - X) @ V)
        info.pg = float(np.linalg.norm(g))
        info.iters = t + 1
        if info.pg < eps * info.g0 or info.pg == 0.0:
            break
    return U, info


# --------------------------------------------------------------------------
# Sec. 4.3: descent by HALS (Cichocki & Phan 2009), stated as mathematics.
def hals_update(X, U, V):
    """One HALS sweep over the columns of U with V fixed.

    With A = X V and B = V^T V, for j = 1..r in order:
    U_:j <- max(0, U_:j + (A_:j - U B_:j) / B_jj), using the columns already
    updated.  Reading R7: floor 0; a column with B_jj = 0 is left unchanged.
    """
    U = np.array(U, dtype=np.float64)
    A = X @ V
    B = V.T @ V
    for j in range(U.shape[1]):
        if B[j, j] <= 0.0:
            continue
        U[:, j] = np.maximum(0.0, U[:, j] + (A[:, j] - U @ B[:, j]) / B[j, j])
    return U


# --------------------------------------------------------------------------
# Algorithm 3: the eNMF iteration after the rotation.
@dataclass
class IterState:
    """Resumable state of Algorithm 3's loops: stage, fixed shift steps, count."""
    stage: str = "asc"          # "asc" (lines 5-11) or "hals" (line 12)
    s_u: float | None = None
    s_v: float | None = None
    k: int = 0
    asc_iters: int = 0
    hals_iters: int = 0
    pbcd_iters: list = field(default_factory=list)


def iterate(X, U, V, n_iter, state=None, eps=PBCD_EPS, pbcd_max_iter=PBCD_MAX_ITER,
            n_shift=N_SHIFT, trace_every=1):
    """Run n_iter alternations of Algorithm 3 from (U, V).

    An alternation (reading R9) is one U-half and one V-half: in the ascent
    stage (while U or V has a negative entry) a shift (Eq. 8 / 9), the mask
    M_+ = [F >= 0] and PBCD for U, then the same for V with X^T; once both are
    nonnegative, a HALS sweep of U then of V.  The objective of Eq. 1 is
    recorded after every V-half (reading R10).  Following Algorithm 3 the HALS
    descent starts only after the ascent loop ends (reading R8).
    Returns (U, V, trace, state).
    """
    X = np.asarray(X, dtype=np.float64)
    U = np.array(U, dtype=np.float64)
    V = np.array(V, dtype=np.float64)
    st = state if state is not None else IterState()
    trace = []
    for _ in range(n_iter):
        if st.stage == "asc" and not (np.any(U < 0) or np.any(V < 0)):
            st.stage = "hals"
        if st.stage == "asc":
            if st.s_u is None:
                st.s_u = shift_step(U, n_shift)
                st.s_v = shift_step(V, n_shift)
            U = shift_negative(U, st.s_u)
            U, iu = pbcd(X, U, V, U >= 0, eps, pbcd_max_iter)
            V = shift_negative(V, st.s_v)
            V, iv = pbcd(X.T, V, U, V >= 0, eps, pbcd_max_iter)
            st.pbcd_iters.append((iu.iters, iv.iters))
            st.asc_iters += 1
        else:
            U = hals_update(X, U, V)
            V = hals_update(X.T, V, U)
            st.hals_iters += 1
        st.k += 1
        if trace_every and (st.k % trace_every == 0):
            trace.append(objective(X, U, V))
    return U, V, np.asarray(trace), st


# --------------------------------------------------------------------------
# App. G: KKT conditions.
@dataclass
class KktReport:
    min_w: float
    min_grad: float
    delta: float       # max(grad_W * W), Table 10
    sigma: float       # sum(grad_W * W), Table 10
    pg_norm: float     # ||P(grad)||_F, projected gradient
    pg_rel: float      # pg_norm / (||XV|| + ||U V^T V|| + ||X^T U|| + ||V U^T U||)


def kkt(X, U, V):
    """KKT measures of App. G for f of Eq. 1.

    grad_U = (U V^T - X) V and grad_V = (U V^T - X)^T U; W stacks U over V.
    delta_W = max(grad_W * W) and sigma_W = sum(grad_W * W) as in Table 10.
    The projected gradient P takes grad_ij where W_ij > 0 and min(0, grad_ij)
    where W_ij = 0 (zero exactly at a KKT point); reading R11 scales its norm
    by the norms of the four terms of the gradient so that it is scale free.
    """
    E = U @ V.T - X
    GU = E @ V
    GV = E.T @ U
    W = np.vstack([U, V])
    G = np.vstack([GU, GV])
    prod = G * W
    P = np.where(W > 0, G, np.minimum(G, 0.0))
    pg = float(np.linalg.norm(P))
    scale = (np.linalg.norm(X @ V) + np.linalg.norm(U @ (V.T @ V))
             + np.linalg.norm(X.T @ U) + np.linalg.norm(V @ (U.T @ U)))
    return KktReport(min_w=float(W.min()), min_grad=float(G.min()),
                     delta=float(prod.max()), sigma=float(prod.sum()),
                     pg_norm=pg, pg_rel=pg / scale if scale > 0 else 0.0)


# --------------------------------------------------------------------------
# Algorithm 3 end to end.
@dataclass
class EnmfResult:
    U: np.ndarray
    V: np.ndarray
    Us: np.ndarray
    Vs: np.ndarray
    sigma: np.ndarray
    R: np.ndarray
    rot: RotateInfo
    trace: np.ndarray
    state: IterState


def enmf(X, r, n_iter, **kw):
    """Algorithm 3: SVD start, Algorithm 1 rotation, ascent loop, then HALS."""
    X = _check(X, r)
    Us, Vs, s = truncated_svd(X, r)
    rk = {k: kw[k] for k in ("rho", "max_iter", "tol") if k in kw}
    U, V, R, rinfo = rotate(Us, Vs, **rk)
    ik = {k: kw[k] for k in ("eps", "pbcd_max_iter", "n_shift") if k in kw}
    U, V, trace, st = iterate(X, U, V, n_iter, **ik)
    return EnmfResult(U, V, Us, Vs, s, R, rinfo, trace, st)


# --------------------------------------------------------------------------
# Row sharding of the V-half (rows of X split over P ranks).
def xtu_sharded(X, U, P):
    """X^T U as the rank-ordered sum of P row-panel partials X_p^T U_p.

    The U-half is row-local (Sec. 4.2: rows do not interact), so row panels
    can live on different ranks; only the n x r partials of X^T U (and the
    r x r partials of U^T U) need a sum across ranks.  Summed in rank order.
    """
    bounds = np.linspace(0, X.shape[0], P + 1).astype(int)
    out = np.zeros((X.shape[1], U.shape[1]))
    for p in range(P):
        a, b = bounds[p], bounds[p + 1]
        out = out + X[a:b].T @ U[a:b]
    return out


# --------------------------------------------------------------------------
# Reduced-precision storage of X (the precision forms; no counterpart in the
# paper, which computes in one precision throughout).  Plain definitions of
# the number formats, written from their published specifications, on
# float64 numbers that hold every value involved exactly.
E4M3_MAX = 448.0             # OCP FP8 E4M3 ("fn"): largest finite value
E4M3_MIN_NORMAL = 2.0 ** -6  # exponent field 1
E4M3_QUANTUM_SUB = 2.0 ** -9  # spacing of the subnormals (exponent field 0)
TILE_K_MIN, TILE_K_MAX = -100, 100   # limits of the tile scale exponent


def e4m3_round(v):
    """Nearest E4M3 value to each v >= 0, ties to the even significand,
    values beyond 448 saturated to 448.  E4M3 has 3 mantissa bits and
    exponent bias 7: normal values 2^(e-7) (1 + m/8), e = 1..15 (e = 15 only
    up to m = 6), subnormals m 2^-9."""
    v = np.asarray(v, dtype=np.float64)
    if np.any(v < 0) or not np.all(np.isfinite(v)):
        raise ValueError("e4m3_round takes finite v >= 0")
    out = np.zeros_like(v)
    sub = v < E4M3_MIN_NORMAL
    # spacing of the grid at v: 2^(floor(log2 v) - 3) in the normal range
    e = np.floor(np.log2(np.where(sub, 1.0, v)))
    # floor(log2) of a float64 power-of-two boundary is exact; guard anyway
    e = np.where(2.0 ** e > v, e - 1, e)
    e = np.where(2.0 ** (e + 1) <= v, e + 1, e)
    quantum = np.where(sub, E4M3_QUANTUM_SUB, 2.0 ** (e - 3))
    out = np.rint(v / quantum) * quantum       # np.rint: half to even
    return np.minimum(out, E4M3_MAX)


def e4m3_code(q):
    """The 8-bit code (sign 0) of each E4M3 value q >= 0."""
    q = np.asarray(q, dtype=np.float64)
    code = np.zeros(q.shape, dtype=np.int64)
    sub = q < E4M3_MIN_NORMAL
    code[sub] = np.rint(q[sub] / E4M3_QUANTUM_SUB).astype(np.int64)
    qn = q[~sub]
    e = np.floor(np.log2(qn)).astype(np.int64)
    m = np.rint((qn / 2.0 ** e - 1.0) * 8).astype(np.int64)
    code[~sub] = ((e + 7) << 3) | m
    return code.astype(np.uint8)


def bf16_round(x32):
    """BF16 of FP32 values (the upper 16 bits of the FP32 pattern), round to
    nearest, ties to even; returned as float64."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def tile_exponent(amax):
    """Least k with amax <= 448 * 2^k, at least TILE_K_MIN (0 maps to it)."""
    if amax <= 0:
        return TILE_K_MIN
    k = math.ceil(math.log2(amax / E4M3_MAX))
    while E4M3_MAX * 2.0 ** (k - 1) >= amax:
        k -= 1
    while E4M3_MAX * 2.0 ** k < amax:
        k += 1
    if k > TILE_K_MAX:
        raise ValueError("entry beyond 448 * 2^100")
    return max(k, TILE_K_MIN)


def quantize_fp8_tiles(X32, tile=128):
    """The FP8 form's split of FP32 X, per tile x tile block (I, J):
    k_IJ = tile_exponent(max of the block); q = e4m3_round(x 2^-k) with
    values below the smallest normal (2^-6) set to 0; X_hi = q 2^k;
    X_lo = bf16(x - X_hi).  Returns (codes uint8, k int array, X_hi, X_lo),
    the last two float64."""
    X32 = np.asarray(X32, dtype=np.float32)
    m, n = X32.shape
    X = X32.astype(np.float64)
    if np.any(X < 0) or not np.all(np.isfinite(X)):
        raise ValueError("X must be finite and nonnegative")
    ti, tj = -(-m // tile), -(-n // tile)
    K = np.zeros((ti, tj), dtype=np.int64)
    Q = np.zeros_like(X)
    for I in range(ti):
        for J in range(tj):
            blk = X[I * tile:(I + 1) * tile, J * tile:(J + 1) * tile]
            k = tile_exponent(float(blk.max()))
            K[I, J] = k
            q = e4m3_round(blk * 2.0 ** -k)
            q[q < E4M3_MIN_NORMAL] = 0.0
            Q[I * tile:(I + 1) * tile, J * tile:(J + 1) * tile] = q
    scale = 2.0 ** np.repeat(np.repeat(K, tile, 0), tile, 1)[:m, :n]
    X_hi = Q * scale
    X_lo = bf16_round((X - X_hi).astype(np.float32))
    return e4m3_code(Q), K, X_hi, X_lo


# --------------------------------------------------------------------------
# Equivalence of two factorisations (Sec. 5, App. F and App. H).
def _cosines(A, B):
    """cos(A_i, B_j) for all column pairs; a zero column has cosine 0."""
    na = np.linalg.norm(A, axis=0)
    nb = np.linalg.norm(B, axis=0)
    G = A.T @ B
    den = np.outer(na, nb)
    return np.where(den > 0, G / np.where(den > 0, den, 1.0), 0.0)


@dataclass
class GeneralTransform:
    R1: np.ndarray
    lam: np.ndarray      # diagonal of Lambda, descending
    R2: np.ndarray
    delta_u: float       # ||U_alg - U_e R1 Lambda R2^T||_F
    delta_v: float       # ||V_alg - V_e R1 Lambda^-1 R2^T||_F


def generalized_transform(Ue, Ve, Ualg, Valg):
    """App. F: R1, Lambda, R2 with U_alg ~ U_e R1 Lambda R2^T and
    V_alg ~ V_e R1 Lambda^-1 R2^T.

    With the thin SVD U_e = P Gamma Q^T, the matrix Z = Q Gamma^-1 P^T U_alg
    (the least-squares map from U_e to U_alg) has the SVD Z = R1 Lambda R2^T;
    the residuals measure how far (U_alg, V_alg) is from such a transform of
    (U_e, V_e) (zero when the two factorisations are equivalent, Sec. 5).
    """
    P, g, Qt = np.linalg.svd(Ue, full_matrices=False)
    Z = Qt.T @ np.diag(1.0 / g) @ P.T @ Ualg
    R1, lam, R2t = np.linalg.svd(Z)
    R2 = R2t.T
    du = float(np.linalg.norm(Ualg - Ue @ R1 @ np.diag(lam) @ R2.T))
    dv = float(np.linalg.norm(Valg - Ve @ R1 @ np.diag(1.0 / lam) @ R2.T))
    return GeneralTransform(R1, lam, R2, du, dv)


def round1(x):
    """Rounding to one decimal place, as the integer k with k / 10 the
    rounded value: floor(10 x + 1/2) (reading of App. H; the paper names no
    tie rule)."""
    return np.floor(10.0 * np.asarray(x, dtype=np.float64) + 0.5).astype(np.int64)


def permutation_check(UA, UB, eps=0.05, keep_frac=0.9):
    """App. H: the columns of U_B that are scaled permutations of columns of U_A.

    Step 1 (candidates): column i of U_A pairs with the column j of U_B of
    largest cos(U_A^(i), U_B^(j)) when that cosine is >= 1 - eps.  Reading: the
    pairs are one to one, taken greedily in decreasing cosine (ties by lower
    i, then lower j).
    Step 2 (cross-similarity pruning): on the candidate columns (in the order
    of U_A's indices) M = cos(U_Asub, U_Asub), N = cos(U_Bsub, U_Bsub) and
    S = cos(U_Asub, U_Bsub); each column of the three is sorted in descending
    order and rounded to one decimal (round1); candidate c is kept when the
    entries of M's column c equal those of N's and S's column c at more than
    keep_frac of the positions.  Reading: every candidate is judged on the
    initial candidate set and the rejected ones are removed together.
    Returns (a_idx, b_idx): the kept pairs, in increasing a_idx.
    """
    S0 = _cosines(UA, UB)
    r = S0.shape[0]
    order = sorted(((S0[i, j], i, j) for i in range(r) for j in range(S0.shape[1])),
                   key=lambda t: (-t[0], t[1], t[2]))
    used_a, used_b, pairs = set(), set(), []
    for c, i, j in order:
        if c < 1.0 - eps:
            break
        if i in used_a or j in used_b:
            continue
        used_a.add(i)
        used_b.add(j)
        pairs.append((i, j))
    pairs.sort()
    if not pairs:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    a = np.array([p[0] for p in pairs])
    b = np.array([p[1] for p in pairs])
    M = round1(-np.sort(-_cosines(UA[:, a], UA[:, a]), axis=0))
    N = round1(-np.sort(-_cosines(UB[:, b], UB[:, b]), axis=0))
    S = round1(-np.sort(-_cosines(UA[:, a], UB[:, b]), axis=0))
    keep = [c for c in range(len(a))
            if np.mean((M[:, c] == N[:, c]) & (M[:, c] == S[:, c])) > keep_frac]
    return a[keep], b[keep]


# --------------------------------------------------------------------------
# App. A.2, Eq. 5, Algorithm 4: the generalized rotation U* R1 Lambda R2.
def quartic_lambda(w11, w21n, w12, w22n, lam_prev):
    """Lambda update of Algorithm 4 for one column: the minimiser over
    lambda > 0 of g(l) = |w21n - l w11|^2 + |w22n - w12 / l|^2, where w21n =
    W21(:,i) + N1(:,i) and w22n = W22(:,i) + N2(:,i).  g'(l) = 0 is the
    quartic a l^4 - b l^3 + c l - d = 0 with a = |w11|^2, b = w21n . w11,
    c = w22n . w12, d = |w12|^2 (App. A.2).  Reading: of its positive real
    roots (numpy's companion-matrix roots, imaginary part below 1e-9 of the
    magnitude), the one with the smallest g; lam_prev when there is none
    (a zero column)."""
    a = float(w11 @ w11)
    b = float(w21n @ w11)
    c = float(w22n @ w12)
    d = float(w12 @ w12)
    if not (a > 0.0 and d > 0.0):
        return lam_prev
    roots = np.roots([a, -b, 0.0, c, -d])
    cand = [z.real for z in roots if abs(z.imag) <= 1e-9 * max(abs(z), 1e-300) and z.real > 0.0]
    if not cand:
        return lam_prev

    def g(lv):
        return float(np.sum((w21n - lv * w11) ** 2) + np.sum((w22n - w12 / lv) ** 2))
    return min(cand, key=g)


def general_w1_update(Ws, m, R1, M, W2, N, lam, rho, gamma):
    """W1 = [W11; W12] of Algorithm 4 (closed forms of App. A.2, per column j):
    W11 = (rho (U* R1 - M1) + gamma lambda_j (W21 + N1)) / (rho + gamma lambda_j^2),
    W12 = (rho (V* R1 - M2) + (gamma / lambda_j) (W22 + N2)) / (rho + gamma / lambda_j^2).
    Rows 0..m-1 are the U block, the rest the V block."""
    W1 = np.empty_like(Ws)
    W1[:m] = (rho * (Ws[:m] @ R1 - M[:m]) + gamma * lam * (W2[:m] + N[:m])) / (rho + gamma * lam ** 2)
    W1[m:] = (rho * (Ws[m:] @ R1 - M[m:]) + (gamma / lam) * (W2[m:] + N[m:])) / (
        rho + gamma / lam ** 2)
    return W1


def general_w2_update(W1, m, N, W3, P, R2, lam, gamma, t):
    """W2 = [W21; W22] of Algorithm 4 (closed forms of App. A.2):
    W21 = (gamma W11 Lambda - gamma N1 + t (W31 + P1) R2^T) / (gamma + t),
    W22 = (gamma W12 Lambda^-1 - gamma N2 + t (W32 + P2) R2^T) / (gamma + t)."""
    W2 = np.empty_like(W1)
    W2[:m] = (gamma * W1[:m] * lam - gamma * N[:m] + t * (W3[:m] + P[:m]) @ R2.T) / (gamma + t)
    W2[m:] = (gamma * W1[m:] / lam - gamma * N[m:] + t * (W3[m:] + P[m:]) @ R2.T) / (gamma + t)
    return W2


@dataclass
class GeneralRotateInfo:
    steps: int = 0
    converged: bool = False
    rho: float = 0.0
    change: float = 0.0


def rotate_general(Us, Vs, rho=None, max_iter=ADMM_MAX_ITER, tol=ADMM_TOL):
    """Algorithm 4: ADMM for Eq. 5 -- orthogonal R1, R2 and diagonal Lambda > 0
    with U* R1 Lambda R2 and V* R1 Lambda^-1 R2 as close to the nonnegative
    orthant as the heuristic gets (App. A.2).

    Splitting (App. A.2): W1 = W_svd R1, W2 = [W11 Lambda; W12 Lambda^-1],
    W3 = W2 R2, with scaled duals M, N, P.  One step, in the order of
    Algorithm 4:
      W3 = prox(W2 R2 - P) with threshold 1/t (the Eq. 7 form);
      W11, W12 from their closed forms (per column j, with lambda_j);
      R1 = polar(W_svd^T (W1 + M));  W21, W22 from their closed forms;
      R2 = polar(W2^T (W3 + P));  each lambda_i from its quartic;
      M += W1 - W_svd R1;  N += W2 - [W11 Lambda; W12 Lambda^-1];
      P += W3 - W2 R2.
    Readings: R1 = R2 = I, Lambda = I, W1 = W2 = W3 = W_svd and zero duals at
    the start; rho = gamma = t = RHO_SCALE / RMS(W_svd) (the scale-free choice
    of Algorithm 1); stop when |R1 - R1'| + |R2 - R2'| + |lambda - lambda'|
    <= tol sqrt(r), or after max_iter steps.  Eq. 5 writes R2 where App. A.1
    writes R2^T; both are orthogonal, and this follows Eq. 5 and Algorithm 4
    (W3 = W2 R2).  Returns (U* R1 Lambda R2, V* R1 Lambda^-1 R2, R1, lambda,
    R2, info).
    """
    Us = np.asarray(Us, dtype=np.float64)
    Vs = np.asarray(Vs, dtype=np.float64)
    m, r = Us.shape
    Ws = np.vstack([Us, Vs])
    if rho is None:
        rms = math.sqrt(float(np.mean(Ws * Ws)))
        rho = RHO_SCALE / rms if rms > 0 else 1.0
    gamma = t = rho
    R1 = np.eye(r)
    R2 = np.eye(r)
    lam = np.ones(r)
    W1 = Ws.copy()
    W2 = Ws.copy()
    W3 = Ws.copy()
    M = np.zeros_like(Ws)
    N = np.zeros_like(Ws)
    P = np.zeros_like(Ws)
    info = GeneralRotateInfo(rho=rho)
    for k in range(max_iter):
        R1o, R2o, lamo = R1, R2, lam.copy()
        # f1: W3 and W1
        W3 = prox_h(W2 @ R2 - P, t)
        W1 = general_w1_update(Ws, m, R1, M, W2, N, lam, rho, gamma)
        # f2: R1 and W2
        R1 = procrustes(Ws.T @ (W1 + M))
        W2 = general_w2_update(W1, m, N, W3, P, R2, lam, gamma, t)
        # f3: R2 and Lambda
        R2 = procrustes(W2.T @ (W3 + P))
        lam = np.array([quartic_lambda(W1[:m, i], W2[:m, i] + N[:m, i], W1[m:, i],
                                       W2[m:, i] + N[m:, i], lam[i]) for i in range(r)])
        # duals
        M = M + W1 - Ws @ R1
        N[:m] = N[:m] + W2[:m] - W1[:m] * lam
        N[m:] = N[m:] + W2[m:] - W1[m:] / lam
        P = P + W3 - W2 @ R2
        info.change = float(np.linalg.norm(R1 - R1o) + np.linalg.norm(R2 - R2o)
                            + np.linalg.norm(lam - lamo))
        info.steps = k + 1
        if info.change <= tol * math.sqrt(r):
            info.converged = True
            break
    T1 = R1 * lam          # R1 Lambda
    T2 = R1 / lam          # R1 Lambda^-1
    return Us @ T1 @ R2, Vs @ T2 @ R2, R1, lam, R2, info


# --------------------------------------------------------------------------
# Sparse X (Sec. 5, the Reuters experiment): X given by its stored entries in
# compressed-row form -- row_ptr (m + 1), col and val (nnz), the entries of
# row i at positions row_ptr[i] .. row_ptr[i+1] - 1 with strictly increasing
# columns.  The method is Algorithm 3 on the matrix these entries define;
# only the products X V and X^T U touch the entries.
def csr_dense(m, n, row_ptr, col, val):
    """The m x n matrix with X[i, col[p]] = val[p] for the stored entries of
    row i and zeros elsewhere."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    X = np.zeros((m, n))
    X[rows, np.asarray(col, dtype=np.int64)] = np.asarray(val, dtype=np.float64)
    return X


def csr_rows_times(row_ptr, col, val, rows, B):
    """(X B)[i, :] for each listed row i, summed over row i's stored entries:
    sum_p val[p] B[col[p], :]."""
    B = np.asarray(B, dtype=np.float64)
    out = np.zeros((len(rows), B.shape[1]))
    for t, i in enumerate(rows):
        a, b = int(row_ptr[i]), int(row_ptr[i + 1])
        c = np.asarray(col[a:b], dtype=np.int64)
        out[t] = np.asarray(val[a:b], dtype=np.float64) @ B[c]
    return out


def csr_cols_times(row_ptr, col, val, cols, B):
    """(X^T B)[j, :] for each listed column j: sum over the stored entries
    (i, j) of val B[i, :]."""
    B = np.asarray(B, dtype=np.float64)
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    out = np.zeros((len(cols), B.shape[1]))
    for t, j in enumerate(cols):
        sel = col == j
        out[t] = val[sel] @ B[rows[sel]]
    return out


def csr_sumsq(val):
    """||X||_F^2 from the stored entries."""
    v = np.asarray(val, dtype=np.float64)
    return float(v @ v)


# --------------------------------------------------------------------------
# Matrix completion (App. C, Algorithm eNMC): only the entries in the mask
# M_E (here: the stored entries of a compressed-row pattern, M_E[i, j] = 1
# for a stored (i, j)) are known.
def objective_masked(X, M, U, V):
    """f^(U, V) = 1/2 ||M_E o (X - U V^T)||_F^2 (App. C)."""
    E = M * (X - U @ V.T)
    return 0.5 * float(np.sum(E * E))


def grad_masked(X, M, U, V):
    """grad_U f^ = (M_E o (U V^T - X)) V (App. C); grad_V is the same with
    X^T, M_E^T and the factors swapped."""
    return (M * (U @ V.T - X)) @ V


def pbcd_masked(X, M, U, V, mask, eps=PBCD_EPS, max_iter=PBCD_MAX_ITER):
    """Algorithm 2 with the mask M_E (App. C): PBCD on U's rows, V fixed.

    g = M_U+ o ((M_E o (U V^T - X)) V).  Reading (the paper changes only the
    gradients): the row step is the exact minimiser of the masked objective
    along -g_i, d_i = ||g_i||^2 / sum_j M_E[i, j] (g_i . v_j)^2, which is
    Eq. 10 when M_E is all ones; d_i = 0 for a zero numerator or denominator.
    U_i <- max(0, U_i - d_i g_i) on the mask; stop when ||g|| < eps ||g_init||
    or after max_iter sweeps (or at an exactly zero gradient).
    """
    U = np.array(U, dtype=np.float64)
    Mk = np.asarray(mask, dtype=np.float64)
    g = Mk * grad_masked(X, M, U, V)
    info = PbcdInfo(g0=float(np.linalg.norm(g)))
    for t in range(max_iter):
        num = np.sum(g * g, axis=1)
        den = np.sum(M * (g @ V.T) ** 2, axis=1)
        d = np.where((num > 0) & (den > 0), num / np.where(den > 0, den, 1.0), 0.0)
        step = np.maximum(U - d[:, None] * g, 0.0)
        U = np.where(Mk > 0, step, U)
        g = Mk * grad_masked(X, M, U, V)
        info.pg = float(np.linalg.norm(g))
        info.iters = t + 1
        if info.pg < eps * info.g0 or info.pg == 0.0:
            break
    return U, info


def masked_als(X, M, r, sweeps=50, lam=1e-3, tol=1e-10):
    """Unconstrained start of Algorithm eNMC: App. C computes a local minimum
    of f^ over all U, V with softImpute-ALS.  Reading: alternating exact
    row least squares with softImpute's ridge,
        u_i = (sum_j M_E[i, j] v_j v_j^T + lam c I)^-1 sum_j M_E[i, j] x_ij v_j
    (c = mean of the Gram's diagonal, 1 when it is 0; lam = 1e-3, the paper
    states no value), then the same for V, from the balanced truncated SVD of
    the zero-filled X; stop when f^ changes by <= tol relative or after
    `sweeps` sweeps.  A row with fewer known entries than r has a singular
    Gram, and without a ridge of this size its solution is fixed only by
    rounding (a 1e-13 change of the start moves U V^T by up to 36 % after 20
    sweeps at lam = 1e-9, by 1e-10 at lam = 1e-3).  Returns (U, V, sweeps_run)."""
    Xz = M * X
    U, V, _ = truncated_svd(Xz, r)
    f_old = objective_masked(X, M, U, V)
    k = 0
    for k in range(1, sweeps + 1):
        for side in (0, 1):
            F, G, Xs, Ms = (U, V, X, M) if side == 0 else (V, U, X.T, M.T)
            Fn = np.empty_like(F)
            for i in range(F.shape[0]):
                sel = Ms[i] > 0
                Gi = G[sel].T @ G[sel]
                c = float(np.trace(Gi)) / r if Gi.size else 0.0
                A = Gi + lam * (c if c > 0 else 1.0) * np.eye(r)
                Fn[i] = np.linalg.solve(A, G[sel].T @ Xs[i, sel])
            if side == 0:
                U = Fn
            else:
                V = Fn
        f = objective_masked(X, M, U, V)
        if abs(f_old - f) <= tol * abs(f):
            break
        f_old = f
    return U, V, k


@dataclass
class EnmcResult:
    U: np.ndarray
    V: np.ndarray
    trace: list
    sweeps: int


def enmc(X, M, r, n_iter, eps=PBCD_EPS, pbcd_max_iter=PBCD_MAX_ITER, n_shift=N_SHIFT,
         als_sweeps=50):
    """Algorithm eNMC (App. C): the masked-ALS start, Algorithm 1's rotation
    (unchanged), then n_iter rounds of: shift U's negative entries (Eq. 8),
    mask, PBCD on U with M_E; the same for V.  Shift steps as in Algorithm 3
    (reading R5: fixed at the first round with a negative entry).  trace: f^
    after every round."""
    X = np.asarray(X, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    U0, V0, sw = masked_als(X, M, r, sweeps=als_sweeps)
    U, V, _, _ = rotate(U0, V0)
    U, V, trace = enmc_rounds(X, M, U, V, n_iter, eps, pbcd_max_iter, n_shift)
    return EnmcResult(U, V, trace, sw)


def enmc_rounds(X, M, U, V, n_iter, eps=PBCD_EPS, pbcd_max_iter=PBCD_MAX_ITER, n_shift=N_SHIFT):
    """The loop of Algorithm eNMC from (U, V): the shift steps fixed from the
    given factors (reading R5), then n_iter rounds of shift, mask and masked
    PBCD on U, then on V.  Returns (U, V, trace of f^ after every round)."""
    U = np.array(U, dtype=np.float64)
    V = np.array(V, dtype=np.float64)
    su = shift_step(U, n_shift) if np.any(U < 0) else 0.0
    sv = shift_step(V, n_shift) if np.any(V < 0) else 0.0
    trace = []
    for _ in range(n_iter):
        U = shift_negative(U, su)
        U, _ = pbcd_masked(X, M, U, V, (U >= 0).astype(np.float64), eps, pbcd_max_iter)
        V = shift_negative(V, sv)
        V, _ = pbcd_masked(X.T, M.T, V, U, (V >= 0).astype(np.float64), eps, pbcd_max_iter)
        trace.append(objective_masked(X, M, U, V))
    return U, V, trace
