"""GPU path vs the FP64 oracle, through the C ABI.

Tolerances: the plain FP64 path must match the oracle's per-iteration
objective to 1e-10 relative; factors element-wise to 1e-9 relative to their
largest entry.  The FP32 form states its error gap to the FP64 oracle.
Discrete decisions (stage switch, PBCD sweep counts) must agree exactly.
"""
import math

import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


def _solver(X, r, dtype=torch.float64):
    from paper_2605_19325_gb300.solver import Solver
    Xt = torch.as_tensor(np.ascontiguousarray(X), dtype=dtype, device="cuda")
    return Solver(Xt, r)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _np(t):
    return t.detach().double().cpu().numpy()


def _set(s, U, V):
    s.U.copy_(torch.as_tensor(U, dtype=s.U.dtype))
    s.V.copy_(torch.as_tensor(V, dtype=s.V.dtype))


# ------------------------------------------------------------------ stages
@pytest.mark.parametrize("shape", [(200, 150, 5), (257, 131, 7), (60, 500, 12), (300, 200, 64)])
def test_svd_start_matches_oracle(shape):
    m, n, r = shape
    X, _, _ = synth.planted(m, n, r, seed=3, zero_frac=0.3, noise=0.01)
    Us, Vs, s = O.truncated_svd(X, r)
    sv = _solver(X, r)
    info = sv.svd_init()
    assert info.residual <= 1e-12
    np.testing.assert_allclose(_np(sv.sigma), s[:r], rtol=1e-12)
    assert _rel(_np(sv.U), Us) < 1e-9
    assert _rel(_np(sv.V), Vs) < 1e-9


def test_rotation_matches_oracle():
    X, r = synth.config_small(0)
    Us, Vs, _ = O.truncated_svd(X, r)
    U, V, R, info = O.rotate(Us, Vs)
    sv = _solver(X, r)
    _set(sv, Us, Vs)
    gi = sv.rotate()
    assert gi.steps == info.steps
    assert gi.rho == pytest.approx(info.rho, rel=1e-13)
    assert _rel(_np(sv.R), R) < 1e-9
    assert _rel(_np(sv.U), U) < 1e-9
    assert _rel(_np(sv.V), V) < 1e-9
    assert gi.neg_mass_out == pytest.approx(O.neg_mass(np.vstack([U, V])), rel=1e-8, abs=1e-12)
    Rg = _np(sv.R)
    # one-sided Jacobi stops when every column cosine is below 1e-15 * max(r, 8),
    # which bounds ||R^T R - I||_F by about r times that
    assert np.linalg.norm(Rg.T @ Rg - np.eye(r)) < 1e-15 * max(r, 8) * r * 4


def test_iterate_trace_matches_oracle():
    X, r = synth.config_small(0)
    Us, Vs, _ = O.truncated_svd(X, r)
    U0, V0, _, _ = O.rotate(Us, Vs)
    Uo, Vo, tr, st = O.iterate(X, U0, V0, 200)
    sv = _solver(X, r)
    _set(sv, U0, V0)
    gtr, info = sv.iterate(200, reset=1)
    assert info.asc_iters == st.asc_iters and info.hals_iters == st.hals_iters
    assert sv.pbcd_counts() == st.pbcd_iters
    assert info.s_u == pytest.approx(st.s_u, rel=1e-14)
    rel = np.abs(_np(gtr) - tr) / np.abs(tr)
    assert rel.max() < OBJ_TOL, rel.max()
    assert _rel(_np(sv.U), Uo) < 1e-9
    assert _rel(_np(sv.V), Vo) < 1e-9


def _pipeline_parity(X, r, n_iter, tol=OBJ_TOL):
    res = O.enmf(X, r, n_iter)
    sv = _solver(X, r)
    sv.svd_init()
    sv.rotate()
    gtr, info = sv.iterate(n_iter, reset=1)
    assert info.asc_iters == res.state.asc_iters
    rel = np.abs(_np(gtr) - res.trace) / np.abs(res.trace)
    assert rel.max() < tol, rel.max()
    return sv, res


def test_full_pipeline_matches_oracle_small():
    X, r = synth.config_small(0)
    _pipeline_parity(X, r, 200)


@pytest.mark.parametrize("shape", [(257, 131, 7), (33, 400, 3), (500, 37, 5), (1000, 700, 16)])
def test_full_pipeline_matches_oracle_ragged(shape):
    """Whole pipeline on ragged shapes.  The SVD start and the rotation agree
    with the oracle to ~1e-13; the ascent stage then amplifies any difference
    of the start by a factor that depends on the input.  The bar is therefore
    the oracle's own conditioning: its trace under a perturbation of the
    rotated start as large as the measured GPU-oracle difference, times 10
    (and never looser than it needs to be: at least 1e-10 is always allowed)."""
    m, n, r = shape
    X, _, _ = synth.planted(m, n, r, seed=7, zero_frac=0.3, noise=0.01)
    n_iter = 60
    res = O.enmf(X, r, n_iter)
    U0, V0 = res.Us @ res.R, res.Vs @ res.R
    sv = _solver(X, r)
    sv.svd_init()
    sv.rotate()
    delta = max(_rel(_np(sv.U), U0), _rel(_np(sv.V), V0))
    assert delta < 1e-9
    rng = np.random.default_rng(0)
    scale_u, scale_v = np.abs(U0).max(), np.abs(V0).max()
    Up = U0 + delta * scale_u * rng.uniform(-1, 1, U0.shape)
    Vp = V0 + delta * scale_v * rng.uniform(-1, 1, V0.shape)
    _, _, tr_p, _ = O.iterate(X, Up, Vp, n_iter)
    self_sens = float(np.max(np.abs(tr_p - res.trace) / np.abs(res.trace)))
    gtr, info = sv.iterate(n_iter, reset=1)
    assert info.asc_iters == res.state.asc_iters
    rel = np.abs(_np(gtr) - res.trace) / np.abs(res.trace)
    assert rel.max() < max(OBJ_TOL, 10 * self_sens), (rel.max(), self_sens, delta)
    # both runs end at the same point of the HALS descent
    assert rel[-1] < max(OBJ_TOL, 10 * self_sens)


@pytest.mark.parametrize("shape", [(1, 40, 1), (40, 1, 1), (2, 2, 2), (64, 64, 1)])
def test_degenerate_shapes(shape):
    m, n, r = shape
    rng = np.random.default_rng(1)
    X = rng.random((m, n)) + 0.1
    res = O.enmf(X, r, 20)
    sv = _solver(X, r)
    sv.svd_init()
    sv.rotate()
    gtr, _ = sv.iterate(20, reset=1)
    rel = np.abs(_np(gtr) - res.trace) / np.maximum(np.abs(res.trace), 1e-300)
    assert rel.max() < 1e-9 or np.abs(_np(gtr) - res.trace).max() < 1e-12 * np.sum(X * X)


def test_residual_and_kkt_match_oracle():
    X, r = synth.config_small(1)
    sv, res = _pipeline_parity(X, r, 100)
    U, V = _np(sv.U), _np(sv.V)
    f_d, rel_d, nx = sv.residual(direct=True)
    f_e, rel_e, _ = sv.residual(direct=False)
    assert f_d == pytest.approx(O.objective(X, U, V), rel=1e-12)
    assert f_e == pytest.approx(O.objective(X, U, V), rel=1e-9)
    assert rel_d == pytest.approx(O.rel_err(X, U, V), rel=1e-12)
    assert nx == pytest.approx(float(np.sum(X * X)), rel=1e-13)
    g = sv.kkt()
    o = O.kkt(X, U, V)
    scale = float(np.linalg.norm(X)) ** 2
    assert g.min_w == o.min_w
    assert g.min_grad == pytest.approx(o.min_grad, abs=1e-10 * scale)
    assert g.delta == pytest.approx(o.delta, abs=1e-10 * scale)
    assert g.sigma == pytest.approx(o.sigma, abs=1e-10 * scale)
    assert g.pg_norm == pytest.approx(o.pg_norm, rel=1e-6, abs=1e-10 * scale)
    assert g.pg_rel == pytest.approx(o.pg_rel, rel=1e-6, abs=1e-14)


# ------------------------------------------------------- method properties
def test_kkt_at_convergence_on_gpu():
    X, r = synth.config_small(0)
    sv = _solver(X, r)
    sv.svd_init()
    sv.rotate()
    sv.iterate(600, reset=1)
    g = sv.kkt()
    assert g.min_w >= 0.0
    assert g.pg_rel < 1e-6


def test_planted_recovery_on_gpu():
    from scipy.optimize import linear_sum_assignment
    X, U0, V0 = synth.planted(120, 90, 4, seed=0, zero_frac=0.3, noise=0.0)
    sv = _solver(X, 4)
    sv.svd_init()
    sv.rotate()
    sv.iterate(1500, reset=1)
    _, rel, _ = sv.residual()
    assert rel < 1e-9
    U = _np(sv.U)
    C = (U / np.linalg.norm(U, axis=0)).T @ (U0 / np.linalg.norm(U0, axis=0))
    ri, ci = linear_sum_assignment(-C)
    assert C[ri, ci].min() > 1 - 1e-9


def test_resume_equals_single_call_and_is_deterministic():
    X, r = synth.config_small(2)
    runs = []
    for split in (False, True):
        sv = _solver(X, r)
        sv.svd_init()
        sv.rotate()
        if split:
            t1, _ = sv.iterate(70, reset=1)
            t2, _ = sv.iterate(50)
            tr = torch.cat([t1, t2])
        else:
            tr, _ = sv.iterate(120, reset=1)
        runs.append((_np(tr), _np(sv.U), _np(sv.V)))
    for a, b in zip(runs[0], runs[1]):
        np.testing.assert_array_equal(a, b)


def test_negative_input_is_rejected():
    from paper_2605_19325_gb300 import binding as B
    X, r = synth.config_small(0)
    X = X.copy()
    X[3, 4] = -1.0
    sv = _solver(X, r)
    with pytest.raises(B.EnmfError) as ei:
        sv.residual()
    assert ei.value.code == 2


# ---------------------------------------------------------- FP32 form
def test_fp32_form_error_gap():
    """FP32 X and factors: the final relative error stays within 1e-3 (relative)
    of the FP64 oracle's, and the trace follows it closely."""
    X, r = synth.config_small(0)
    res = O.enmf(X, r, 200)
    sv = _solver(X, r, dtype=torch.float32)
    sv.svd_init()
    sv.rotate()
    gtr, _ = sv.iterate(200, reset=1)
    _, rel, _ = sv.residual()
    ref = O.rel_err(X, res.U, res.V)
    assert abs(rel - ref) / ref < 1e-3
    # The trace is the Gram expansion 1/2|X|^2 - <X^T U, V> + 1/2 <U^T U, V^T V>
    # with FP32 cross terms: its error is about the FP32 unit roundoff times
    # the cancellation factor |X|^2 / f, so that is the bar (8 units).
    t = _np(gtr)
    tol = 8 * 2.0 ** -24 * float(np.sum(X * X)) / res.trace[-20:]
    assert np.all(np.abs(t[-20:] - res.trace[-20:]) / res.trace[-20:] < tol)


# ------------------------------------------------- full-size, sampled
def test_dense_config_full_size_sampled_rows():
    """8192 x 6144, r = 32 (the dense planted workload): one HALS alternation
    on the GPU from its own state, checked row by row against the oracle's
    update on sampled rows (the oracle cannot run the whole size quickly)."""
    X, r = synth.config_dense(0)
    sv = _solver(X, r)
    sv.svd_init()
    sv.rotate()
    tr, info = sv.iterate(20, reset=1)
    t = _np(tr)
    assert np.all(np.isfinite(t))
    hals = t[info.asc_iters:]
    assert np.all(np.diff(hals) <= 1e-12 * hals[:-1])
    U0, V0 = _np(sv.U), _np(sv.V)
    sv.iterate(1)
    U1, V1 = _np(sv.U), _np(sv.V)
    rows = np.random.default_rng(0).choice(X.shape[0], 12, replace=False)
    G = V0.T @ V0
    for i in rows:
        a = X[i] @ V0
        u = U0[i].copy()
        for j in range(r):
            if G[j, j] > 0:
                u[j] = max(0.0, u[j] + (a[j] - u @ G[:, j]) / G[j, j])
        np.testing.assert_allclose(U1[i], u, rtol=1e-9, atol=1e-12 * np.abs(U1).max())
    cols = np.random.default_rng(1).choice(X.shape[1], 12, replace=False)
    Gu = U1.T @ U1
    for j0 in cols:
        a = X[:, j0] @ U1
        v = V0[j0].copy()
        for j in range(r):
            if Gu[j, j] > 0:
                v[j] = max(0.0, v[j] + (a[j] - v @ Gu[:, j]) / Gu[j, j])
        np.testing.assert_allclose(V1[j0], v, rtol=1e-9, atol=1e-12 * np.abs(V1).max())
