"""The equivalence tools (App. F, App. H) on the GPU against the oracle.

enmf_equiv_transform and enmf_perm_check get the same factor matrices as
oracle.generalized_transform and oracle.permutation_check:

* App. F: R1 Lambda R2^T (unique, unlike R1 and R2 themselves, which an SVD
  fixes only up to column signs) and Lambda agree with the oracle's, R1 and
  R2 are orthogonal, and delta_u, delta_v agree; on an equivalent pair (an
  invertible map) and on a pair with a component outside range(U_e);
* App. H: the matched columns are the oracle's, index for index, on a scaled
  permutation, with unrelated columns, and where the pruning step acts.
FP64 factors within 1e-10 (relative); FP32 factors within 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(m, n, r, dt):
    from paper_2605_19325_gb300.solver import Solver
    X = torch.ones(m, n, dtype=dt, device="cuda")
    return Solver(X, r)


def _dev(A, dt):
    return torch.as_tensor(np.ascontiguousarray(A), dtype=dt, device="cuda")


def _np(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
@pytest.mark.parametrize("m,n,r", [(300, 200, 5), (1000, 700, 32), (129, 257, 64)])
def test_transform_matches_oracle(dt, tol, m, n, r):
    from oracle import enmf_oracle as O
    rng = np.random.default_rng(r)
    Ue = rng.random((m, r)) * (rng.random((m, r)) > 0.3) + 0.01
    Ve = rng.random((n, r)) * (rng.random((n, r)) > 0.3) + 0.01
    A = rng.standard_normal((r, r)) + 3 * np.eye(r)
    E = 1e-3 * rng.standard_normal((m, r))
    for Ua, Va in ((Ue @ A, Ve @ np.linalg.inv(A).T), (Ue @ A + E, Ve @ np.linalg.inv(A).T)):
        # the oracle runs on exactly the values the GPU sees
        Ue_, Ve_, Ua_, Va_ = (_np(_dev(M, dt)) for M in (Ue, Ve, Ua, Va))
        g = O.generalized_transform(Ue_, Ve_, Ua_, Va_)
        sv = _ctx(m, n, r, dt)
        R1, lam, R2, du, dv = sv.equiv_transform(_dev(Ua, dt), _dev(Va, dt), _dev(Ue, dt),
                                                 _dev(Ve, dt))
        R1, lam, R2 = _np(R1), _np(lam), _np(R2)
        Z = R1 @ np.diag(lam) @ R2.T
        Zo = g.R1 @ np.diag(g.lam) @ g.R2.T
        assert np.abs(Z - Zo).max() <= tol * np.abs(Zo).max() * 10, np.abs(Z - Zo).max()
        np.testing.assert_allclose(lam, g.lam, rtol=tol * 10)
        for R in (R1, R2):
            assert np.abs(R.T @ R - np.eye(r)).max() <= 1e-12
        scale_u = np.linalg.norm(Ua_)
        assert abs(du - g.delta_u) <= tol * scale_u, (du, g.delta_u)
        assert abs(dv - g.delta_v) <= tol * np.linalg.norm(Va_) * 10, (dv, g.delta_v)
        sv.close()


def _perm_cases():
    rng = np.random.default_rng(11)
    U = rng.random((200, 10)) * (rng.random((200, 10)) > 0.3)
    U[0:10, :] = 0.0
    perm = rng.permutation(10)
    yield "permutation", U, U[:, perm] * rng.uniform(0.2, 5.0, 10)
    UB = U[:, perm].copy()
    UB[:, 3] = 0.0
    UB[:, 7] = 0.0
    UB[0:5, 3] = 1.0
    UB[5:10, 7] = 1.0
    yield "unrelated", U, UB
    Q, _ = np.linalg.qr(rng.standard_normal((300, 4)))
    UA = np.abs(Q)
    UA /= np.linalg.norm(UA, axis=0)
    UB = UA.copy()
    UB[:, 0] = UA[:, 0] + 0.3 * UA[:, 1]
    yield "pruned", UA, UB


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_perm_check_matches_oracle(dt):
    from oracle import enmf_oracle as O
    for name, UA, UB in _perm_cases():
        m, r = UA.shape
        UA_, UB_ = _np(_dev(UA, dt)), _np(_dev(UB, dt))
        a, b = O.permutation_check(UA_, UB_)
        expect = [-1] * r
        for i, j in zip(a, b):
            expect[i] = int(j)
        sv = _ctx(m, r + 8, r, dt)
        got, kept = sv.perm_check(_dev(UB, dt), UA=_dev(UA, dt))
        assert got == expect, (name, got, expect)
        assert kept == len(a)
        sv.close()
