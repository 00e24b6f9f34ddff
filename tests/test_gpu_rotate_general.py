"""The generalized rotation (Eq. 5, Algorithm 4) on the GPU against the oracle.

enmf_rotate_general gets the oracle's own SVD start (FP64 form) and is
compared with oracle.rotate_general on the same start:

* after 1, 5 and 30 ADMM steps (tol = 0, so both run exactly that many):
  R1, Lambda, R2 and the rotated factors within 1e-9;
* with the default stopping rule: the same step count, R1 and R2 orthogonal,
  Lambda > 0, U V^T = U* V*^T to 1e-12, and the negative mass the oracle's;
* the FP32-factor form keeps the level set and orthogonality to FP32 accuracy
  and moves the factors toward the orthant like the oracle.
Shapes include an odd rank (a padded Jacobi column) and the paper's small
exact-NMF example (50 x 40, r = 10, sparsity 0.1).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(60, 45, 6, 0.01), (300, 200, 16, 0.01), (129, 257, 49, 0.01), (50, 40, 10, 0.0)]


def _start(m, n, r, noise, seed=0):
    from oracle import enmf_oracle as O
    X, _, _ = synth.planted(m, n, r, seed=seed, zero_frac=0.1, noise=noise)
    Us, Vs, _ = O.truncated_svd(X, r)
    return X, Us, Vs


def _gpu(X, Us, Vs, r, max_iter, tol, dt=torch.float64):
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    sv = Solver(torch.as_tensor(X, dtype=dt, device="cuda"), r)
    sv.U.copy_(torch.as_tensor(Us, dtype=dt))
    sv.V.copy_(torch.as_tensor(Vs, dtype=dt))
    info, R1, lam, R2 = sv.rotate_general(B.enmf_admm_opts(0.0, 3.0, max_iter, tol))
    out = tuple(t.double().cpu().numpy() for t in (sv.U, sv.V, R1, lam, R2)) + (info,)
    sv.close()
    return out


@pytest.mark.parametrize("m,n,r,noise", SHAPES)
@pytest.mark.parametrize("steps", [1, 5, 30])
def test_general_rotation_steps_match_oracle(m, n, r, noise, steps):
    from oracle import enmf_oracle as O
    X, Us, Vs = _start(m, n, r, noise)
    U, V, R1, lam, R2, info = _gpu(X, Us, Vs, r, steps, 0.0)
    Uo, Vo, R1o, lamo, R2o, io = O.rotate_general(Us, Vs, max_iter=steps, tol=0.0)
    assert info.steps == io.steps == steps
    np.testing.assert_allclose(lam, lamo, rtol=1e-9)
    np.testing.assert_allclose(R1, R1o, atol=1e-9)
    np.testing.assert_allclose(R2, R2o, atol=1e-9)
    np.testing.assert_allclose(U, Uo, atol=1e-9 * np.abs(Uo).max())
    np.testing.assert_allclose(V, Vo, atol=1e-9 * np.abs(Vo).max())


@pytest.mark.parametrize("m,n,r,noise", SHAPES)
def test_general_rotation_default_rule(m, n, r, noise):
    from oracle import enmf_oracle as O
    X, Us, Vs = _start(m, n, r, noise)
    U, V, R1, lam, R2, info = _gpu(X, Us, Vs, r, 200, 1e-12)
    Uo, Vo, R1o, lamo, R2o, io = O.rotate_general(Us, Vs)
    assert info.steps == io.steps
    for R in (R1, R2):
        assert np.abs(R.T @ R - np.eye(r)).max() < 1e-12
    assert np.all(lam > 0)
    P = Us @ Vs.T
    assert np.abs(U @ V.T - P).max() <= 1e-12 * np.abs(P).max()
    nm = O.neg_mass(np.vstack([U, V]))
    nmo = O.neg_mass(np.vstack([Uo, Vo]))
    assert info.neg_mass_out == pytest.approx(nm, rel=1e-9, abs=1e-12)
    assert abs(nm - nmo) <= 1e-6 * O.neg_mass(np.vstack([Us, Vs])) + 1e-12, (nm, nmo)


@pytest.mark.parametrize("m,n,r,noise", SHAPES[:2])
def test_general_rotation_fp32_form(m, n, r, noise):
    from oracle import enmf_oracle as O
    X, Us, Vs = _start(m, n, r, noise)
    U, V, R1, lam, R2, info = _gpu(X, Us, Vs, r, 60, 0.0, torch.float32)
    for R in (R1, R2):
        assert np.abs(R.T @ R - np.eye(r)).max() < 1e-10
    P = Us @ Vs.T
    assert np.abs(U @ V.T - P).max() <= 1e-5 * np.abs(P).max()
    start = O.neg_mass(np.vstack([Us, Vs]))
    nm = O.neg_mass(np.vstack([U, V]))
    _, _, _, _, _, io = O.rotate_general(Us, Vs, max_iter=60, tol=0.0)
    Uo, Vo = O.rotate_general(Us, Vs, max_iter=60, tol=0.0)[:2]
    nmo = O.neg_mass(np.vstack([Uo, Vo]))
    assert nm < start and abs(nm - nmo) <= 1e-2 * start, (start, nm, nmo)
