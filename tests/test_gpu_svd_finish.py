"""The SVD start's fp32_finish option (FP32 factors).

With fp32_finish = 1 the start is made from the FP32 Jacobi SVD of the last
Rayleigh-Ritz matrix instead of that SVD finished by FP64 sweeps.  Both are
the same truncated SVD up to the FP32 Jacobi's stopping tolerance (pair
cosines below 4e-5 at l = 42): the singular values agree to that level and
the rank-r products U V^T (a rotation-free quantity) to it as well, and both
stay within the oracle's truncated SVD by the same margin.  FP64 factors
ignore the option.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _start(X, r, finish, dtype):
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    s = Solver(torch.as_tensor(X.astype(dtype), device="cuda"), r)
    tol = 1e-12 if dtype == np.float64 else 1e-5
    s.svd_init(B.enmf_svd_opts(10, 40, tol, 0x5eed, finish))
    U, V = s.U.double().cpu().numpy(), s.V.double().cpu().numpy()
    sig = s.sigma.cpu().numpy().copy() if getattr(s, "sigma", None) is not None else None
    s.close()
    return U, V, sig


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(600, 400, 32), (300, 900, 12), (200, 170, 64)])
def test_fp32_finish_start_matches_the_fp64_finished_one(shape):
    m, n, r = shape
    X, _, _ = synth.planted(m, n, r, seed=3, dist="uniform", zero_frac=0.3, noise=0.01)
    U0, V0, s0 = _start(X, r, 0, np.float32)
    U1, V1, s1 = _start(X, r, 1, np.float32)
    P0, P1 = U0 @ V0.T, U1 @ V1.T
    scale = np.linalg.norm(P0)
    assert np.linalg.norm(P1 - P0) <= 1e-4 * scale
    # both against the exact truncated SVD of X (FP64)
    u, s, vt = np.linalg.svd(X, full_matrices=False)
    Pt = (u[:, :r] * s[:r]) @ vt[:r]
    e0 = np.linalg.norm(P0 - Pt) / scale
    e1 = np.linalg.norm(P1 - Pt) / scale
    assert e1 <= max(2 * e0, 1e-4), (e0, e1)
    if s0 is not None and s1 is not None:
        np.testing.assert_allclose(s1, s0, rtol=1e-4)


@pytest.mark.gpu
def test_fp64_factors_ignore_fp32_finish():
    X, _, _ = synth.planted(300, 200, 8, seed=4, dist="uniform", zero_frac=0.3, noise=0.01)
    U0, V0, _ = _start(X, 8, 0, np.float64)
    U1, V1, _ = _start(X, 8, 1, np.float64)
    assert np.array_equal(U0, U1) and np.array_equal(V0, V1)
