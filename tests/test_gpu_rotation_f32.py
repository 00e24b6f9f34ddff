"""The FP32-factor rotation (Algorithm 1 in one persistent kernel) against the oracle.

The FP32 forms rotate their SVD start with a different kernel from the FP64
form (FP32 rows, FP64 partial sums of M = W^T B, a scaled Newton-Schulz polar
factor).  Here it gets the oracle's own start, rounded to FP32, and its output
is compared with oracle.rotate on exactly those FP32 values:

* after 1, 4 and 20 ADMM steps R agrees with the oracle's R within 1e-4;
* after the default 200 steps R is orthogonal to FP32 accuracy, U R and V R are
  the start times the returned R, the negative mass is the oracle's within 1 %
  of the start's, and R is within the FP32 rotation's stated gap of 5e-3 of
  the oracle's R.  The test also prints how far the oracle's own R moves when
  rounding of FP32 size is injected into the Procrustes input of every step
  (the ADMM amplifies a difference made at any step).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(300, 200, 5), (500, 400, 16), (700, 600, 32), (900, 700, 49), (1000, 800, 64)]


def _start(m, n, r, seed):
    from oracle import enmf_oracle as O
    X, _, _ = synth.planted(m, n, r, seed=seed, dist="uniform", zero_frac=0.3, noise=0.01)
    Us, Vs, _ = O.truncated_svd(X, r)
    return X, Us.astype(np.float32), Vs.astype(np.float32)


def _gpu_rotate(X, Us, Vs, r, max_iter):
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    sv = Solver(torch.as_tensor(X.astype(np.float32), device="cuda"), r)
    sv.U.copy_(torch.as_tensor(Us))
    sv.V.copy_(torch.as_tensor(Vs))
    info = sv.rotate(B.enmf_admm_opts(0.0, 3.0, max_iter, 1e-12))
    out = (sv.U.double().cpu().numpy(), sv.V.double().cpu().numpy(), sv.R.cpu().numpy(), info)
    sv.close()
    return out


@pytest.mark.parametrize("m,n,r", SHAPES)
@pytest.mark.parametrize("steps", [1, 4, 20])
def test_fp32_rotation_first_steps_match_oracle(m, n, r, steps):
    from oracle import enmf_oracle as O
    X, Us, Vs = _start(m, n, r, seed=r)
    U, V, R, info = _gpu_rotate(X, Us, Vs, r, steps)
    Uo, Vo, Ro, io = O.rotate(Us.astype(np.float64), Vs.astype(np.float64), max_iter=steps)
    assert info.steps == io.steps == steps
    assert info.rho == pytest.approx(io.rho, rel=1e-6)
    # M = W^T B is summed from FP32 products (relative error ~1e-7) and the
    # polar factor amplifies a perturbation of M by up to ~sigma_1 / sigma_r of M
    assert np.abs(R - Ro).max() < 1e-4, np.abs(R - Ro).max()
    scale = np.abs(Uo).max()
    assert np.abs(U - Uo).max() < 1e-4 * scale * np.sqrt(r)


@pytest.mark.parametrize("m,n,r", SHAPES)
def test_fp32_rotation_default_steps_against_oracle(m, n, r, monkeypatch):
    from oracle import enmf_oracle as O
    X, Us, Vs = _start(m, n, r, seed=r)
    U, V, R, info = _gpu_rotate(X, Us, Vs, r, 200)
    U64, V64 = Us.astype(np.float64), Vs.astype(np.float64)
    Uo, Vo, Ro, io = O.rotate(U64, V64)
    # The oracle's own response to rounding of FP32 size made at every step:
    # the same loop with each Procrustes input M multiplied entrywise by
    # 1 + 2^-24 g (g standard normal), three noise seeds.
    exact = O.procrustes
    sens = 0.0
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        monkeypatch.setattr(O, "procrustes",
                            lambda M: exact(M * (1 + 2.0 ** -24 * rng.standard_normal(M.shape))))
        _, _, Rp, _ = O.rotate(U64, V64)
        sens = max(sens, float(np.abs(Rp - Ro).max()))
    monkeypatch.setattr(O, "procrustes", exact)
    assert info.steps == io.steps
    assert np.abs(R.T @ R - np.eye(r)).max() < 2e-6
    # the factors returned are the start times the returned R
    np.testing.assert_allclose(U, U64 @ R, rtol=0, atol=2e-6 * np.abs(U64).max() * np.sqrt(r))
    np.testing.assert_allclose(V, V64 @ R, rtol=0, atol=2e-6 * np.abs(V64).max() * np.sqrt(r))
    err = float(np.abs(R - Ro).max())
    print(f"r={r}: |R - R_oracle| = {err:.2e}, oracle per-step rounding sensitivity {sens:.2e}")
    # The stated gap of the FP32 rotation after the 200 steps: 5e-3 in R.
    # Measured 1.1e-3 (r = 32) and 1.7e-3 (r = 64), 20 to 50 times the
    # oracle's response to FP32-size rounding of M alone; the polar factor's
    # FP32 Newton-Schulz iterations add rounding in directions its own
    # iteration does not correct, and the 200 steps amplify it.
    assert err < max(5e-3, 4 * sens), f"|R - R_oracle| = {err:.2e}, oracle sensitivity {sens:.2e}"
    nm_o = O.neg_mass(np.vstack([Uo, Vo]))
    nm_g = O.neg_mass(np.vstack([U, V]))
    w = O.neg_mass(np.vstack([U64, V64]))
    # the negative mass reached is the oracle's up to 1 % of the start's
    assert abs(nm_g - nm_o) <= 1e-2 * w, (nm_g, nm_o, w, sens)
