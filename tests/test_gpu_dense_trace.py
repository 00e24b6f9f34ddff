"""The dense planted workload at full size (8192 x 6144, r = 32) against the oracle.

The oracle's results for this workload are stored in
tests/golden/dense_8192x6144_r32.json (written by make_dense_trace.py beside
it, which calls only the oracle): the top singular values, sampled rows of the
rotated start and of the final factors, and f of Eq. 1 after each of the 500
alternations of Algorithm 3.  The plain FP64 GPU form runs the whole pipeline
(SVD start, Algorithm 1, ascent stage, HALS) from X and is compared with it:

* sigma to 1e-12 relative;
* the rotated start's sampled rows: their largest relative difference
  delta_gpu is the start difference the GPU run carries into the iteration;
* the objective trace, alternation by alternation, to 1e-10 relative, or -- the
  iteration amplifying start differences -- to 10 x the oracle's own trace
  response to a start perturbation of that size (the stored sensitivity at
  1e-9 of the SVD start, scaled by delta_gpu over the rotated-start
  difference that perturbation made); the assertion message reports both;
* the same ascent-stage length.

The BF16 precision form on the same matrix states its final relative-error gap
to the oracle's final value, which must be within 1e-3.
"""
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "dense_8192x6144_r32.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def X64():
    X, r = synth.config_dense(0)
    return X


def _rowdiff(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)))


def test_dense_fp64_trace_against_the_oracle(golden, X64):
    from paper_2605_19325_gb300.solver import Solver
    r = 32
    sv = Solver(torch.as_tensor(X64, device="cuda"), r)
    sv.svd_init()
    sig = sv.sigma.cpu().numpy()
    np.testing.assert_allclose(sig, golden["sigma"], rtol=1e-12)
    sv.rotate()
    ri, rj = golden["rows_i"], golden["rows_j"]
    U = sv.U.cpu().numpy()
    V = sv.V.cpu().numpy()
    delta_gpu = max(_rowdiff(U[ri], golden["rotated_U_rows"]),
                    _rowdiff(V[rj], golden["rotated_V_rows"]))
    tr, info = sv.iterate(golden["n_iter"], reset=1)
    t = tr.cpu().numpy()
    ref = np.asarray(golden["trace"])
    rel = np.abs(t - ref) / ref
    # the oracle's trace response per unit of rotated-start difference, from
    # its own run with a perturbed start
    sens = golden["max_rel_sensitivity"] * max(delta_gpu, 1e-15) / \
        golden["rotated_rows_difference_perturbed"]
    bar = max(1e-10, 10 * sens)
    msg = (f"max rel trace diff {rel.max():.3e} (at alternation {int(rel.argmax())}); "
           f"start difference {delta_gpu:.2e}; oracle sensitivity {golden['max_rel_sensitivity']:.2e} "
           f"at {golden['delta']:.0e} -> bar {bar:.2e}")
    print(msg)
    assert info.asc_iters == golden["asc_iters"], msg
    assert rel.max() < bar, msg
    U1 = sv.U.cpu().numpy()
    V1 = sv.V.cpu().numpy()
    fin = max(_rowdiff(U1[ri], golden["final_U_rows"]), _rowdiff(V1[rj], golden["final_V_rows"]))
    # the final factors move with the start like the oracle's own do
    fbar = max(1e-9, 10 * golden["final_rows_difference_perturbed"] *
               max(delta_gpu, 1e-15) / golden["rotated_rows_difference_perturbed"])
    assert fin < fbar, (fin, fbar, msg)
    sv.close()


def test_dense_bf16_form_final_gap(golden, X64):
    from paper_2605_19325_gb300.solver import Solver
    r = 32
    X32 = torch.as_tensor(X64.astype(np.float32), device="cuda")
    sv = Solver(X32, r, x_stream=torch.bfloat16)
    sv.svd_init()
    sv.rotate()
    sv.iterate(golden["n_iter"], trace=False, reset=1)
    _, rel, _ = sv.residual()
    gap = abs(rel - golden["rel_err_final"]) / golden["rel_err_final"]
    print(f"BF16 form: final rel. error {rel:.9f}, oracle {golden['rel_err_final']:.9f}, gap {gap:.2e}")
    assert gap < 1e-3
    sv.close()
