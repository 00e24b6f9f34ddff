"""Writes tests/golden/dense_8192x6144_r32.json from the FP64 oracle alone.

The dense planted workload (8192 x 6144, r = 32, Exponential(1) factors with
50% zeros, 1% relative noise; the stand-in for the dense synthetic benchmark of
Sec. 5.1) is too large for the oracle to run inside a GPU test, so its results
are stored here:

* sigma: the top 32 singular values (Sec. 4, the SVD start);
* rows_U, rows_V: 16 sampled rows of the rotated factors U* R, V* R
  (Algorithm 1's output) and of U, V after the 500 alternations;
* trace: f of Eq. 1 after each of 500 alternations of Algorithm 3
  (ascent stage, then HALS), from the oracle's own start;
* trace_perturbed: the same from an SVD start whose entries are multiplied by
  1 + 1e-9 g (g standard normal, seed 5), the size of the difference allowed
  between the GPU's SVD start and the oracle's; max_rel_sensitivity is the
  largest relative difference between the two traces -- how much the method
  itself amplifies a start difference of that size on this workload -- and
  the two *_rows_difference_perturbed entries are the largest relative row
  differences of the sampled rows after the rotation and after the last
  alternation between the two runs.

Run: python tests/golden/make_dense_trace.py   (about half an hour on 8 cores)
"""
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import enmf_oracle as O  # noqa: E402

N_ITER = 500
DELTA = 1e-9
ROWS = 16


def main(out=os.path.join(HERE, "dense_8192x6144_r32.json")):
    t0 = time.time()
    X, r = synth.config_dense(0)
    Us, Vs, s = O.truncated_svd(X, r)
    U, V, R, rinfo = O.rotate(Us, Vs)
    ri = np.random.default_rng(0).choice(X.shape[0], ROWS, replace=False)
    rj = np.random.default_rng(1).choice(X.shape[1], ROWS, replace=False)
    U1, V1, tr, st = O.iterate(X, U, V, N_ITER)
    rng = np.random.default_rng(5)
    Us2 = Us * (1 + DELTA * rng.standard_normal(Us.shape))
    Vs2 = Vs * (1 + DELTA * rng.standard_normal(Vs.shape))
    U2, V2, _, _ = O.rotate(Us2, Vs2)
    U3, V3, tr2, st2 = O.iterate(X, U2, V2, N_ITER)
    sens = float(np.max(np.abs(tr2 - tr) / tr))
    def rowdiff(a, b):
        return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))
    start_d = max(rowdiff(U2[ri], U[ri]), rowdiff(V2[rj], V[rj]))
    final_d = max(rowdiff(U3[ri], U1[ri]), rowdiff(V3[rj], V1[rj]))
    doc = {
        "source": "oracle/enmf_oracle.py (enmf pipeline: truncated_svd, rotate, iterate); "
                  "Sec. 4, Algorithm 1, Algorithm 3, Eq. 1",
        "workload": "synth.config_dense(0): 8192x6144, r=32",
        "n_iter": N_ITER,
        "sigma": s[:r].tolist(),
        "rows_i": ri.tolist(), "rows_j": rj.tolist(),
        "rotated_U_rows": U[ri].tolist(), "rotated_V_rows": V[rj].tolist(),
        "final_U_rows": U1[ri].tolist(), "final_V_rows": V1[rj].tolist(),
        "admm_steps": rinfo.steps, "rho": rinfo.rho,
        "asc_iters": st.asc_iters, "hals_iters": st.hals_iters,
        "trace": tr.tolist(),
        "rel_err_final": math.sqrt(2 * tr[-1]) / float(np.linalg.norm(X)),
        "delta": DELTA,
        "trace_perturbed": tr2.tolist(),
        "asc_iters_perturbed": st2.asc_iters,
        "max_rel_sensitivity": sens,
        "rotated_rows_difference_perturbed": start_d,
        "final_rows_difference_perturbed": final_d,
        "seconds": time.time() - t0,
    }
    with open(out, "w") as f:
        json.dump(doc, f, indent=0)
    print(out, f"sensitivity {sens:.3e}", f"{doc['seconds']:.0f} s")


if __name__ == "__main__":
    main()
