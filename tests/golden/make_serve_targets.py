"""Writes serve_targets_seed0_16.json: the FP64 oracle's converged relative
error on the first 16 requests of the request stream (seed 0), and the band
the oracle itself reaches when its SVD start is perturbed at FP32 rounding size.

For request q (X = the request's planted matrix rounded to FP32, as served):
  rel_f64        ||X - U V^T||_F / ||X||_F after Algorithm 3 with 500
                 alternations (oracle.enmf);
  rel_perturbed  the same after multiplying every entry of U*, V* by
                 (1 + 1e-7 z), z standard normal (seeds 1..4), then Algorithm 1
                 and 500 alternations.
A reduced-precision form rounds at about 1e-7 relative in its factors, so it
cannot be held closer to rel_f64 than the oracle's own response to such a
perturbation (reading R27 of the method's open points: planted requests at
rank 64 move by percents under it).

Calls only oracle/ and synth (the seeded inputs).  Run from the repository
root:  python tests/golden/make_serve_targets.py   (about 10 minutes on 8 cores).
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N_REQ = 16
N_ALT = 500
SEEDS = (1, 2, 3, 4)
DELTA = 1e-7


def one(i):
    import synth
    from oracle import enmf_oracle as O
    q = synth.request_stream(N_REQ, seed=0)[i]
    X = synth.request_matrix(q, dtype=np.float32).astype(np.float64)
    Us, Vs, _ = O.truncated_svd(X, q.r)
    U, V, _, _ = O.rotate(Us, Vs)
    U1, V1, _, _ = O.iterate(X, U, V, N_ALT)
    rel = O.rel_err(X, U1, V1)
    pert = []
    for sd in SEEDS:
        rng = np.random.default_rng(sd)
        Us2 = Us * (1 + DELTA * rng.standard_normal(Us.shape))
        Vs2 = Vs * (1 + DELTA * rng.standard_normal(Vs.shape))
        U2, V2, _, _ = O.rotate(Us2, Vs2)
        U3, V3, _, _ = O.iterate(X, U2, V2, N_ALT)
        pert.append(O.rel_err(X, U3, V3))
    return {"rid": q.rid, "m": q.m, "n": q.n, "r": q.r, "rel_f64": rel, "rel_perturbed": pert}


def main():
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = pool.map(one, range(N_REQ))
    out = {
        "what": "FP64 oracle relative error after Algorithm 3 (500 alternations) on requests "
                "0..15 of synth.request_stream(seed=0), X rounded to FP32; rel_perturbed: the "
                "same from an SVD start perturbed by 1e-7 relative (seeds 1..4)",
        "n_alt": N_ALT,
        "delta": DELTA,
        "requests": rows,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "serve_targets_seed0_16.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
