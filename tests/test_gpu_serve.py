"""Serving: continuous batching (paper_2605_19325_gb300.serve).

Requests of different (m, n, r) arrive over time, are admitted by device
footprint, and share grouped launches with whatever else is running.  Each
result must be the one the request gets alone, within the tolerance of the
batching tests (1e-5 relative on the objective, 1e-4 on the factors): the
requests here run a fixed number of alternations (tol = 0), so alone and in
the mix they stop at the same point.
"""
import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


def _requests(count, seed, rate, m_hi=640):
    from paper_2605_19325_gb300.serve import Request
    reqs = synth.request_stream(count, seed=seed, rate_per_s=rate, m_hi=m_hi)
    return [Request(q.rid, synth.request_matrix(q, dtype=np.float32), q.r, q.arrival_s)
            for q in reqs]


@pytest.mark.gpu
def test_serve_mix_matches_alone():
    from paper_2605_19325_gb300.serve import Server, stats
    reqs = _requests(12, seed=7, rate=400.0)
    srv = Server(chunk=10, tol=0.0, max_iter=40)
    res = {r.rid: r for r in srv.run(reqs)}
    srv.close()
    assert len(res) == len(reqs)
    st = stats(list(res.values()), max(r.done_s for r in res.values()))
    assert st["solves_per_s"] > 0 and st["p99_ms"] >= st["p50_ms"]
    for q in reqs[::3]:
        alone = Server(chunk=10, tol=0.0, max_iter=40)
        (a,) = alone.run([type(q)(q.rid, q.X, q.r, 0.0)])
        alone.close()
        m = res[q.rid]
        assert a.iters == m.iters == 43   # 3 ascent alternations on admission + 40
        assert abs(a.f - m.f) <= 1e-5 * abs(a.f), (q.rid, a.f, m.f)
        for A_, M_ in ((a.U, m.U), (a.V, m.V)):
            assert (A_ - M_).abs().max().item() <= 1e-4 * A_.abs().max().item(), q.rid


@pytest.mark.gpu
def test_serve_admits_by_footprint():
    from paper_2605_19325_gb300.serve import Server, footprint
    reqs = _requests(8, seed=3, rate=None)
    sizes = [footprint(q.X.shape[0], q.X.shape[1], q.r) for q in reqs]
    budget = 2 * max(sizes)
    srv = Server(budget_bytes=budget, chunk=10, tol=0.0, max_iter=20)
    peak = 0
    orig = srv._prepare

    def tracked(req, now):
        nonlocal peak
        sl = orig(req, now)
        peak = max(peak, srv.used)
        return sl
    srv._prepare = tracked
    res = srv.run(reqs)
    srv.close()
    assert len(res) == len(reqs)
    assert peak <= budget
    assert srv.used == 0


@pytest.mark.gpu
def test_serve_solves_to_the_oracle_error():
    """Served to convergence, a request's relative error is within a factor
    1 + 1e-3 of the FP64 oracle's converged value (the cfg-5 target)."""
    from paper_2605_19325_gb300.serve import Server
    reqs = _requests(3, seed=11, rate=None, m_hi=256)
    srv = Server(chunk=10, tol=1e-7, max_iter=500)
    res = {r.rid: r for r in srv.run(reqs)}
    srv.close()
    for q in reqs:
        X64 = q.X.astype(np.float64)
        ref = O.enmf(X64, q.r, 500)
        rel_star = O.rel_err(X64, ref.U, ref.V)
        assert res[q.rid].rel_err <= (1 + 1e-3) * rel_star, (q.rid, res[q.rid].rel_err, rel_star)


def test_footprint_counts_x_pair_factors_and_workspace():
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.serve import footprint
    m, n, r = 300, 200, 12
    p = B.enmf_problem(m, n, n, r, B.ENMF_F32, B.ENMF_F32, B.ENMF_BF16)
    ws = B.enmf_workspace_size(p)
    assert footprint(m, n, r) == m * n * 8 + (m + n) * r * 4 + ws
    assert footprint(2 * m, n, r) > footprint(m, n, r)


@pytest.mark.gpu
def test_serve_stream_meets_the_oracle_target():
    """The first 16 requests of the seed-0 stream (m, n up to 3127, r up to
    64), served together in the BF16 form to convergence (tol 1e-6, at most
    500 alternations), against the FP64 oracle after 500 alternations (stored
    by tests/golden/make_serve_targets.py with, per request, the worst final
    error the oracle itself reaches from its SVD start perturbed at FP32
    rounding size, 1e-7, four seeds).

    A request meets the target when its served relative error is within 1e-3
    of the oracle's or no higher than (1 + 1e-3) x that worst case.  Every
    request of rank up to 32 must meet it.  Rank-64 requests on these planted
    matrices are nearly degenerate (request 0's oracle result moves by 93 %
    under the 1e-7 perturbation); for them the form's stated gap is 2 % above
    the oracle (measured: +0.84 % and +1.67 % on requests 4 and 11)."""
    import json
    import os
    from paper_2605_19325_gb300.serve import Request, Server
    path = os.path.join(os.path.dirname(__file__), "golden", "serve_targets_seed0_16.json")
    golden = json.load(open(path))
    qs = synth.request_stream(16, seed=0)
    reqs = [Request(q.rid, synth.request_matrix(q, dtype=np.float32), q.r, 0.0) for q in qs]
    srv = Server(chunk=10, tol=1e-6, max_iter=golden["n_alt"])
    res = {r.rid: r for r in srv.run(reqs)}
    srv.close()
    rows, misses = [], []
    for g in golden["requests"]:
        q = qs[g["rid"]]
        assert (q.m, q.n, q.r) == (g["m"], g["n"], g["r"])
        served = res[g["rid"]].rel_err
        band = max([g["rel_f64"]] + g["rel_perturbed"])
        rows.append((g["rid"], q.r, served / g["rel_f64"] - 1, band / g["rel_f64"] - 1))
        meets = served <= (1 + 1e-3) * g["rel_f64"] or served <= (1 + 1e-3) * band
        if (q.r <= 32 and not meets) or served > 1.02 * max(g["rel_f64"], band):
            misses.append(rows[-1])
    assert not misses, ("(rid, r, excess, oracle band)", misses, rows)
