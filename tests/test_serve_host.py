"""Host logic of the serving loop, on the CPU.

`serve.Server` is run unchanged against fakes of the library binding and of
the per-request solver, which stand in for the device work. The fake batch moves
each member's objective geometrically toward a floor, one factor per
alternation, and reports the HALS stage from the tenth alternation on. The checks cover the loop's own rules:

* admission is FIFO by arrival and never takes the footprint in use above the
  budget, except for a lone request that could never fit;
* a batch never holds more than max_members;
* a member retires when its objective settles (relative change <= tol over one
  chunk, in the HALS stage, after min_iter), or at max_iter;
* every request gets exactly one result, and the footprint returns to zero.
"""
import contextlib
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_19325_gb300 import serve  # noqa: E402


class _Info:
    def __init__(self, iters, stage):
        self.iters = iters
        self.stage = stage


class FakeBinding:
    """The binding calls serve.py makes, with per-member state on the host."""

    ENMF_F32, ENMF_BF16 = 1, 2

    def __init__(self, rates):
        self.rates = rates              # rid -> objective decay per alternation
        self.batches = {}
        self.next_id = 0
        self.max_seen = {}
        self.rotated = []               # request ids, in grouped-rotation order
        self.started = []               # request ids, in grouped SVD-start order

    def enmf_problem(self, m, n, ldx, r, *dtypes):
        return (m, n, r)

    def enmf_workspace_size(self, p):
        m, n, r = p
        return 1000 + (m + n) * r

    def enmf_admm_opts(self, *fields):
        return fields

    def enmf_svd_opts(self, *fields):
        return fields

    def enmf_batch_create(self, max_members, stream=None):
        self.next_id += 1
        self.batches[self.next_id] = {"max": max_members, "members": {}, "next": 0}
        return self.next_id

    def enmf_batch_destroy(self, b):
        self.batches.pop(b)

    def enmf_batch_add(self, b, ctx, X, U, V):
        bt = self.batches[b]
        assert len(bt["members"]) < bt["max"]
        slot = bt["next"]
        bt["next"] += 1
        bt["members"][slot] = {"rid": ctx, "iters": 0, "f": 1.0}
        self.max_seen[b] = max(self.max_seen.get(b, 0), len(bt["members"]))
        return slot

    def enmf_batch_remove(self, b, slot):
        del self.batches[b]["members"][slot]

    def enmf_batch_size(self, b):
        return len(self.batches[b]["members"])

    def enmf_batch_tune(self, b):
        return None

    def enmf_svd_init_group(self, ctxs, Xs, Us, Vs, sigmas=None, opts=None):
        self.started.extend(ctxs)
        return [], []

    def enmf_rotate_group(self, ctxs, Us, Vs, opts=None):
        self.rotated.extend(ctxs)
        return []

    def enmf_batch_step(self, b, n_alt):
        # the objective approaches 0.5 geometrically: f = 0.5 + 0.5 rate^iters
        for mb in self.batches[b]["members"].values():
            mb["iters"] += n_alt
            mb["f"] = 0.5 + 0.5 * self.rates[mb["rid"]] ** mb["iters"]

    def enmf_batch_member(self, b, slot):
        mb = self.batches[b]["members"][slot]
        stage = 1 if mb["iters"] >= 10 else 0
        return _Info(mb["iters"], stage), mb["f"]

    def enmf_batch_states(self, b, cap):
        assert len(self.batches[b]["members"]) <= cap
        return {slot: self.enmf_batch_member(b, slot) for slot in self.batches[b]["members"]}


class FakeSolver:
    def __init__(self, Xt, r, stream=None, x_stream=None):
        self.X = Xt
        self.ctx = Xt.rid
        self.U = torch.zeros(Xt.shape[0], r)
        self.V = torch.zeros(Xt.shape[1], r)

    def svd_init(self, opts=None):
        pass

    def rotate(self, opts=None):
        pass

    def residual(self):
        return 0.0, 0.01, 0.0

    def close(self):
        pass


class _HostArray:
    """What serve.py's host-to-device copy returns here: shape and request id."""

    def __init__(self, a, rid):
        self.shape = a.shape
        self.rid = rid

    def to(self, *args, **kwargs):
        return self


def _fake_torch(rid_of):
    t = types.SimpleNamespace()
    t.bfloat16 = torch.bfloat16
    t.cuda = types.SimpleNamespace(stream=lambda s: contextlib.nullcontext())
    t.from_numpy = lambda a: _HostArray(a, rid_of[id(a)])
    return t


def _run(monkeypatch, reqs, rates, budget, max_members=128, chunk=10, tol=1e-5, max_iter=500):
    B = FakeBinding(rates)
    rid_of = {}
    # serve.py passes np.ascontiguousarray(req.X, float32) to torch.from_numpy;
    # keep the arrays float32 and contiguous so it is the same object
    for q in reqs:
        rid_of[id(q.X)] = q.rid
    monkeypatch.setattr(serve, "B", B)
    monkeypatch.setattr(serve, "Solver", FakeSolver)
    monkeypatch.setattr(serve, "torch", _fake_torch(rid_of))
    srv = serve.Server(budget_bytes=budget, max_members=max_members, chunk=chunk, tol=tol,
                       max_iter=max_iter, stream=object(), tune=True)
    admitted, used_after = [], []
    orig = srv._prepare

    def spy(req, now):
        sl = orig(req, now)
        admitted.append(req.rid)
        # footprint in use and requests on the device once this one is prepared
        used_after.append((srv.used, len(srv.active) + len(srv._new) + 1))
        return sl

    srv._prepare = spy
    results = srv.run(reqs)
    srv.close()
    return srv, B, results, admitted, used_after


def _requests(shapes, arrivals):
    out = []
    for rid, ((m, n, r), t) in enumerate(zip(shapes, arrivals)):
        X = np.zeros((m, n), dtype=np.float32)
        out.append(serve.Request(rid, X, r, t))
    return out


def _fp(m, n, r):
    return m * n * 4 + 2 * m * n * 2 + (m + n) * r * 4 + 1000 + (m + n) * r


def test_admission_keeps_within_budget_and_fifo(monkeypatch):
    shapes = [(64, 48, 4), (80, 40, 8), (70, 70, 16), (64, 64, 4), (90, 30, 32), (50, 50, 8)]
    reqs = _requests(shapes, [0.0] * len(shapes))
    budget = _fp(70, 70, 16) + _fp(80, 40, 8) + 10
    rates = {q.rid: 0.5 for q in reqs}
    srv, B, results, admitted, used_after = _run(monkeypatch, reqs, rates, budget)
    assert admitted == [q.rid for q in reqs]                    # FIFO
    assert sorted(B.rotated) == sorted(admitted)                # every admission rotated once
    assert B.started == admitted                                # and started once, in order
    assert all(u <= budget for u, _ in used_after)
    assert sorted(r.rid for r in results) == [q.rid for q in reqs]
    assert srv.used == 0 and not srv.active


def test_lone_request_beyond_budget_is_still_served(monkeypatch):
    reqs = _requests([(100, 100, 8), (20, 20, 4)], [0.0, 0.0])
    budget = _fp(20, 20, 4) + 1                                 # the first never fits
    srv, B, results, admitted, used_after = _run(monkeypatch, reqs, {0: 0.5, 1: 0.5}, budget)
    assert admitted == [0, 1]
    assert used_after[0][1] == 1                                 # admitted alone
    assert len(results) == 2


def test_batch_never_exceeds_max_members(monkeypatch):
    reqs = _requests([(64, 64, 8)] * 7, [0.0] * 7)
    srv, B, results, admitted, _ = _run(monkeypatch, reqs, {i: 0.5 for i in range(7)},
                                        budget=10 ** 12, max_members=3)
    assert max(B.max_seen.values()) == 3
    assert len(results) == 7


def test_retirement_rules(monkeypatch):
    """A fast-settling member retires after min_iter at a chunk boundary; one
    whose objective never settles retires at max_iter."""
    reqs = _requests([(64, 64, 8), (64, 64, 8)], [0.0, 0.0])
    rates = {0: 0.1, 1: 0.999}      # rid 1 moves by ~0.5 % per chunk: never within tol
    srv, B, results, _, _ = _run(monkeypatch, reqs, rates, budget=10 ** 12, chunk=10,
                                 tol=1e-5, max_iter=200)
    by = {r.rid: r for r in results}
    assert by[1].iters == 200
    assert by[0].iters < 200 and by[0].iters >= 20 and by[0].iters % 10 == 0
    assert [r.rid for r in results][0] == 0                     # completion order
