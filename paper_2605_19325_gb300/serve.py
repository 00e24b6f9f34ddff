"""Serving: continuous batching of eNMF solves on one GPU.

Requests (X, r) arrive over time.  A request is admitted when its device
footprint fits the memory budget:
  X in FP32, its BF16 pair X_hi / X_lo, U and V, and the context workspace
  (enmf_workspace_size).
On admission it gets the SVD start and the rotation -- for all requests
admitted in one step together: one enmf_svd_init_group call, then one grouped
rotation launch per padded rank (enmf_rotate_group) -- and then joins the
batch of its padded rank (16, 32, 48 or 64).  Every batch advances all its members
together, `chunk` alternations per step, in grouped launches under a
replayed CUDA graph (enmf_batch_step).  So requests that arrive while others
are running share the device with them, and each finished request frees its
slot and memory for the next.

A member is done when its objective, sampled after every step, has changed
by less than `tol` (relative) over the last step while in the HALS stage, or
after `max_iter` alternations.  X, U, V and the iteration state stay resident
on the device from admission to completion.

Everything runs on one CUDA stream, so the cooperative launches of different
batches never run concurrently on the device.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np
import torch

from . import binding as B
from .solver import Solver


@dataclasses.dataclass
class Request:
    rid: int
    X: np.ndarray        # m x n, nonnegative, host
    r: int
    arrival_s: float = 0.0


@dataclasses.dataclass
class Result:
    rid: int
    m: int
    n: int
    r: int
    iters: int
    f: float
    rel_err: float
    U: torch.Tensor      # host copies
    V: torch.Tensor
    arrival_s: float
    admitted_s: float
    done_s: float

    @property
    def latency_s(self):
        return self.done_s - self.arrival_s


def footprint(m, n, r):
    """Device bytes a request holds while it is served."""
    p = B.enmf_problem(m, n, n, r, B.ENMF_F32, B.ENMF_F32, B.ENMF_BF16)
    return m * n * 4 + 2 * m * n * 2 + (m + n) * r * 4 + B.enmf_workspace_size(p)


class _Slot:
    __slots__ = ("req", "solver", "rp", "slot", "bytes", "f_prev", "admitted_s")


class Server:
    def __init__(self, budget_bytes=None, max_members=128, chunk=10, tol=1e-5, max_iter=500,
                 min_iter=20, stream=None, tune=True, fp32_finish=0):
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = int(0.6 * free)
        self.budget = budget_bytes
        self.max_members = max_members
        self.chunk = chunk
        self.tol = tol
        self.max_iter = max_iter
        self.min_iter = min_iter
        self.tune = tune
        self.fp32_finish = fp32_finish   # enmf_svd_opts.fp32_finish of the SVD starts
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.batches = {}            # padded rank -> batch handle
        self.tuned = {}      # padded rank -> batch size when its sweeps were last tuned
        self.pending = collections.deque()
        self.active = []
        self._new = []
        self.used = 0
        self.results = []
        self.steps = 0
        # host wall time spent admitting (SVD start + rotation), stepping the
        # batches and retiring finished requests
        self.time_s = {"admit": 0.0, "step": 0.0, "retire": 0.0}

    # ------------------------------------------------------------- requests
    def submit(self, req: Request):
        self.pending.append(req)

    def _batch(self, rp):
        b = self.batches.get(rp)
        if b is None:
            b = B.enmf_batch_create(self.max_members, stream=self.stream)
            self.batches[rp] = b
        return b

    @staticmethod
    def _rank_pad(r):
        return 16 if r <= 16 else 32 if r <= 32 else 48 if r <= 48 else 64

    def _prepare(self, req, now):
        """Device copy of X and the context of one request (its SVD start runs
        with the step's other admissions, in _admit)."""
        m, n = req.X.shape
        with torch.cuda.stream(self.stream):
            Xt = torch.from_numpy(np.ascontiguousarray(req.X, dtype=np.float32)).to(
                "cuda", non_blocking=False)
            s = Solver(Xt, req.r, stream=self.stream, x_stream=torch.bfloat16)
        sl = _Slot()
        sl.req = req
        sl.solver = s
        sl.rp = self._rank_pad(req.r)
        sl.bytes = footprint(m, n, req.r)
        sl.f_prev = None
        sl.admitted_s = now
        self.used += sl.bytes
        return sl

    def _admit(self, now):
        new = self._new = []            # prepared in this step, not yet in a batch
        joining = collections.Counter()
        while self.pending and self.pending[0].arrival_s <= now:
            req = self.pending[0]
            need = footprint(req.X.shape[0], req.X.shape[1], req.r)
            if (self.active or new) and self.used + need > self.budget:
                break                   # wait for memory to free up
            rp = self._rank_pad(req.r)
            b = self.batches.get(rp)
            if (B.enmf_batch_size(b) if b is not None else 0) + joining[rp] >= self.max_members:
                break
            self.pending.popleft()
            new.append(self._prepare(req, now))
            joining[rp] += 1
        # the SVD starts of the step's new requests in one call (their
        # FP64-finished Rayleigh-Ritz SVDs side by side; with fp32_finish the
        # stream's chaotic requests land elsewhere often enough to cost served
        # accuracy, so it is off by default), then their rotations, grouped
        # by padded rank
        if new:
            B.enmf_svd_init_group([sl.solver.ctx for sl in new], [sl.solver.X for sl in new],
                                  [sl.solver.U for sl in new], [sl.solver.V for sl in new],
                                  None, B.enmf_svd_opts(10, 40, 1e-5, 0x5eed, self.fp32_finish))
        for rp in sorted(joining):
            sls = [sl for sl in new if sl.rp == rp]
            B.enmf_rotate_group([sl.solver.ctx for sl in sls], [sl.solver.U for sl in sls],
                                [sl.solver.V for sl in sls])
        for sl in new:
            sl.slot = B.enmf_batch_add(self._batch(sl.rp), sl.solver.ctx, sl.solver.X,
                                       sl.solver.U, sl.solver.V)
            self.active.append(sl)
        self._new = []

    def _retire(self, now):
        keep = []
        states = {rp: B.enmf_batch_states(b, self.max_members)
                  for rp, b in self.batches.items() if B.enmf_batch_size(b) > 0}
        for sl in self.active:
            b = self.batches[sl.rp]
            info, f = states[sl.rp][sl.slot]
            done = info.iters >= self.max_iter
            if (not done and info.stage == 1 and info.iters >= self.min_iter
                    and sl.f_prev is not None):
                done = abs(sl.f_prev - f) <= self.tol * abs(f)
            sl.f_prev = f
            if not done:
                keep.append(sl)
                continue
            B.enmf_batch_remove(b, sl.slot)
            s = sl.solver
            _, rel, _ = s.residual()
            t = time.perf_counter() - self.t0
            self.results.append(Result(sl.req.rid, s.X.shape[0], s.X.shape[1], sl.req.r,
                                       info.iters, f, rel, s.U.cpu(), s.V.cpu(),
                                       sl.req.arrival_s, sl.admitted_s, t))
            s.close()
            self.used -= sl.bytes
        self.active = keep

    # ----------------------------------------------------------------- loop
    def run(self, requests=()):
        """Serve `requests` (sorted by arrival) and whatever was submitted;
        return the results in completion order."""
        for req in sorted(requests, key=lambda q: q.arrival_s):
            self.submit(req)
        self.t0 = time.perf_counter()
        while self.pending or self.active:
            now = time.perf_counter() - self.t0
            t = time.perf_counter()
            self._admit(now)
            self.time_s["admit"] += time.perf_counter() - t
            if not self.active:
                if self.pending:
                    wait = self.pending[0].arrival_s - (time.perf_counter() - self.t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            t = time.perf_counter()
            for rp, b in self.batches.items():
                size = B.enmf_batch_size(b)
                if size == 0:
                    continue
                # (re)tune the grouped sweeps when the batch is new or its
                # membership has changed by half since the last tuning
                last = self.tuned.get(rp)
                if self.tune and (last is None or abs(size - last) * 2 > max(last, 4)):
                    B.enmf_batch_tune(b)
                    self.tuned[rp] = size
                B.enmf_batch_step(b, self.chunk)
            self.steps += 1
            t2 = time.perf_counter()
            self._retire(t2 - self.t0)
            t3 = time.perf_counter()
            self.time_s["step"] += t2 - t
            self.time_s["retire"] += t3 - t2
        return self.results

    def close(self):
        for b in self.batches.values():
            B.enmf_batch_destroy(b)
        self.batches = {}


def stats(results, wall_s):
    """solves/s and latency percentiles (ms) of a finished run."""
    lat = np.array([r.latency_s for r in results]) * 1e3
    return {"solves": len(results), "wall_s": wall_s,
            "solves_per_s": len(results) / wall_s if wall_s > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None}
