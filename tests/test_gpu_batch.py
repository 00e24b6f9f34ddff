"""Batching: many problems iterated by grouped launches (enmf_batch_*).

Each member of a batch must give the result it gives alone.  Alone and in a
mix, a member's half steps are the same computation (its own group of
blocks, its own fixed-order Gram sums, its own PBCD decisions), but the
grouped tensor-core sweep cuts the members' concatenated work into stream-K
ranges that depend on the whole batch, so the FP32 sums of a sweep output
are taken in a different order: each differs by a few units of 2^-24
relative.  Over the alternations of HALS (a contraction near the solution)
that stays at the level of the per-step rounding; the stated tolerance is
1e-5 relative on the objective and 1e-4 on the factors (max abs difference
over max abs entry).

A member's ascent stage (the first n_shift = 3 alternations from its start)
runs alone when it is added, with the X_lo term refreshed in every
alternation, exactly as enmf_iterate runs a fresh ascent stage; the batch
steps then continue its descent.
"""
N_SHIFT = 3
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


def _prepared(m, n, r, seed):
    """A tensor-core-form solver after the SVD start and the rotation."""
    from paper_2605_19325_gb300.solver import Solver
    X, _, _ = synth.planted(m, n, r, seed=seed, noise=0.01)
    Xt = torch.as_tensor(X, dtype=torch.float32, device="cuda")
    s = Solver(Xt, r, x_stream=torch.bfloat16)
    s.svd_init()
    s.rotate()
    return s


SHAPES = [(300, 200, 12, 1), (700, 1100, 16, 2), (129, 257, 9, 3), (1500, 640, 14, 4)]


def _run_batch(solvers, starts, n_alt, chunk=10, correct_every=10):
    from paper_2605_19325_gb300 import binding as B
    b = B.enmf_batch_create(8, correct_every=correct_every)
    try:
        slots = []
        for s, (U0, V0) in zip(solvers, starts):
            s.U.copy_(U0)
            s.V.copy_(V0)
            slots.append(B.enmf_batch_add(b, s.ctx, s.X, s.U, s.V))
        for _ in range(n_alt // chunk):
            B.enmf_batch_step(b, chunk)
        out = []
        for s, slot in zip(solvers, slots):
            info, f = B.enmf_batch_member(b, slot)
            out.append((info.iters, f, s.U.clone(), s.V.clone()))
        for slot in slots:
            B.enmf_batch_remove(b, slot)
        torch.cuda.synchronize()
        return out
    finally:
        B.enmf_batch_destroy(b)


def test_batch_member_alone_and_in_mix():
    solvers = [_prepared(*sh) for sh in SHAPES]
    starts = [(s.U.clone(), s.V.clone()) for s in solvers]
    n_alt = 40
    mix = _run_batch(solvers, starts, n_alt)
    for i, s in enumerate(solvers):
        alone = _run_batch([s], [starts[i]], n_alt)[0]
        k_a, f_a, U_a, V_a = alone
        k_m, f_m, U_m, V_m = mix[i]
        assert k_a == k_m == n_alt + N_SHIFT
        assert abs(f_a - f_m) <= 1e-5 * abs(f_a), (i, f_a, f_m)
        for A_, M_ in ((U_a, U_m), (V_a, V_m)):
            scale = A_.abs().max().item()
            assert (A_ - M_).abs().max().item() <= 1e-4 * scale, i
    for s in solvers:
        s.close()


def test_batch_matches_enmf_iterate():
    """A one-member batch runs the same alternations as enmf_iterate on the
    same context (the ascent stage when added, then the batch steps): the same
    stage sequence and, within the same tolerance, the same objective and
    factors.  Both refresh the X_lo term every alternation here, so that the
    batch's correction phase (anchored at the member's first batch step) and
    the call's (anchored at its first alternation) cannot differ."""
    from paper_2605_19325_gb300 import binding as B
    s = _prepared(700, 1100, 16, 2)
    U0, V0 = s.U.clone(), s.V.clone()
    tr, info = s.iterate(N_SHIFT + 30, reset=1, correct_every=1)
    f_it = float(tr[-1].item())
    U_it, V_it = s.U.clone(), s.V.clone()
    (k, f_b, U_b, V_b), = _run_batch([s], [(U0, V0)], 30, correct_every=1)
    assert k == N_SHIFT + 30
    assert abs(f_b - f_it) <= 1e-5 * abs(f_it), (f_b, f_it)
    scale = U_it.abs().max().item()
    assert (U_b - U_it).abs().max().item() <= 1e-4 * scale
    s.close()


def test_batch_rejects_other_padded_rank_and_bad_step():
    from paper_2605_19325_gb300 import binding as B
    s16 = _prepared(200, 150, 10, 5)     # padded to 16
    s32 = _prepared(200, 150, 20, 6)     # padded to 32
    b = B.enmf_batch_create(4)
    try:
        slot = B.enmf_batch_add(b, s16.ctx, s16.X, s16.U, s16.V)
        with pytest.raises(B.EnmfError) as ei:
            B.enmf_batch_add(b, s32.ctx, s32.X, s32.U, s32.V)
        assert ei.value.code == 1
        with pytest.raises(B.EnmfError):
            B.enmf_batch_step(b, 7)          # not a multiple of correct_every
        B.enmf_batch_step(b, 10)
        info, f = B.enmf_batch_member(b, slot)
        assert info.iters == N_SHIFT + 10 and np.isfinite(f)
        g, ms = B.enmf_batch_tune(b)
        assert g > 0 and ms > 0
        B.enmf_batch_step(b, 10)              # after tuning: still iterating
        info, f2 = B.enmf_batch_member(b, slot)
        assert info.iters == N_SHIFT + 20 and f2 <= f * (1 + 1e-6)
        B.enmf_batch_remove(b, slot)
    finally:
        B.enmf_batch_destroy(b)
        s16.close()
        s32.close()
