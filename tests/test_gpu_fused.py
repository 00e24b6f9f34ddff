"""The fused single-pass HALS alternation (fused.cu) against the oracle.

In the HALS stage of the BF16 tensor-core form one kernel reads X once per
alternation: X V, the HALS update of U's rows (Sec. 4.3), X^T U with the new U.
With the X_lo correction refreshed every alternation (correct_every = 1) the
alternation computes, from the staged split X_hi + X_lo (exact in FP64 as Xs)
and the factors' 16-bit pairs (F2 = hi + lo, exact in FP64):

    U1 = HALS(U0; A = Xs F2(V0), B)     V1 = HALS(V0; A' = Xs^T F2(U1), B')

with B, B' the Grams of the factors.  The oracle's hals_update(Xs, U0, F2(V0))
computes the same update with B = F2(V0)^T F2(V0), which differs from the
kernel's V0^T V0 by the pair's rounding (2^-17 relative), so the bar is 5e-5 of
the largest entry.  The V-half is checked from the GPU's own U1 in the same
way.  Shapes span several 128-row panels with a ragged last panel, empty column
slices (n below the cluster's width) and both rank pads (32, 64).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(1000, 700, 20), (100, 900, 24), (1300, 2100, 49), (333, 6144, 32), (2053, 4096, 64)]


def _np(t):
    return t.detach().double().cpu().numpy()


def _solver(X, r):
    from paper_2605_19325_gb300.solver import Solver
    return Solver(torch.as_tensor(X.astype(np.float32), device="cuda"), r, x_stream=torch.bfloat16)


def _pair(F):
    from oracle import enmf_oracle as O
    F32 = np.asarray(F, dtype=np.float32)
    hi = O.bf16_round(F32).astype(np.float64)
    lo = O.bf16_round((F32.astype(np.float64) - hi).astype(np.float32)).astype(np.float64)
    return hi + lo


def _inputs(m, n, r, seed=0):
    X, _, _ = synth.planted(m, n, r, seed=seed, dist="uniform", zero_frac=0.3, noise=0.01)
    return X


@pytest.mark.parametrize("m,n,r", SHAPES)
def test_fused_alternation_matches_oracle(m, n, r):
    from oracle import enmf_oracle as O
    from paper_2605_19325_gb300 import binding as B
    X = _inputs(m, n, r)
    sv = _solver(X, r)
    assert B.enmf_set_fused(sv.ctx, 1)
    sv.svd_init()
    sv.rotate()
    _, info = sv.iterate(6, reset=1, correct_every=1)      # ascent, then fused HALS
    assert info.stage == 1
    hi, lo, _ = sv.staged()
    Xs = _np(hi) + _np(lo)
    U0, V0 = _np(sv.U), _np(sv.V)
    tr, _ = sv.iterate(1, correct_every=1)
    U1, V1 = _np(sv.U), _np(sv.V)
    Uo = O.hals_update(Xs, U0, _pair(V0))
    assert np.abs(U1 - Uo).max() <= 5e-5 * np.abs(Uo).max(), np.abs(U1 - Uo).max() / np.abs(Uo).max()
    Vo = O.hals_update(Xs.T, V0, _pair(U1))
    assert np.abs(V1 - Vo).max() <= 5e-5 * np.abs(Vo).max(), np.abs(V1 - Vo).max() / np.abs(Vo).max()
    # The trace is 1/2 |X|^2 - <Xs^T U, V> + 1/2 <U^T U, V^T V>: |X|^2 of the
    # FP32 X, the cross term through the split (X - Xs is X_lo's rounding).
    # X^T U is accumulated in FP32 by the tensor cores over m rows, L =
    # 2 ceil(m / 16) additions per entry (hi and lo products), each within
    # 2^-23 relative (the accumulation need not round to nearest), so the
    # cross term is within L 2^-23 <|Xs|, |U||V|^T>; the Grams add FP32 sums.
    f = float(_np(tr)[0])
    X32 = X.astype(np.float32).astype(np.float64)
    fo = O.objective(X32, U1, V1)
    split = abs(float(np.sum((X32 - Xs) * (U1 @ V1.T))))
    L = 2 * ((m + 15) // 16)
    acc = L * 2.0 ** -23 * float(np.sum(np.abs(Xs) * (np.abs(U1) @ np.abs(V1).T)))
    assert abs(f - fo) <= split + acc + 8 * 2.0 ** -24 * float(np.sum(X32 * X32)), (f, fo, split, acc)
    sv.close()


@pytest.mark.parametrize("m,n,r", [(1000, 700, 20), (1300, 2100, 49)])
def test_fused_and_two_pass_agree_and_fused_is_deterministic(m, n, r):
    """The same 120 alternations with and without the fused pass end within the
    FP32 accumulation differences of each other; two fused runs are equal bit
    for bit."""
    from paper_2605_19325_gb300 import binding as B
    X = _inputs(m, n, r, seed=1)
    runs = []
    for fused in (True, True, False):
        sv = _solver(X, r)
        B.enmf_set_fused(sv.ctx, fused)
        sv.svd_init()
        sv.rotate()
        tr, _ = sv.iterate(120, reset=1)
        runs.append((_np(tr), _np(sv.U), _np(sv.V), sv.residual()[1]))
        sv.close()
    for a, b in zip(runs[0][:3], runs[1][:3]):
        np.testing.assert_array_equal(a, b)
    # the direct residuals at the end agree to FP32 accumulation differences
    assert abs(runs[0][3] - runs[2][3]) <= 1e-5 * runs[2][3], (runs[0][3], runs[2][3])
    # The traces are Gram expansions 1/2 |X|^2 - <X^T U, V> + 1/2 <U^T U, V^T V>
    # with FP32 cross terms: each is within a few units of 2^-24 |X|^2 of f
    # (the cancellation against |X|^2 / 2), so that is the bar between them.
    nx2 = float(np.sum(X.astype(np.float32).astype(np.float64) ** 2))
    assert np.max(np.abs(runs[0][0] - runs[2][0])) <= 16 * 2.0 ** -24 * nx2


def test_fused_form_final_gap_to_the_oracle():
    """Whole solve in the BF16 form with the fused pass: final relative error
    within 1e-3 of the FP64 oracle's on a planted problem."""
    from oracle import enmf_oracle as O
    m, n, r = 900, 640, 24
    X = _inputs(m, n, r, seed=2)
    res = O.enmf(X, r, 200)
    from paper_2605_19325_gb300 import binding as B
    sv = _solver(X, r)
    assert B.enmf_set_fused(sv.ctx, 1)
    sv.svd_init()
    sv.rotate()
    sv.iterate(200, reset=1)
    _, rel, _ = sv.residual()
    ref = O.rel_err(X, res.U, res.V)
    assert abs(rel - ref) <= 1e-3 * ref, (rel, ref)
    sv.close()


def test_fused_availability():
    from paper_2605_19325_gb300 import binding as B
    X = _inputs(300, 200, 5)
    sv = _solver(X, 5)                 # rank pad 16: two-pass sweeps only
    assert not B.enmf_set_fused(sv.ctx, 1)
    sv.close()
    X = _inputs(300, 200, 20)
    sv = _solver(X, 20)
    assert B.enmf_set_fused(sv.ctx, 1)
    sv.close()


def test_fused_graph_replay_repeats_the_captured_call():
    """A second identical call replays the captured alternation graph (fused
    kernels included) and must reproduce the first call's results bit for bit;
    the first call ran the graph it had just captured."""
    from paper_2605_19325_gb300 import binding as B
    X = _inputs(1000, 700, 20, seed=3)
    sv = _solver(X, 20)
    assert B.enmf_set_fused(sv.ctx, 1)
    sv.svd_init()
    sv.rotate()
    U0, V0 = sv.U.clone(), sv.V.clone()
    runs = []
    for _ in range(3):
        sv.U.copy_(U0)
        sv.V.copy_(V0)
        tr, info = sv.iterate(60, reset=1)
        runs.append((_np(tr), _np(sv.U), _np(sv.V)))
    for k in (1, 2):
        for a, b in zip(runs[0], runs[k]):
            np.testing.assert_array_equal(a, b)
    sv.close()
