"""Programmatic dependent launches in the captured alternation loop.

With enmf_set_overlap, the tensor-core sweeps start while the half step before
them still runs (requesting their first X tiles) and the half steps start while
the sweep before them drains; each kernel waits for its predecessor before it
touches anything they share.  The arithmetic is unchanged, so every setting
must give the same trace and factors bit for bit, with and without the
profiling events that break the chain of kernel nodes.  The driver must
accept the attribute (the flags stay in effect after the capture).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _run(X, r, U0, V0, flags, prof=0, n_iter=60):
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    s = Solver(torch.as_tensor(X, device="cuda"), r, x_stream=torch.bfloat16)
    assert B.enmf_set_overlap(s.ctx, flags) == flags
    if prof:
        B.enmf_profile(s.ctx, prof)
    s.U.copy_(U0)
    s.V.copy_(V0)
    t, info = s.iterate(n_iter, reset=1)
    # a second call replays the captured graph
    t2, _ = s.iterate(n_iter)
    in_effect = B.enmf_set_overlap(s.ctx, -1)
    out = (np.concatenate([t.cpu().numpy(), t2.cpu().numpy()]), s.U.cpu().numpy(), s.V.cpu().numpy(), in_effect)
    s.close()
    return out


@pytest.mark.gpu
def test_overlap_settings_are_bit_identical():
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.config_dense(1, dtype=np.float32)
    s = Solver(torch.as_tensor(X, device="cuda"), r, x_stream=torch.bfloat16)
    s.svd_init()
    s.rotate()
    U0, V0 = s.U.clone(), s.V.clone()
    s.close()
    t0, U_ref, V_ref, _ = _run(X, r, U0, V0, 0)
    assert np.all(np.isfinite(t0))
    for flags, prof in ((3, 0), (1, 0), (2, 0), (3, 4)):
        t, U, V, eff = _run(X, r, U0, V0, flags, prof)
        assert eff == flags, f"the driver refused the attribute (flags {flags} -> {eff})"
        assert np.array_equal(t, t0), (flags, prof, np.max(np.abs(t - t0)))
        assert np.array_equal(U, U_ref) and np.array_equal(V, V_ref), (flags, prof)


@pytest.mark.gpu
def test_overlap_flags_are_checked():
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.config_small(1)
    s = Solver(torch.as_tensor(X.astype(np.float32), device="cuda"), r, x_stream=torch.bfloat16)
    assert B.enmf_set_overlap(s.ctx, -1) == 1          # the default
    with pytest.raises(RuntimeError):
        B.enmf_set_overlap(s.ctx, 4)
    assert B.enmf_set_overlap(s.ctx, 0) == 0
    s.close()
