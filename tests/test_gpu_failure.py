"""Failure paths on the GPU, made without a fault.

* A bounded device wait on an event that never happens gives up and reports a
  timeout (a flag that nothing sets; an mbarrier phase that nothing completes).
* A context whose grid barriers are given a one-cycle spin limit times out in
  its cooperative kernels: the call returns ENMF_ETIMEOUT, the context is
  poisoned (later calls return the same code), and the CUDA context stays
  usable: a new context solves normally afterwards.
* A workspace larger than the device returns ENMF_ENOMEM and leaks nothing.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


@pytest.mark.gpu
@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_on_an_event_that_never_happens(kind):
    from paper_2605_19325_gb300 import binding as B
    assert B.enmf_probe_wait(kind, 2_000_000) == 5      # about 1 ms, then ETIMEOUT
    torch.cuda.synchronize()                              # the CUDA context is fine
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0


def _small_solver():
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.config_small(0)
    return X, r, Solver(torch.as_tensor(X, device="cuda"), r)


@pytest.mark.gpu
def test_barrier_timeout_poisons_the_context_only():
    from oracle import enmf_oracle as O
    from paper_2605_19325_gb300 import binding as B
    X, r, sv = _small_solver()
    sv.svd_init()
    sv.rotate()
    B.enmf_set_wait_limit(sv.ctx, 1)
    with pytest.raises(B.EnmfError) as ei:
        sv.iterate(6, reset=1)
    assert ei.value.code == 5
    for call in (lambda: sv.residual(), lambda: sv.iterate(1), lambda: sv.kkt(),
                 lambda: B.enmf_set_wait_limit(sv.ctx, 0)):
        with pytest.raises(B.EnmfError) as ei:
            call()
        assert ei.value.code == 5
    sv.close()
    torch.cuda.synchronize()
    # a fresh context on the same device works and matches the oracle
    X, r, sv2 = _small_solver()
    sv2.svd_init()
    sv2.rotate()
    tr, _ = sv2.iterate(20, reset=1)
    ref = O.enmf(X, r, 20)
    t = tr.cpu().numpy()
    assert np.max(np.abs(t - ref.trace) / ref.trace) < 1e-10
    sv2.close()


@pytest.mark.gpu
def test_default_wait_limit_restored_keeps_results():
    """Setting the limit back to the default (0) changes nothing in the results."""
    from paper_2605_19325_gb300 import binding as B
    X, r, a = _small_solver()
    a.svd_init()
    a.rotate()
    B.enmf_set_wait_limit(a.ctx, 4_000_000_000)
    B.enmf_set_wait_limit(a.ctx, 0)
    ta, _ = a.iterate(15, reset=1)
    X, r, b = _small_solver()
    b.svd_init()
    b.rotate()
    tb, _ = b.iterate(15, reset=1)
    np.testing.assert_array_equal(ta.cpu().numpy(), tb.cpu().numpy())
    with pytest.raises(B.EnmfError) as ei:
        B.enmf_set_wait_limit(a.ctx, -1)
    assert ei.value.code == 1
    a.close()
    b.close()


@pytest.mark.gpu
def test_oversized_workspace_returns_enomem_and_leaks_nothing():
    from paper_2605_19325_gb300 import binding as B
    m = n = 1 << 28      # the workspace alone is about a terabyte
    p = B.enmf_problem(m, n, n, 4, B.ENMF_F64, B.ENMF_F64, 0)
    need = B.enmf_workspace_size(p)
    free0, total = torch.cuda.mem_get_info()
    assert need > total
    with pytest.raises(B.EnmfError) as ei:
        B.enmf_create(p)
    assert ei.value.code == 3
    torch.cuda.synchronize()
    # nothing stays allocated (the driver's own bookkeeping may move a few MiB)
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
