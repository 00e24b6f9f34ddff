"""The grouped SVD start (enmf_svd_init_group) against enmf_svd_init.

Each problem runs its own power iterations and stopping test; only the
FP32-then-FP64 Rayleigh-Ritz SVDs that finish the FP32-factor starts share one
launch (one CTA per problem, the arithmetic of its own launch).  So the
starts, singular values and records must equal one enmf_svd_init per problem
bit for bit, across ranks (so widths l) and forms in one group, with and
without fp32_finish.  Argument checks come before any launch.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

SHAPES = [(64, 70, 4, np.float32), (300, 129, 8, np.float32), (1000, 700, 32, np.float32),
          (200, 170, 64, np.float32), (400, 300, 12, np.float64), (90, 2000, 20, np.float32)]


def _solver(m, n, r, dt, seed):
    from paper_2605_19325_gb300.solver import Solver
    X, _, _ = synth.planted(m, n, r, seed=seed, dist="uniform", zero_frac=0.3, noise=0.01,
                            dtype=dt)
    return Solver(torch.as_tensor(X, device="cuda"), r)


@pytest.mark.gpu
@pytest.mark.parametrize("finish", [0, 1])
def test_group_start_equals_one_start_per_problem(finish):
    from paper_2605_19325_gb300 import binding as B
    solo = [_solver(m, n, r, dt, i) for i, (m, n, r, dt) in enumerate(SHAPES)]
    group = [_solver(m, n, r, dt, i) for i, (m, n, r, dt) in enumerate(SHAPES)]
    res_solo = []
    for s in solo:
        tol = 1e-12 if s.X.dtype == torch.float64 else 1e-5
        opts = B.enmf_svd_opts(10, 40, tol, 0x5eed, finish)
        info, code = B.enmf_svd_init(s.ctx, s.X, s.U, s.V, s.sigma, opts)
        res_solo.append((info.iters, info.rank, info.residual, code))
    # one group call per tolerance class (the options are shared by the group)
    for dtype in (torch.float32, torch.float64):
        gs = [g for g in group if g.X.dtype == dtype]
        tol = 1e-12 if dtype == torch.float64 else 1e-5
        opts = B.enmf_svd_opts(10, 40, tol, 0x5eed, finish)
        infos, codes = B.enmf_svd_init_group([g.ctx for g in gs], [g.X for g in gs],
                                             [g.U for g in gs], [g.V for g in gs],
                                             [g.sigma for g in gs], opts)
        for g, info, code in zip(gs, infos, codes):
            g.res = (info.iters, info.rank, info.residual, code)
    torch.cuda.synchronize()
    for s, g, rs in zip(solo, group, res_solo):
        assert torch.equal(s.U, g.U) and torch.equal(s.V, g.V)
        assert torch.equal(s.sigma, g.sigma)
        assert rs == g.res
    for s in solo + group:
        s.close()


@pytest.mark.gpu
def test_group_start_argument_checks():
    from paper_2605_19325_gb300 import binding as B
    a = _solver(100, 80, 8, np.float32, 0)
    U0 = a.U.clone()
    with pytest.raises(B.EnmfError) as ei:
        B.enmf_svd_init_group([a.ctx, a.ctx], [a.X, a.X], [a.U, a.U], [a.V, a.V])
    assert ei.value.code == 1
    other = torch.cuda.Stream()
    from paper_2605_19325_gb300.solver import Solver
    b = Solver(torch.rand(60, 50, device="cuda"), 4, stream=other)
    with pytest.raises(B.EnmfError) as ei:
        B.enmf_svd_init_group([a.ctx, b.ctx], [a.X, b.X], [a.U, b.U], [a.V, b.V])
    assert ei.value.code == 1
    assert torch.equal(a.U, U0)
    a.close()
    b.close()


@pytest.mark.gpu
def test_group_start_bad_options_fail_every_problem():
    from paper_2605_19325_gb300 import binding as B
    a = _solver(100, 80, 8, np.float32, 0)
    b = _solver(90, 70, 4, np.float32, 1)
    U0 = a.U.clone()
    with pytest.raises(B.EnmfError) as ei:
        B.enmf_svd_init_group([a.ctx, b.ctx], [a.X, b.X], [a.U, b.U], [a.V, b.V],
                              opts=B.enmf_svd_opts(10, 0, 1e-5, 0x5eed, 0))
    assert ei.value.code == 1
    assert torch.equal(a.U, U0)
    a.close()
    b.close()
