"""The grouped FP32 rotation (enmf_rotate_group) against enmf_rotate.

Every problem of a group gets the blocks its own launch would have, its own
partial sums in the same order and its polar factor on its own first block,
so the rotated factors, R's effect and the step records must equal those of
one enmf_rotate per problem bit for bit -- for shapes from a few rows to one
that needs several passes of its blocks, for groups that fill more than one
grid, and after a problem's stop rule has held early (it then idles through
the barriers of the others).  The call's argument checks come before any
launch.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _start(m, n, r, seed):
    from paper_2605_19325_gb300.solver import Solver
    X, _, _ = synth.planted(m, n, r, seed=seed, dist="uniform", zero_frac=0.3, noise=0.01,
                            dtype=np.float32)
    s = Solver(torch.as_tensor(X, device="cuda"), r)
    s.svd_init()
    return s


def _info(i):
    return (i.steps, i.converged, i.rho, i.dR, i.neg_mass_in, i.neg_mass_out)


SHAPES_16 = [(64, 70, 4, 0), (300, 129, 8, 1), (1000, 2000, 16, 2), (90, 4096, 5, 3),
             (3000, 3500, 12, 4)]
SHAPES_64 = [(200, 170, 64, 5), (1500, 900, 50, 6), (64, 64, 64, 7)]


@pytest.mark.gpu
@pytest.mark.parametrize("shapes", [SHAPES_16, SHAPES_64], ids=["pad16", "pad64"])
def test_group_equals_one_rotation_per_problem(shapes):
    from paper_2605_19325_gb300 import binding as B
    solo, group = [], []
    for (m, n, r, seed) in shapes:
        a = _start(m, n, r, seed)
        b = _start(m, n, r, seed)
        assert torch.equal(a.U, b.U) and torch.equal(a.V, b.V)
        solo.append(a)
        group.append(b)
    infos_solo, codes = [], []
    for a in solo:
        info, code = B.enmf_rotate(a.ctx, a.U, a.V)
        infos_solo.append(_info(info))
        codes.append(code)
    infos, gcode = B.enmf_rotate_group([b.ctx for b in group], [b.U for b in group],
                                       [b.V for b in group])
    assert gcode == next((c for c in codes if c), 0)
    torch.cuda.synchronize()
    for a, b, isolo, ig in zip(solo, group, infos_solo, infos):
        assert torch.equal(a.U, b.U) and torch.equal(a.V, b.V)
        assert isolo == _info(ig)
    for s in solo + group:
        s.close()


@pytest.mark.gpu
def test_group_spans_several_grids_and_early_stops():
    """Many mid-sized rank-32 problems (more blocks than one grid holds) and a
    loose tolerance, so that some problems stop before max_iter."""
    from paper_2605_19325_gb300 import binding as B
    shapes = [(1200 + 97 * i, 1500 + 61 * i, 24 + (i % 9), 20 + i) for i in range(14)]
    opts = B.enmf_admm_opts(0.0, 3.0, 200, 1e-2, 0)
    solo, group = [], []
    for (m, n, r, seed) in shapes:
        solo.append(_start(m, n, r, seed))
        group.append(_start(m, n, r, seed))
    infos_solo = [_info(B.enmf_rotate(a.ctx, a.U, a.V, opts=opts)[0]) for a in solo]
    infos, _ = B.enmf_rotate_group([b.ctx for b in group], [b.U for b in group],
                                   [b.V for b in group], opts=opts)
    assert any(i[0] < 200 for i in infos_solo), "no problem stopped early"
    for a, b, isolo, ig in zip(solo, group, infos_solo, infos):
        assert torch.equal(a.U, b.U) and torch.equal(a.V, b.V)
        assert isolo == _info(ig)
    for s in solo + group:
        s.close()


@pytest.mark.gpu
def test_group_argument_checks():
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    a = _start(100, 80, 8, 0)
    b = _start(120, 90, 40, 1)          # rank pad 48: another class
    X64 = torch.rand(50, 40, dtype=torch.float64, device="cuda")
    c = Solver(X64, 4)                  # FP64 factors
    U0, V0 = a.U.clone(), a.V.clone()
    for ctxs, Us, Vs in (([a.ctx, b.ctx], [a.U, b.U], [a.V, b.V]),
                         ([a.ctx, c.ctx], [a.U, c.U], [a.V, c.V]),
                         ([a.ctx, a.ctx], [a.U, a.U], [a.V, a.V])):
        with pytest.raises(B.EnmfError) as ei:
            B.enmf_rotate_group(ctxs, Us, Vs)
        assert ei.value.code == 1
    with pytest.raises(B.EnmfError):
        B.enmf_rotate_group([a.ctx], [a.U], [a.V], opts=B.enmf_admm_opts(0.0, 3.0, 200, 1e-12, 1))
    # nothing ran
    assert torch.equal(a.U, U0) and torch.equal(a.V, V0)
    for s in (a, b, c):
        s.close()
