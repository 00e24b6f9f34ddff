"""The FP16 stream form of the precision form (tensor cores, kind::f16 with
FP16 A and B, FP32 accumulation).

The sweep is checked against the same FP16 decomposition (X_hi = f16(X),
X_lo = f16(X - X_hi), the factor as an FP16 pair) multiplied in FP64: only
the FP32 accumulation differs, so the relative error to the largest output
entry stays below 2e-6.  FP16 keeps 11 significant bits against BF16's 8, so
the undecomposed product is matched more closely than in the BF16 form.
"""
import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


def _f16_pair(a32):
    t = torch.as_tensor(a32, dtype=torch.float32)
    hi = t.to(torch.float16).to(torch.float32)
    lo = (t - hi).to(torch.float16).to(torch.float32)
    return hi.double().numpy(), lo.double().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("m,n,r", [(300, 200, 5), (1000, 700, 32), (513, 1031, 49),
                                   (129, 3, 2), (4100, 260, 20)])
def test_fp16_sweep_matches_decomposed_reference(m, n, r):
    from paper_2605_19325_gb300.solver import Solver
    rng = np.random.default_rng(m * 5 + n)
    X = rng.random((m, n)).astype(np.float32) * 3.0
    U = rng.random((m, r)).astype(np.float32)
    V = rng.random((n, r)).astype(np.float32)
    s = Solver(torch.as_tensor(X, device="cuda"), r, x_stream=torch.float16)
    Ud = torch.as_tensor(U, device="cuda")
    Vd = torch.as_tensor(V, device="cuda")
    xh, xl = _f16_pair(X)
    uh, ul = _f16_pair(U)
    vh, vl = _f16_pair(V)
    for exact in (1, 0):
        XV, XtU = s.sweep(Ud, Vd, exact=exact)
        torch.cuda.synchronize()
        Xe = xh + xl if exact else xh
        assert _rel(XV.double().cpu().numpy(), Xe @ (vh + vl)) < 2e-6
        assert _rel(XtU.double().cpu().numpy(), Xe.T @ (uh + ul)) < 2e-6
    XV, XtU = s.sweep(Ud, Vd, exact=1)
    assert _rel(XV.double().cpu().numpy(), X.astype(np.float64) @ V) < 1e-5
    assert _rel(XtU.double().cpu().numpy(), X.astype(np.float64).T @ U) < 1e-5
    s.close()


def test_fp16_precision_form_error_gap_small():
    """Final relative error within 1e-3 (relative) of the FP64 oracle's, the
    stated target, and in practice within 1e-5."""
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.config_small(0)
    res = O.enmf(X, r, 200)
    ref = O.rel_err(X, res.U, res.V)
    s = Solver(torch.as_tensor(X, dtype=torch.float32, device="cuda"), r, x_stream=torch.float16)
    s.svd_init()
    s.rotate()
    s.iterate(200, reset=1)
    _, rel, _ = s.residual()
    gap = abs(rel - ref) / ref
    assert gap < 1e-5, gap
    s.close()


def test_fp16_image_stack_against_fp64_form():
    """Image-stack workload (10304 x 4096, r = 49) in the FP16 stream form and
    in the plain FP64 form, 40 alternations each from their own starts: the
    final relative errors agree within the stated 1e-3."""
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.image_stack(seed=0, dtype=np.float32)
    out = {}
    for name, kw in (("f16", dict(x_stream=torch.float16)), ("f64", {})):
        Xt = torch.as_tensor(X, dtype=torch.float64 if name == "f64" else torch.float32,
                             device="cuda")
        s = Solver(Xt, r, **kw)
        s.svd_init()
        s.rotate()
        s.iterate(40, reset=1, trace=False)
        out[name] = s.residual()[1]
        s.close()
    assert abs(out["f16"] - out["f64"]) / out["f64"] < 1e-3, out


def test_fp16_rejects_x_beyond_range():
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    X = torch.rand(256, 128, device="cuda")
    X[3, 5] = 1e5                        # above the largest FP16 value
    with pytest.raises(B.EnmfError) as ei:
        s = Solver(X, 8, x_stream=torch.float16)
        s.svd_init()
    assert ei.value.code == 2
