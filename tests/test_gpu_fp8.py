"""The FP8 stream form of the precision form: X_hi as E4M3 codes with one
power-of-two scale per 128 x 128 tile, streamed through the tensor cores
(codes converted to exact BF16 values in shared memory), X_lo = bf16(X - X_hi)
applied every few alternations.

Staging is byte work and is compared bit for bit with the oracle's split of
the same FP32 X.  The sweep is compared with the oracle's decomposition
multiplied in FP64: the factor enters as its BF16 pair, so only the FP32
accumulation differs and the relative error to the largest output entry
stays below 2e-6 (the bound of the 16-bit forms).  The form's final relative
error is stated against the FP64 oracle and against the FP32 form.
"""
import numpy as np
import pytest

import synth
from oracle import enmf_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP8 = getattr(torch, "float8_e4m3fn", None)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


def _bf16_pair(a32):
    t = torch.as_tensor(a32, dtype=torch.float32)
    hi = t.to(torch.bfloat16).to(torch.float32)
    lo = (t - hi).to(torch.bfloat16).to(torch.float32)
    return hi.double().numpy(), lo.double().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _accum_bound(rows_out, red):
    """Relative error bound of the sweep's FP32 accumulation for nonnegative
    operands (relative to the exact sum of the nonnegative terms).  Each
    addition into an FP32 accumulator errs by less than one unit in the last
    place, 2^-23 relative (tensor-core accumulation may truncate rather than
    round, so no sqrt-growth is assumed).  Additions per output: the K steps
    of 16 a CTA's stream-K segment of the tile accumulates (at most the
    tile's k-blocks, at most the units per CTA plus one), one per partial
    slot summed, the hi + lo and the X_lo term."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nkb = -(-red // 128)
    units = -(-rows_out // 128) * nkb
    grid = min(units, sms)
    seg = min(nkb, -(-units // grid) + 1)
    parts = -(-nkb // max(1, units // grid)) + 1
    return max(2e-6, (8 * seg + parts + 3) * 2.0 ** -23)


def _tiled_magnitudes(m, n, seed):
    """Nonnegative FP32 X whose 128 x 128 tiles span many binades, with an
    all-zero tile row, a tile below the exponent floor and sparse entries."""
    rng = np.random.default_rng(seed)
    X = rng.random((m, n)) ** 2
    X[rng.random((m, n)) < 0.2] = 0.0
    ti, tj = -(-m // 128), -(-n // 128)
    scale = 2.0 ** rng.integers(-40, 40, (ti, tj)).astype(float)
    X *= np.repeat(np.repeat(scale, 128, 0), 128, 1)[:m, :n]
    if ti > 2:
        X[128:256, :] = 0.0
    if tj > 1:
        X[:min(m, 128), 128:256] *= 2.0 ** -110
    return X.astype(np.float32)


def _staged_numpy(s):
    hi, lo, ex = s.staged()
    return (hi.cpu().numpy(), lo.float().double().cpu().numpy(), ex.cpu().numpy())


@pytest.mark.parametrize("m,n", [(300, 200), (1025, 700), (129, 1031), (64, 40)])
def test_fp8_staging_is_bit_exact(m, n):
    from paper_2605_19325_gb300.solver import Solver
    X = _tiled_magnitudes(m, n, m + 3 * n)
    s = Solver(torch.as_tensor(X, device="cuda"), 4, x_stream=FP8)
    codes, lo, ex = _staged_numpy(s)
    s.close()
    c_ref, K_ref, _, lo_ref = O.quantize_fp8_tiles(X)
    np.testing.assert_array_equal(ex, K_ref)
    np.testing.assert_array_equal(codes, c_ref)
    np.testing.assert_array_equal(lo, lo_ref)


@pytest.mark.parametrize("m,n,r", [(300, 200, 5), (1000, 700, 32), (513, 1031, 49),
                                   (129, 3, 2), (4100, 260, 20), (700, 900, 40),
                                   (1025, 4096, 64)])
def test_fp8_sweep_matches_decomposed_reference(m, n, r):
    from paper_2605_19325_gb300.solver import Solver
    rng = np.random.default_rng(m * 7 + n)
    X = (rng.random((m, n)) * 3.0).astype(np.float32)
    X[:, : n // 3] *= 1e3                      # tiles of different scale
    U = rng.random((m, r)).astype(np.float32)
    V = rng.random((n, r)).astype(np.float32)
    s = Solver(torch.as_tensor(X, device="cuda"), r, x_stream=FP8)
    Ud = torch.as_tensor(U, device="cuda")
    Vd = torch.as_tensor(V, device="cuda")
    _, _, xh, xl = O.quantize_fp8_tiles(X)
    uh, ul = _bf16_pair(U)
    vh, vl = _bf16_pair(V)
    for exact in (1, 0, 1):
        XV, XtU = s.sweep(Ud, Vd, exact=exact)
        torch.cuda.synchronize()
        Xe = xh + xl if exact else xh
        assert _rel(XV.double().cpu().numpy(), Xe @ (vh + vl)) < 2e-6, exact
        assert _rel(XtU.double().cpu().numpy(), Xe.T @ (uh + ul)) < 2e-6, exact
    # against the undecomposed product: X_hi + X_lo keeps 12 significant bits
    XV, XtU = s.sweep(Ud, Vd, exact=1)
    Xd = X.astype(np.float64)
    assert _rel(XV.double().cpu().numpy(), Xd @ V) < 1e-4
    assert _rel(XtU.double().cpu().numpy(), Xd.T @ U) < 1e-4
    s.close()


def test_fp8_sweep_twice_is_deterministic():
    from paper_2605_19325_gb300.solver import Solver
    rng = np.random.default_rng(5)
    X = rng.random((2000, 3000)).astype(np.float32)
    s = Solver(torch.as_tensor(X, device="cuda"), 32, x_stream=FP8)
    U = torch.rand(2000, 32, device="cuda")
    V = torch.rand(3000, 32, device="cuda")
    a = s.sweep(U, V, exact=1)
    b = s.sweep(U, V, exact=1)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    s.close()


def test_fp8_precision_form_error_gap():
    """Final relative error within the stated 1e-3 (relative) of the FP64
    oracle's on the small planted workload."""
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.config_small(0)
    res = O.enmf(X, r, 200)
    ref = O.rel_err(X, res.U, res.V)
    s = Solver(torch.as_tensor(X, dtype=torch.float32, device="cuda"), r, x_stream=FP8)
    s.svd_init()
    s.rotate()
    s.iterate(200, reset=1)
    _, rel, _ = s.residual()
    gap = abs(rel - ref) / ref
    print(f"FP8 form: rel_err {rel:.9g}, oracle {ref:.9g}, gap {gap:.3g}")
    assert gap < 1e-3, gap
    s.close()


def test_fp8_spectrogram_against_fp32_form():
    """Spectrogram-shaped X (1025 x 16384, r = 64) in the FP8 form and in the
    FP32 form, 60 alternations each from their own starts: the final relative
    errors agree within the stated 1e-3."""
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.spectrogram(n=16384, seed=1, dtype=np.float32)
    out = {}
    for name, kw in (("fp8", dict(x_stream=FP8)), ("f32", {})):
        s = Solver(torch.as_tensor(X, device="cuda"), r, **kw)
        s.svd_init()
        s.rotate()
        s.iterate(60, reset=1, trace=False)
        out[name] = s.residual()[1]
        s.close()
    print("spectrogram 1025 x 16384:", out)
    assert abs(out["fp8"] - out["f32"]) / out["f32"] < 1e-3, out


def test_fp8_full_size_spectrogram_sampled():
    """Full-size spectrogram workload (1025 x 131072, r = 64), in the launch
    configuration the benchmark times: staging of sampled row and column
    panels bit-exact, and sampled rows of X V and columns of X^T U against
    the oracle's decomposition in FP64, within the FP32 accumulation bound of
    the launch (131072-long reductions split into stream-K segments of about
    60 k-blocks: 5.9e-5 for X V, 1e-5 for X^T U)."""
    from paper_2605_19325_gb300.solver import Solver
    X, r = synth.spectrogram(seed=0, dtype=np.float32)
    m, n = X.shape
    rng = np.random.default_rng(3)
    U = rng.random((m, r)).astype(np.float32)
    V = rng.random((n, r)).astype(np.float32)
    s = Solver(torch.as_tensor(X, device="cuda"), r, x_stream=FP8)
    hi, lo, ex = s.staged()
    XV, XtU = s.sweep(torch.as_tensor(U, device="cuda"), torch.as_tensor(V, device="cuda"),
                      exact=1)
    torch.cuda.synchronize()
    uh, ul = _bf16_pair(U)
    vh, vl = _bf16_pair(V)
    for I in (0, 4, 8):                          # row panels (8: the one-row panel)
        P = X[I * 128:(I + 1) * 128]
        c, K, ph, pl = O.quantize_fp8_tiles(P)
        np.testing.assert_array_equal(hi[I * 128:(I + 1) * 128].cpu().numpy(), c)
        np.testing.assert_array_equal(ex[I].cpu().numpy(), K[0])
        np.testing.assert_array_equal(lo[I * 128:(I + 1) * 128].float().double().cpu().numpy(), pl)
        rows = rng.choice(P.shape[0], min(8, P.shape[0]), replace=False)
        want = (ph[rows] + pl[rows]) @ (vh + vl)
        got = XV[I * 128 + torch.as_tensor(rows, device="cuda")].double().cpu().numpy()
        assert _rel(got, want) < _accum_bound(m, n), I
    for J in (0, 517, 1023):                     # column panels
        P = X[:, J * 128:(J + 1) * 128]
        c, K, ph, pl = O.quantize_fp8_tiles(P)
        np.testing.assert_array_equal(ex[:, J].cpu().numpy(), K[:, 0])
        cols = rng.choice(128, 8, replace=False)
        want = (ph[:, cols] + pl[:, cols]).T @ (uh + ul)
        got = XtU[J * 128 + torch.as_tensor(cols, device="cuda")].double().cpu().numpy()
        assert _rel(got, want) < _accum_bound(n, m), J
    s.close()


def test_fp8_rejects_negative_x_and_batching():
    from paper_2605_19325_gb300 import binding as B
    from paper_2605_19325_gb300.solver import Solver
    X = torch.rand(256, 300, device="cuda")
    X[7, 9] = -1.0
    with pytest.raises(B.EnmfError) as ei:
        s = Solver(X, 8, x_stream=FP8)
        s.svd_init()
    assert ei.value.code == 2
    X = torch.rand(256, 300, device="cuda")
    s = Solver(X, 8, x_stream=FP8)
    b = B.enmf_batch_create(4)
    try:
        with pytest.raises(B.EnmfError) as ei:
            B.enmf_batch_add(b, s.ctx, X, s.U, s.V)
        assert ei.value.code == 1
    finally:
        B.enmf_batch_destroy(b)
        s.close()
