"""Allocation-free residual (enmf_residual_noalloc) against enmf_residual.

The allocation-free call forms every entry of X - U V^T with the same
arithmetic as enmf_residual(direct = 1); only the order of the FP64 sums
differs.  Each sum has N = m n nonnegative terms, so either order is within
(N - 1) 2^-53 of the exact sum, relatively: the two results agree within
2 N 2^-53.  Two calls in a row must agree bit for bit (the panel sums are
combined in a fixed order), and calls after the first must not change the
device's free memory.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2605_19325_gb300 import build
    build.build()


def _inputs(m, n, r, xdt, fdt, ldx=None, seed=0):
    X, U0, V0 = synth.planted(m, n, r, seed=seed, noise=0.05)
    rng = np.random.default_rng(seed + 1)
    U = U0 * rng.uniform(0.8, 1.2, U0.shape)
    V = V0 * rng.uniform(0.8, 1.2, V0.shape)
    ldx = ldx or n
    buf = torch.zeros((m, ldx), dtype=torch.float64)
    buf[:, :n] = torch.from_numpy(X)
    Xd = buf.to(device="cuda", dtype=xdt)[:, :n]
    Ud = torch.from_numpy(U).to(device="cuda", dtype=fdt).contiguous()
    Vd = torch.from_numpy(V).to(device="cuda", dtype=fdt).contiguous()
    return Xd, Ud, Vd


def _ctx_residual(X, U, V):
    from paper_2605_19325_gb300 import binding as B
    m, n = X.shape
    p = B.enmf_problem(m, n, X.stride(0), U.shape[1], B._dtype_code(X), B._dtype_code(U), 0)
    ctx = B.enmf_create(p)
    try:
        return B.enmf_residual(ctx, X, U, V, direct=1)
    finally:
        B.enmf_destroy(ctx)


CASES = [
    (300, 200, 5, torch.float64, torch.float64, None),
    (1000, 700, 32, torch.float32, torch.float32, None),
    (513, 1031, 49, torch.bfloat16, torch.float32, None),
    (129, 3, 2, torch.float16, torch.float32, None),
    (1, 64, 1, torch.float64, torch.float64, None),
    (4100, 260, 20, torch.float32, torch.float32, None),   # ragged last panel
    (200, 130, 7, torch.float64, torch.float64, 136),      # row stride > n
]


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,r,xdt,fdt,ldx", CASES)
def test_noalloc_matches_context_residual(m, n, r, xdt, fdt, ldx):
    from paper_2605_19325_gb300 import binding as B
    X, U, V = _inputs(m, n, r, xdt, fdt, ldx)
    ref = np.array(_ctx_residual(X, U, V))
    out_a = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    out_b = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    B.enmf_residual_noalloc(X, U, V, out_a)
    B.enmf_residual_noalloc(X, U, V, out_b)
    torch.cuda.synchronize()
    a, b = out_a.cpu().numpy(), out_b.cpu().numpy()
    assert np.array_equal(a, b), (a, b)
    tol = 2.0 * m * n * 2.0 ** -53 + 1e-15
    assert np.all(np.abs(a - ref) <= tol * np.abs(ref)), (a, ref, tol)
    assert a[0] > 0 and a[2] > 0


def _oracle_bound(X, U, V, f_dtype):
    """f of Eq. 1 by the oracle on the tensors' exact values, and a bound on
    the allowed difference: the entries x - u.v are formed with a dot product
    in the factors' type (r fused multiply-adds: each entry within
    gamma_r (|U| |V|^T)_ij of exact, gamma_r = r u / (1 - r u)), so f moves by at
    most gamma_r sum |E| (|U||V|^T) + gamma_r^2 sum (|U||V|^T)^2 / 2; the FP64
    sums of m n terms add 2 m n 2^-53 f."""
    from oracle import enmf_oracle as O
    Xh = X.double().cpu().numpy()
    Uh = U.double().cpu().numpy()
    Vh = V.double().cpu().numpy()
    m, n = Xh.shape
    r = Uh.shape[1]
    f = O.objective(Xh, Uh, Vh)
    u = 2.0 ** -24 if f_dtype == torch.float32 else 2.0 ** -53
    g = r * u / (1 - r * u)
    P = np.abs(Uh) @ np.abs(Vh).T
    E = Xh - Uh @ Vh.T
    bound = g * float(np.sum(np.abs(E) * P)) + 0.5 * g * g * float(np.sum(P * P))
    return f, O.rel_err(Xh, Uh, Vh), float(np.sum(Xh * Xh)), bound + 2 * m * n * 2.0 ** -53 * f


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,r,xdt,fdt,ldx", CASES)
def test_noalloc_matches_the_oracle(m, n, r, xdt, fdt, ldx):
    """The allocation-free residual against the oracle's f of Eq. 1, computed
    in FP64 from the same (exactly converted) X, U and V, within the rounding
    bound of the factors' dot product; two calls in a row."""
    from paper_2605_19325_gb300 import binding as B
    X, U, V = _inputs(m, n, r, xdt, fdt, ldx, seed=3)
    f, rel, nx2, bound = _oracle_bound(X, U, V, fdt)
    for _ in range(2):
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        B.enmf_residual_noalloc(X, U, V, out)
        torch.cuda.synchronize()
        a = out.cpu().numpy()
        assert abs(a[0] - f) <= bound, (a[0], f, bound)
        assert abs(a[2] - nx2) <= 2 * m * n * 2.0 ** -53 * nx2, (a[2], nx2)
        # rel = sqrt(2 f) / ||X||: the relative bound halves through the root
        assert abs(a[1] - rel) <= (0.5 * bound / f + 4 * m * n * 2.0 ** -53) * rel, (a[1], rel)


@pytest.mark.gpu
def test_noalloc_calls_leave_free_memory_unchanged():
    from paper_2605_19325_gb300 import binding as B
    X, U, V = _inputs(640, 300, 12, torch.float32, torch.float32)
    out = torch.empty((3,), dtype=torch.float64, device="cuda")
    B.enmf_residual_noalloc(X, U, V, out)      # first call: one-time set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        B.enmf_residual_noalloc(X, U, V, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.gpu
def test_noalloc_empty_inputs():
    from paper_2605_19325_gb300 import binding as B
    for m, n in ((0, 5), (5, 0)):
        X = torch.zeros((m, n), dtype=torch.float64, device="cuda")
        U = torch.zeros((m, 2), dtype=torch.float64, device="cuda")
        V = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        B.enmf_residual_noalloc(X, U, V, out)
        torch.cuda.synchronize()
        assert out.cpu().tolist() == [0.0, 0.0, 0.0]


def test_noalloc_rejects_bad_arguments_before_any_launch():
    """Checked on the host before any CUDA call, so this runs without a GPU."""
    from paper_2605_19325_gb300 import binding as B
    lib = B.lib()
    dummy = C.c_void_p(256)
    fn = lib.enmf_residual_noalloc
    big = B.ENMF_RESIDUAL_NOALLOC_MAX_ROWS + 1
    assert fn(dummy, B.ENMF_F64, big, 4, 4, dummy, dummy, 2, B.ENMF_F64, dummy, None) == 1
    assert fn(dummy, B.ENMF_F64, 10, 4, 3, dummy, dummy, 2, B.ENMF_F64, dummy, None) == 1  # ldx < n
    assert fn(dummy, B.ENMF_F64, 10, 4, 4, dummy, dummy, 0, B.ENMF_F64, dummy, None) == 1  # r = 0
    assert fn(dummy, B.ENMF_F64, 10, 4, 4, dummy, dummy, 65, B.ENMF_F64, dummy, None) == 1
    assert fn(dummy, B.ENMF_F32, 10, 4, 4, dummy, dummy, 2, B.ENMF_F64, dummy, None) == 1
    assert fn(dummy, B.ENMF_F64, 10, 4, 4, dummy, dummy, 2, B.ENMF_F64, None, None) == 1
    assert fn(None, B.ENMF_F64, 10, 4, 4, dummy, dummy, 2, B.ENMF_F64, dummy, None) == 1
    with pytest.raises(B.EnmfError, match="ENMF_RESIDUAL_NOALLOC_MAX_ROWS"):
        X = torch.zeros((big, 1), dtype=torch.float64)
        U = torch.zeros((big, 1), dtype=torch.float64)
        V = torch.zeros((1, 1), dtype=torch.float64)
        B.enmf_residual_noalloc(X, U, V, torch.zeros(3, dtype=torch.float64),
                                stream=_FakeStream())


class _FakeStream:
    cuda_stream = 0


def test_noalloc_wrapper_checks_tensors_before_calling_the_library(monkeypatch):
    """Each malformed tensor argument is refused on the host: the C entry point
    sees only pointers, so these would otherwise read or write out of bounds."""
    from paper_2605_19325_gb300 import binding as B

    def no_call():
        raise AssertionError("the library was called")

    monkeypatch.setattr(B, "lib", no_call)
    f64, f32 = torch.float64, torch.float32
    X = torch.zeros((10, 6), dtype=f64)
    U = torch.zeros((10, 3), dtype=f64)
    V = torch.zeros((6, 3), dtype=f64)
    out = torch.zeros(3, dtype=f64)
    bad = [
        (X, U.t().contiguous().t(), V, out),                    # U not contiguous
        (X, torch.zeros((3, 10), dtype=f64), V, out),           # U transposed shape
        (X, U, torch.zeros((5, 3), dtype=f64), out),            # V too short
        (X, U, torch.zeros((6, 4), dtype=f64), out),            # rank mismatch
        (X, U, V.to(f32), out),                                 # mixed factor dtypes
        (X, U, V, torch.zeros(3, dtype=f32)),                   # out3 not float64
        (X, U, V, torch.zeros(2, dtype=f64)),                   # out3 too short
        (X, U, V, torch.zeros(6, dtype=f64)[::2]),              # out3 strided
        (X.t(), torch.zeros((6, 3), dtype=f64), torch.zeros((10, 3), dtype=f64), out),
        (torch.zeros(1, 6, dtype=f64).expand(10, 6), U, V, out),   # row stride 0 < n
        (torch.zeros(60, dtype=f64), U, V, out),                # X not a matrix
        (X, U, V, out),                                         # tensors not on the GPU
    ]
    for args in bad:
        with pytest.raises(ValueError):
            B.enmf_residual_noalloc(*args)
