"""ctypes binding of libenmf.so: the C ABI of include/enmf.h, same names.

Argument marshalling only -- every step of the factorisation runs in the CUDA
kernels of the library.  Tensors are passed as device pointers; PyTorch is
used for device memory and streams.  If the library is missing this module
raises on import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libenmf.so")

ENMF_F64, ENMF_F32, ENMF_BF16, ENMF_F16, ENMF_E4M3, ENMF_CSR = 0, 1, 2, 3, 4, 5
ENMF_MAX_RANK = 64
ENMF_RESIDUAL_NOALLOC_MAX_ROWS = 262144
ENMF_STATE_BYTES = 128

STATUS = {0: "ok", 1: "EINVAL", 2: "EDOMAIN", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT",
          6: "ENOTCONV", 7: "EBUSY", 8: "ESTATE"}


class EnmfError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class enmf_problem(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("ldx", C.c_int64), ("r", C.c_int32),
                ("x_dtype", C.c_int32), ("f_dtype", C.c_int32), ("stream_dtype", C.c_int32),
                ("nnz", C.c_int64)]


class enmf_csr(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class CsrMatrix:
    """X of the sparse form (x_dtype ENMF_CSR): compressed rows in CUDA
    tensors -- row_ptr int64 (m + 1), col int32 (nnz), val float32 or float64
    (nnz, the factors' type) -- with shape (m, n).  Wherever the C ABI takes X
    it gets the address of this object's enmf_csr descriptor (data_ptr()).
    Only shapes, types, devices and contiguity are checked here; the entries
    themselves are checked by the library on the device."""

    def __init__(self, row_ptr, col, val, shape):
        m, n = int(shape[0]), int(shape[1])
        for name, t, dt in (("row_ptr", row_ptr, "torch.int64"), ("col", col, "torch.int32")):
            if not t.is_cuda or not t.is_contiguous() or t.dim() != 1 or str(t.dtype) != dt:
                raise ValueError(f"{name} must be a contiguous 1-D CUDA {dt} tensor")
        if str(val.dtype) not in ("torch.float32", "torch.float64"):
            raise ValueError("val must be float32 or float64")
        if not val.is_cuda or not val.is_contiguous() or val.dim() != 1:
            raise ValueError("val must be a contiguous 1-D CUDA tensor")
        if row_ptr.numel() != m + 1 or col.numel() != val.numel():
            raise ValueError("row_ptr must have m + 1 entries and col, val nnz entries each")
        if not (row_ptr.device == col.device == val.device):
            raise ValueError("row_ptr, col and val must be on one device")
        self.row_ptr, self.col, self.val = row_ptr, col, val
        self.shape = (m, n)
        self.nnz = int(val.numel())
        self.dtype = val.dtype
        self.device = val.device
        self.is_cuda = True
        self.desc = enmf_csr(row_ptr.data_ptr(), col.data_ptr() if self.nnz else None,
                             val.data_ptr() if self.nnz else None)

    def data_ptr(self):
        return C.addressof(self.desc)


class enmf_svd_opts(C.Structure):
    _fields_ = [("oversample", C.c_int32), ("max_iters", C.c_int32), ("tol", C.c_double),
                ("seed", C.c_uint64), ("fp32_finish", C.c_int32)]


class enmf_svd_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("rank", C.c_int32), ("residual", C.c_double)]


class enmf_admm_opts(C.Structure):
    _fields_ = [("rho", C.c_double), ("rho_scale", C.c_double), ("max_iter", C.c_int32),
                ("tol", C.c_double), ("f64", C.c_int32)]


class enmf_rotate_info(C.Structure):
    _fields_ = [("steps", C.c_int32), ("converged", C.c_int32), ("rho", C.c_double),
                ("dR", C.c_double), ("neg_mass_in", C.c_double), ("neg_mass_out", C.c_double)]


class enmf_iter_opts(C.Structure):
    _fields_ = [("n_iter", C.c_int32), ("pbcd_max_iter", C.c_int32), ("eps", C.c_double),
                ("n_shift", C.c_int32), ("trace", C.c_void_p), ("reset", C.c_int32),
                ("sync_info", C.c_int32), ("correct_every", C.c_int32)]


class enmf_iter_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("asc_iters", C.c_int32), ("hals_iters", C.c_int32),
                ("stage", C.c_int32), ("s_u", C.c_double), ("s_v", C.c_double)]


class enmf_kkt_report(C.Structure):
    _fields_ = [("min_w", C.c_double), ("min_grad", C.c_double), ("delta", C.c_double),
                ("sigma", C.c_double), ("pg_norm", C.c_double), ("pg_rel", C.c_double)]


class enmf_nmc_start_opts(C.Structure):
    _fields_ = [("max_sweeps", C.c_int32), ("lam", C.c_double), ("tol", C.c_double),
                ("svd_max_iters", C.c_int32)]


class enmf_nmc_start_info(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("f", C.c_double)]


_SIGS = {
    "enmf_nmc_start": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(enmf_nmc_start_opts), C.POINTER(enmf_nmc_start_info)]),
    "enmf_nmc_iterate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(enmf_iter_opts), C.POINTER(enmf_iter_info)]),
    "enmf_nmc_objective": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_double)]),
    "enmf_workspace_size": (C.c_int, [C.POINTER(enmf_problem), C.POINTER(C.c_size_t)]),
    "enmf_create": (C.c_int, [C.POINTER(enmf_problem), C.c_void_p, C.POINTER(C.c_void_p)]),
    "enmf_destroy": (None, [C.c_void_p]),
    "enmf_status_string": (C.c_char_p, [C.c_int]),
    "enmf_svd_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(enmf_svd_opts), C.POINTER(enmf_svd_info)]),
    "enmf_rotate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.POINTER(enmf_admm_opts), C.POINTER(enmf_rotate_info)]),
    "enmf_svd_init_group": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.c_int32,
                                      C.POINTER(enmf_svd_opts), C.POINTER(enmf_svd_info),
                                      C.POINTER(C.c_int)]),
    "enmf_rotate_group": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p), C.c_int32,
                                    C.POINTER(enmf_admm_opts), C.POINTER(enmf_rotate_info)]),
    "enmf_iterate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(enmf_iter_opts), C.POINTER(enmf_iter_info)]),
    "enmf_pbcd_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32,
                                   C.POINTER(C.c_int32)]),
    "enmf_residual": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_double), C.c_int32]),
    "enmf_kkt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.POINTER(enmf_kkt_report)]),
    "enmf_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                             C.POINTER(enmf_svd_opts), C.POINTER(enmf_admm_opts),
                             C.POINTER(enmf_iter_opts), C.POINTER(C.c_double)]),
    "enmf_stage_x": (C.c_int, [C.c_void_p, C.c_void_p]),
    "enmf_stage_copy": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "enmf_state_export": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "enmf_state_import": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "enmf_sweep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_int32]),
    "enmf_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "enmf_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                    C.c_int32]),
    "enmf_probe_fma_peak": (C.c_int, [C.c_int32, C.POINTER(C.c_double)]),
    "enmf_launch_count": (C.c_longlong, []),
    "enmf_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "enmf_set_fused": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "enmf_set_overlap": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "enmf_rotate_general": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(enmf_admm_opts),
                                      C.POINTER(enmf_rotate_info)]),
    "enmf_equiv_transform": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_double)]),
    "enmf_perm_check": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                  C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "enmf_fused_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32)]),
    "enmf_fused_stamps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "enmf_probe_wait": (C.c_int, [C.c_int32, C.c_int64, C.POINTER(C.c_int32)]),
    "enmf_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "enmf_batch_destroy": (None, [C.c_void_p]),
    "enmf_batch_add": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.POINTER(C.c_int32)]),
    "enmf_batch_remove": (C.c_int, [C.c_void_p, C.c_int32]),
    "enmf_batch_size": (C.c_int32, [C.c_void_p]),
    "enmf_batch_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "enmf_batch_member": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_double)]),
    "enmf_batch_tune": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "enmf_batch_states": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p,
                                    C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_int32)]),
    "enmf_residual_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                                        C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                        C.c_void_p]),
    "enmf_version": (C.c_char_p, []),
}

EXPORTED = tuple(_SIGS)


def load(path=LIB_PATH):
    """Load libenmf.so and declare its signatures; raise if it is missing."""
    if not os.path.exists(path):
        raise ImportError(f"libenmf.so not built ({path}); run paper_2605_19325_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(code, where):
    if code != 0:
        raise EnmfError(code, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------- C ABI mirror
def enmf_workspace_size(problem):
    out = C.c_size_t(0)
    check(lib().enmf_workspace_size(C.byref(problem), C.byref(out)), "enmf_workspace_size")
    return out.value


def enmf_create(problem, stream=None):
    h = C.c_void_p()
    check(lib().enmf_create(C.byref(problem), _stream(stream), C.byref(h)), "enmf_create")
    return h


def enmf_destroy(ctx):
    lib().enmf_destroy(ctx)


def enmf_svd_init(ctx, X, U, V, sigma=None, opts=None):
    info = enmf_svd_info()
    code = lib().enmf_svd_init(ctx, _ptr(X), _ptr(U), _ptr(V), _ptr(sigma),
                               C.byref(opts) if opts is not None else None, C.byref(info))
    if code not in (0, 6):
        check(code, "enmf_svd_init")
    return info, code


def enmf_rotate(ctx, U, V, R=None, opts=None):
    info = enmf_rotate_info()
    code = lib().enmf_rotate(ctx, _ptr(U), _ptr(V), _ptr(R),
                             C.byref(opts) if opts is not None else None, C.byref(info))
    if code not in (0, 6):
        check(code, "enmf_rotate")
    return info, code


def enmf_svd_init_group(ctxs, Xs, Us, Vs, sigmas=None, opts=None):
    """The SVD start for several contexts (one stream); returns (infos,
    per-problem status codes)."""
    n = len(ctxs)
    cs = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    xs = (C.c_void_p * n)(*[X.data_ptr() for X in Xs])
    us = (C.c_void_p * n)(*[U.data_ptr() for U in Us])
    vs = (C.c_void_p * n)(*[V.data_ptr() for V in Vs])
    ss = (C.c_void_p * n)(*[(s.data_ptr() if s is not None else None) for s in sigmas]) \
        if sigmas is not None else None
    infos = (enmf_svd_info * n)()
    status = (C.c_int * n)()
    check(lib().enmf_svd_init_group(cs, xs, us, vs, ss, n,
                                    C.byref(opts) if opts is not None else None, infos, status),
          "enmf_svd_init_group")
    for code in status:
        if code not in (0, 6):
            check(code, "enmf_svd_init_group")
    return list(infos), list(status)


def enmf_rotate_group(ctxs, Us, Vs, opts=None):
    """Algorithm 1 for several contexts at once (FP32 factors, one rank pad,
    one stream); returns (per-problem infos, status), status 0 or ENOTCONV
    (6) as enmf_rotate."""
    n = len(ctxs)
    cs = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    us = (C.c_void_p * n)(*[U.data_ptr() for U in Us])
    vs = (C.c_void_p * n)(*[V.data_ptr() for V in Vs])
    infos = (enmf_rotate_info * n)()
    code = lib().enmf_rotate_group(cs, us, vs, n, C.byref(opts) if opts is not None else None,
                                   infos)
    if code not in (0, 6):
        check(code, "enmf_rotate_group")
    return list(infos), code


def enmf_stage_x(ctx, X):
    check(lib().enmf_stage_x(ctx, _ptr(X)), "enmf_stage_x")


def enmf_stage_copy(ctx, hi=None, lo=None, tile_exp=None):
    """Copy the staged X_hi / X_lo (m x n dense) and, in the FP8 form, the
    per-tile exponents (int32) into the given tensors (any may be None)."""
    check(lib().enmf_stage_copy(ctx, _ptr(hi), _ptr(lo), _ptr(tile_exp)), "enmf_stage_copy")


def enmf_state_export(ctx):
    """The context's iteration state as ENMF_STATE_BYTES bytes."""
    buf = (C.c_char * ENMF_STATE_BYTES)()
    n = C.c_size_t(ENMF_STATE_BYTES)
    check(lib().enmf_state_export(ctx, buf, C.byref(n)), "enmf_state_export")
    return bytes(buf[:n.value])


def enmf_state_import(ctx, blob):
    """Load an exported iteration state into a context of the same problem."""
    buf = C.create_string_buffer(bytes(blob), len(blob))
    check(lib().enmf_state_import(ctx, buf, len(blob)), "enmf_state_import")


def enmf_sweep(ctx, X, U, V, XV=None, XtU=None, exact=1):
    check(lib().enmf_sweep(ctx, _ptr(X), _ptr(U), _ptr(V), _ptr(XV), _ptr(XtU), exact),
          "enmf_sweep")


def enmf_iterate(ctx, X, U, V, n_iter, trace=None, reset=0, eps=1e-4, pbcd_max_iter=5,
                 n_shift=3, sync_info=1, correct_every=10):
    o = enmf_iter_opts(n_iter, pbcd_max_iter, eps, n_shift,
                       None if trace is None else trace.data_ptr(), reset, sync_info,
                       correct_every)
    info = enmf_iter_info()
    check(lib().enmf_iterate(ctx, _ptr(X), _ptr(U), _ptr(V), C.byref(o),
                             C.byref(info) if sync_info else None), "enmf_iterate")
    return info


def enmf_nmc_start(ctx, X, U, V, max_sweeps=50, lam=1e-3, tol=1e-10, svd_max_iters=0):
    o = enmf_nmc_start_opts(max_sweeps, lam, tol, svd_max_iters)
    info = enmf_nmc_start_info()
    code = lib().enmf_nmc_start(ctx, _ptr(X), _ptr(U), _ptr(V), C.byref(o), C.byref(info))
    if code not in (0, 6):
        check(code, "enmf_nmc_start")
    return info


def enmf_nmc_iterate(ctx, X, U, V, n_iter, trace=None, reset=0, eps=1e-4, pbcd_max_iter=5,
                     n_shift=3, sync_info=1):
    o = enmf_iter_opts(n_iter, pbcd_max_iter, eps, n_shift,
                       None if trace is None else trace.data_ptr(), reset, sync_info, 10)
    info = enmf_iter_info()
    check(lib().enmf_nmc_iterate(ctx, _ptr(X), _ptr(U), _ptr(V), C.byref(o),
                                 C.byref(info) if sync_info else None), "enmf_nmc_iterate")
    return info


def enmf_nmc_objective(ctx, X, U, V):
    out = (C.c_double * 2)()
    check(lib().enmf_nmc_objective(ctx, _ptr(X), _ptr(U), _ptr(V), out), "enmf_nmc_objective")
    return out[0], out[1]


def enmf_pbcd_counts(ctx, cap=8192):
    buf = (C.c_int32 * cap)()
    cnt = C.c_int32(0)
    check(lib().enmf_pbcd_counts(ctx, buf, cap, C.byref(cnt)), "enmf_pbcd_counts")
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(min(cnt.value, cap // 2))]


def enmf_residual(ctx, X, U, V, direct=1):
    out = (C.c_double * 3)()
    check(lib().enmf_residual(ctx, _ptr(X), _ptr(U), _ptr(V), out, direct), "enmf_residual")
    return out[0], out[1], out[2]


def enmf_kkt(ctx, X, U, V):
    rep = enmf_kkt_report()
    check(lib().enmf_kkt(ctx, _ptr(X), _ptr(U), _ptr(V), C.byref(rep)), "enmf_kkt")
    return rep


def enmf_profile(ctx, every):
    check(lib().enmf_profile(ctx, every), "enmf_profile")


def enmf_profile_read(ctx, reset=1):
    ms = C.c_double(0)
    n = C.c_int64(0)
    check(lib().enmf_profile_read(ctx, C.byref(ms), C.byref(n), reset), "enmf_profile_read")
    return ms.value, n.value


def enmf_probe_fma_peak(dtype):
    out = C.c_double(0)
    check(lib().enmf_probe_fma_peak(dtype, C.byref(out)), "enmf_probe_fma_peak")
    return out.value


def enmf_launch_count():
    return int(lib().enmf_launch_count())


def enmf_batch_create(max_members, stream=None, pbcd_max_iter=5, eps=1e-4, n_shift=3,
                      correct_every=10):
    o = enmf_iter_opts(0, pbcd_max_iter, eps, n_shift, None, 0, 0, correct_every)
    h = C.c_void_p()
    check(lib().enmf_batch_create(C.byref(o), max_members, _stream(stream), C.byref(h)),
          "enmf_batch_create")
    return h


def enmf_batch_destroy(b):
    lib().enmf_batch_destroy(b)


def enmf_batch_add(b, ctx, X, U, V):
    slot = C.c_int32(-1)
    check(lib().enmf_batch_add(b, ctx, _ptr(X), _ptr(U), _ptr(V), C.byref(slot)), "enmf_batch_add")
    return slot.value


def enmf_batch_remove(b, slot):
    check(lib().enmf_batch_remove(b, slot), "enmf_batch_remove")


def enmf_batch_size(b):
    return int(lib().enmf_batch_size(b))


def enmf_batch_step(b, n_alt):
    check(lib().enmf_batch_step(b, n_alt), "enmf_batch_step")


def enmf_batch_member(b, slot):
    info = enmf_iter_info()
    f = C.c_double(0)
    check(lib().enmf_batch_member(b, slot, C.byref(info), C.byref(f)), "enmf_batch_member")
    return info, f.value


def enmf_batch_states(b, cap):
    """{slot: (enmf_iter_info, f)} for every member, read in one copy."""
    slots = (C.c_int32 * cap)()
    infos = (enmf_iter_info * cap)()
    f = (C.c_double * cap)()
    n = C.c_int32(0)
    check(lib().enmf_batch_states(b, slots, infos, f, cap, C.byref(n)), "enmf_batch_states")
    return {slots[i]: (infos[i], f[i]) for i in range(n.value)}


def enmf_batch_tune(b):
    g = C.c_int32(0)
    ms = C.c_float(0)
    check(lib().enmf_batch_tune(b, C.byref(g), C.byref(ms)), "enmf_batch_tune")
    return g.value, ms.value


def enmf_set_wait_limit(ctx, cycles):
    """Spin limit (SM cycles) of the context's grid barriers; 0 = default."""
    check(lib().enmf_set_wait_limit(ctx, int(cycles)), "enmf_set_wait_limit")


def enmf_rotate_general(ctx, U, V, R1, lam, R2, opts=None):
    """Algorithm 4 in place on U, V; R1, lam, R2 device FP64 outputs."""
    info = enmf_rotate_info()
    code = lib().enmf_rotate_general(ctx, _ptr(U), _ptr(V), _ptr(R1), _ptr(lam), _ptr(R2),
                                     C.byref(opts) if opts is not None else None, C.byref(info))
    if code not in (0, 6):
        check(code, "enmf_rotate_general")
    return info, code


def enmf_equiv_transform(ctx, Ue, Ve, Ua, Va, R1, lam, R2):
    """App. F transform into the device tensors R1, lam, R2; returns (delta_u, delta_v)."""
    d = (C.c_double * 2)()
    check(lib().enmf_equiv_transform(ctx, _ptr(Ue), _ptr(Ve), _ptr(Ua), _ptr(Va), _ptr(R1),
                                     _ptr(lam), _ptr(R2), d), "enmf_equiv_transform")
    return d[0], d[1]


def enmf_perm_check(ctx, UA, UB, r, eps=0.05, keep_frac=0.9):
    """App. H permutation check: list (length r) of matched U_B columns or -1."""
    out = (C.c_int32 * r)()
    kept = C.c_int32(0)
    check(lib().enmf_perm_check(ctx, _ptr(UA), _ptr(UB), eps, keep_frac, out, C.byref(kept)),
          "enmf_perm_check")
    return list(out), kept.value


def enmf_set_fused(ctx, on):
    """Use the fused single-pass HALS alternation (1) or not (0, default);
    returns whether the context can run it."""
    av = C.c_int32(0)
    check(lib().enmf_set_fused(ctx, 1 if on else 0, C.byref(av)), "enmf_set_fused")
    return bool(av.value)


def enmf_set_overlap(ctx, flags=-1):
    """Programmatic dependent launches in the captured loop (bit 0: sweeps
    after half steps, bit 1: half steps after sweeps); flags < 0 only reads.
    Returns the flags in effect."""
    cur = C.c_int32(0)
    check(lib().enmf_set_overlap(ctx, int(flags), C.byref(cur)), "enmf_set_overlap")
    return cur.value


def enmf_fused_shape(ctx):
    """(available, CTAs per cluster, clusters, columns per CTA, stages, smem KB)."""
    out = (C.c_int32 * 6)()
    check(lib().enmf_fused_shape(ctx, out), "enmf_fused_shape")
    return tuple(out)


def enmf_fused_stamps(ctx):
    """The fused pass's phase stamps (ns) as a list, empty when not recorded."""
    n = C.c_int64(0)
    check(lib().enmf_fused_stamps(ctx, None, 0, C.byref(n)), "enmf_fused_stamps")
    if n.value == 0:
        return []
    buf = (C.c_longlong * n.value)()
    check(lib().enmf_fused_stamps(ctx, buf, n.value, C.byref(n)), "enmf_fused_stamps")
    return list(buf)


def enmf_probe_wait(kind, cycles):
    """Status (0 ok, 5 ETIMEOUT) of a bounded wait on an event that never occurs."""
    st = C.c_int32(-1)
    check(lib().enmf_probe_wait(int(kind), int(cycles), C.byref(st)), "enmf_probe_wait")
    return st.value


def enmf_solve(ctx, X_ptr, U_ptr, V_ptr, n_iter):
    """Whole Algorithm 3 through one call; pointers may be host or device."""
    out = (C.c_double * 3)()
    check(lib().enmf_solve(ctx, C.c_void_p(X_ptr), C.c_void_p(U_ptr), C.c_void_p(V_ptr),
                           n_iter, None, None, None, out), "enmf_solve")
    return out[0], out[1], out[2]


_TORCH_DT = None


def _dtype_code(t):
    global _TORCH_DT
    if _TORCH_DT is None:
        import torch
        _TORCH_DT = {torch.float64: ENMF_F64, torch.float32: ENMF_F32,
                     torch.bfloat16: ENMF_BF16, torch.float16: ENMF_F16}
    if t.dtype not in _TORCH_DT:
        raise ValueError(f"unsupported dtype {t.dtype}")
    return _TORCH_DT[t.dtype]


def _noalloc_args(X, U, V, out3):
    """Host-side checks of enmf_residual_noalloc's tensors.

    The C entry point sees only pointers and sizes, so a wrong shape, a
    transposed or strided factor, or a short or mistyped out3 would become an
    out-of-bounds device access.  Every such case raises ValueError here,
    before the library is called.  Returns (m, n, ldx, r)."""
    if isinstance(X, CsrMatrix):
        raise ValueError("enmf_residual_noalloc takes a dense X")
    if X.dim() != 2:
        raise ValueError("X must be a matrix")
    m, n = X.shape
    if U.dim() != 2 or V.dim() != 2:
        raise ValueError("U and V must be matrices")
    r = U.shape[1]
    if tuple(U.shape) != (m, r):
        raise ValueError(f"U has shape {tuple(U.shape)}, expected ({m}, r)")
    if tuple(V.shape) != (n, r):
        raise ValueError(f"V has shape {tuple(V.shape)}, expected ({n}, {r})")
    if U.dtype != V.dtype:
        raise ValueError(f"U and V differ in dtype ({U.dtype} vs {V.dtype})")
    if not (U.is_contiguous() and V.is_contiguous()):
        raise ValueError("U and V must be contiguous (row-major, leading dimension r)")
    if m > 0 and n > 0:
        if n > 1 and X.stride(1) != 1:
            raise ValueError("X must be a row-major matrix (unit column stride)")
        if m > 1 and X.stride(0) < n:
            raise ValueError(f"X row stride {X.stride(0)} is below n = {n} (rows overlap)")
    ldx = X.stride(0) if m > 1 else n
    ldx = max(ldx, n)
    if out3.dtype != _float64() or not out3.is_contiguous() or out3.numel() < 3:
        raise ValueError("out3 must be a contiguous float64 tensor of at least 3 elements")
    _dtype_code(X)
    _dtype_code(U)
    return m, n, ldx, r


def _float64():
    import torch
    return torch.float64


def enmf_residual_noalloc(X, U, V, out3, stream=None):
    """Allocation-free residual into the device tensor out3 (3 doubles).

    Enqueues on `stream` (default: the current torch stream) and returns
    without synchronising.  X is (m, n) with unit column stride; U (m, r) and
    V (n, r) are contiguous and of one dtype; out3 is a contiguous float64
    tensor; all four live on the current CUDA device.  Bad arguments raise
    ValueError (or EnmfError for m beyond the row limit) before any launch."""
    import torch
    m, n, ldx, r = _noalloc_args(X, U, V, out3)
    if m > ENMF_RESIDUAL_NOALLOC_MAX_ROWS:
        raise EnmfError(1, f"enmf_residual_noalloc: m = {m} exceeds "
                           f"ENMF_RESIDUAL_NOALLOC_MAX_ROWS = {ENMF_RESIDUAL_NOALLOC_MAX_ROWS}")
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t in (("X", X), ("U", U), ("V", V), ("out3", out3)):
        if t.device.type != "cuda" or t.device.index != dev:
            raise ValueError(f"{name} must be on the current CUDA device (cuda:{dev}), "
                             f"not {t.device}")
    code = lib().enmf_residual_noalloc(
        _ptr(X), _dtype_code(X), m, n, ldx, _ptr(U), _ptr(V), r,
        _dtype_code(U), _ptr(out3), _stream(stream))
    check(code, "enmf_residual_noalloc")
