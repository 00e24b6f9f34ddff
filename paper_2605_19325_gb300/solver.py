"""Python convenience layer over the C ABI: one Solver per (X, r) problem.

Only marshalling: tensors are allocated with PyTorch on the current CUDA
device and their pointers handed to libenmf.  All arithmetic happens in the
library's CUDA kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B

_XDT = {torch.float64: B.ENMF_F64, torch.float32: B.ENMF_F32, torch.bfloat16: B.ENMF_BF16,
        torch.float16: B.ENMF_F16}


def problem_for(X, r, f_dtype=None, stream=None):
    """C problem descriptor for X (m x n, row-major) at rank r.

    stream=torch.bfloat16 (or torch.float16) selects the precision form: the
    iteration's X sweeps run on the tensor cores over a BF16 (FP16) copy of X,
    with the X_lo correction when X is FP32.  stream=torch.float8_e4m3fn (FP32
    X only) selects the FP8 form: e4m3 codes with a power-of-two scale per
    128 x 128 tile, and a BF16 X_lo correction.  X may also be a
    binding.CsrMatrix (the sparse form, compressed rows)."""
    if isinstance(X, B.CsrMatrix):
        if stream not in (None,):
            raise ValueError("the sparse form has no tensor-core stream")
        if f_dtype is not None and f_dtype != X.dtype:
            raise ValueError("the sparse form's factors have the values' type")
        fdt = B.ENMF_F64 if X.dtype == torch.float64 else B.ENMF_F32
        return B.enmf_problem(X.shape[0], X.shape[1], X.shape[1], r, B.ENMF_CSR, fdt, 0,
                              X.nnz), X.dtype
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be a row-major matrix (unit column stride)")
    xdt = _XDT.get(X.dtype)
    if xdt is None:
        raise ValueError(f"unsupported X dtype {X.dtype}")
    if f_dtype is None:
        f_dtype = torch.float64 if X.dtype == torch.float64 else torch.float32
    fdt = B.ENMF_F64 if f_dtype == torch.float64 else B.ENMF_F32
    sdt = {torch.bfloat16: B.ENMF_BF16, torch.float16: B.ENMF_F16,
           torch.float8_e4m3fn: B.ENMF_E4M3}.get(stream, 0)
    return B.enmf_problem(X.shape[0], X.shape[1], X.stride(0), r, xdt, fdt, sdt), f_dtype


@dataclass
class SolveResult:
    U: torch.Tensor
    V: torch.Tensor
    sigma: torch.Tensor
    R: torch.Tensor
    trace: torch.Tensor
    svd: object
    rot: object
    it: object


class Solver:
    """eNMF on one matrix: svd_init -> rotate -> iterate (Algorithm 3)."""

    def __init__(self, X: torch.Tensor, r: int, f_dtype=None, stream=None, x_stream=None):
        if not X.is_cuda:
            raise ValueError("X must be a CUDA tensor")
        self.X = X
        self.r = r
        self.problem, self.f_dtype = problem_for(X, r, f_dtype, x_stream)
        self.stream = stream
        self.ctx = B.enmf_create(self.problem, stream)
        if x_stream in (torch.bfloat16, torch.float16, torch.float8_e4m3fn):
            B.enmf_stage_x(self.ctx, X)
        dev = X.device
        self.U = torch.zeros(X.shape[0], r, dtype=self.f_dtype, device=dev)
        self.V = torch.zeros(X.shape[1], r, dtype=self.f_dtype, device=dev)
        self.sigma = torch.zeros(r, dtype=torch.float64, device=dev)
        self.R = torch.zeros(r, r, dtype=torch.float64, device=dev)

    def close(self):
        if self.ctx is not None:
            B.enmf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def svd_init(self, opts=None):
        info, code = B.enmf_svd_init(self.ctx, self.X, self.U, self.V, self.sigma, opts)
        return info

    def rotate(self, opts=None):
        info, code = B.enmf_rotate(self.ctx, self.U, self.V, self.R, opts)
        return info

    def iterate(self, n_iter, trace=True, reset=0, **kw):
        tr = torch.zeros(max(n_iter, 1), dtype=torch.float64, device=self.X.device) if trace else None
        info = B.enmf_iterate(self.ctx, self.X, self.U, self.V, n_iter, trace=tr, reset=reset, **kw)
        return (tr[:n_iter] if trace else None), info

    def nmc_start(self, **kw):
        """The masked-ALS start of Algorithm eNMC (App. C) in place on U, V
        (sparse form: the stored entries are the known ones)."""
        return B.enmf_nmc_start(self.ctx, self.X, self.U, self.V, **kw)

    def nmc_iterate(self, n_iter, trace=True, reset=0, **kw):
        """n_iter rounds of Algorithm eNMC; returns (f^ per round, info)."""
        tr = torch.zeros(max(n_iter, 1), dtype=torch.float64, device=self.X.device) if trace else None
        info = B.enmf_nmc_iterate(self.ctx, self.X, self.U, self.V, n_iter, trace=tr, reset=reset, **kw)
        return (tr[:n_iter] if trace else None), info

    def nmc_objective(self):
        return B.enmf_nmc_objective(self.ctx, self.X, self.U, self.V)

    def rotate_general(self, opts=None):
        """Algorithm 4 (Eq. 5) in place on U, V: returns (info, R1, lam, R2)."""
        dev = self.X.device
        R1 = torch.empty(self.r, self.r, dtype=torch.float64, device=dev)
        R2 = torch.empty(self.r, self.r, dtype=torch.float64, device=dev)
        lam = torch.empty(self.r, dtype=torch.float64, device=dev)
        info, code = B.enmf_rotate_general(self.ctx, self.U, self.V, R1, lam, R2, opts)
        return info, R1, lam, R2

    def residual(self, direct=True):
        return B.enmf_residual(self.ctx, self.X, self.U, self.V, 1 if direct else 0)

    def kkt(self):
        return B.enmf_kkt(self.ctx, self.X, self.U, self.V)

    def sweep(self, U=None, V=None, exact=1):
        """(X V, X^T U) for the given (or current) factors, in this form."""
        U = self.U if U is None else U
        V = self.V if V is None else V
        XV = torch.empty(self.X.shape[0], self.r, dtype=self.f_dtype, device=self.X.device)
        XtU = torch.empty(self.X.shape[1], self.r, dtype=self.f_dtype, device=self.X.device)
        B.enmf_sweep(self.ctx, self.X, U, V, XV, XtU, exact)
        return XV, XtU

    def export_state(self):
        """The iteration state (stage, shift steps, counters) as bytes; with
        copies of U and V it resumes the iteration in another Solver of the
        same problem (import_state, then iterate(..., reset=0))."""
        return B.enmf_state_export(self.ctx)

    def import_state(self, blob):
        B.enmf_state_import(self.ctx, blob)

    def staged(self):
        """The staged decomposition of X (tensor-core forms): X_hi (e4m3 codes
        as uint8 in the FP8 form, else BF16 / FP16), X_lo (16-bit, None when X
        was given in the stream type) and the FP8 form's per-tile exponents
        (int32, else None), copied to new device tensors."""
        m, n = self.X.shape
        dev = self.X.device
        sdt = self.problem.stream_dtype
        hi_dt = {B.ENMF_E4M3: torch.uint8, B.ENMF_F16: torch.float16}.get(sdt, torch.bfloat16)
        lo_dt = torch.float16 if sdt == B.ENMF_F16 else torch.bfloat16
        hi = torch.empty(m, n, dtype=hi_dt, device=dev)
        lo = (torch.empty(m, n, dtype=lo_dt, device=dev)
              if self.X.dtype == torch.float32 else None)
        exps = (torch.empty((m + 127) // 128, (n + 127) // 128, dtype=torch.int32, device=dev)
                if sdt == B.ENMF_E4M3 else None)
        B.enmf_stage_copy(self.ctx, hi, lo, exps)
        return hi, lo, exps

    def pbcd_counts(self):
        return B.enmf_pbcd_counts(self.ctx)

    def equiv_transform(self, Ua, Va, Ue=None, Ve=None):
        """App. F: (R1, lam, R2, delta_u, delta_v) relating (Ue, Ve) (default:
        this solver's U, V) to another factorisation (Ua, Va) of the same
        problem."""
        Ue = self.U if Ue is None else Ue
        Ve = self.V if Ve is None else Ve
        dev = self.X.device
        R1 = torch.empty(self.r, self.r, dtype=torch.float64, device=dev)
        R2 = torch.empty(self.r, self.r, dtype=torch.float64, device=dev)
        lam = torch.empty(self.r, dtype=torch.float64, device=dev)
        du, dv = B.enmf_equiv_transform(self.ctx, Ue, Ve, Ua, Va, R1, lam, R2)
        return R1, lam, R2, du, dv

    def perm_check(self, UB, UA=None, eps=0.05, keep_frac=0.9):
        """App. H: for each column of UA (default: this solver's U) the
        matched column of UB, or -1; and the number of matches."""
        UA = self.U if UA is None else UA
        return B.enmf_perm_check(self.ctx, UA, UB, self.r, eps, keep_frac)


def solve(X: torch.Tensor, r: int, n_iter: int, f_dtype=None, x_stream=None) -> SolveResult:
    """Algorithm 3 end to end on the GPU."""
    s = Solver(X, r, f_dtype, x_stream=x_stream)
    try:
        si = s.svd_init()
        ri = s.rotate()
        tr, ii = s.iterate(n_iter, reset=1)
        return SolveResult(s.U, s.V, s.sigma, s.R, tr, si, ri, ii)
    finally:
        s.close()
