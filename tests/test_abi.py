"""The C ABI library builds, loads and exports every entry point of include/*.h.

CPU only: nvcc cross-compiles for sm_103a without a GPU and the library loads
without touching a device.  No compute call is made here.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_19325_gb300 import build
    return build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(enmf_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_five_calls():
    names = declared_functions()
    for f in ("enmf_svd_init", "enmf_rotate", "enmf_iterate", "enmf_residual", "enmf_kkt"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2605_19325_gb300 import binding
    assert set(declared_functions()) <= set(binding.EXPORTED)
    lib = binding.load(libpath)
    assert lib.enmf_version().decode().startswith("enmf")


def test_status_strings_and_invalid_arguments(libpath):
    """Argument checks run before any device work, so they work without a GPU."""
    from paper_2605_19325_gb300 import binding as B
    lib = B.load(libpath)
    assert lib.enmf_status_string(0) == b"ok"
    assert b"invalid" in lib.enmf_status_string(1)
    bad = [B.enmf_problem(0, 5, 5, 1, B.ENMF_F64, B.ENMF_F64),      # m = 0
           B.enmf_problem(5, 5, 4, 1, B.ENMF_F64, B.ENMF_F64),      # ldx < n
           B.enmf_problem(5, 5, 5, 6, B.ENMF_F64, B.ENMF_F64),      # r > min(m, n)
           B.enmf_problem(500, 500, 500, 65, B.ENMF_F64, B.ENMF_F64),  # r > max rank
           B.enmf_problem(5, 5, 5, 2, B.ENMF_F32, B.ENMF_F64)]      # FP64 factors need FP64 X
    for p in bad:
        size = ctypes.c_size_t(0)
        assert lib.enmf_workspace_size(ctypes.byref(p), ctypes.byref(size)) == 1
        h = ctypes.c_void_p()
        assert lib.enmf_create(ctypes.byref(p), None, ctypes.byref(h)) == 1
    # null context
    assert lib.enmf_iterate(None, None, None, None, None, None) == 1
    assert lib.enmf_stage_copy(None, None, None, None) == 1
    size = ctypes.c_size_t(B.ENMF_STATE_BYTES)
    buf = ctypes.create_string_buffer(B.ENMF_STATE_BYTES)
    assert lib.enmf_state_export(None, buf, ctypes.byref(size)) == 1
    assert lib.enmf_state_import(None, buf, B.ENMF_STATE_BYTES) == 1


def test_fp8_form_problem_rules_and_footprint(libpath):
    """The FP8 form takes F32 X and F32 factors only; its staged X (one-byte
    codes, a BF16 X_lo and one exponent per 128 x 128 tile) is smaller than
    the BF16 form's BF16 pair by about m n bytes."""
    from paper_2605_19325_gb300 import binding as B
    lib = B.load(libpath)

    def ws(p):
        size = ctypes.c_size_t(0)
        code = lib.enmf_workspace_size(ctypes.byref(p), ctypes.byref(size))
        return code, size.value

    m, n = 1025, 4096
    for bad in (B.enmf_problem(m, n, n, 64, B.ENMF_BF16, B.ENMF_F32, B.ENMF_E4M3),
                B.enmf_problem(m, n, n, 64, B.ENMF_F64, B.ENMF_F64, B.ENMF_E4M3),
                B.enmf_problem(m, n, n, 64, B.ENMF_F32, B.ENMF_F64, B.ENMF_E4M3),
                B.enmf_problem(m, n, n, 64, B.ENMF_E4M3, B.ENMF_F32, B.ENMF_E4M3),
                B.enmf_problem(65535 * 128 + 1, 64, 64, 4, B.ENMF_F32, B.ENMF_F32, B.ENMF_E4M3)):
        assert ws(bad)[0] == 1
    c8, s8 = ws(B.enmf_problem(m, n, n, 64, B.ENMF_F32, B.ENMF_F32, B.ENMF_E4M3))
    c16, s16 = ws(B.enmf_problem(m, n, n, 64, B.ENMF_F32, B.ENMF_F32, B.ENMF_BF16))
    assert c8 == 0 and c16 == 0
    assert s16 - s8 >= m * n - 2 ** 20
    assert s8 >= m * n + 2 * m * n + ((m + 127) // 128) * ((n + 127) // 128) * 4


def test_state_blob_size_matches_header(libpath):
    from paper_2605_19325_gb300 import binding as B
    text = open(os.path.join(ROOT, "include", "enmf.h")).read()
    m = re.search(r"#define ENMF_STATE_BYTES (\d+)", text)
    assert m and int(m.group(1)) == B.ENMF_STATE_BYTES


def test_sparse_form_problem_rules_and_footprint(libpath):
    """The sparse form (ENMF_CSR): FP32 or FP64 factors, no tensor-core
    stream, 0 <= nnz <= m n, indices below 2^31; ldx is ignored.  Its
    workspace adds the transpose (n + 1 column pointers, nnz row indices and
    nnz values)."""
    from paper_2605_19325_gb300 import binding as B
    lib = B.load(libpath)

    def ws(p):
        size = ctypes.c_size_t(0)
        code = lib.enmf_workspace_size(ctypes.byref(p), ctypes.byref(size))
        return code, size.value

    m, n, r, nnz = 5000, 3000, 16, 200000
    code64, w64 = ws(B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_F64, 0, nnz))
    code32, w32 = ws(B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_F32, 0, nnz))
    assert code64 == 0 and code32 == 0
    code0, w0 = ws(B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_F32, 0, 0))
    assert code0 == 0
    assert w32 - w0 >= nnz * 8          # row indices and FP32 values
    for p in (B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_F32, 0, -1),
              B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_F32, 0, m * n + 1),
              B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_F32, B.ENMF_BF16, nnz),
              B.enmf_problem(m, n, 0, r, B.ENMF_CSR, B.ENMF_BF16, 0, nnz),
              B.enmf_problem(1 << 31, n, 0, r, B.ENMF_CSR, B.ENMF_F32, 0, nnz)):
        assert ws(p)[0] == 1   # ENMF_EINVAL
