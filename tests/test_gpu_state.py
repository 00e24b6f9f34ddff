"""Checkpoint of Algorithm 3's loop state (enmf_state_export / _import) on the GPU.

A context that imports another context's exported state, given copies of that
context's U and V, must continue the iteration exactly as the exporting
context would have: the same trace and the same factors, bit for bit, as one
uninterrupted call.  Checked for the plain FP64 form and for the BF16
tensor-core form (whose call prologue rebuilds the Gram of V and V's 16-bit
pair from the imported factor).  A corrupt state buffer is refused.
"""
import struct

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


def _np(t):
    return t.detach().cpu().numpy()


def _make(X, r, form):
    from paper_2605_19325_gb300.solver import Solver
    if form == "f64":
        return Solver(torch.as_tensor(X, dtype=torch.float64, device="cuda"), r)
    Xd = torch.as_tensor(X.astype(np.float32), device="cuda")
    return Solver(Xd, r, x_stream=torch.bfloat16)


# (form, alternations before the checkpoint, after it): the BF16 split is a
# multiple of the X_lo correction period (10), so both runs refresh the
# correction term at the same alternations.
@pytest.mark.gpu
@pytest.mark.parametrize("form,n1,n2", [("f64", 7, 45), ("f64", 0, 30), ("bf16", 20, 40)])
def test_state_export_import_resumes_bit_for_bit(form, n1, n2):
    X, r = synth.config_small(1)
    ref = _make(X, r, form)
    ref.svd_init()
    ref.rotate()
    U0, V0 = ref.U.clone(), ref.V.clone()
    t_ref, i_ref = ref.iterate(n1 + n2, reset=1)
    # the same start, interrupted after n1 alternations
    a = _make(X, r, form)
    a.U.copy_(U0)
    a.V.copy_(V0)
    if n1 > 0:
        t1, _ = a.iterate(n1, reset=1)
    else:
        # nothing iterated yet: a state to export needs one call (0 alternations)
        t1, _ = a.iterate(0, reset=1)
        t1 = t1[:0]
    blob = a.export_state()
    Uc, Vc = a.U.clone(), a.V.clone()
    a.close()
    b = _make(X, r, form)
    b.U.copy_(Uc)
    b.V.copy_(Vc)
    b.import_state(blob)
    t2, i2 = b.iterate(n2, reset=0)
    np.testing.assert_array_equal(np.concatenate([_np(t1), _np(t2)]), _np(t_ref))
    np.testing.assert_array_equal(_np(b.U), _np(ref.U))
    np.testing.assert_array_equal(_np(b.V), _np(ref.V))
    assert (i2.iters, i2.asc_iters, i2.hals_iters, i2.stage) == \
        (i_ref.iters, i_ref.asc_iters, i_ref.hals_iters, i_ref.stage)
    assert (i2.s_u, i2.s_v) == (i_ref.s_u, i_ref.s_v)
    b.close()
    ref.close()


# StateBlob layout: magic, version (u32); m, n (i64); r, x_dtype, f_dtype,
# stream_dtype, stage, k, asc_iters, hals_iters, negU, negV (i32); s_u, s_v,
# maxneg_u, maxneg_v, f_last (f64); padding to 128 bytes.
_FMT = "<IIqq10i5d"
_FIELDS = ["magic", "version", "m", "n", "r", "x_dtype", "f_dtype", "stream_dtype", "stage",
           "k", "asc_iters", "hals_iters", "negU", "negV", "s_u", "s_v", "maxneg_u",
           "maxneg_v", "f_last"]


def _edit(blob, **kw):
    vals = dict(zip(_FIELDS, struct.unpack_from(_FMT, blob)))
    vals.update(kw)
    out = bytearray(blob)
    struct.pack_into(_FMT, out, 0, *[vals[f] for f in _FIELDS])
    return bytes(out)


@pytest.mark.gpu
def test_state_import_rejects_corrupt_buffers():
    from paper_2605_19325_gb300 import binding as B
    X, r = synth.config_small(0)
    a = _make(X, r, "f64")
    a.svd_init()
    a.rotate()
    a.iterate(5, reset=1)
    blob = a.export_state()
    assert len(blob) == B.ENMF_STATE_BYTES
    vals = dict(zip(_FIELDS, struct.unpack_from(_FMT, blob)))
    assert (vals["m"], vals["n"], vals["r"], vals["k"]) == (200, 150, 5, 5)
    a.import_state(blob)          # its own state is accepted
    bad = [dict(magic=0), dict(version=99), dict(m=201), dict(r=4), dict(stage=2),
           dict(k=-1), dict(asc_iters=-1), dict(hals_iters=-3), dict(asc_iters=9),
           dict(negU=2), dict(negV=-1), dict(s_u=float("nan")), dict(s_v=-1.0),
           dict(maxneg_u=float("inf")), dict(maxneg_v=float("nan")),
           dict(f_last=float("nan"))]
    for kw in bad:
        with pytest.raises(B.EnmfError) as ei:
            a.import_state(_edit(blob, **kw))
        assert ei.value.code == 1, kw
    with pytest.raises(B.EnmfError):
        a.import_state(blob[:64])
    # the context is still usable after the refusals
    a.import_state(blob)
    tr, info = a.iterate(3)
    assert info.iters == 8 and np.all(np.isfinite(_np(tr)))
    a.close()
