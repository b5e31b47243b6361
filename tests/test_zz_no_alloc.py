"""The allocation-free Schur entry point (fixed device array for its intermediate field)
against dw_apply(DW_OP_SCHUR), which allocates its intermediate on first use.

Collected last on purpose: it must pass after every other test of the session as well
as alone (it keeps no state besides the per-device address of its array)."""
import pytest
import torch

from paper_0706_2298_gb300 import dwsolve as dw
from paper_0706_2298_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {dw.DW_F64: 1e-15, dw.DW_F32: 1e-6}


def _packed(ctx, prec, L, seed):
    src = synth.gaussian_source(L, seed).to("cuda").contiguous()
    out = ctx.empty_field(prec)
    dw.dw_pack(ctx, prec, 1, src, out)
    return out


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("prec", [dw.DW_F64, dw.DW_F32])
def test_static_schur_matches_dw_apply_twice(prec):
    L = (8, 8, 8, 8)
    U = synth.random_gauge(L, 11)
    ctx = dw.dw_create(L, -0.1, 1.3, U, (4, 4, 4, 4))
    x1, x2 = _packed(ctx, prec, L, 21), _packed(ctx, prec, L, 22)
    ref1, ref2 = ctx.empty_field(prec), ctx.empty_field(prec)
    dw.dw_apply(ctx, prec, dw.DW_OP_SCHUR, 1, x1, ref1)
    dw.dw_apply(ctx, prec, dw.DW_OP_SCHUR, 1, x2, ref2)
    y1, y2 = ctx.empty_field(prec), ctx.empty_field(prec)
    y1.fill_(float("nan"))
    y2.fill_(float("nan"))
    # two calls in a row on different inputs: the second reuses the array the first filled
    dw.dw_apply_schur_static(ctx, prec, x1, y1)
    dw.dw_apply_schur_static(ctx, prec, x2, y2)
    torch.cuda.synchronize()
    assert torch.isfinite(y1).all() and torch.isfinite(y2).all()
    assert _rel(y1, ref1) <= TOL[prec]
    assert _rel(y2, ref2) <= TOL[prec]
    assert _rel(y1, ref2) > 1e-3     # the two results are not the same field


def test_static_schur_volume_limit():
    # 24 x 16^3 = 98304 sites: an FP64 packed field (18.9 MB) exceeds the 16 MiB array,
    # an FP32 one (9.4 MB) fits
    L = (24, 16, 16, 16)
    U = synth.random_gauge(L, 12)
    ctx = dw.dw_create(L, 0.0, 1.0, U, (4, 4, 4, 4))
    x64 = _packed(ctx, dw.DW_F64, L, 23)
    y64 = ctx.empty_field(dw.DW_F64)
    with pytest.raises(dw.DwError, match="fixed"):
        dw.dw_apply_schur_static(ctx, dw.DW_F64, x64, y64)
    x32 = _packed(ctx, dw.DW_F32, L, 23)
    ref, y = ctx.empty_field(dw.DW_F32), ctx.empty_field(dw.DW_F32)
    dw.dw_apply(ctx, dw.DW_F32, dw.DW_OP_SCHUR, 1, x32, ref)
    dw.dw_apply_schur_static(ctx, dw.DW_F32, x32, y)
    torch.cuda.synchronize()
    assert _rel(y, ref) <= TOL[dw.DW_F32]


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second device to make the current device differ")
def test_static_schur_rejects_other_device():
    """A context lives on the device current at dw_create; with another device current the
    entry point refuses instead of launching kernels on one device with memory of the other."""
    L = (8, 8, 8, 8)
    with torch.cuda.device(0):
        ctx = dw.dw_create(L, -0.1, 1.3, synth.random_gauge(L, 11), (4, 4, 4, 4))
        x = _packed(ctx, dw.DW_F32, L, 21)
        y = ctx.empty_field(dw.DW_F32)
    with torch.cuda.device(1):
        with pytest.raises(dw.DwError, match="not the context's device"):
            dw.dw_apply_schur_static(ctx, dw.DW_F32, x, y)
