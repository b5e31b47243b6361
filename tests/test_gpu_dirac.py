"""GPU parity of the packed layout, the Wilson-clover operator, its even-odd
Schur complement and the Schwarz preconditioner against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_0706_2298_gb300 import dwsolve as dw
from paper_0706_2298_gb300 import synth
from oracle.dirac import WilsonClover
from oracle.sap import SchwarzOracle

from .gpu_util import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

# (lattice, Schwarz block, m0, c_sw, antiperiodic): cubic and non-cubic lattices,
# several block shapes (including 2-site extents), both boundary conditions
CASES = [
    ((8, 8, 8, 8), (4, 4, 4, 4), -0.2, 1.0, True),
    ((8, 4, 4, 8), (4, 2, 2, 4), 0.1, 1.9, True),
    ((4, 4, 8, 4), (2, 2, 4, 2), -0.1, 1.3, False),
    ((12, 8, 8, 4), (2, 4, 4, 2), 0.0, 1.0, True),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "".join(map(str, c[1])))
def case(request):
    L, sb, m0, csw, ap = request.param
    U = synth.random_gauge(L, 3)
    ctx = dw.dw_create(L, m0, csw, U, sb, ap)
    D = WilsonClover(L, U.numpy(), m0, csw, ap)
    return L, sb, ctx, D


def test_pack_roundtrip(case):
    L, sb, ctx, D = case
    psi = synth.gaussian_source(L, 5, nrhs=2).numpy()
    p64 = to_packed(ctx, dw.DW_F64, psi)
    assert np.array_equal(from_packed(ctx, dw.DW_F64, p64, 2), psi)
    p32 = to_packed(ctx, dw.DW_F32, psi)
    back = from_packed(ctx, dw.DW_F32, p32, 2)
    assert np.array_equal(back, psi.astype(np.complex64).astype(np.complex128))


@pytest.mark.parametrize("prec,tol", [(dw.DW_F64, 1e-14), (dw.DW_F32, 2e-6)])
def test_dirac_full(case, prec, tol):
    L, sb, ctx, D = case
    psi = synth.gaussian_source(L, 6).numpy()
    x = to_packed(ctx, prec, psi)
    y = ctx.empty_field(prec)
    dw.dw_apply(ctx, prec, dw.DW_OP_FULL, 1, x, y)
    assert rel(from_packed(ctx, prec, y), D.apply(psi)) <= tol


def test_dirac_full_double_float(case):
    """DW_F64X: FP64 fields, D computed in double-float arithmetic on the FP32 pipes."""
    L, sb, ctx, D = case
    psi = synth.gaussian_source(L, 6).numpy()
    x = to_packed(ctx, dw.DW_F64, psi)
    y = ctx.empty_field(dw.DW_F64)
    dw.dw_apply(ctx, dw.DW_F64X, dw.DW_OP_FULL, 1, x, y)
    assert rel(from_packed(ctx, dw.DW_F64, y), D.apply(psi)) <= 5e-14


@pytest.mark.parametrize("prec,tol", [(dw.DW_F64, 1e-14), (dw.DW_F32, 5e-6)])
def test_dirac_schur(case, prec, tol):
    L, sb, ctx, D = case
    psi = synth.gaussian_source(L, 7).numpy()
    x = to_packed(ctx, prec, psi)
    y = ctx.empty_field(prec)
    dw.dw_apply(ctx, prec, dw.DW_OP_SCHUR, 1, x, y)
    assert rel(from_packed(ctx, prec, y), D.schur(psi)) <= tol


def test_dirac_multi_rhs(case):
    L, sb, ctx, D = case
    psi = synth.gaussian_source(L, 8, nrhs=3).numpy()
    x = to_packed(ctx, dw.DW_F64, psi)
    y = ctx.empty_field(dw.DW_F64, 3)
    dw.dw_apply(ctx, dw.DW_F64, dw.DW_OP_FULL, 3, x, y)
    assert rel(from_packed(ctx, dw.DW_F64, y, 3), D.apply(psi)) <= 1e-14


@pytest.mark.parametrize("prec,tol", [(dw.DW_F64, 1e-12), (dw.DW_F32, 1e-4)])
@pytest.mark.parametrize("ncy,nmr", [(1, 1), (4, 4), (2, 7)])
def test_sap(case, prec, tol, ncy, nmr):
    L, sb, ctx, D = case
    sap = SchwarzOracle(D, sb)
    rho = synth.gaussian_source(L, 9).numpy()
    x = to_packed(ctx, prec, rho)
    y = ctx.empty_field(prec)
    dw.sap_precondition(ctx, prec, ncy, nmr, 1, x, y)
    assert rel(from_packed(ctx, prec, y), sap.apply(rho, ncy, nmr)) <= tol


def test_sap_zero_cycles(case):
    L, sb, ctx, D = case
    rho = synth.gaussian_source(L, 10).numpy()
    x = to_packed(ctx, dw.DW_F32, rho)
    y = ctx.empty_field(dw.DW_F32)
    y.fill_(1.0)
    dw.sap_precondition(ctx, dw.DW_F32, 0, 4, 1, x, y)
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0


def test_sap_staged_matches_generic(case):
    """The staged FP32 Schwarz kernel and the generic kernel compute the same M_sap."""
    import os
    L, sb, ctx, D = case
    rho = synth.gaussian_source(L, 12).numpy()
    x = to_packed(ctx, dw.DW_F32, rho)
    out = {}
    for flag in ("0", "1"):
        os.environ["DW_SAP_STAGED"] = flag
        y = ctx.empty_field(dw.DW_F32)
        dw.sap_precondition(ctx, dw.DW_F32, 4, 4, 1, x, y)
        out[flag] = from_packed(ctx, dw.DW_F32, y)
    os.environ.pop("DW_SAP_STAGED")
    assert rel(out["1"], out["0"]) <= 2e-5
