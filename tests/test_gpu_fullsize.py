"""Parity at the benchmark's full size (48 x 24^3, m0 = 0, c_sw = 1) in the benchmark's launch
configuration: the FP32 and double-float Wilson-clover operators against the FP64 oracle, and
the mixed-precision DFL+SAP+GCR solve (Ns = 20 BF16 basis on 4^4 blocks, 11 inverse-iteration
steps, N_kv = 16, ncy = nmr = 4) reaching a true relative residual of 1e-10 measured with the
oracle's D."""
import numpy as np
import pytest
import torch

from oracle.dirac import WilsonClover
from paper_0706_2298_gb300 import dwsolve as dw
from paper_0706_2298_gb300 import synth

from .gpu_util import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

L = (48, 24, 24, 24)


@pytest.fixture(scope="module")
def full():
    U = synth.random_gauge(L, 1, device="cuda").cpu()
    ctx = dw.dw_create(L, 0.0, 1.0, U, (4, 4, 4, 4))
    D = WilsonClover(L, U.numpy(), 0.0, 1.0)
    return ctx, D


def test_operator_full_size(full):
    ctx, D = full
    psi = synth.gaussian_source(L, 99).numpy()
    want = D.apply(psi)
    x32 = to_packed(ctx, dw.DW_F32, psi)
    y32 = ctx.empty_field(dw.DW_F32)
    dw.dw_apply(ctx, dw.DW_F32, dw.DW_OP_FULL, 1, x32, y32)
    assert rel(from_packed(ctx, dw.DW_F32, y32), want) <= 2e-6
    x64 = to_packed(ctx, dw.DW_F64, psi)
    y64 = ctx.empty_field(dw.DW_F64)
    dw.dw_apply(ctx, dw.DW_F64X, dw.DW_OP_FULL, 1, x64, y64)
    assert rel(from_packed(ctx, dw.DW_F64, y64), want) <= 5e-14


def test_solve_full_size(full):
    ctx, D = full
    dfl = dw.deflation_build(ctx, (4, 4, 4, 4), 20, 11, 4, 4, synth.start_fields(L, 20, 3).cuda(),
                             basis_prec=dw.DW_BF16, iter_prec=dw.DW_F32)
    eta = synth.gaussian_source(L, 2)
    psi = torch.empty_like(eta, device="cuda")
    p = dw.sol_params(tol=1e-10, nkv=16, ncy=4, nmr=4, mixed=1)
    rc, infos = dw.gcr_solve(ctx, dfl, p, 1, eta.cuda(), psi)
    assert rc == dw.DW_OK and infos[0].relres <= 1e-10
    e = eta.numpy()
    res = np.linalg.norm(e - D.apply(psi.cpu().numpy())) / np.linalg.norm(e)
    assert res <= 1.05e-10, res
