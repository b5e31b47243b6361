"""GPU parity of the batched (multi right-hand side) path: multi-RHS D and
M_sap, the lockstep DFL+SAP+GCR solve of the 12 spin-colour point sources,
its CUDA-graph replay, and the autotuner."""
import numpy as np
import pytest
import torch

from oracle.dirac import WilsonClover
from oracle.sap import SchwarzOracle
from paper_0706_2298_gb300 import dwsolve as dw
from paper_0706_2298_gb300 import synth

from .gpu_util import from_packed, rel, to_packed

pytestmark = pytest.mark.gpu

L = (8, 8, 8, 8)


@pytest.fixture(scope="module")
def setup():
    U = synth.random_gauge(L, 5)
    ctx = dw.dw_create(L, -0.2, 1.0, U, (4, 4, 4, 4))
    D = WilsonClover(L, U.numpy(), -0.2, 1.0)
    return ctx, D


@pytest.mark.parametrize("prec,tol", [(dw.DW_F32, 2e-6), (dw.DW_F64, 1e-14)])
@pytest.mark.parametrize("nrhs", [2, 5, 12])
def test_dirac_multi_rhs(setup, prec, tol, nrhs):
    ctx, D = setup
    psi = synth.gaussian_source(L, 20, nrhs=nrhs).numpy()
    x = to_packed(ctx, prec, psi)
    y = ctx.empty_field(prec, nrhs)
    dw.dw_apply(ctx, prec, dw.DW_OP_FULL, nrhs, x, y)
    out = from_packed(ctx, prec, y, nrhs)
    for r in range(nrhs):
        assert rel(out[r], D.apply(psi[r])) <= tol


def test_sap_multi_rhs(setup):
    ctx, D = setup
    nrhs = 4
    sap = SchwarzOracle(D, (4, 4, 4, 4))
    rho = synth.gaussian_source(L, 21, nrhs=nrhs).numpy()
    x = to_packed(ctx, dw.DW_F32, rho)
    y = ctx.empty_field(dw.DW_F32, nrhs)
    dw.sap_precondition(ctx, dw.DW_F32, 4, 4, nrhs, x, y)
    out = from_packed(ctx, dw.DW_F32, y, nrhs)
    for r in range(nrhs):
        single = ctx.empty_field(dw.DW_F32)
        dw.sap_precondition(ctx, dw.DW_F32, 4, 4, 1, x[r * ctx.V * 24:(r + 1) * ctx.V * 24], single)
        assert rel(out[r], from_packed(ctx, dw.DW_F32, single)) <= 1e-6
        assert rel(out[r], sap.apply(rho[r], 4, 4)) <= 1e-4


@pytest.fixture(scope="module")
def dfl(setup):
    ctx, D = setup
    return dw.deflation_build(ctx, (4, 4, 4, 4), 8, 4, 4, 4, synth.start_fields(L, 8, 3).cuda(),
                              basis_prec=dw.DW_BF16, iter_prec=dw.DW_F32)


def test_batched_point_source_solve(setup, dfl):
    """All 12 spin-colour point sources solved in one lockstep batch (twice: the second
    solve replays the captured M_sap graphs) to ||eta - D psi|| <= 1e-10 ||eta||."""
    ctx, D = setup
    eta = synth.point_sources(L)
    p = dw.sol_params(tol=1e-10, nkv=16, mixed=1)
    for _ in range(2):
        psi = torch.empty_like(eta, device="cuda")
        rc, infos = dw.gcr_solve(ctx, dfl, p, 12, eta.cuda(), psi)
        assert rc == dw.DW_OK
        psi = psi.cpu().numpy()
        for r in range(12):
            res = np.linalg.norm(eta[r].numpy() - D.apply(psi[r])) / np.linalg.norm(eta[r].numpy())
            assert res <= 1.05e-10, (r, res)
            assert infos[r].status == dw.DW_OK and infos[r].iterations > 0


def test_batched_equals_sequential(setup, dfl):
    import os
    ctx, D = setup
    eta = synth.gaussian_source(L, 22, nrhs=3)
    p = dw.sol_params(tol=1e-10, nkv=16, mixed=1)
    psi_b = torch.empty_like(eta, device="cuda")
    rc, _ = dw.gcr_solve(ctx, dfl, p, 3, eta.cuda(), psi_b)
    assert rc == dw.DW_OK
    os.environ["DW_BATCH"] = "0"
    psi_s = torch.empty_like(eta, device="cuda")
    rc2, _ = dw.gcr_solve(ctx, dfl, p, 3, eta.cuda(), psi_s)
    os.environ.pop("DW_BATCH")
    assert rc2 == dw.DW_OK
    # both are solutions to 1e-10; they agree to the conditioning of D times the tolerance
    assert rel(psi_b.cpu().numpy(), psi_s.cpu().numpy()) <= 1e-8


def test_multi_rhs_little_solver_matches_per_rhs(setup, dfl):
    """14 right-hand sides batched: the little solves of each step run in two multi-RHS
    cooperative launches (12 + 2); the result equals the batch with one little solve per
    right-hand side, and every solution meets the tolerance with the oracle D."""
    import os
    ctx, D = setup
    eta = synth.gaussian_source(L, 23, nrhs=14)
    p = dw.sol_params(tol=1e-10, nkv=16, mixed=1)
    psi_m = torch.empty_like(eta, device="cuda")
    rc, infos = dw.gcr_solve(ctx, dfl, p, 14, eta.cuda(), psi_m)
    assert rc == dw.DW_OK and all(i.status == dw.DW_OK for i in infos)
    os.environ["DW_LITTLE_MRHS"] = "0"
    psi_s = torch.empty_like(eta, device="cuda")
    rc2, _ = dw.gcr_solve(ctx, dfl, p, 14, eta.cuda(), psi_s)
    os.environ.pop("DW_LITTLE_MRHS")
    assert rc2 == dw.DW_OK
    pm = psi_m.cpu().numpy()
    assert rel(pm, psi_s.cpu().numpy()) <= 1e-8
    for r in (0, 11, 12, 13):
        res = np.linalg.norm(eta[r].numpy() - D.apply(pm[r])) / np.linalg.norm(eta[r].numpy())
        assert res <= 1.05e-10, (r, res)


def test_autotune(setup):
    ctx, D = setup
    rep = dw.dw_autotune(ctx, 4)
    assert rep["rgroup"] in (0, 1, 2, 3) and rep["sap_staged"] in (0, 1)
    assert all(v > 0 for v in rep["dirac_mrhs_ms"].values())


def test_little_solver_autotune(setup, dfl):
    """The shape sweep of the cooperative little solver keeps a configuration it timed, and the
    solver still reaches the tolerance with it."""
    ctx, D = setup
    rep = dw.dfl_autotune(dfl)
    assert rep["tuned"] and rep["grid"] > 0 and rep["ring"] in (0, 1)
    assert all(v > 0 for v in rep["us_per_iteration"].values())
    eta = synth.gaussian_source(L, 25)
    psi = torch.empty_like(eta, device="cuda")
    rc, _ = dw.gcr_solve(ctx, dfl, dw.sol_params(tol=1e-10, mixed=1), 1, eta.cuda(), psi)
    assert rc == dw.DW_OK
    r = np.linalg.norm(eta.numpy() - D.apply(psi.cpu().numpy())) / np.linalg.norm(eta.numpy())
    assert r <= 1.05e-10
