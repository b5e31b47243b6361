"""Pins of the oracle's Schwarz procedure, little solver and outer solvers.

* One SAP cycle with exact block solves is block Gauss-Seidel on the
  black/white partition of the dense matrix D (black first).
* nmr MR steps: residual never increases; many steps reach the exact
  block solve.
* The even-odd little solve (A.2)-(A.4) equals the dense solve A^{-1} w;
  global-mode deflation (A.3) lowers the little GCR iteration count.
* DFL+SAP+GCR and SAP+GCR reach ||eta - D psi|| <= 1e-10 ||eta|| and agree
  with the dense solution.
"""
import numpy as np
import pytest

from paper_0706_2298_gb300 import synth
from oracle.deflation import BlockSubspace, block_gram_schmidt, build_subspace
from oracle.dirac import WilsonClover
from oracle.krylov import mr
from oracle.lattice import norm
from oracle.little import EOLittle, IllConditioned
from oracle.sap import Blocking, SchwarzOracle
from oracle.solver import solve_dfl_sap, solve_plain, solve_sap

L4 = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def setup4():
    U = synth.random_gauge(L4, 31).numpy()
    D = WilsonClover(L4, U, -0.1, 1.0)
    return D, D.dense()


def test_sap_exact_is_block_gauss_seidel(setup4):
    D, M = setup4
    sap = SchwarzOracle(D, (2, 2, 2, 2))
    rho = synth.gaussian_source(L4, 3).numpy()
    xi = sap.apply(rho, ncy=1, nmr=0, exact=True)
    # block Gauss-Seidel from the dense matrix: black rows first, then white
    colour = np.repeat(sap.blk.colour_of_site.ravel(), 12)
    B, W = colour == 0, colour == 1
    r = rho.reshape(-1)
    x = np.zeros_like(r)
    x[B] = np.linalg.solve(M[np.ix_(B, B)], r[B])
    res = r - M @ x
    x[W] += np.linalg.solve(M[np.ix_(W, W)], res[W])
    assert np.linalg.norm(xi.reshape(-1) - x) <= 1e-12 * np.linalg.norm(x)


def test_block_mr_converges_to_exact(setup4):
    D, _ = setup4
    sap = SchwarzOracle(D, (2, 2, 2, 2))
    r = synth.gaussian_source(L4, 4).numpy()
    exact = sap.block_mr(r, 0, 0, exact=True)
    approx = sap.block_mr(r, 0, 150)
    assert norm(approx - exact) <= 1e-10 * norm(exact)


def test_mr_residual_monotone(setup4):
    D, _ = setup4
    b = synth.gaussian_source(L4, 5).numpy()
    prev = norm(b)
    for n in range(1, 8):
        _, r = mr(D.apply, b, n)
        assert norm(r) <= prev * (1 + 1e-14)
        prev = norm(r)


def test_sap_reduces_residual(setup4):
    D, _ = setup4
    sap = SchwarzOracle(D, (2, 2, 2, 2))
    rho = synth.gaussian_source(L4, 6).numpy()
    r_prev = norm(rho)
    for ncy in (1, 2, 4):
        r = norm(rho - D.apply(sap.apply(rho, ncy, 4)))
        assert r < r_prev
        r_prev = r


@pytest.fixture(scope="module")
def setup8():
    L = (8, 8, 8, 8)
    U = synth.random_gauge(L, 1).numpy()
    D = WilsonClover(L, U, -0.2, 1.0)
    sap = SchwarzOracle(D, (4, 4, 4, 4))
    start = synth.start_fields(L, 6, 3).numpy()
    sub = build_subspace(D, (4, 4, 4, 4), (4, 4, 4, 4), start, 3, 4, 4)
    return D, sap, sub


def test_little_eo_solve_equals_dense(setup8):
    D, sap, sub = setup8
    lit = EOLittle(sub)
    w = sub.restrict(synth.gaussian_source(D.L, 7).numpy())
    v, info = lit.solve(w, tol=1e-12)
    vd = sub.little_solve(w)
    assert info.converged
    assert np.linalg.norm(v - vd) <= 1e-9 * np.linalg.norm(vd)


def test_global_mode_deflation_lowers_iterations(setup8):
    D, sap, sub = setup8
    w = sub.restrict(synth.gaussian_source(D.L, 8).numpy())
    _, i_defl = EOLittle(sub).solve(w, tol=1e-12)
    _, i_plain = EOLittle(sub, deflate=False).solve(w, tol=1e-12)
    assert i_defl.iterations < i_plain.iterations


def test_ill_conditioned_diagonal_block_detected(setup8):
    D, sap, sub = setup8
    with pytest.raises(IllConditioned):
        EOLittle(sub, cond_max=1.0)


def test_outer_solvers_reach_tolerance(setup4):
    D, M = setup4
    sap = SchwarzOracle(D, (2, 2, 2, 2))
    start = synth.start_fields(L4, 4, 3).numpy()
    sub = build_subspace(D, (2, 2, 2, 2), (2, 2, 2, 2), start, 3, 4, 4)
    eta = synth.gaussian_source(L4, 2).numpy()
    x = np.linalg.solve(M, eta.reshape(-1)).reshape(eta.shape)
    psi, info = solve_dfl_sap(D, sap, sub, EOLittle(sub), eta, tol=1e-10)
    assert info.converged
    assert norm(eta - D.apply(psi)) <= 1e-10 * norm(eta)
    assert norm(psi - x) <= 1e-8 * norm(x)
    psi2, info2 = solve_sap(D, sap, eta, tol=1e-10)
    assert info2.converged
    assert norm(psi2 - x) <= 1e-8 * norm(x)


def test_plain_gcr_matches_dense(setup4):
    D, M = setup4
    eta = synth.gaussian_source(L4, 9).numpy()
    psi, info = solve_plain(D, eta, tol=1e-11)
    x = np.linalg.solve(M, eta.reshape(-1))
    assert info.converged
    assert np.linalg.norm(psi.reshape(-1) - x) <= 1e-8 * np.linalg.norm(x)
