"""Pins of the oracle's block projection, projectors and little operator.

* Free-field deficit of constant block modes, exact to all orders:
  for blocks b_0 x ... x b_3 and a plane wave u e^{ipx},
      eps_p = 1 - prod_mu sin^2(b_mu p_mu / 2) / (b_mu^2 sin^2(p_mu / 2)),
  whose leading term is (1/12) p^2 (b^2 - 1) for a = 1, eq. (4.4).
* Projector identities (3.5)-(3.8), deflated solution (3.10), Schur
  complement inverse (3.14).
* Little operator support (Fig. 4 / A.1) and, for a complete block basis,
  Phi A Phi^dag = D.
* bfloat16 rounding on hand-checked values.
"""
import json
import os

import numpy as np
import pytest

from paper_0706_2298_gb300 import synth
from oracle.deflation import BlockSubspace, block_gram_schmidt, round_bf16
from oracle.dirac import WilsonClover
from oracle.krylov import gcr
from oracle.lattice import norm
from oracle.sap import Blocking


def _exact_deficit(p, b):
    f = 1.0
    for mu in range(4):
        s = np.sin(p[mu] / 2)
        f *= 1.0 if abs(s) < 1e-15 else np.sin(b[mu] * p[mu] / 2) ** 2 / (b[mu] ** 2 * s ** 2)
    return 1.0 - f


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 1, 0, 2), (2, 3, 1, 0)])
def test_free_field_constant_mode_deficit(n):
    L = (8, 8, 4, 8)
    b = (4, 2, 2, 4)
    D = WilsonClover(L, synth.unit_gauge(L).numpy(), 0.0, 0.0)
    V = D.V
    # 12 global fields spanning the constant spinors, mixed by a random matrix so that
    # the block Gram-Schmidt has real work to do
    rng = np.random.default_rng(3)
    M = rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12))
    fields = np.broadcast_to(M.reshape(12, 1, 4, 3), (12, V, 4, 3)).copy()
    blk = Blocking(L, b)
    sub = BlockSubspace(D, b, block_gram_schmidt(blk, fields))
    p = np.array([(2 * n[0] + 1) * np.pi / L[0]] + [2 * np.pi * n[k] / L[k] for k in (1, 2, 3)])
    x = np.indices(L).reshape(4, -1).T
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi = np.exp(1j * (x @ p))[:, None, None] * u[None]
    assert abs(sub.deficit(psi) - _exact_deficit(p, b)) < 1e-13


def test_deficit_small_momentum_expansion():
    """The exact free-field deficit reproduces (4.4): eps = p^2 (b^2 - 1)/12 + O(p^4 b^4)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "eq_4_4_free_deficit.json")) as f:
        coef = json.load(f)["leading_coefficient"]
    b = (4, 4, 4, 4)
    for t in (1e-2, 3e-3):
        p = t * np.array([1.0, 0.5, -0.7, 0.2])
        lead = coef * np.sum(p ** 2) * (16 - 1)
        assert abs(_exact_deficit(p, b) - lead) < 5 * (t * 4) ** 4


@pytest.fixture(scope="module")
def small():
    L = (4, 4, 4, 4)
    U = synth.random_gauge(L, 21).numpy()
    D = WilsonClover(L, U, -0.1, 1.0)
    bs = (2, 2, 2, 2)
    blk = Blocking(L, bs)
    fields = synth.start_fields(L, 3, 5).numpy()
    sub = BlockSubspace(D, bs, block_gram_schmidt(blk, fields), fields)
    return D, sub


def test_block_gram_schmidt(small):
    D, sub = small
    ph = sub.phi.reshape(sub.Nb, sub.Ns, -1)
    G = np.einsum("bki,bli->bkl", ph.conj(), ph)
    assert np.abs(G - np.eye(sub.Ns)[None]).max() < 1e-13
    for l in range(sub.Ns):                      # span contains the restricted input fields
        f = sub.global_fields[l]
        assert norm(f - sub.project(f)) ** 2 <= 1e-26 * norm(f) ** 2


def test_projector_identities(small):
    D, sub = small
    psi = synth.gaussian_source(D.L, 9).numpy()
    P, PL, PR = sub.project, sub.P_L, sub.P_R
    scale = norm(psi)
    tol = 1e-11 * scale
    assert norm(PL(PL(psi)) - PL(psi)) < tol                    # (3.5)
    assert norm(PR(PR(psi)) - PR(psi)) < tol
    assert norm(PL(D.apply(psi)) - D.apply(PR(psi))) < tol      # (3.6)
    assert norm(P(PL(psi))) < tol                               # (3.7)
    assert norm(PR(P(psi))) < tol
    q = psi - P(psi)
    assert norm(PL(q) - q) < tol                                # (3.8)
    prp = PR(psi)
    assert norm((prp - P(prp)) - q) < tol                       # (1-P) P_R = 1-P


def test_deflated_solution_and_schur(small):
    D, sub = small
    eta = synth.gaussian_source(D.L, 10).numpy()
    # (3.10)/(3.11): chi solves P_L D chi = P_L eta; psi = P_R chi + Phi A^-1 Phi^dag eta solves D psi = eta
    chi, info = gcr(lambda v: sub.P_L(D.apply(v)), sub.P_L(eta), tol=1e-12, nkv=32)
    assert info.converged
    psi = sub.P_R(chi) + sub.prolong(sub.little_solve(sub.restrict(eta)))
    assert norm(D.apply(psi) - eta) < 1e-10 * norm(eta)
    # (3.14): for u in S-perp, P_L D (1-P) D^-1 u = u
    Dm = D.dense()
    v = synth.gaussian_source(D.L, 12).numpy()
    u = v - sub.project(v)
    w = np.linalg.solve(Dm, u.reshape(-1)).reshape(u.shape)
    assert norm(sub.P_L(D.apply(w - sub.project(w))) - u) < 1e-11 * norm(u)


def test_little_operator_support():
    """(A.1)/Fig. 4: B_{LL'} vanishes unless L' = L or a nearest neighbour."""
    L = (8, 4, 4, 4)
    U = synth.random_gauge(L, 22).numpy()
    D = WilsonClover(L, U, 0.0, 1.0)
    bs = (2, 2, 2, 2)
    blk = Blocking(L, bs)
    fields = synth.start_fields(L, 2, 6).numpy()
    sub = BlockSubspace(D, bs, block_gram_schmidt(blk, fields), fields)
    bc = blk.block_coords.T
    for La in range(blk.Nb):
        for Lb in range(blk.Nb):
            d = [(bc[Lb][m] - bc[La][m]) % blk.nb[m] for m in range(4)]
            d = [min(v, blk.nb[m] - v) for m, v in enumerate(d)]
            nb = sum(d) <= 1
            mag = np.abs(sub.block_matrix(La, Lb)).max()
            assert (mag > 1e-3) if nb else (mag == 0.0)


@pytest.mark.slow
def test_complete_block_basis_reproduces_D():
    """With Ns = 12|L| the block basis is a unitary change of basis: Phi A Phi^dag = D."""
    L = (4, 4, 4, 4)
    U = synth.random_gauge(L, 23).numpy()
    D = WilsonClover(L, U, -0.1, 1.0)
    bs = (2, 2, 2, 2)
    blk = Blocking(L, bs)
    Ns = 12 * blk.vol
    fields = synth.start_fields(L, Ns, 7).numpy()
    sub = BlockSubspace(D, bs, block_gram_schmidt(blk, fields), fields)
    eta = synth.gaussian_source(L, 13).numpy()
    lhs = sub.prolong((sub.A @ sub.restrict(eta).reshape(-1)).reshape(sub.Nb, Ns))
    assert norm(lhs - D.apply(eta)) < 1e-12 * norm(eta)


def test_round_bf16_hand_values():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1.0 / 3.0, -2.5, 0.0])
    expect = np.array([1.0, 1.0, 1 + 2 ** -6, 171.0 / 512.0, -2.5, 0.0])
    assert np.array_equal(round_bf16(x), expect)
