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


# ----------------------------------------------------------------------------- inverse iteration (5.1)
class _LinearPreconditioner:
    """Stand-in for M_sap with a known linear action (a dense matrix), so that the steps of
    the inverse iteration can be checked against matrix powers."""

    def __init__(self, A):
        self.A = A
        self.calls = 0

    def apply(self, fields, ncy, nmr):
        self.calls += 1
        f = np.asarray(fields)
        return (f.reshape(f.shape[0], -1) @ self.A.T).reshape(f.shape)


def _plane_wave_span(L, p0):
    """Orthonormal basis of {u exp(i p.x)}: momenta (+-p0, 0, 0, 0), u any spin-colour vector."""
    x0 = np.indices(L)[0].reshape(-1)
    cols = []
    for s in (1, -1):
        ph = np.exp(1j * s * p0 * x0) / np.sqrt(x0.size)
        for k in range(12):
            v = np.zeros((x0.size, 12), dtype=np.complex128)
            v[:, k] = ph
            cols.append(v.reshape(-1))
    return np.array(cols).T


def test_inverse_iteration_is_normalised_power():
    """(5.1) with a linear stand-in M = D^{-1}: n steps give D^{-n} psi_l / ||D^{-n} psi_l||
    for every field separately (each step normalises each field, not the set)."""
    from oracle.deflation import inverse_iteration
    L = (4, 4, 2, 2)
    D = WilsonClover(L, synth.random_gauge(L, 31).numpy(), 0.3, 1.0)
    Dm = D.dense()
    M = _LinearPreconditioner(np.linalg.inv(Dm))
    start = synth.start_fields(L, 3, 5).numpy()
    start[1] *= 7.0                       # unequal norms: a joint normalisation would show
    from scipy.linalg import lu_factor, lu_solve
    lu = lu_factor(Dm)
    for n in (0, 1, 3):
        M.calls = 0
        got = inverse_iteration(M, start, n, 4, 4)
        assert M.calls == n
        for l in range(3):
            w = start[l].reshape(-1)
            for _ in range(n):
                w = lu_solve(lu, w)
            if n:
                w = w / np.linalg.norm(w)
            assert np.linalg.norm(got[l].reshape(-1) - w) <= 1e-11 * np.linalg.norm(w)
            if n:
                assert abs(np.linalg.norm(got[l]) - 1.0) <= 1e-13


def test_inverse_iteration_free_field_reaches_lowest_modes():
    """Free field on 4^4 (antiperiodic time): the smallest |lambda| of D is taken on the plane
    waves with p = (+-pi/4, 0, 0, 0), |lambda| = |m0 + 1 - cos(pi/4) + i sin(pi/4)|, and the next
    |lambda| is 1.6415 (p0 = pi/4 with one spatial pi/2).  With M = D^{-1} the fields converge to
    that 24-dimensional span at the rate (0.7132/1.6415)^n; with the Schwarz procedure itself
    (4 cycles, 4 MR steps) they become dominated by it (deficit far below the start's 0.99) and
    ||D psi|| approaches the lower end of the spectrum."""
    from oracle.deflation import inverse_iteration
    from oracle.sap import SchwarzOracle
    L = (4, 4, 4, 4)
    m0 = -0.2
    D = WilsonClover(L, synth.unit_gauge(L).numpy(), m0, 1.0)
    lam_min = abs(m0 + 1 - np.cos(np.pi / 4) + 1j * np.sin(np.pi / 4))
    Q = _plane_wave_span(L, np.pi / 4)
    # the span is an invariant subspace of D on which |lambda| = lam_min
    DQ = D.apply(Q.T.reshape(24, D.V, 4, 3)).reshape(24, -1).T
    assert np.linalg.norm(DQ - Q @ (Q.conj().T @ DQ)) <= 1e-12 * np.linalg.norm(DQ)
    assert np.allclose(np.abs(np.linalg.eigvals(Q.conj().T @ DQ)), lam_min, atol=1e-12)

    def deficit(f):
        f = f.reshape(-1)
        return np.linalg.norm(f - Q @ (Q.conj().T @ f)) / np.linalg.norm(f)

    start = synth.start_fields(L, 2, 3).numpy()
    assert min(deficit(s) for s in start) > 0.9
    exact = inverse_iteration(_LinearPreconditioner(np.linalg.inv(D.dense())), start, 25, 0, 0)
    bound = 10 * (lam_min / 1.6415) ** 25
    assert max(deficit(s) for s in exact) <= bound
    sap = SchwarzOracle(D, (2, 2, 2, 2))
    got = inverse_iteration(sap, start, 11, 4, 4)
    assert max(deficit(s) for s in got) <= 0.2
    for s in got:
        assert lam_min <= norm(D.apply(s)) / norm(s) <= 1.2 * lam_min


def test_bootstrap_iteration_tight_tolerance_is_exact_inverse_iteration():
    """Section 5.3 bootstrapped steps: solved to 1e-11, each step is psi <- D^{-1} psi / |.| (the
    dense LU inverse), whatever the subspace used to deflate the solver; a loose tolerance gives a
    field nearer the low modes than one plain Schwarz step (smaller ||D psi|| / ||psi||, (5.2))."""
    from scipy.linalg import lu_factor, lu_solve
    from oracle.deflation import bootstrap_iteration, inverse_iteration
    from oracle.sap import SchwarzOracle
    L = (4, 4, 4, 4)
    D = WilsonClover(L, synth.random_gauge(L, 32).numpy(), -0.1, 1.0)
    start = synth.start_fields(L, 3, 6).numpy()
    f0 = inverse_iteration(SchwarzOracle(D, (2, 2, 2, 2)), start, 2, 4, 4)
    got = bootstrap_iteration(D, (2, 2, 2, 2), (2, 2, 2, 2), f0, 1, 1e-11)
    lu = lu_factor(D.dense())
    for l in range(3):
        w = lu_solve(lu, f0[l].reshape(-1))
        w /= np.linalg.norm(w)
        assert np.linalg.norm(got[l].reshape(-1) - w) <= 1e-8
    loose = bootstrap_iteration(D, (2, 2, 2, 2), (2, 2, 2, 2), f0, 1, 1e-2)
    plain = inverse_iteration(SchwarzOracle(D, (2, 2, 2, 2)), f0, 1, 4, 4)
    for l in range(3):
        assert norm(D.apply(loose[l])) < norm(D.apply(plain[l]))
