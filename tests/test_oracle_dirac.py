"""Pins of the oracle's Wilson-clover operator against facts fixed by the
mathematics: the Clifford algebra, gamma_5-hermiticity, gauge covariance,
the free-field plane-wave solution, the field strength of a constant
abelian field and of a single excited link (worked out by hand), and a
dense 4^4 brute-force check."""
import numpy as np
import pytest

from paper_0706_2298_gb300 import synth
from oracle.dirac import WilsonClover, field_strength
from oracle.krylov import gcr
from oracle.lattice import GAMMA, GAMMA5

L8 = (8, 8, 8, 8)
L4 = (4, 4, 4, 4)


def _g5(p):
    return np.einsum("st,...tc->...sc", GAMMA5, p)


@pytest.fixture(scope="module")
def D8():
    U = synth.random_gauge(L8, 1).numpy()
    return WilsonClover(L8, U, -0.2, 1.0)


@pytest.fixture(scope="module")
def D4():
    U = synth.random_gauge(L4, 7).numpy()
    return WilsonClover(L4, U, -0.2, 1.0)


@pytest.fixture(scope="module")
def dense4(D4):
    return D4.dense()


def test_clifford_and_gamma5():
    for m in range(4):
        assert np.allclose(GAMMA[m], GAMMA[m].conj().T)
        for n in range(4):
            assert np.allclose(GAMMA[m] @ GAMMA[n] + GAMMA[n] @ GAMMA[m], 2.0 * (m == n) * np.eye(4))
    # chiral basis: gamma_5 = diag(1, 1, -1, -1)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


def test_gamma5_hermiticity(D8):
    eta = synth.gaussian_source(L8, 2).numpy()
    chi = synth.gaussian_source(L8, 3).numpy()
    lhs = np.vdot(chi, _g5(D8.apply(_g5(eta))))
    rhs = np.vdot(D8.apply(chi), eta)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gauge_covariance(D8):
    V = D8.V
    Om = synth.random_su3(V, 11).numpy().reshape(L8 + (3, 3))
    U = D8.U
    Up = np.empty_like(U)
    for mu in range(4):
        Om_f = np.roll(Om, -1, axis=mu)
        Up[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(Om_f, -1, -2))
    Dp = WilsonClover(L8, Up.reshape(V, 4, 3, 3), D8.m0, D8.csw)
    psi = synth.gaussian_source(L8, 4).numpy()
    Omf = Om.reshape(V, 3, 3)
    rot = lambda p: np.einsum("xab,xsb->xsa", Omf, p)
    lhs = Dp.apply(rot(psi))
    rhs = rot(D8.apply(psi))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 3), (3, 1, 1, 2)])
def test_free_field_plane_wave(n):
    """U = 1: D (u e^{ipx}) = [m0 + sum(1 - cos p) + i sum gamma_mu sin p_mu] u e^{ipx},
    with p_0 = (2 n_0 + 1) pi / L0 (antiperiodic) and p_k = 2 pi n_k / L_k."""
    L = (6, 4, 4, 8)
    m0 = -0.3
    D = WilsonClover(L, synth.unit_gauge(L).numpy(), m0, 1.7)
    p = np.array([(2 * n[0] + 1) * np.pi / L[0]] + [2 * np.pi * n[k] / L[k] for k in (1, 2, 3)])
    x = np.indices(L).reshape(4, -1).T
    phase = np.exp(1j * (x @ p))
    rng = np.random.default_rng(0)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi = phase[:, None, None] * u[None]
    Dp = (m0 + np.sum(1 - np.cos(p))) * np.eye(4) + 1j * np.einsum("m,mst->st", np.sin(p), GAMMA)
    expect = phase[:, None, None] * (Dp @ u)[None]
    assert np.allclose(D.apply(psi), expect, atol=1e-13)


def test_free_field_spectrum_dense():
    L = (4, 2, 2, 2)
    m0 = 0.1
    D = WilsonClover(L, synth.unit_gauge(L).numpy(), m0, 1.0)
    ev = np.linalg.eigvals(D.dense())
    lam = []
    for n0 in range(L[0]):
        for n1 in range(L[1]):
            for n2 in range(L[2]):
                for n3 in range(L[3]):
                    p = np.array([(2 * n0 + 1) * np.pi / L[0], 2 * np.pi * n1 / L[1],
                                  2 * np.pi * n2 / L[2], 2 * np.pi * n3 / L[3]])
                    a = m0 + np.sum(1 - np.cos(p))
                    b = np.sqrt(np.sum(np.sin(p) ** 2))
                    lam += [a + 1j * b] * 6 + [a - 1j * b] * 6
    key = lambda z: np.sort_complex(np.round(z.real, 8) + 1j * np.round(z.imag, 8))
    assert np.allclose(key(ev), key(np.array(lam)), atol=1e-7)


def test_constant_abelian_field_clover():
    """U_1(x) = exp(i theta x0), other links 1, theta = 2 pi / L0: every plaquette in
    the (0,1) plane is e^{i theta}, so F_01 = i sin(theta) and, with
    sigma_01 = diag(s_1, -s_1) in the chiral basis,
    C(x) = (4 + m0) - (c_sw / 2) sin(theta) diag(s_1, -s_1) (x) 1_3 on every site."""
    L = (6, 4, 4, 4)
    th = 2 * np.pi / L[0]
    U = synth.unit_gauge(L).numpy().reshape(L + (4, 3, 3)).copy()
    x0 = np.indices(L)[0]
    U[..., 1, :, :] = np.exp(1j * th * x0)[..., None, None] * np.eye(3)
    m0, csw = 0.05, 1.9
    D = WilsonClover(L, U.reshape(-1, 4, 3, 3), m0, csw)
    s1 = np.array([[0, 1], [1, 0]])
    sig01 = np.block([[s1, np.zeros((2, 2))], [np.zeros((2, 2)), -s1]])
    expect = (4 + m0) * np.eye(12) - 0.5 * csw * np.sin(th) * np.kron(sig01, np.eye(3))
    assert np.allclose(D.C, expect[None, None, None, None], atol=1e-14)


def test_single_link_field_strength():
    """Only U_1(y) = W != 1.  Worked by hand: for a plane (mu, nu) containing
    direction 1, the two plaquettes through the link contribute W or W^dag to
    the leaves at their corners; F_{mu nu} = (Q - Q^dag)/8 vanishes at y and
    y+1 and is +-(W - W^dag)/8 at the corners shifted off the link."""
    L = (4, 4, 4, 4)
    y = (1, 2, 1, 2)
    W = synth.random_su3(1, 5).numpy()[0]
    U = synth.unit_gauge(L).numpy().reshape(L + (4, 3, 3)).copy()
    U[y + (1,)] = W
    A = (W - W.conj().T) / 8.0

    def site(*d):
        return tuple((y[i] + d[i]) % L[i] for i in range(4))

    def unit(mu, s=1):
        e = [0, 0, 0, 0]
        e[mu] = s
        return e

    e1 = unit(1)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(U, mu, nu)
            expect = np.zeros(L + (3, 3), dtype=complex)
            if 1 in (mu, nu):
                other = nu if mu == 1 else mu
                sgn = 1.0 if mu == 1 else -1.0      # link along mu: +A at y+nu; along nu: -A at y+mu
                for s, val in ((1, sgn * A), (-1, -sgn * A)):
                    d = unit(other, s)
                    expect[site(*d)] += val
                    expect[site(*[d[i] + e1[i] for i in range(4)])] += val
            assert np.allclose(F, expect, atol=1e-15), (mu, nu)


def test_clover_hermitian_and_chiral(D8):
    C = D8.C.reshape(-1, 12, 12)
    assert np.allclose(C, np.conj(np.swapaxes(C, -1, -2)), atol=1e-15)
    G5 = np.kron(GAMMA5, np.eye(3))
    assert np.allclose(G5 @ C, C @ G5, atol=1e-15)


def test_even_odd_schur(D8):
    """D acting on (psi_e, -C_oo^{-1} D_oe psi_e) is (D^ psi_e, 0)."""
    pe = D8.even(synth.gaussian_source(L8, 6).numpy())
    po = -D8.odd(D8.apply_clover_inv(D8.D_oe(pe)))
    full = D8.apply(pe + po)
    assert np.linalg.norm(D8.odd(full)) <= 1e-13 * np.linalg.norm(full)
    assert np.allclose(D8.even(full), D8.schur(pe), atol=1e-13)
    # block decomposition of D
    psi = synth.gaussian_source(L8, 8).numpy()
    pe, po = D8.even(psi), D8.odd(psi)
    blocks = D8.even(D8.apply_clover(pe)) + D8.D_eo(po) + D8.D_oe(pe) + D8.odd(D8.apply_clover(po))
    assert np.allclose(blocks, D8.apply(psi), atol=1e-13)


def test_dense_4x4(D4, dense4):
    """Brute force on 4^4: spectrum closed under conjugation (gamma_5-hermiticity makes
    the characteristic polynomial real) and GCR solution = dense solve."""
    ev = np.linalg.eigvals(dense4)
    # every eigenvalue has its complex conjugate in the spectrum
    dist = np.abs(ev[:, None] - np.conj(ev)[None, :]).min(axis=1)
    assert dist.max() < 1e-8
    eta = synth.gaussian_source(L4, 2).numpy()
    x_dense = np.linalg.solve(dense4, eta.reshape(-1)).reshape(eta.shape)
    x, info = gcr(D4.apply, eta, tol=1e-12, nkv=16)
    assert info.converged
    cond = np.linalg.cond(dense4)
    assert np.linalg.norm(x - x_dense) <= 10 * cond * 1e-12 * np.linalg.norm(x_dense)


def test_low_modes_free_field_closed_form():
    """Lowest eigenvalues of D^dag D for the free field: on the plane wave with momentum p (p0
    antiperiodic), D = m0 + sum(1 - cos p) + i sum gamma sin p, so D^dag D = (m0 + sum(1 - cos p))^2 +
    sum sin^2 p on all 12 spin-colour components; the 12 lowest eigenvalues form one multiplet per
    minimising momentum (here p = (+-pi/4, 0, 0, 0): 24 equal eigenvalues)."""
    from oracle.dirac import low_modes
    L = (4, 2, 2, 2)
    m0 = -0.2
    D = WilsonClover(L, synth.unit_gauge(L).numpy(), m0, 1.0)
    w, v = low_modes(D, 30)
    vals = []
    for n0 in range(L[0]):
        for n in np.ndindex(*L[1:]):
            p = [(2 * n0 + 1) * np.pi / L[0]] + [2 * np.pi * n[k] / L[k + 1] for k in range(3)]
            vals.append((m0 + sum(1 - np.cos(x) for x in p)) ** 2 + sum(np.sin(x) ** 2 for x in p))
    vals = np.sort(np.repeat(vals, 12))
    assert np.allclose(w, vals[:30], rtol=1e-12, atol=1e-12)
    # eigenvectors: D^dag D v = w v (D^dag = gamma5 D gamma5), orthonormal
    g5 = np.diag([1, 1, -1, -1]).astype(complex)
    for i in (0, 23, 29):
        x = v[i]
        y = np.einsum("st,vtc->vsc", g5, D.apply(np.einsum("st,vtc->vsc", g5, D.apply(x))))
        assert np.linalg.norm(y - w[i] * x) <= 1e-11 * np.linalg.norm(y)
    G = v.reshape(30, -1).conj() @ v.reshape(30, -1).T
    assert np.allclose(G, np.eye(30), atol=1e-12)
