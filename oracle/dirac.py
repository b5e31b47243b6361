"""O(a)-improved Wilson-Dirac operator (Sheikholeslami-Wohlert), FP64.

The paper uses "the O(a)-improved Wilson formulation" with a clover
coefficient c_sw (Section 2.1) and defines it only by reference.  The
textbook form written out here is

    D psi(x) = (4 + m0) psi(x) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) psi(x)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                              + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ],

    F_{mu nu}(x) = (1/8) (Q_{mu nu}(x) - Q_{nu mu}(x)),

with Q_{mu nu}(x) the sum of the four plaquette loops in the (mu, nu)
plane that start and end at x, all with the orientation mu -> nu.  The
fermion field is antiperiodic in time: the links U_0(x) with x0 = L0-1 are
multiplied by -1 inside the hopping term only.  In terms of the hopping
parameter kappa = 1/(2 m0 + 8) this is D = D_kappa / (2 kappa).

Fields: gauge U complex128[V, 4, 3, 3]; quark fields complex128[..., V, 4, 3]
(canonical layouts of ``paper_0706_2298_gb300.synth``).
"""
from __future__ import annotations

import numpy as np

from .lattice import GAMMA, SIGMA, Lattice

_I4 = np.eye(4, dtype=np.complex128)


def _dag(m: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(m, -1, -2))


def field_strength(U_grid: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Clover-leaf field strength F_{mu nu}(x), complex128[L0, L1, L2, L3, 3, 3].

    U_grid: (L0, L1, L2, L3, 4, 3, 3) gauge field (periodic, no fermion sign).
    """
    S = Lattice.shift
    Um = U_grid[..., mu, :, :]
    Un = U_grid[..., nu, :, :]
    Um_m = S(Um, mu, -1)            # U_mu(x - mu)
    Un_m = S(Un, nu, -1)            # U_nu(x - nu)
    leaf1 = Um @ S(Un, mu, 1) @ _dag(S(Um, nu, 1)) @ _dag(Un)
    leaf2 = Un @ _dag(S(Um_m, nu, 1)) @ _dag(S(Un, mu, -1)) @ Um_m
    leaf3 = _dag(Um_m) @ _dag(S(S(Un, mu, -1), nu, -1)) @ S(Um_m, nu, -1) @ Un_m
    leaf4 = _dag(Un_m) @ S(Um, nu, -1) @ S(Un_m, mu, 1) @ _dag(Um)
    Q = leaf1 + leaf2 + leaf3 + leaf4
    return (Q - _dag(Q)) / 8.0


class WilsonClover:
    """The Wilson-clover operator on a given gauge field (FP64 reference)."""

    def __init__(self, L, U, m0: float, csw: float, antiperiodic: bool = True):
        self.lat = Lattice(L, antiperiodic)
        self.L = self.lat.L
        self.V = self.lat.V
        self.m0 = float(m0)
        self.csw = float(csw)
        U = np.asarray(U, dtype=np.complex128)
        self.U = U.reshape(self.L + (4, 3, 3))
        # fermion links: antiperiodic sign on the time links of the last time slice
        Uf = self.U.copy()
        if antiperiodic:
            Uf[self.L[0] - 1, :, :, :, 0] *= -1.0
        self.Uf = [np.ascontiguousarray(Uf[..., mu, :, :]) for mu in range(4)]
        self.C = self.clover_matrices()
        self._Cinv = None

    # -- clover term ----------------------------------------------------------
    def clover_matrices(self) -> np.ndarray:
        """C(x) = (4 + m0) + c_sw (i/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x).

        Returns complex128[L0, L1, L2, L3, 12, 12], index 3*spin + colour.
        (i/4) sum over all ordered pairs equals (i/2) sum over mu < nu.
        """
        C = np.zeros(self.L + (12, 12), dtype=np.complex128)
        for mu in range(4):
            for nu in range(mu + 1, 4):
                F = field_strength(self.U, mu, nu)
                T = np.einsum("st,xyzwcd->xyzwsctd", SIGMA[mu, nu], F).reshape(self.L + (12, 12))
                C += 0.5j * self.csw * T
        C += (4.0 + self.m0) * np.eye(12)
        return C

    @property
    def Cinv(self) -> np.ndarray:
        if self._Cinv is None:
            self._Cinv = np.linalg.inv(self.C)
        return self._Cinv

    # -- field helpers -----------------------------------------------------------
    def _grid(self, psi):
        psi = np.asarray(psi, dtype=np.complex128)
        single = psi.ndim == 3
        g = psi.reshape((-1,) + self.L + (4, 3))
        return g, single, psi.shape

    @staticmethod
    def _back(g, shape):
        return g.reshape(shape)

    def _clover_apply(self, M, psi):
        g, _, shape = self._grid(psi)
        b = g.reshape(g.shape[:5] + (12, 1))
        return np.matmul(M[None], b).reshape(shape)

    def apply_clover(self, psi):
        """C(x) psi(x)."""
        return self._clover_apply(self.C, psi)

    def apply_clover_inv(self, psi):
        """C(x)^{-1} psi(x)."""
        return self._clover_apply(self.Cinv, psi)

    def hop(self, psi):
        """-1/2 sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]."""
        g, _, shape = self._grid(psi)
        out = np.zeros_like(g)
        for mu in range(4):
            U = self.Uf[mu][None]                                   # (1, L0..L3, 3, 3)
            # (U psi)[s, a] = sum_b U[a, b] psi[s, b]  ->  psi @ U^T
            fwd = np.matmul(Lattice.shift(g, mu, 1, lead=1), np.swapaxes(U, -1, -2))
            out -= 0.5 * np.matmul(_I4 - GAMMA[mu], fwd)
            bwd = np.matmul(g, np.conj(U))                          # U^dag psi at y
            bwd = Lattice.shift(bwd, mu, -1, lead=1)                # ... taken at y = x - mu
            out -= 0.5 * np.matmul(_I4 + GAMMA[mu], bwd)
        return out.reshape(shape)

    def apply(self, psi):
        """D psi."""
        return self.apply_clover(psi) + self.hop(psi)

    # -- even-odd decomposition ----------------------------------------------------
    def _mask(self, psi, sel):
        g, _, shape = self._grid(psi)
        return (g * sel[None, ..., None, None]).reshape(shape)

    def even(self, psi):
        return self._mask(psi, self.lat.even)

    def odd(self, psi):
        return self._mask(psi, self.lat.odd)

    def D_eo(self, psi):
        """Hopping from odd to even sites: (even part of) hop(odd part of psi)."""
        return self.even(self.hop(self.odd(psi)))

    def D_oe(self, psi):
        return self.odd(self.hop(self.even(psi)))

    def schur(self, psi):
        """Even-odd Schur complement on even sites: C_ee - D_eo C_oo^{-1} D_oe.

        Takes a field (odd part ignored) and returns a field zero on odd sites.
        """
        pe = self.even(psi)
        return self.even(self.apply_clover(pe)) - self.D_eo(self.odd(self.apply_clover_inv(self.D_oe(pe))))

    def dense(self, chunk: int = 768) -> np.ndarray:
        """The 12V x 12V matrix of D (small lattices only), columns = D e_j."""
        n = 12 * self.V
        M = np.zeros((n, n), dtype=np.complex128)
        for j0 in range(0, n, chunk):
            j1 = min(n, j0 + chunk)
            E = np.zeros((j1 - j0, n), dtype=np.complex128)
            E[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
            M[:, j0:j1] = self.apply(E.reshape(-1, self.V, 4, 3)).reshape(j1 - j0, n).T
        return M


def low_modes(D: WilsonClover, k: int):
    """The k lowest eigenvalues and eigenvectors of D^dag D (Section 2.2 works with this hermitian
    operator): the dense Hermitian eigendecomposition, the definition.  Small lattices only.
    Returns (w[k] ascending, v[k, V, 4, 3])."""
    M = D.dense()
    w, v = np.linalg.eigh(M.conj().T @ M)
    return w[:k], v[:, :k].T.reshape(k, D.V, 4, 3)
