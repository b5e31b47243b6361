"""Deflation subspace, projectors and the little Dirac operator (FP64).

* (3.1)  P psi = sum_k phi_k (phi_k, psi)                 orthogonal projector
* (3.2)  A_kl = (phi_k, D phi_l)                          little Dirac operator
* (3.3)  P_L psi = psi - sum_kl D phi_k (A^-1)_kl (phi_l, psi)
* (3.4)  P_R psi = psi - sum_kl phi_k (A^-1)_kl (phi_l, D psi)
* (3.15) deficit eps = ||(1 - P) psi||^2 for a normalised psi
* (4.1)  block projection:  P psi = sum_L sum_l phi^L_l (phi^L_l, psi)
* (4.2)  psi^L_l = psi_l restricted to L, then Gram-Schmidt on every block
* (5.1)  inverse iteration psi_l <- "D^-1" psi_l, the inverse replaced by
         M_sap (Section 5.3); normalised after every step [reading: the
         paper leaves the normalisation open; it only fixes the scale]
* (5.1) bootstrapped (Section 5.3): later steps replace "D^-1" by the
         deflated solver built on the current fields, stopped early
* (A.1)  B_{LL'} = (phi^L_k, D phi^{L'}_l), nonzero for L' = L or a neighbour

Basis layout: ``phi[L, l, s, spin, colour]`` with ``s`` the site within
block L in lexicographic order (``Blocking.sites``).  The global index of
basis vector (L, l) is ``k = L * Ns + l``.
"""
from __future__ import annotations

import numpy as np

from .dirac import WilsonClover
from .lattice import norm
from .sap import Blocking, SchwarzOracle

BF16_MANTISSA = 8


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round real or complex FP64 values to bfloat16 (round to nearest even) and back.

    Rounds through FP32 first (as a BF16 store of an FP32 value does);
    bfloat16 keeps the top 16 bits of the FP32 pattern.
    """
    if np.iscomplexobj(x):
        return round_bf16(x.real) + 1j * round_bf16(x.imag)
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def block_gram_schmidt(blk: Blocking, fields: np.ndarray, passes: int = 2, rank_tol: float = 1e-12):
    """Restrict global fields to the blocks (4.2) and orthonormalise per block.

    fields: complex128[Ns, V, 4, 3].  Modified Gram-Schmidt in the order
    l = 1..Ns, ``passes`` sweeps of re-orthogonalisation, then normalisation.
    Returns phi complex128[Nb, Ns, vol, 4, 3].  Raises on rank loss.
    """
    Ns = fields.shape[0]
    v = fields.reshape(Ns, -1, 12)[:, blk.sites, :]              # (Ns, Nb, vol, 12)
    v = np.ascontiguousarray(np.transpose(v, (1, 0, 2, 3))).reshape(blk.Nb, Ns, -1)
    for l in range(Ns):
        n0 = np.sqrt(np.einsum("bi,bi->b", v[:, l].conj(), v[:, l]).real)
        for _ in range(passes):
            for j in range(l):
                c = np.einsum("bi,bi->b", v[:, j].conj(), v[:, l])
                v[:, l] -= c[:, None] * v[:, j]
        n1 = np.sqrt(np.einsum("bi,bi->b", v[:, l].conj(), v[:, l]).real)
        if np.any(n1 <= rank_tol * np.maximum(n0, 1e-300)):
            raise np.linalg.LinAlgError("rank loss in block Gram-Schmidt")
        v[:, l] /= n1[:, None]
    return v.reshape(blk.Nb, Ns, blk.vol, 4, 3)


class BlockSubspace:
    """Domain-decomposed deflation subspace with its little Dirac operator."""

    def __init__(self, D: WilsonClover, bs, phi: np.ndarray, global_fields: np.ndarray | None = None):
        self.D = D
        self.blk = Blocking(D.L, bs)
        self.phi = phi                                     # (Nb, Ns, vol, 4, 3)
        self.Nb, self.Ns = phi.shape[0], phi.shape[1]
        self.N = self.Nb * self.Ns
        self.global_fields = global_fields
        self._A = None

    # -- (4.1) ----------------------------------------------------------------------
    def restrict(self, psi):
        """c[L, l] = (phi^L_l, psi); psi (V,4,3) or (B,V,4,3) -> (Nb,Ns) or (B,Nb,Ns)."""
        psi = np.asarray(psi)
        single = psi.ndim == 3
        p = psi.reshape(-1, self.D.V, 12)[:, self.blk.sites, :]        # (B, Nb, vol, 12)
        ph = self.phi.reshape(self.Nb, self.Ns, self.blk.vol, 12)
        c = np.einsum("LlsA,BLsA->BLl", ph.conj(), p)
        return c[0] if single else c

    def prolong(self, c):
        """sum_L sum_l phi^L_l c[L, l] as a global field."""
        c = np.asarray(c)
        single = c.ndim == 2
        cb = c.reshape(-1, self.Nb, self.Ns)
        ph = self.phi.reshape(self.Nb, self.Ns, self.blk.vol, 12)
        loc = np.einsum("LlsA,BLl->BLsA", ph, cb)
        out = np.zeros((cb.shape[0], self.D.V, 12), dtype=np.complex128)
        out[:, self.blk.sites, :] = loc
        out = out.reshape(-1, self.D.V, 4, 3)
        return out[0] if single else out

    def project(self, psi):
        """P psi (4.1)."""
        return self.prolong(self.restrict(psi))

    def deficit(self, psi):
        """||(1-P) psi||^2 / ||psi||^2 (3.15)."""
        return norm(psi - self.project(psi)) ** 2 / norm(psi) ** 2

    # -- (3.2) / (A.1) ----------------------------------------------------------------------
    def basis_field(self, L, l):
        c = np.zeros((self.Nb, self.Ns), dtype=np.complex128)
        c[L, l] = 1.0
        return self.prolong(c)

    @property
    def A(self):
        """Dense little Dirac operator A[k, k'] = (phi_k, D phi_k'), k = L*Ns + l."""
        if self._A is None:
            A = np.zeros((self.N, self.N), dtype=np.complex128)
            for l in range(self.Ns):
                cols = np.zeros((self.Nb, self.Nb, self.Ns), dtype=np.complex128)
                cols[np.arange(self.Nb), np.arange(self.Nb), l] = 1.0
                Dphi = self.D.apply(self.prolong(cols))                    # (Nb, V, 4, 3)
                r = self.restrict(Dphi)                                    # (Nb(col L'), Nb, Ns)
                for Lp in range(self.Nb):
                    A[:, Lp * self.Ns + l] = r[Lp].reshape(-1)
            self._A = A
        return self._A

    def block_matrix(self, L, Lp):
        """B_{L L'} (A.1), an Ns x Ns block of A."""
        s = self.Ns
        return self.A[L * s:(L + 1) * s, Lp * s:(Lp + 1) * s]

    def little_solve(self, w):
        """v = A^{-1} w (dense; the definition of the little solve)."""
        return np.linalg.solve(self.A, w.reshape(self.N)).reshape(self.Nb, self.Ns)

    # -- (3.3), (3.4) ---------------------------------------------------------------------
    def P_L(self, psi):
        return psi - self.D.apply(self.prolong(self.little_solve(self.restrict(psi))))

    def P_R(self, psi):
        return psi - self.prolong(self.little_solve(self.restrict(self.D.apply(psi))))


def inverse_iteration(sap: SchwarzOracle, fields: np.ndarray, n_inv: int, ncy: int, nmr: int):
    """psi_l <- M_sap psi_l, normalised, n_inv times (5.1); the Ns fields are independent."""
    out = np.array(fields, dtype=np.complex128, copy=True)
    for _ in range(n_inv):
        out = sap.apply(out, ncy, nmr)
        out /= np.sqrt(np.einsum("lvsc,lvsc->l", out.conj(), out).real)[:, None, None, None]
    return out


def build_subspace(D: WilsonClover, sap_bs, dfl_bs, start, n_inv, ncy, nmr, bf16: bool = False):
    """Plain subspace generation: inverse iteration, block restriction, block GS.

    With ``bf16=True`` the orthonormal basis is rounded to bfloat16 (the
    stored basis of the mixed-precision path) and everything downstream uses
    the rounded fields.
    """
    sap = SchwarzOracle(D, sap_bs)
    fields = inverse_iteration(sap, start, n_inv, ncy, nmr)
    blk = Blocking(D.L, dfl_bs)
    phi = block_gram_schmidt(blk, fields)
    if bf16:
        phi = round_bf16(phi)
    return BlockSubspace(D, dfl_bs, phi, fields)


def bootstrap_iteration(D: WilsonClover, sap_bs, dfl_bs, fields: np.ndarray, n_boot: int, tol: float,
                        ncy: int = 4, nmr: int = 4, nkv: int = 16):
    """The bootstrapped steps of the subspace generation (Section 5.3): n_boot times, the block
    subspace of the current fields (restriction and Gram-Schmidt (4.2), little operator (A.1),
    even-odd little system with global-mode deflation (A.2)-(A.3)) deflates the Dirac equation,
    D chi_l = psi_l is solved by DFL+SAP+GCR (Section 6) to ||psi_l - D chi_l|| <= tol ||psi_l||,
    and psi_l <- chi_l / ||chi_l||.  With tol -> 0 every step is exact inverse iteration."""
    from .little import EOLittle
    from .solver import solve_dfl_sap
    sap = SchwarzOracle(D, sap_bs)
    out = np.array(fields, dtype=np.complex128, copy=True)
    for _ in range(n_boot):
        phi = block_gram_schmidt(Blocking(D.L, dfl_bs), out)
        sub = BlockSubspace(D, dfl_bs, phi, out)
        little = EOLittle(sub)
        for l in range(out.shape[0]):
            chi, _ = solve_dfl_sap(D, sap, sub, little, out[l], tol=tol, nkv=nkv, ncy=ncy, nmr=nmr)
            out[l] = chi / norm(chi)
    return out
