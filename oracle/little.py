"""Solution of the little Dirac equation (Appendix A), FP64.

* (A.2) even-odd preconditioning on the block lattice.  Blocks are even
  or odd by the parity of their block-coordinate sum.  With B the little
  operator split into even/odd block rows and columns, B v = w becomes

      w~_e = B_ee^{-1} (w_e - B_eo B_oo^{-1} w_o)
      B^ v_e = w~_e,   B^ = 1 - B_ee^{-1} B_eo B_oo^{-1} B_oe     ("symmetric" form)
      v_o  = B_oo^{-1} (w_o - B_oe v_e)

  B_ee and B_oo are block diagonal (nearest-neighbour blocks have opposite
  parity), so their inverses are per-block Ns x Ns inverses.  The program
  must check that the diagonal blocks are safely invertible; an
  ill-conditioned block raises ``IllConditioned`` (the caller then falls
  back to the full little system).
* (A.3) global-mode deflation: the even-block components of the Ns global
  fields, g_l[L, k] = (phi^L_k, psi_l) for even L, orthonormalised, span a
  "little deflation subspace"; the Ns x Ns operator A~ = g^dag B^ g is
  inverted exactly and Section 3's projectors are applied with D -> B^.
* (A.4) the deflated equation P~_L B^ chi = P~_L w~_e is solved by GCR;
  v_e = P~_R chi + g A~^{-1} g^dag w~_e.
"""
from __future__ import annotations

import numpy as np

from .deflation import BlockSubspace
from .krylov import gcr


class IllConditioned(np.linalg.LinAlgError):
    pass


def _blockdiag_inverse(A, blocks, Ns, cond_max):
    """Inverse of the block-diagonal part of A over ``blocks`` (dense, in block order)."""
    n = len(blocks)
    out = np.zeros((n * Ns, n * Ns), dtype=np.complex128)
    for i, L in enumerate(blocks):
        B = A[L * Ns:(L + 1) * Ns, L * Ns:(L + 1) * Ns]
        if np.linalg.cond(B) > cond_max:
            raise IllConditioned(f"diagonal little block {L} is ill-conditioned")
        out[i * Ns:(i + 1) * Ns, i * Ns:(i + 1) * Ns] = np.linalg.inv(B)
    return out


class EOLittle:
    def __init__(self, sub: BlockSubspace, global_fields=None, deflate: bool = True,
                 cond_max: float = 1e12):
        self.sub = sub
        Ns = sub.Ns
        col = sub.blk.block_colour
        self.even_blocks = np.nonzero(col == 0)[0]
        self.odd_blocks = np.nonzero(col == 1)[0]
        if not sub.blk.even_counts():
            raise ValueError("even-odd little operator needs an even number of blocks per direction")

        def ix(blocks):
            return (blocks[:, None] * Ns + np.arange(Ns)[None, :]).reshape(-1)

        self.ie, self.io = ix(self.even_blocks), ix(self.odd_blocks)
        A = sub.A
        self.Bee = A[np.ix_(self.ie, self.ie)]
        self.Beo = A[np.ix_(self.ie, self.io)]
        self.Boe = A[np.ix_(self.io, self.ie)]
        self.Boo = A[np.ix_(self.io, self.io)]
        self.Bee_inv = _blockdiag_inverse(A, self.even_blocks, Ns, cond_max)
        self.Boo_inv = _blockdiag_inverse(A, self.odd_blocks, Ns, cond_max)
        ne = len(self.ie)
        self.Bhat = np.eye(ne) - self.Bee_inv @ self.Beo @ self.Boo_inv @ self.Boe
        self.g = None
        if deflate:
            gf = global_fields if global_fields is not None else sub.global_fields
            G = sub.restrict(gf).reshape(gf.shape[0], -1)[:, self.ie].T      # (N/2, Ns)
            self.g, _ = np.linalg.qr(G)                                       # orthonormal columns
            self.Atil = self.g.conj().T @ self.Bhat @ self.g

    # -- pieces ------------------------------------------------------------------------
    def apply_bhat(self, ve):
        return self.Bhat @ ve

    def _coarse(self, u):
        """g A~^{-1} g^dag u."""
        return self.g @ np.linalg.solve(self.Atil, self.g.conj().T @ u)

    def PL(self, u):
        return u - self.Bhat @ self._coarse(u)

    def PR(self, u):
        return u - self._coarse(self.Bhat @ u)

    # -- the solve ----------------------------------------------------------------------
    def solve(self, w, tol=1e-12, nkv=16, maxit=10000):
        """v ~= B^{-1} w via (A.2)-(A.4); w, v shaped (Nb, Ns).  Returns (v, GCR info)."""
        wf = np.asarray(w).reshape(-1)
        we, wo = wf[self.ie], wf[self.io]
        wt = self.Bee_inv @ (we - self.Beo @ (self.Boo_inv @ wo))
        if self.g is None:
            ve, info = gcr(self.apply_bhat, wt, tol=tol, nkv=nkv, maxit=maxit)
        else:
            chi, info = gcr(lambda u: self.PL(self.Bhat @ u), self.PL(wt), tol=tol, nkv=nkv, maxit=maxit)
            ve = self.PR(chi) + self._coarse(wt)
        vo = self.Boo_inv @ (wo - self.Boe @ ve)
        v = np.zeros_like(wf)
        v[self.ie], v[self.io] = ve, vo
        return v.reshape(self.sub.Nb, self.sub.Ns), info
