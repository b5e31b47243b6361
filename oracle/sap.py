"""Block decomposition and the Schwarz alternating procedure (FP64).

Blocks (Section 4): the lattice is divided into non-overlapping rectangular
blocks of size bs = (b0, b1, b2, b3).  Blocks are numbered
lexicographically by their block coordinates (x0 slowest) and coloured by
the parity of the block-coordinate sum: colour 0 ("black") and 1 ("white").
With an even number of blocks in every direction, face-adjacent blocks have
opposite colours.

M_sap (Section 6.1; the paper defines it by reference to its earlier work
on Schwarz preconditioning) is read as the multiplicative Schwarz sweep

    xi = 0, r = rho
    repeat ncy times, for colour in (black, white):
        for every block L of that colour:  delta_L ~= D_L^{-1} r|_L
        xi += delta,  r = rho - D xi

where D_L is D restricted to L with the hops that leave L dropped
(Dirichlet block boundary).  The approximate block inverse is nmr
minimal-residual steps on the even-odd preconditioned block operator
D^_L = C_ee - D_eo,L C_oo^{-1} D_oe,L followed by the odd-site
reconstruction.  Blocks of one colour never touch, so they are processed
together with per-block inner products.
"""
from __future__ import annotations

import numpy as np

from .dirac import WilsonClover


class Blocking:
    def __init__(self, L, bs):
        self.L = tuple(int(v) for v in L)
        self.bs = tuple(int(v) for v in bs)
        for mu in range(4):
            if self.L[mu] % self.bs[mu] != 0:
                raise ValueError("block size must divide the lattice")
        self.nb = tuple(self.L[mu] // self.bs[mu] for mu in range(4))
        self.Nb = int(np.prod(self.nb))
        self.vol = int(np.prod(self.bs))
        x = np.indices(self.L)
        bc = x // np.array(self.bs).reshape(4, 1, 1, 1, 1)
        n = self.nb
        self.site_block = ((bc[0] * n[1] + bc[1]) * n[2] + bc[2]) * n[3] + bc[3]     # grid of block ids
        bcoord = np.array(np.unravel_index(np.arange(self.Nb), self.nb))             # (4, Nb)
        self.block_coords = bcoord
        self.block_colour = bcoord.sum(axis=0) % 2
        flat = self.site_block.ravel()
        # canonical site indices of every block, in lexicographic (x0 slowest) order
        order = np.argsort(flat, kind="stable")
        self.sites = order.reshape(self.Nb, self.vol)
        self.colour_of_site = self.block_colour[self.site_block]

    def even_counts(self) -> bool:
        return all(v % 2 == 0 for v in self.nb)

    def block_dot(self, a_grid, b_grid):
        """Per-block inner products (a, b)_L, complex128[B, Nb]; fields shaped (B, L0..L3, 4, 3)."""
        s = (np.conj(a_grid) * b_grid).sum(axis=(-1, -2)).reshape(a_grid.shape[0], -1)
        ids = self.site_block.ravel()
        out = np.zeros((a_grid.shape[0], self.Nb), dtype=np.complex128)
        for i in range(s.shape[0]):
            out[i] = (np.bincount(ids, s[i].real, self.Nb)
                      + 1j * np.bincount(ids, s[i].imag, self.Nb))
        return out

    def per_site(self, vals):
        """Broadcast per-block values (B, Nb) to the grid, (B, L0..L3, 1, 1)."""
        return vals[:, self.site_block][..., None, None]


class SchwarzOracle:
    """The Schwarz alternating procedure on top of a WilsonClover operator."""

    def __init__(self, D: WilsonClover, bs):
        self.D = D
        self.blk = Blocking(D.L, bs)
        if not self.blk.even_counts():
            raise ValueError("SAP needs an even number of blocks in every direction")
        self._sel = [self.blk.colour_of_site == c for c in (0, 1)]

    def _grid(self, psi):
        return psi.reshape((-1,) + self.D.L + (4, 3))

    def _mask(self, g, sel):
        return g * sel[None, ..., None, None]

    def block_op(self, g, colour):
        """D_L on all blocks of a colour (Dirichlet): mask D mask."""
        sel = self._sel[colour]
        return self._mask(self.D.apply(self._mask(g, sel)), sel)

    def _hop_c(self, g, colour, dst, src):
        sel = self._sel[colour]
        return self._mask(self.D.hop(self._mask(g, sel & src)), sel & dst)

    def block_mr(self, r, colour, nmr, exact=False):
        """Approximate block solves D_L delta = r|_L on all blocks of ``colour``.

        nmr MR steps on the even-odd block operator with per-block scalars,
        then odd reconstruction.  ``exact=True`` replaces this with dense
        block solves (used only to pin the sweep against block Gauss-Seidel).
        """
        D, lat = self.D, self.D.lat
        g = self._grid(r)
        sel = self._sel[colour]
        if exact:
            return self._exact_block_solve(g, colour).reshape(r.shape)
        E, O = lat.even, lat.odd
        b = self._mask(g, sel)
        be, bo = self._mask(b, E), self._mask(b, O)
        # r^_e = b_e - D_eo,L C_oo^{-1} b_o
        rh = be - self._hop_c(D.apply_clover_inv(bo), colour, E, O)
        x = np.zeros_like(rh)

        def dhat(v):
            t = D.apply_clover_inv(self._hop_c(v, colour, O, E))
            return self._mask(D.apply_clover(v), E & sel) - self._hop_c(t, colour, E, O)

        for _ in range(nmr):
            p = dhat(rh)
            pr = self.blk.block_dot(p, rh)
            pp = self.blk.block_dot(p, p).real
            alpha = np.where(pp > 0, pr / np.where(pp > 0, pp, 1.0), 0.0)
            a = self.blk.per_site(alpha)
            x = x + a * rh
            rh = rh - a * p
        # x_o = C_oo^{-1} (b_o - D_oe,L x_e)
        xo = D.apply_clover_inv(bo - self._hop_c(x, colour, O, E))
        xo = self._mask(xo, O & sel)
        return (x + xo).reshape(r.shape)

    def _exact_block_solve(self, g, colour):
        D = self.D
        out = np.zeros_like(g)
        for L_id in np.nonzero(self.blk.block_colour == colour)[0]:
            sites = self.blk.sites[L_id]
            n = len(sites) * 12
            cols = np.zeros((n,) + g.shape[1:], dtype=np.complex128)
            flat = cols.reshape(n, -1, 4, 3)
            for j in range(n):
                flat[j, sites[j // 12], (j % 12) // 3, j % 3] = 1.0
            Dc = D.apply(cols.reshape(n, -1, 4, 3)).reshape(n, -1, 12)[:, sites, :].reshape(n, n).T
            for bi in range(g.shape[0]):
                rhs = g[bi].reshape(-1, 12)[sites].reshape(n)
                sol = np.linalg.solve(Dc, rhs)
                o = out[bi].reshape(-1, 12)
                o[sites] = sol.reshape(-1, 12)
        return out

    def apply(self, rho, ncy, nmr, exact=False):
        """xi = M_sap rho."""
        g = self._grid(rho)
        xi = np.zeros_like(g)
        r = g.copy()
        for _ in range(ncy):
            for colour in (0, 1):
                delta = self._grid(self.block_mr(r, colour, nmr, exact=exact))
                xi = xi + delta
                r = g - self._grid(self.D.apply(xi.reshape(rho.shape)))
        return xi.reshape(rho.shape)
