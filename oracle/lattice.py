"""Lattice geometry and Dirac matrices (FP64, numpy).

Conventions (the paper defines the operator only by reference to the
O(a)-improved Wilson formulation, Section 2.1; these are the textbook
choices):

* L = (L0, L1, L2, L3), L0 = time; fields are numpy arrays with the four
  lattice axes first, ``(L0, L1, L2, L3, ...)``; site index with x0 slowest.
* Euclidean chiral basis
      gamma_0 = [[0, -1], [-1, 0]],  gamma_k = [[0, -i s_k], [i s_k, 0]]
  so that gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).
* sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu].
"""
from __future__ import annotations

import numpy as np

_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_PAULI = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def _chiral(e: np.ndarray) -> np.ndarray:
    return np.block([[_Z2, e], [e.conj().T, _Z2]])


GAMMA = np.stack([_chiral(-_I2)] + [_chiral(-1j * s) for s in _PAULI])   # (4, 4, 4)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
SIGMA = np.zeros((4, 4, 4, 4), dtype=np.complex128)
for _m in range(4):
    for _n in range(4):
        SIGMA[_m, _n] = 0.5j * (GAMMA[_m] @ GAMMA[_n] - GAMMA[_n] @ GAMMA[_m])


class Lattice:
    """Periodic 4D lattice with (anti)periodic fermion boundary in time."""

    def __init__(self, L, antiperiodic: bool = True):
        self.L = tuple(int(v) for v in L)
        self.V = int(np.prod(self.L))
        self.antiperiodic = bool(antiperiodic)
        x = np.indices(self.L)                       # (4, L0, L1, L2, L3)
        self.coords = x
        self.parity = (x.sum(axis=0) % 2).astype(np.int64)   # site parity
        self.even = self.parity == 0
        self.odd = ~self.even

    # fields -----------------------------------------------------------------
    def spinor_shape(self):
        return self.L + (4, 3)

    def to_grid(self, f: np.ndarray) -> np.ndarray:
        """(..., V, k...) canonical array -> (..., L0, L1, L2, L3, k...)."""
        f = np.asarray(f)
        return f.reshape(f.shape[:-3] + self.L + f.shape[-2:]) if f.shape[-3] == self.V and f.ndim >= 3 else f

    @staticmethod
    def shift(f: np.ndarray, mu: int, s: int, lead: int = 0) -> np.ndarray:
        """f(x + s*mu) for a field with ``lead`` leading batch axes (periodic)."""
        return np.roll(f, -s, axis=lead + mu)


def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    """(a, b) = sum conj(a) b over all components."""
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm(a: np.ndarray) -> float:
    return float(np.sqrt(np.vdot(a.ravel(), a.ravel()).real))
