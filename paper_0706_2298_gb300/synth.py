"""Seeded synthetic inputs: gauge fields, quark sources, random start fields.

This module only draws random numbers and builds input fields.  It holds
none of the solver's arithmetic (no Dirac operator, no Schwarz sweep, no
projection); both the CUDA path and the FP64 checker take their inputs
from here.

Canonical layouts (shared by every caller):

* lattice ``L = (L0, L1, L2, L3)`` with ``L0`` the time extent;
  site index ``((x0*L1 + x1)*L2 + x2)*L3 + x3`` (x0 slowest);
* gauge field: ``complex128[V, 4, 3, 3]``, ``U[x, mu]`` is the link from
  ``x`` to ``x + mu``, colour matrix row-major;
* quark field: ``complex128[..., V, 4, 3]`` (spin, colour).

The paper's ensembles (two-flavour QCD at beta=5.3, Section 2.1) are not
available; the stand-in is a random SU(3) field ``U = exp(i*eps*X)`` with
``X`` a Gaussian traceless Hermitian matrix, followed by APE smearing with
reunitarisation, which gives smooth fields whose low Dirac modes show the
local coherence of Section 5.1 to a useful degree.

Random numbers come from torch's CPU Mersenne-Twister generator seeded per
(seed, kind), so the draws are identical on every machine; the smearing may
run on any device (the CUDA run changes only the last bits).
"""
from __future__ import annotations

import math
from typing import Sequence

import torch

_KIND = {"gauge": 11, "source": 23, "start": 37, "transform": 41, "basis": 53, "misc": 61}


def volume(L: Sequence[int]) -> int:
    return int(L[0]) * int(L[1]) * int(L[2]) * int(L[3])


def _gen(seed: int, kind: str) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed((int(seed) * 1000003 + _KIND[kind]) & 0x7FFFFFFFFFFFFFFF)
    return g


def complex_gaussian(shape, seed: int, kind: str = "misc") -> torch.Tensor:
    """i.i.d. complex normals with E|z|^2 = 1 (real and imaginary parts N(0, 1/2))."""
    g = _gen(seed, kind)
    re = torch.randn(*shape, generator=g, dtype=torch.float64)
    im = torch.randn(*shape, generator=g, dtype=torch.float64)
    return torch.complex(re, im) * math.sqrt(0.5)


def _traceless_hermitian(n: int, seed: int, kind: str) -> torch.Tensor:
    G = complex_gaussian((n, 3, 3), seed, kind)
    H = 0.5 * (G + G.conj().transpose(-1, -2))
    tr = torch.diagonal(H, dim1=-2, dim2=-1).sum(-1) / 3.0
    return H - tr[:, None, None] * torch.eye(3, dtype=H.dtype)


def _exp_i_hermitian(X: torch.Tensor, eps: float) -> torch.Tensor:
    """exp(i*eps*X) for Hermitian X through its eigendecomposition (exactly unitary)."""
    w, Q = torch.linalg.eigh(X)
    ph = torch.polar(torch.ones_like(w), eps * w)
    return (Q * ph[..., None, :]) @ Q.conj().transpose(-1, -2)


def reunitarize(U: torch.Tensor) -> torch.Tensor:
    """Gram-Schmidt of rows 0 and 1; row 2 = conj(row0 x row1); result has det 1."""
    r0 = U[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = U[..., 1, :]
    r1 = r1 - (r0.conj() * r1).sum(-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.linalg.cross(r0, r1, dim=-1).conj()
    return torch.stack([r0, r1, r2], dim=-2)


def _shift(f: torch.Tensor, mu: int, s: int) -> torch.Tensor:
    """f(x + s*mu) on a field shaped (L0, L1, L2, L3, ...), periodic."""
    return torch.roll(f, shifts=-s, dims=mu)


def ape_smear(U: torch.Tensor, L: Sequence[int], steps: int, alpha: float) -> torch.Tensor:
    """APE smearing, all links updated together from the previous step.

    V_mu(x) = (1-alpha) U_mu(x) + alpha/6 * sum_{nu != mu} [staples], then
    reunitarisation.  Periodic boundary conditions for the gauge field.
    """
    L0, L1, L2, L3 = (int(v) for v in L)
    W = U.reshape(L0, L1, L2, L3, 4, 3, 3)
    for _ in range(steps):
        new = []
        for mu in range(4):
            Umu = W[..., mu, :, :]
            st = torch.zeros_like(Umu)
            for nu in range(4):
                if nu == mu:
                    continue
                Unu = W[..., nu, :, :]
                # upper staple  U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                st = st + Unu @ _shift(Umu, nu, 1) @ _shift(Unu, mu, 1).conj().transpose(-1, -2)
                # lower staple  U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
                Unu_m = _shift(Unu, nu, -1)
                st = st + Unu_m.conj().transpose(-1, -2) @ _shift(Umu, nu, -1) @ _shift(_shift(Unu, nu, -1), mu, 1)
            new.append(reunitarize((1.0 - alpha) * Umu + (alpha / 6.0) * st))
        W = torch.stack(new, dim=4)
    return W.reshape(-1, 4, 3, 3)


def random_gauge(L: Sequence[int], seed: int, eps: float = 0.3, ape_steps: int = 5,
                 alpha: float = 0.5, device: str | torch.device = "cpu") -> torch.Tensor:
    """Smeared random SU(3) field, complex128[V, 4, 3, 3] on ``device``."""
    V = volume(L)
    X = _traceless_hermitian(V * 4, seed, "gauge")
    # the eigendecomposition runs on the CPU (batched 3x3 eigh on CUDA asks for huge workspaces)
    U = _exp_i_hermitian(X, eps).reshape(V, 4, 3, 3).to(device)
    if ape_steps > 0:
        U = ape_smear(U, L, ape_steps, alpha)
    return U.contiguous()


def unit_gauge(L: Sequence[int]) -> torch.Tensor:
    V = volume(L)
    return torch.eye(3, dtype=torch.complex128).expand(V, 4, 3, 3).contiguous()


def random_su3(n: int, seed: int, eps: float = 1.0) -> torch.Tensor:
    """n random SU(3) matrices (used as gauge transformations in tests)."""
    return _exp_i_hermitian(_traceless_hermitian(n, seed, "transform"), eps)


def gaussian_source(L: Sequence[int], seed: int, nrhs: int | None = None) -> torch.Tensor:
    """Complex Gaussian quark field(s), complex128[(nrhs,) V, 4, 3]."""
    V = volume(L)
    shape = (V, 4, 3) if nrhs is None else (nrhs, V, 4, 3)
    return complex_gaussian(shape, seed, "source")


def point_sources(L: Sequence[int], x: Sequence[int] = (0, 0, 0, 0)) -> torch.Tensor:
    """The 12 spin-colour unit sources at site x, complex128[12, V, 4, 3]."""
    V = volume(L)
    L0, L1, L2, L3 = L
    site = ((x[0] * L1 + x[1]) * L2 + x[2]) * L3 + x[3]
    eta = torch.zeros(12, V, 4, 3, dtype=torch.complex128)
    for s in range(4):
        for c in range(3):
            eta[3 * s + c, site, s, c] = 1.0
    return eta


def start_fields(L: Sequence[int], Ns: int, seed: int) -> torch.Tensor:
    """Ns random start fields for the subspace generation, complex128[Ns, V, 4, 3]."""
    return complex_gaussian((Ns, volume(L), 4, 3), seed, "start")
