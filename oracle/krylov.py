"""Krylov solvers used by the method, FP64.

GCR: the paper solves both the deflated Dirac equation (6.2) and the little
system (A.4) with the GCR algorithm, chosen because it tolerates inexact
(flexible) preconditioning (Section 6.2).  The paper cites Saad for the
algorithm; the textbook flexible GCR(nkv) with restarts is written here:

    rho_0 = eta - Op x
    for k = 0 .. nkv-1:
        xi_k  = M rho_k                   (M = 1 when unpreconditioned)
        chi_k = Op xi_k
        chi_k -= sum_{j<k} (chi_j, chi_k) chi_j      (modified Gram-Schmidt)
        c_k = ||chi_k||,  chi_k /= c_k
        a_k = (chi_k, rho_k),  rho_{k+1} = rho_k - a_k chi_k
    x += sum_k beta_k xi_k  with  beta_k = (a_k - sum_{j>k} b_kj beta_j) / c_k
    restart from the recomputed residual eta - Op x.

MR: minimal-residual steps x += alpha r, r -= alpha Op r, alpha = (Op r, r)/|Op r|^2,
used for the block solves inside the Schwarz procedure (Section 6.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .lattice import norm, vdot


@dataclass
class GcrInfo:
    iterations: int = 0
    restarts: int = 0
    converged: bool = False
    residuals: list = field(default_factory=list)   # true relative residual at each restart


def gcr_cycle(op, rho, nkv, prec=None, stop=None):
    """One GCR cycle from residual ``rho``; returns (update, new residual, steps).

    ``stop(rnorm)`` may end the cycle early.  The returned residual is the
    recursively updated one (the caller recomputes the true residual).
    """
    xis, chis = [], []
    a = np.zeros(nkv, dtype=np.complex128)
    b = np.zeros((nkv, nkv), dtype=np.complex128)
    c = np.zeros(nkv)
    rho = rho.copy()
    k_done = 0
    for k in range(nkv):
        xi = prec(rho) if prec is not None else rho.copy()
        chi = op(xi)
        for j in range(k):
            b[j, k] = vdot(chis[j], chi)
            chi = chi - b[j, k] * chis[j]
        c[k] = norm(chi)
        chi = chi / c[k]
        a[k] = vdot(chi, rho)
        rho = rho - a[k] * chi
        xis.append(xi)
        chis.append(chi)
        k_done = k + 1
        if stop is not None and stop(norm(rho)):
            break
    beta = np.zeros(k_done, dtype=np.complex128)
    for k in range(k_done - 1, -1, -1):
        beta[k] = (a[k] - np.dot(b[k, k + 1:k_done], beta[k + 1:k_done])) / c[k]
    upd = np.zeros_like(rho)
    for k in range(k_done):
        upd = upd + beta[k] * xis[k]
    return upd, rho, k_done


def gcr(op, eta, tol=1e-10, nkv=16, maxit=100000, prec=None, x0=None):
    """Restarted (flexible) GCR for Op x = eta to ||eta - Op x|| <= tol ||eta||."""
    info = GcrInfo()
    x = np.zeros_like(eta) if x0 is None else x0.copy()
    en = norm(eta)
    if en == 0.0:
        info.converged = True
        return x, info
    while True:
        rho = eta - op(x)
        rn = norm(rho)
        info.residuals.append(rn / en)
        if rn <= tol * en:
            info.converged = True
            return x, info
        if info.iterations >= maxit:
            return x, info
        n = min(nkv, maxit - info.iterations)
        upd, _, steps = gcr_cycle(op, rho, n, prec, stop=lambda r: r <= tol * en)
        x = x + upd
        info.iterations += steps
        info.restarts += 1


def mr(op, b, nmr):
    """nmr minimal-residual steps from x = 0; returns (x, r = b - Op x)."""
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(nmr):
        p = op(r)
        pp = vdot(p, p).real
        if pp == 0.0:
            break
        alpha = vdot(p, r) / pp
        x = x + alpha * r
        r = r - alpha * p
    return x, r
