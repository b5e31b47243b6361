"""Solvers for the Wilson-clover equation D psi = eta (3.9), FP64.

``solve_plain``      the definition: unpreconditioned restarted GCR on D
                     (any convergent method reaches the same unique psi).
``solve_dfl_sap``    the paper's DFL+SAP+GCR (Sections 3.2, 6.1, 6.2, A.5),
                     read as follows.  Every restart:

        rho = eta - D psi                    (recomputed "with high precision", A.5)
        c   = A^{-1} Phi^dag rho             (little solve, outer tolerance)
        psi += Phi c;  rho = eta - D psi     (now Phi^dag rho ~ 0, i.e. P_L rho = rho)
        stop if ||rho|| <= tol ||eta||
        one flexible GCR cycle on  P_L D M_sap phi = rho  (6.2):
            xi_k = M_sap rho_k,  chi_k = P_L D xi_k  (little solve to the
            adapted tolerance  tol_in * ||rho_0|| / ||D xi_k||, capped)
        psi += sum_k beta_k xi_k

  The final P_R of (3.10)/(6.2) is folded into the next restart: after
  psi' = psi + zeta the deflation correction adds -Phi A^{-1} Phi^dag D zeta,
  so psi'' = psi + P_R zeta (+ the new Phi A^{-1} Phi^dag rho part).
  [reading: the paper gives the ingredients, not this ordering; any ordering
  converges to the same psi.]
``solve_sap``        SAP+GCR without deflation (the middle column of Table 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dirac import WilsonClover
from .krylov import gcr, gcr_cycle
from .lattice import norm
from .little import EOLittle
from .sap import SchwarzOracle
from .deflation import BlockSubspace


@dataclass
class SolveInfo:
    converged: bool = False
    restarts: int = 0
    gcr_iterations: int = 0
    little_iterations: list = field(default_factory=list)
    residuals: list = field(default_factory=list)


def solve_plain(D: WilsonClover, eta, tol=1e-10, nkv=16, maxit=200000):
    return gcr(D.apply, eta, tol=tol, nkv=nkv, maxit=maxit)


def solve_sap(D: WilsonClover, sap: SchwarzOracle, eta, tol=1e-10, nkv=32, ncy=4, nmr=4, maxres=200):
    info = SolveInfo()
    psi = np.zeros_like(eta)
    en = norm(eta)
    for _ in range(maxres):
        rho = eta - D.apply(psi)
        rn = norm(rho)
        info.residuals.append(rn / en)
        if rn <= tol * en:
            info.converged = True
            break
        upd, _, k = gcr_cycle(D.apply, rho, nkv, prec=lambda r: sap.apply(r, ncy, nmr),
                              stop=lambda r: r <= tol * en)
        psi = psi + upd
        info.gcr_iterations += k
        info.restarts += 1
    return psi, info


def solve_dfl_sap(D: WilsonClover, sap: SchwarzOracle, sub: BlockSubspace, little: EOLittle, eta,
                  tol=1e-10, nkv=16, ncy=4, nmr=4, little_tol_out=1e-12, little_tol_in=1e-6,
                  little_tol_cap=1e-1, little_nkv=16, maxres=100):
    info = SolveInfo()
    psi = np.zeros_like(eta)
    en = norm(eta)

    def lsolve(w, t):
        v, li = little.solve(w, tol=t, nkv=little_nkv)
        info.little_iterations.append(li.iterations)
        return v

    for _ in range(maxres):
        rho = eta - D.apply(psi)
        c = lsolve(sub.restrict(rho), little_tol_out)
        psi = psi + sub.prolong(c)
        rho = eta - D.apply(psi)
        rn = norm(rho)
        info.residuals.append(rn / en)
        if rn <= tol * en:
            info.converged = True
            break

        def op(xi, r0=rn):
            w = D.apply(xi)
            t = min(little_tol_cap, little_tol_in * r0 / max(norm(w), 1e-300))
            return w - D.apply(sub.prolong(lsolve(sub.restrict(w), t)))

        upd, _, k = gcr_cycle(op, rho, nkv, prec=lambda r: sap.apply(r, ncy, nmr),
                              stop=lambda r: r <= tol * en)
        psi = psi + upd
        info.gcr_iterations += k
        info.restarts += 1
    return psi, info
