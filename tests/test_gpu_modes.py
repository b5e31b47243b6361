"""GPU parity of the low-mode solver (Chebyshev-accelerated subspace iteration on D^+ D, the paper's
Section 2.2 method) against the oracle's dense eigendecomposition, and of the block-subspace deficits
(3.15) used for the local-coherence measurement of Section 5.2."""
import numpy as np
import pytest
import torch

from oracle.deflation import BlockSubspace
from oracle.dirac import WilsonClover, low_modes
from oracle.sap import Blocking
from paper_0706_2298_gb300 import dwsolve as dw
from paper_0706_2298_gb300 import synth

pytestmark = pytest.mark.gpu

L = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def setup():
    U = synth.random_gauge(L, 33)
    ctx = dw.dw_create(L, -0.1, 1.0, U, (2, 2, 2, 2))
    D = WilsonClover(L, U.numpy(), -0.1, 1.0)
    w, v = low_modes(D, 12)
    return ctx, D, w, v


@pytest.mark.parametrize("prec,tol,etol,vtol", [(dw.DW_F64, 1e-10, 1e-9, 1e-8), (dw.DW_F32, 1e-9, 1e-9, 1e-7)])
def test_lowmodes_match_dense_eigendecomposition(setup, prec, tol, etol, vtol):
    """FP64 filter; FP32 filter, which hands over to FP64 when its rounding stalls the residuals."""
    ctx, D, w, v = setup
    nev, nbuf = 6, 6
    assert np.min(np.diff(w[:nev + 1])) > 1e-6 * w[nev]      # non-degenerate: vectors are unique up to a phase
    start = synth.start_fields(L, nev + nbuf, 41).cuda()
    modes = torch.empty((nev, ctx.V, 4, 3), dtype=torch.complex128, device="cuda")
    rc, ev, rs, it = dw.lowmodes_solve(ctx, nev, nbuf, start, modes, degree=16, tol=tol, maxit=200, prec=prec)
    assert rc == dw.DW_OK and it >= 1
    assert np.allclose(ev, w[:nev], rtol=etol, atol=0)
    assert max(r / e for r, e in zip(rs, ev)) <= tol
    m = modes.cpu().numpy()
    for i in range(nev):
        overlap = abs(np.vdot(v[i].reshape(-1), m[i].reshape(-1)))
        assert overlap >= 1 - vtol, (i, overlap)


def test_deficits_match_oracle(setup):
    """eps = |(1 - P) psi|^2 / |psi|^2 for a block subspace of 4 low modes on 2^4 blocks."""
    ctx, D, w, v = setup
    start = torch.from_numpy(np.ascontiguousarray(v[:4])).cuda()
    d = dw.deflation_build(ctx, (2, 2, 2, 2), 4, 0, 4, 4, start, basis_prec=dw.DW_F64, iter_prec=dw.DW_F64)
    basis = torch.empty((4, ctx.V, 4, 3), dtype=torch.complex128, device="cuda")
    dw.dfl_basis_export(d, basis)
    torch.cuda.synchronize()
    bl = basis.cpu().numpy()
    blk = Blocking(L, (2, 2, 2, 2))
    sub = BlockSubspace(D, (2, 2, 2, 2), np.stack([bl[:, blk.sites[b]] for b in range(blk.Nb)]))
    fields = np.concatenate([v[4:12], synth.gaussian_source(L, 42, nrhs=2).numpy()])
    eps = dw.dfl_deficits(d, torch.from_numpy(np.ascontiguousarray(fields)).cuda())
    ref = [sub.deficit(f) for f in fields]
    assert np.allclose(eps, ref, rtol=1e-10, atol=1e-14)
    # the generating modes themselves lie in the subspace
    eps0 = dw.dfl_deficits(d, start)
    assert max(eps0) <= 1e-24 * 1e4
