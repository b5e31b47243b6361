"""Helpers shared by the GPU tests: marshal canonical fields to packed device fields."""
import numpy as np
import torch

from paper_0706_2298_gb300 import dwsolve as dw


def to_packed(ctx, prec, psi):
    """canonical complex128[(nrhs,) V, 4, 3] (CPU or GPU) -> packed device field(s)."""
    psi = torch.as_tensor(psi)
    nrhs = 1 if psi.dim() == 3 else psi.shape[0]
    dev = psi.to("cuda").contiguous()
    out = ctx.empty_field(prec, nrhs)
    dw.dw_pack(ctx, prec, nrhs, dev, out)
    return out


def from_packed(ctx, prec, packed, nrhs=1):
    out = torch.empty((nrhs, ctx.V, 4, 3), dtype=torch.complex128, device="cuda")
    dw.dw_unpack(ctx, prec, nrhs, packed, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return o[0] if nrhs == 1 else o


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
