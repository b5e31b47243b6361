"""Small driver for profiling single kernels with ncu: builds the 48x24^3
operator, then applies D and M_sap a few times (FP32 by default).

    python -m paper_0706_2298_gb300.profile_driver [--L 48,24,24,24] [--prec f32|f64] [--sap 2] [--dirac 3]
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    import torch
    from paper_0706_2298_gb300 import dwsolve as dw
    from paper_0706_2298_gb300 import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--L", default="48,24,24,24")
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--dirac", type=int, default=3)
    ap.add_argument("--sap", type=int, default=2)
    ap.add_argument("--ncy", type=int, default=1)
    args = ap.parse_args()
    L = tuple(int(v) for v in args.L.split(","))
    prec = dw.DW_F32 if args.prec == "f32" else dw.DW_F64
    U = synth.random_gauge(L, 1, device="cuda").cpu()
    ctx = dw.dw_create(L, 0.0, 1.0, U, (4, 4, 4, 4))
    eta = synth.gaussian_source(L, 2).cuda()
    x, y = ctx.empty_field(prec), ctx.empty_field(prec)
    dw.dw_pack(ctx, prec, 1, eta, x)
    for _ in range(args.dirac):
        dw.dw_apply(ctx, prec, dw.DW_OP_FULL, 1, x, y)
    for _ in range(args.sap):
        dw.sap_precondition(ctx, prec, args.ncy, 4, 1, x, y)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
