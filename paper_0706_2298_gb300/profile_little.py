"""Driver for profiling the little solver with ncu: 48x24^3 operator, Ns = 20 subspace on 4^4
blocks (4 inverse-iteration steps), then a few FP32 little solves to 1e-6.

    python -m paper_0706_2298_gb300.profile_little [--solves 3]
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
    ap.add_argument("--solves", type=int, default=3)
    args = ap.parse_args()
    L = tuple(int(v) for v in args.L.split(","))
    U = synth.random_gauge(L, 1, device="cuda").cpu()
    ctx = dw.dw_create(L, 0.0, 1.0, U, (4, 4, 4, 4))
    d = dw.deflation_build(ctx, (4, 4, 4, 4), 20, 4, 4, 4, synth.start_fields(L, 20, 3).cuda())
    w = torch.randn(d.Nb * d.Ns * 2, dtype=torch.float32, device="cuda")
    v = torch.empty_like(w)
    import time
    for _ in range(args.solves):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, it, rr = dw.little_dirac_solve(d, dw.DW_F32, w, v, 1e-6, 2000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        print(f"little solve rc {rc} iterations {it} relres {rr:.3e} time {dt * 1e3:.3f} ms "
              f"({dt * 1e6 / max(it, 1):.1f} us/iteration)", flush=True)


if __name__ == "__main__":
    main()
