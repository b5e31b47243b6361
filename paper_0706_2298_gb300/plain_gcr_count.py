"""Iteration count of plain (unpreconditioned) FP64 GCR on a benchmark workload, on the GPU.

Plain restarted GCR(16) on D is the oracle's own solve (its definition of psi = D^{-1} eta); the
oracle itself needs many hours for it at 48 x 24^3 on a CPU, so its reference timing measures a
bounded number of its GCR iterations on the host and scales them by the iteration count that
the same algorithm needs on the same workload, which this script measures with the library
(gcr_solve without deflation and with ncy = 0, i.e. M = 1, everything FP64) and records in
plain_gcr_counts.json.  At 8^4 the count equals that of the oracle's full run (GPU test).

    python -m paper_0706_2298_gb300.plain_gcr_count [--workload 24^3x48]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)
OUT = os.path.join(HERE, "plain_gcr_counts.json")


def measure(wl, maxit=200000):
    import torch
    from paper_0706_2298_gb300 import dwsolve as dw
    from paper_0706_2298_gb300 import synth
    L = wl["L"]
    U = synth.random_gauge(L, wl["gauge_seed"], device="cuda").cpu()
    ctx = dw.dw_create(L, wl["m0"], wl["csw"], U, wl["sap_bs"])
    eta = synth.gaussian_source(L, wl["source_seed"]).cuda()
    psi = torch.empty_like(eta)
    p = dw.sol_params(tol=wl["tol"], nkv=wl["nkv"], nmx=maxit, ncy=0, nmr=0, mixed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, infos = dw.gcr_solve(ctx, None, p, 1, eta, psi)
    t = time.perf_counter() - t0
    return {"iterations": infos[0].iterations, "relres": infos[0].relres, "converged": rc == dw.DW_OK,
            "gpu_seconds": t, "algorithm": f"GCR({wl['nkv']}) on D, no preconditioner, FP64, tol {wl['tol']:g}",
            "L": list(L), "m0": wl["m0"], "csw": wl["csw"]}


def main():
    import bench
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="24^3x48")
    a = ap.parse_args()
    bench.load_masses()
    rec = measure(bench.WORKLOADS[a.workload])
    print(json.dumps(rec), flush=True)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    data[a.workload] = rec
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1)


if __name__ == "__main__":
    main()
