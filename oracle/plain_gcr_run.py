"""Run the oracle's definition of the solve -- unpreconditioned restarted GCR on D (FP64, numpy)
-- on one of the benchmark workloads and record its iteration count, true residuals and wall time.

TEST INFRASTRUCTURE ONLY (part of the oracle): it produces the measured baseline that the
benchmark's CPU and reference legs quote, from the oracle alone.  Writes JSON incrementally
(after every `--chunk` GCR cycles) so that a long run can be followed.

    python -m oracle.plain_gcr_run --L 48,24,24,24 --m0 0 --out oracle/plain_gcr_48x24c3.json
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import time

import numpy as np

from .dirac import WilsonClover
from .krylov import gcr
from .lattice import norm


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def main():
    from paper_0706_2298_gb300 import synth      # seeded inputs only (no arithmetic of the method)
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", default="48,24,24,24")
    ap.add_argument("--m0", type=float, default=0.0)
    ap.add_argument("--csw", type=float, default=1.0)
    ap.add_argument("--gauge-seed", type=int, default=1)
    ap.add_argument("--source-seed", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--nkv", type=int, default=16)
    ap.add_argument("--chunk", type=int, default=5, help="GCR cycles between progress records")
    ap.add_argument("--max-iterations", type=int, default=200000)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    L = tuple(int(v) for v in a.L.split(","))
    t0 = time.perf_counter()
    U = synth.random_gauge(L, a.gauge_seed).numpy()
    eta = synth.gaussian_source(L, a.source_seed).numpy()
    D = WilsonClover(L, U, a.m0, a.csw)
    t_setup = time.perf_counter() - t0
    en = norm(eta)
    rec = {"what": "oracle plain (unpreconditioned) restarted GCR on D, FP64 numpy",
           "L": list(L), "m0": a.m0, "csw": a.csw, "gauge_seed": a.gauge_seed, "source_seed": a.source_seed,
           "tol": a.tol, "nkv": a.nkv, "host": platform.node(), "cpu_model": cpu_model(), "nproc": os.cpu_count(),
           "setup_s": t_setup, "progress": [], "converged": False}
    x = np.zeros_like(eta)
    its = 0
    t1, c1 = time.perf_counter(), time.process_time()
    while its < a.max_iterations:
        n = min(a.chunk * a.nkv, a.max_iterations - its)
        x, info = gcr(D.apply, eta, tol=a.tol, nkv=a.nkv, maxit=n, x0=x)
        its += info.iterations
        rel = norm(eta - D.apply(x)) / en
        rec["progress"].append({"iterations": its, "true_relres": rel, "seconds": time.perf_counter() - t1})
        rec["converged"] = bool(rel <= a.tol)
        rec["iterations"] = its
        rec["solve_s"] = time.perf_counter() - t1
        rec["threads_busy"] = (time.process_time() - c1) / max(rec["solve_s"], 1e-9)
        with open(a.out + ".tmp", "w") as f:
            json.dump(rec, f, indent=1)
        os.replace(a.out + ".tmp", a.out)
        if rec["converged"] or info.iterations == 0:
            break


if __name__ == "__main__":
    main()
