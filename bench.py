#!/usr/bin/env python
"""Seconds per solve of D psi = eta to ||eta - D psi|| <= 1e-10 ||eta||.

Workload (default "24^3x48"): 48 x 24^3 lattice, smeared random SU(3)
field (U = exp(0.3 i X), 5 APE steps, alpha = 0.5), c_sw = 1, bare mass at
the most nearly critical value found by the unpreconditioned CG count scan
(workload_masses.json), one Gaussian source.  Solver: flexible GCR (restart
16) with FP64-class restart steps (double-float arithmetic), right-
preconditioned by M_sap (4^4 blocks, ncy = 4, nmr = 4, FP32), deflated by
Ns = 20 block fields on 4^4 blocks stored in BF16 (11 inverse-iteration
steps), little operator FP32 with FP64 assembly.
One step = one solve from psi = 0 with eta and all operator data resident
in HBM.  The same algorithm in plain FP64 is timed beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torch.distributed.run: every rank solves its own
right-hand sides (independent replicas, weak scaling, no collective in the
data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "24^3x48": dict(L=(48, 24, 24, 24), m0=-0.0, csw=1.0, sap_bs=(4, 4, 4, 4), dfl_bs=(4, 4, 4, 4), Ns=20,
                    n_inv=11, ncy=4, nmr=4, nkv=16, tol=1e-10, gauge_seed=1, source_seed=2, start_seed=3),
    "8^4": dict(L=(8, 8, 8, 8), m0=-0.2, csw=1.0, sap_bs=(4, 4, 4, 4), dfl_bs=(4, 4, 4, 4), Ns=8,
                n_inv=11, ncy=4, nmr=4, nkv=16, tol=1e-10, gauge_seed=1, source_seed=2, start_seed=3),
    # 64 x 32^3, 8^4 deflation blocks, Ns = 20, 12 point sources batched
    "32^3x64": dict(L=(64, 32, 32, 32), m0=0.0, csw=1.0, sap_bs=(4, 4, 4, 4), dfl_bs=(8, 8, 8, 8), Ns=20,
                    n_inv=11, ncy=4, nmr=4, nkv=16, tol=1e-10, gauge_seed=1, source_seed=2, start_seed=3),
    # 96 x 48^3, 8^4 deflation blocks, Ns = 32 (BF16 basis 16 GB); the 12 point sources one after the
    # other (a lockstep batch of 12 would need 12 x 32 Krylov fields at once)
    "48^3x96": dict(L=(96, 48, 48, 48), m0=0.0, csw=1.0, sap_bs=(4, 4, 4, 4), dfl_bs=(8, 8, 8, 8), Ns=32,
                    n_inv=11, ncy=4, nmr=4, nkv=16, tol=1e-10, gauge_seed=1, source_seed=2, start_seed=3,
                    batch=False, generation=False, table1=False),
}
# Mass of the 24^3x48 workload: the most nearly critical value of a CGNR iteration-count scan
# (workload_masses.json, written by tune_mass.py; the 2000-iteration rule is out of reach for
# these smeared fields, the count peaks at m0 = 0).
MASS_FILE = os.path.join(ROOT, "paper_0706_2298_gb300", "workload_masses.json")


# The benchmark's metric, printed identically by both arms (ours and the oracle reference arm).
METRIC = "s/solve to rel. residual 1e-10 vs plain FP64 path; D_w HBM GB/s & % of peak"
# Iteration counts of the oracle's own solve (plain, unpreconditioned GCR(16) on D, FP64) to 1e-10:
# the oracle's full run where it finishes in minutes (oracle/plain_gcr_run.py), else the count of
# the same algorithm on the GPU (paper_0706_2298_gb300/plain_gcr_count.py; equal to the oracle's
# at 8^4, checked by a GPU test).
ORACLE_RUN = {"8^4": os.path.join(ROOT, "oracle", "plain_gcr_8c4.json")}
PLAIN_COUNTS = os.path.join(ROOT, "paper_0706_2298_gb300", "plain_gcr_counts.json")

# DRAM bytes per little-GCR iteration of the cooperative kernel, from one ncu capture of the
# current kernel (dram__bytes_read.sum + dram__bytes_write.sum of one launch / its iterations):
# 48x24^3, Ns = 20: (76.61 + 3.65) MB over 41 iterations (cold cache: the first iteration reads
# the little operator from HBM, the rest hit L2).  Remove an entry when the kernel changes.
LITTLE_TRAFFIC = {("24^3x48", 20): 80.84e6 / 41}


def aggregate_ranks(t_ms, steps, world, device="cpu"):
    """Timed region of the slowest rank and the whole-job seconds per solve (every rank solved
    `steps` systems of its own: all ranks' solves over the slowest rank's time)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(t_ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    return t_ms, (t_ms / 1e3) / (steps * world)


def load_masses():
    if os.path.exists(MASS_FILE):
        with open(MASS_FILE) as f:
            for k, v in json.load(f).items():
                if k in WORKLOADS:
                    WORKLOADS[k]["m0"] = v["m0"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_gcr_sample(U, eta, wl, iterations, warmup=1):
    """The oracle's own solve -- unpreconditioned restarted GCR on D, FP64 numpy, as it stands --
    on the workload for a bounded number of GCR iterations (`warmup` untimed D applications
    first).  Returns (seconds per GCR iteration, iterations run, true relative residual)."""
    from oracle.dirac import WilsonClover
    from oracle.krylov import gcr
    from oracle.lattice import norm
    D = WilsonClover(wl["L"], U, wl["m0"], wl["csw"])
    for _ in range(max(warmup, 0)):
        D.apply(eta)
    t0, c0 = time.perf_counter(), time.process_time()
    x, info = gcr(D.apply, eta, tol=wl["tol"], nkv=wl["nkv"], maxit=iterations)
    t, cpu = time.perf_counter() - t0, time.process_time() - c0
    rel = norm(eta - D.apply(x)) / norm(eta)
    ORACLE_THREADS.append(cpu / max(t, 1e-9))
    return t / max(info.iterations, 1), info.iterations, float(rel)


# threads busy on average during the oracle samples (process CPU time / wall time)
ORACLE_THREADS = []


def oracle_cores():
    return max(1, round(max(ORACLE_THREADS))) if ORACLE_THREADS else 1


def oracle_run_record(workload):
    """Iteration count of the oracle's solve (plain GCR to 1e-10) on this workload: its own full run
    (oracle/plain_gcr_run.py) if recorded, else the GPU count of the same algorithm."""
    p = ORACLE_RUN.get(workload)
    if p and os.path.exists(p):
        with open(p) as f:
            rec = json.load(f)
        if rec.get("converged"):
            rec["source"] = (f"the oracle's full run ({rec['solve_s']:.0f} s wall on {rec.get('cpu_model', '?')}, "
                             f"{rec.get('threads_busy', 0):.1f} threads busy)")
            return rec
    if os.path.exists(PLAIN_COUNTS):
        with open(PLAIN_COUNTS) as f:
            rec = json.load(f).get(workload)
        if rec and rec.get("converged"):
            rec["source"] = (f"the same algorithm run to {rec['relres']:.2e} on the GPU in FP64 "
                             f"(plain_gcr_count.py; at 8^4 the GPU count is within 1% of the oracle's full run "
                             f"on the same inputs)")
            return rec
    return None


def _oracle_small_solve(seed):
    """One whole oracle solve at 8^4 (plain GCR to 1e-10); returns (seconds, iterations, residual)."""
    sys.path.insert(0, ROOT)
    from oracle.dirac import WilsonClover
    from oracle.lattice import norm
    from oracle.solver import solve_plain
    from paper_0706_2298_gb300 import synth
    wl = WORKLOADS["8^4"]
    D = WilsonClover(wl["L"], synth.random_gauge(wl["L"], wl["gauge_seed"]).numpy(), wl["m0"], wl["csw"])
    eta = synth.gaussian_source(wl["L"], seed).numpy()
    t0, c0 = time.perf_counter(), time.process_time()
    x, info = solve_plain(D, eta, tol=wl["tol"], nkv=wl["nkv"])
    t, cpu = time.perf_counter() - t0, time.process_time() - c0
    return t, info.iterations, float(norm(eta - D.apply(x)) / norm(eta)), cpu / max(t, 1e-9)


def oracle_small_solves(nproc):
    """Whole oracle solves at 8^4, measured: one on one core, then nproc independent solves in nproc
    processes started with spawn (all cores); s/solve single-thread and all-cores."""
    import multiprocessing as mp
    t1, its, rel, thr = _oracle_small_solve(1002)
    ctx = mp.get_context("spawn")
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"                  # one thread per process: nproc processes on nproc cores
    try:
        t0 = time.perf_counter()
        with ctx.Pool(nproc) as pool:
            res = pool.map(_oracle_small_solve, [2000 + k for k in range(nproc)])
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"workload": "8^4, m0 = -0.2, c_sw = 1, plain GCR(16) to 1e-10 (whole solves, measured)",
            "one_process_s_per_solve": t1, "one_process_threads_busy": thr, "iterations": its, "true_relres": rel,
            "all_cores_s_per_solve": wall / nproc, "all_cores_processes": nproc, "threads_per_process": 1,
            "all_cores_max_relres": max(r[2] for r in res)}


def l2_copy_bandwidth(torch, mb=32, reps=100):
    """Measured L2-resident copy bandwidth: a 2 x `mb` MB working set (inside the 129 MB L2) copied
    back and forth `reps` times from one captured CUDA graph (no launch gaps); bytes read + written
    per copy over the CUDA-event time of a replay, best of 5 replays."""
    n = mb * (1 << 20) // 4
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(4):
            b.copy_(a)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(reps // 2):
            b.copy_(a)
            a.copy_(b)
    graph.replay()
    torch.cuda.synchronize()
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        best = t if best is None else min(best, t)
    del graph
    return {"gbs": 2 * n * 4 / best / 1e9,
            "how": f"{reps} copies of a {mb} MB fp32 buffer back and forth in one CUDA graph, best of 5 (CUDA events)"}


def fp32_peak_tflops():
    """FP32 CUDA-core peak from the unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop/FMA x
    2.07 GHz (maximum SM clock) = 80.5 TFLOP/s."""
    return {"tflops": 152 * 128 * 2 * 2.07e9 / 1e12, "how": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}


def sap_flops_per_site(nmr):
    """Algorithmic FP32 flops per lattice site of the colour a Schwarz pass processes (counting the
    Wilson hop as 1320 and the clover term as 552 flops per site): even-odd preparation
    (A_oo^-1, D_eo: 948 per block site), nmr MR steps (one D^ application 1884 + two inner products
    and two updates 168 per block site), odd reconstruction (948) and the residual update (one D,
    1872)."""
    return 948 + nmr * (1884 + 168) + 948 + 1872


def run_reference(args, wl, rank):
    """The reference arm: the oracle (plain FP64 numpy, as it stands) on the host cores.  A step is
    one GCR iteration of the oracle's own solve (unpreconditioned GCR on D) at the workload's size;
    s/solve = measured seconds per iteration x the iteration count of the oracle's full run to
    1e-10 on this workload (oracle/plain_gcr_run.py, whose record names its host)."""
    from paper_0706_2298_gb300 import synth
    if rank != 0:
        return
    L = wl["L"]
    rec = oracle_run_record(args.workload)
    base = {"impl": "reference", "metric": METRIC, "unit": "s/solve", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload, "L": list(L), "m0": wl["m0"]}}
    if rec is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no converged oracle run recorded for {args.workload}"}),
              flush=True)
        return
    U = synth.random_gauge(L, wl["gauge_seed"]).numpy()
    eta = synth.gaussian_source(L, wl["source_seed"]).numpy()
    t_it, n_it, rel = oracle_gcr_sample(U, eta, wl, max(args.steps, 1), warmup=args.warmup)
    val = t_it * rec["iterations"]
    sample = (f"{n_it} GCR iterations of the oracle's plain GCR({wl['nkv']}) on D at {args.workload} "
              f"(true relres after them {rel:.3e}; {t_it:.3f} s per iteration, numpy) x "
              f"{rec['iterations']} iterations to {wl['tol']:g}, from {rec['source']}")
    line = dict(base, value=val, ms_per_step=1e3 * t_it,
                cpu_baseline={"value": val, "unit": "s/solve", "cores": oracle_cores(), "kind": "oracle", "sample": sample,
                              "cpu_model": cpu_model(), "nproc": os.cpu_count()},
                e2e={"value": val, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    print(json.dumps(line), flush=True)


def profile_case(args, wl):
    """Small fixed launch sequences for ncu captures of single kernels (not a benchmark):
    'dirac-sap': 3 D applications and 2 M_sap (ncy = 1) in --prec;  'little': --solves FP32
    little solves to 1e-6 with an Ns-field subspace (4 inverse-iteration steps);  'little12': the
    same with 12 systems in one multi-RHS solve;  'batch12': one
    batched solve of the 12 point sources;  'ptnet': one 16 -> 16 network layer on the tensor cores
    and one on the CUDA cores."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_0706_2298_gb300 import dwsolve as dw
    from paper_0706_2298_gb300 import synth
    L = wl["L"]
    U = synth.random_gauge(L, wl["gauge_seed"], device="cuda").cpu()
    ctx = dw.dw_create(L, wl["m0"], wl["csw"], U, wl["sap_bs"])
    if args.profile_case == "ptnet":
        # one 16 -> 16 network layer on the tensor cores and one on the CUDA cores
        w = torch.randn(9 * 64 * 64 * 2, dtype=torch.float32, device="cuda") * 0.05
        hin = torch.randn(16 * synth.volume(L) * 24, dtype=torch.float32, device="cuda")
        hout = torch.empty_like(hin)
        dw.ptnet_layer16(ctx, w, 0, 1, hin, hout)
        dw.ptnet_layer16(ctx, w, 0, 0, hin, hout)
    elif args.profile_case == "dirac-sap":
        prec = dw.DW_F32 if args.prec == "f32" else dw.DW_F64
        x, y = ctx.empty_field(prec), ctx.empty_field(prec)
        dw.dw_pack(ctx, prec, 1, synth.gaussian_source(L, 2).cuda(), x)
        for _ in range(3):
            dw.dw_apply(ctx, prec, dw.DW_OP_FULL, 1, x, y)
        for _ in range(2):
            dw.sap_precondition(ctx, prec, 1, wl["nmr"], 1, x, y)
    else:
        n_inv = 4 if args.profile_case in ("little", "little12") else wl["n_inv"]
        d = dw.deflation_build(ctx, wl["dfl_bs"], wl["Ns"], n_inv, wl["ncy"], wl["nmr"],
                               synth.start_fields(L, wl["Ns"], wl["start_seed"]).cuda())
        if args.profile_case == "little12":
            # the 12 systems of a point-source batch in one multi-RHS little solve (FP32, 1e-6)
            w = torch.randn(12 * d.Nb * d.Ns * 2, dtype=torch.float32, device="cuda")
            v = torch.empty_like(w)
            for _ in range(args.solves):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, its, rr = dw.little_dirac_solve_batch(d, dw.DW_F32, 12, w, v, 1e-6, 2000)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                print(f"12-system little solve rc {rc} iterations {max(its)} {dt * 1e6 / max(max(its), 1):.1f} "
                      "us/iteration", flush=True)
        elif args.profile_case == "little":
            w = torch.randn(d.Nb * d.Ns * 2, dtype=torch.float32, device="cuda")
            v = torch.empty_like(w)
            for _ in range(args.solves):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, it, rr = dw.little_dirac_solve(d, dw.DW_F32, w, v, 1e-6, 2000)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                print(f"little solve rc {rc} iterations {it} relres {rr:.3e} {dt * 1e6 / max(it, 1):.1f} us/iteration",
                      flush=True)
        else:
            eta = synth.point_sources(L).cuda()
            psi = torch.empty_like(eta)
            dw.dw_autotune(ctx, 12)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("batched_solve")
            rc, _ = dw.gcr_solve(ctx, d, dw.sol_params(tol=wl["tol"], nkv=wl["nkv"], mixed=1), 12, eta, psi)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            print("batched solve rc", rc, flush=True)
    torch.cuda.synchronize()
    print("ok", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="24^3x48", choices=list(WORKLOADS))
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-batch", action="store_true", help="skip the 12 point-source batched solve")
    ap.add_argument("--coherence", action="store_true",
                    help="also measure local coherence (24 low modes of D^+D, about two minutes at 48x24^3)")
    ap.add_argument("--no-ptnet", action="store_true", help="skip the network-layer timing")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip the solver comparison over masses and the subspace generation variants")
    ap.add_argument("--profile-case", choices=["dirac-sap", "little", "little12", "batch12", "ptnet"], default=None,
                    help="run a small fixed launch sequence for an ncu capture and exit")
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"], help="--profile-case dirac-sap precision")
    ap.add_argument("--solves", type=int, default=1, help="--profile-case little: number of little solves")
    args = ap.parse_args()
    load_masses()
    wl = WORKLOADS[args.workload]
    if args.profile_case:
        profile_case(args, wl)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    if world > 1:
        dist.barrier()
    from paper_0706_2298_gb300 import dwsolve as dw
    from paper_0706_2298_gb300 import synth

    L = wl["L"]
    V = synth.volume(L)
    # ---- inputs (seeded, synthetic); the smearing runs on the GPU, draws are on the CPU generator
    U = synth.random_gauge(L, wl["gauge_seed"], device="cuda").cpu()
    ctx = dw.dw_create(L, wl["m0"], wl["csw"], U, wl["sap_bs"])
    eta_h = synth.gaussian_source(L, wl["source_seed"] + 1000 * rank)
    eta = eta_h.cuda()
    start = synth.start_fields(L, wl["Ns"], wl["start_seed"]).cuda()
    psi = torch.empty_like(eta)

    t0 = time.perf_counter()
    dfl = dw.deflation_build(ctx, wl["dfl_bs"], wl["Ns"], wl["n_inv"], wl["ncy"], wl["nmr"], start,
                             basis_prec=dw.DW_BF16, iter_prec=dw.DW_F32)
    t_build = time.perf_counter() - t0
    little_tune = dw.dfl_autotune(dfl)          # grid size and hop variant of the little solver
    p_mixed = dw.sol_params(tol=wl["tol"], nkv=wl["nkv"], ncy=wl["ncy"], nmr=wl["nmr"], mixed=1)

    def solve():
        rc, infos = dw.gcr_solve(ctx, dfl, p_mixed, 1, eta, psi)
        if rc != dw.DW_OK:
            raise RuntimeError(f"solve did not converge: {infos[0].as_dict()}")
        return infos[0]

    for _ in range(max(args.warmup, 0)):
        solve()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(os.path.join(os.environ.get("DW_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_r{rank}.csv"))
    clocks.start()
    n0 = dw.dw_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    torch.cuda.nvtx.range_push("timed_solve")
    infos = [solve() for _ in range(args.steps)]
    torch.cuda.nvtx.range_pop()
    ev1.record()
    torch.cuda.synchronize()
    launches = dw.dw_launch_count() - n0
    t_ms, value = aggregate_ranks(ev0.elapsed_time(ev1), args.steps, world, device="cuda")
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_per_step = t_ms / args.steps
    iters = statistics.median([i.iterations for i in infos])

    # ---- true residual of the last timed solve, by the library's FP64 D (not its double-float D)
    x64, y64 = ctx.empty_field(dw.DW_F64), ctx.empty_field(dw.DW_F64)
    dw.dw_pack(ctx, dw.DW_F64, 1, psi, x64)
    dw.dw_apply(ctx, dw.DW_F64, dw.DW_OP_FULL, 1, x64, y64)
    dw.dw_pack(ctx, dw.DW_F64, 1, eta, x64)
    relres64 = float(torch.linalg.norm(x64 - y64) / torch.linalg.norm(x64))
    del x64, y64

    # ---- rooflines from the library's CUDA-event phase timers over the timed solves
    hbm, peak_kind = peaks()
    l2 = l2_copy_bandwidth(torch)
    fp32_peak = fp32_peak_tflops()
    # dominant kernel: the cooperative little GCR (A.2-A.4).  Algorithmic bytes per little-GCR
    # iteration (FP32): the eight off-diagonal Ns x Ns blocks of every block row of the little
    # operator (both parities, read once by the two hops) and the 2 Ns global-mode vectors g, B^g
    # of the A.3 projection (Ne Ns complex each).  The operator (66 MB) is L2-resident.
    Nb, Ns = dfl.Nb, dfl.Ns
    lit_bytes = Nb * 8 * Ns * Ns * 8 + 2 * Ns * (Nb // 2) * Ns * 8
    t_little = sum(i.t_little for i in infos)
    n_lit = sum(i.little_iterations for i in infos)
    lit_s = t_little / max(n_lit, 1)
    roof = {"kernel": f"little_gcr_coop_kernel<float,{Ns}>", "bound": "l2", "achieved": lit_bytes / lit_s / 1e9,
            "peak": l2["gbs"], "unit": "GB/s", "frac": lit_bytes / lit_s / 1e9 / l2["gbs"],
            "traffic": LITTLE_TRAFFIC.get((args.workload, Ns)), "peak_kind": "measured here: " + l2["how"],
            "per": "little GCR iteration", "us_per_iteration": lit_s * 1e6, "algorithmic_bytes": lit_bytes,
            "l2_resident": True, "hbm_peak": hbm, "frac_of_hbm": lit_bytes / lit_s / 1e9 / hbm,
            "iterations_per_solve": n_lit / max(len(infos), 1)}
    # the Schwarz block kernel (second largest): 960 algorithmic bytes per site processed
    t_sap = sum(i.t_sap for i in infos)
    n_sap_launch = sum(i.iterations for i in infos) * 2 * wl["ncy"]
    sap_launch_s = t_sap / max(n_sap_launch, 1)
    # per site processed (FP32): links 4 x 12 reals, clover (A or A^-1) 72 reals, r in/out, delta out, xi in/out
    sap_bytes = (V // 2) * 4 * (48 + 72 + 24 * 5)
    sap_flops = (V // 2) * sap_flops_per_site(wl["nmr"])
    roof_sap = {"kernel": "sap_staged_kernel<128>", "bound": "hbm+alu", "achieved": sap_bytes / sap_launch_s / 1e9,
                "peak": hbm, "unit": "GB/s", "frac": sap_bytes / sap_launch_s / 1e9 / hbm,
                "launch_us": sap_launch_s * 1e6, "algorithmic_bytes_per_launch": sap_bytes,
                "alu": {"achieved": sap_flops / sap_launch_s / 1e12, "peak": fp32_peak["tflops"], "unit": "TFLOP/s",
                        "frac": sap_flops / sap_launch_s / 1e12 / fp32_peak["tflops"],
                        "peak_kind": fp32_peak["how"], "flops_per_launch": sap_flops}}

    # ---- D_w bandwidth: FP32 and FP64 applications, L2 flushed before each timed launch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    dirac = {}
    for prec, name, rb in ((dw.DW_F32, "f32", 4), (dw.DW_F64, "f64", 8)):
        x = ctx.empty_field(prec)
        y = ctx.empty_field(prec)
        dw.dw_pack(ctx, prec, 1, eta, x)
        ts = []
        for it in range(13):
            flush.fill_(float(it))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dw.dw_apply(ctx, prec, dw.DW_OP_FULL, 1, x, y)
            b.record()
            torch.cuda.synchronize()
            if it >= 3:
                ts.append(a.elapsed_time(b) / 1e3)
        t = statistics.median(ts)
        algo = V * rb * (24 + 24 + 4 * 18 + 72)      # psi in + out, 4 links (18 reals), clover 72 reals
        dirac[name] = {"us": t * 1e6, "gbs": algo / t / 1e9, "frac_of_measured": algo / t / 1e9 / hbm,
                       "frac_of_8tbs": algo / t / 8e12, "algorithmic_bytes": algo}
        del x, y
    del flush

    # ---- plain FP64 path (same algorithm, FP64 everywhere, FP64 basis)
    plain = None
    dw.dw_release_workspace(ctx)           # the mixed solver's cached fields are not needed meanwhile
    if not args.no_plain:
        dfl64 = dw.deflation_build(ctx, wl["dfl_bs"], wl["Ns"], wl["n_inv"], wl["ncy"], wl["nmr"], start,
                                   basis_prec=dw.DW_F64, iter_prec=dw.DW_F64)
        p64 = dw.sol_params(tol=wl["tol"], nkv=wl["nkv"], ncy=wl["ncy"], nmr=wl["nmr"], mixed=0)
        psi64 = torch.empty_like(eta)
        rc, inf64 = dw.gcr_solve(ctx, dfl64, p64, 1, eta, psi64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        n_plain = max(1, min(args.steps, 3))
        for _ in range(n_plain):
            rc, inf64 = dw.gcr_solve(ctx, dfl64, p64, 1, eta, psi64)
        b.record()
        torch.cuda.synchronize()
        plain = {"s_per_solve": a.elapsed_time(b) / 1e3 / n_plain, "iterations": inf64[0].iterations,
                 "relres": inf64[0].relres, "converged": rc == dw.DW_OK}
        del dfl64
        dw.dw_release_workspace(ctx)

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    eta_pin = eta_h.pin_memory()
    psi_pin = torch.empty_like(eta_h).pin_memory()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        eta.copy_(eta_pin, non_blocking=True)
        rc, _ = dw.gcr_solve(ctx, dfl, p_mixed, 1, eta, psi)
        psi_pin.copy_(psi, non_blocking=True)
    b.record()
    torch.cuda.synchronize()
    e2e = {"value": a.elapsed_time(b) / 1e3 / args.steps, "unit": "s/solve",
           "h2d_bytes_per_step": eta_h.numel() * 16, "d2h_bytes_per_step": eta_h.numel() * 16}

    # ---- 12 spin-colour point sources: one lockstep batch (captured M_sap graphs) vs one at a time
    batch = None
    if not args.no_batch:
        tune = dw.dw_autotune(ctx, 12)
        eta12 = synth.point_sources(L).cuda()
        psi12 = torch.empty_like(eta12)
        res = {}
        for mode in (("batched", "sequential") if wl.get("batch", True) else ("sequential",)):
            if mode == "sequential":
                os.environ["DW_BATCH"] = "0"
            rc, inf12 = dw.gcr_solve(ctx, dfl, p_mixed, 12, eta12, psi12)      # warm-up (captures graphs)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n0b = dw.dw_launch_count()
            a.record()
            rc, inf12 = dw.gcr_solve(ctx, dfl, p_mixed, 12, eta12, psi12)
            b.record()
            torch.cuda.synchronize()
            os.environ.pop("DW_BATCH", None)
            res[mode] = {"s_per_rhs": a.elapsed_time(b) / 1e3 / 12, "s_total": a.elapsed_time(b) / 1e3,
                         "converged": rc == dw.DW_OK, "max_relres": max(i.relres for i in inf12),
                         "gcr_iterations_max": max(i.iterations for i in inf12),
                         "launches": dw.dw_launch_count() - n0b}
        batch = {"workload": f"{args.workload}, 12 point sources (spin-colour unit vectors at the origin)",
                 **res, "speedup_batched": (res["sequential"]["s_total"] / res["batched"]["s_total"]
                                            if "batched" in res else None),
                 "autotune": tune}
        del eta12, psi12
        dw.dw_release_workspace(ctx)

    # ---- subspace generation variants (Section 5.3): plain inverse iteration vs bootstrapped steps
    gen = None
    # (skipped at 96x48^3: the extra Ns = 32 subspaces would need a second 65 GB FP64 basis beside
    # the benchmark's own)
    if not args.no_table1 and wl.get("generation", True):
        gen = {}
        for name, kw in (("plain n_inv=11", dict(n_inv=11)), ("plain n_inv=5", dict(n_inv=5)),
                         ("bootstrap 3 plain + 2 boot (tol 1e-2)", dict(n_inv=3, boot_steps=2, boot_tol=1e-2,
                                                                          boot_nmx=16))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dv = dw.deflation_build(ctx, wl["dfl_bs"], wl["Ns"], kw.pop("n_inv"), wl["ncy"], wl["nmr"], start,
                                    basis_prec=dw.DW_BF16, iter_prec=dw.DW_F32, **kw)
            tb = time.perf_counter() - t0
            rc, inf = dw.gcr_solve(ctx, dv, p_mixed, 1, eta, psi)
            gen[name] = {"build_s": tb, "solve_gcr_steps": inf[0].iterations, "solve_s": inf[0].seconds,
                         "mean_Dpsi_over_psi": dv.info.rho_out,
                         "boot_gcr_steps_per_field": dv.info.boot_gcr_steps / wl["Ns"], "converged": rc == dw.DW_OK}
            del dv

    # ---- Table 1 analogue (Section 6.3): three solvers at several bare masses, one deflation
    # subspace generated at the workload mass and reused at the others (Section 6.4)
    table1 = None
    if not args.no_table1 and wl.get("table1", True):    # (four extra contexts: not at 96x48^3)
        table1 = []
        for dm in (0.0, 0.02, 0.05, 0.1):
            m = wl["m0"] + dm
            cm = ctx if dm == 0.0 else dw.dw_create(L, m, wl["csw"], U, wl["sap_bs"])
            t0 = time.perf_counter()
            dm_ = dfl if dm == 0.0 else dw.dfl_retarget(dfl, cm)
            t_rt = time.perf_counter() - t0
            row = {"m0": m, "retarget_s": t_rt if dm else 0.0}
            for name, fn in (
                    ("DFL+SAP+GCR mixed", lambda: dw.gcr_solve(cm, dm_, p_mixed, 1, eta, psi)),
                    ("SAP+GCR mixed", lambda: dw.gcr_solve(cm, None, dw.sol_params(tol=wl["tol"], nkv=32,
                                                                                   ncy=wl["ncy"], nmr=wl["nmr"],
                                                                                   mixed=1, nmx=20000), 1, eta, psi)),
                    ("EO+BiCGstab FP64", lambda: dw.bicgstab_solve(cm, wl["tol"], 20000, eta, psi))):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = fn()
                torch.cuda.synchronize()
                ts = time.perf_counter() - t0
                if name.startswith("EO"):
                    row[name] = {"iterations": res[1], "s": ts, "relres": res[2], "converged": res[0] == dw.DW_OK}
                else:
                    row[name] = {"iterations": res[1][0].iterations, "s": ts, "relres": res[1][0].relres,
                                 "converged": res[0] == dw.DW_OK}
            table1.append(row)
            if dm:
                del dm_, cm

    # ---- network layer (learned subspace generation): the 16 -> 16 channel layer on the tensor cores
    # (tcgen05, BF16 operands, FP32 accumulation) and on the CUDA cores (FP32), one set of 16 fields
    ptl = None
    if not args.no_ptnet:
        import numpy as _np
        wl1 = (_np.random.default_rng(5).normal(size=(9, 64, 64, 2)) * 0.05).astype(_np.float32)
        wdev = torch.from_numpy(wl1.reshape(-1)).cuda()
        hin = torch.randn(16 * V * 24, dtype=torch.float32, device="cuda")
        hout = torch.empty_like(hin)
        flops = 9 * 2 * 128 * 128 * 3 * V          # real-form GEMM: 885 kflop per site
        bf16_peak = 1889.1
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pk):
            with open(pk) as f:
                bf16_peak = json.load(f).get("bf16_tflops", bf16_peak)
        ptl = {"flops_per_layer": flops}
        for name, tc in (("tensor_cores_bf16", 1), ("tensor_cores_bf16_tile32", 1), ("cuda_cores_fp32", 0)):
            if name.endswith("tile32"):
                os.environ["DW_TC_TILE"] = "32"
            for _ in range(2):
                dw.ptnet_layer16(ctx, wdev, 0, tc, hin, hout)
            ts = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                dw.ptnet_layer16(ctx, wdev, 0, tc, hin, hout)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            os.environ.pop("DW_TC_TILE", None)
            t = statistics.median(ts)
            ptl[name] = {"ms": t * 1e3, "tflops": flops / t / 1e12}
        ptl["tensor_cores_bf16"]["frac_of_bf16_peak"] = ptl["tensor_cores_bf16"]["tflops"] / bf16_peak
        ptl["bf16_peak_tflops"] = bf16_peak
        ptl["speedup_tensor_cores"] = ptl["cuda_cores_fp32"]["ms"] / ptl["tensor_cores_bf16"]["ms"]
        del hin, hout, wdev

    # ---- local coherence (Section 5.2): low modes of D^+ D by Chebyshev-accelerated subspace
    # iteration, a block subspace (4^4 blocks) from half of them, deficits (3.15) of the others
    coherence = None
    dw.dw_release_workspace(ctx)
    if args.coherence:
        nev, nbuf = 24, 8
        st = synth.start_fields(L, nev + nbuf, 4242).cuda()
        modes = torch.empty((nev, V, 4, 3), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, ev, rs, its = dw.lowmodes_solve(ctx, nev, nbuf, st, modes, degree=24, tol=1e-4, maxit=80,
                                            prec=dw.DW_F32)
        torch.cuda.synchronize()
        t_modes = time.perf_counter() - t0
        del st
        build = modes[0::2].contiguous()
        held = modes[1::2].contiguous()
        dc = dw.deflation_build(ctx, wl["dfl_bs"], nev // 2, 0, wl["ncy"], wl["nmr"], build, basis_prec=dw.DW_F64,
                                iter_prec=dw.DW_F64)
        eps = dw.dfl_deficits(dc, held)
        eps_gen = dw.dfl_deficits(dfl, held)          # the benchmark's inverse-iterated subspace (Ns = 20)
        coherence = {"modes": nev, "converged": rc == dw.DW_OK, "iterations": its, "seconds": t_modes,
                     "eigenvalues_DdagD": ev, "max_rel_residual": max(r / e for r, e in zip(rs, ev)),
                     "blocks": list(wl["dfl_bs"]), "built_from": "modes 0, 2, ..., 22 (12 fields)",
                     "deficits_held_out": {"min": min(eps), "mean": sum(eps) / len(eps), "max": max(eps)},
                     "deficits_held_out_in_generated_subspace": {"min": min(eps_gen),
                                                                 "mean": sum(eps_gen) / len(eps_gen),
                                                                 "max": max(eps_gen)}}
        del dc, modes, build, held

    # ---- CPU oracle sample (rank 0, N = 1 only): the oracle's own solve on the host cores
    cpu = None
    rec = oracle_run_record(args.workload)
    if rank == 0 and world == 1 and not args.no_cpu and rec is not None:
        n_s = 4
        t_it, n_it, rel = oracle_gcr_sample(U.numpy(), eta_h.numpy() if rank == 0 else None, wl, n_s)
        cpu = {"value": t_it * rec["iterations"], "unit": "s/solve", "cores": oracle_cores(), "kind": "oracle",
               "sample": f"{n_it} GCR iterations of the oracle's plain GCR({wl['nkv']}) on D at {args.workload} "
                         f"({t_it:.2f} s per iteration, numpy, true relres after them {rel:.3e}) x "
                         f"{rec['iterations']} iterations to {wl['tol']:g}, from {rec['source']}",
               "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "iteration_count": {k: rec.get(k) for k in ("iterations", "source")},
               "whole_solves": oracle_small_solves(min(os.cpu_count() or 1, 16))}

    if rank == 0:
        line = {"metric": METRIC,
                "value": value, "unit": "s/solve", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+bf16 (double-float restarts)", "data": "synthetic",
                "config": {"workload": args.workload, "L": list(L), "m0": wl["m0"], "csw": wl["csw"],
                           "sap_bs": list(wl["sap_bs"]), "dfl_bs": list(wl["dfl_bs"]), "Ns": wl["Ns"],
                           "n_inv": wl["n_inv"], "nkv": wl["nkv"], "ncy": wl["ncy"], "nmr": wl["nmr"],
                           "tol": wl["tol"], "l2": "inputs larger than L2 (solve working set > 2 GB)",
                           "parallelism": f"replicas x{world}"},
                "gcr_iterations": iters, "relres": max(i.relres for i in infos), "relres_fp64_check": relres64,
                "little_iterations_per_solve": statistics.median([i.little_iterations for i in infos]),
                "phase_s": {k: statistics.median([getattr(i, k) for i in infos])
                            for k in ("t_sap", "t_dirac", "t_project", "t_little", "t_orth", "t_restart")},
                "dfl_build_s": t_build, "little_autotune": little_tune, "plain_fp64": plain,
                "speedup_vs_plain_fp64": (plain["s_per_solve"] / value) if plain else None,
                "dirac": dirac, "roofline": roof, "roofline_sap": roof_sap, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "batch12": batch, "subspace_generation": gen,
                "table1": table1, "local_coherence": coherence, "ptnet_layer16": ptl}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
