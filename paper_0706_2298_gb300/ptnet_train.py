"""Training and evaluation of the gauge-covariant parallel-transport network that proposes
the deflation fields (the learned part of the subspace generation, Section 5.1 procedure).

Training pairs come from the plain procedure (5.1) on several seeded gauge fields: x = the Ns
fields after k0 inverse-iteration steps psi <- M_sap psi / |psi|, y = the same fields after
n_inv steps.  The network (3 layers, 1 -> 16 -> 16 -> 1 channels, the library's CUDA forward,
backward and Adam kernels) is trained to map x to y.  On held-out gauge fields three subspaces
are compared:

  plain n_inv   the full plain procedure (the method without the network);
  plain k0      the plain procedure stopped after k0 steps (the same number of Schwarz sweeps
                as the learned generation, i.e. the method without the network at equal cost);
  learned       k0 plain steps, then the network (judged by the quality measure (5.2) against
                its input, with the plain procedure as fallback).

Reported per subspace: the quality measure (5.2) of the generated fields (mean |D psi|/|psi|,
measured by the library's judge for the learned build), the deficit |(1 - P) v|/|v| of
approximate low modes v (fields after many inverse-iteration steps from independent starts),
the FGCR and little GCR iteration counts and the times of one mixed-precision solve to 1e-10,
and the build time.

    python -m paper_0706_2298_gb300.ptnet_train [--L 32,16,16,16] [--train-seeds 8] ...
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def init_weights(channels: int = 16, seed: int = 0, scale: float = 0.1):
    """Near-identity start (flat complex64 layout [layer][9][4 cout][4 cin] as float32 pairs):
    the site term passes the input through (spin kept, channels mixed evenly), hops small."""
    import torch
    rng = np.random.default_rng(seed)
    parts = []
    for cin, cout in ((1, channels), (channels, channels), (channels, 1)):
        w = (rng.normal(size=(9, 4 * cout, 4 * cin)) + 1j * rng.normal(size=(9, 4 * cout, 4 * cin)))
        w *= scale / np.sqrt(9 * 4 * cin)
        eye = np.kron(np.ones((cout, cin)) / np.sqrt(cin * cout), np.eye(4))
        w[0] += eye
        parts.append(w.reshape(-1))
    flat = np.concatenate(parts).astype(np.complex64)
    return torch.from_numpy(flat.view(np.float32).copy()).cuda()


def make_pairs(dw, synth, ctx, L, Ns, k0, n_inv, ncy, nmr, start_seed):
    """(x, y): Ns packed FP32 fields after k0 and after n_inv plain inverse-iteration steps."""
    start = synth.start_fields(L, Ns, start_seed).cuda()
    x = ctx.empty_field(dw.DW_F32, Ns)
    dw.dw_pack(ctx, dw.DW_F32, Ns, start, x)
    dw.dfl_inverse_iteration(ctx, ncy, nmr, k0, Ns, x)
    y = x.clone()
    dw.dfl_inverse_iteration(ctx, ncy, nmr, n_inv - k0, Ns, y)
    return x, y


def train(dw, samples, W, steps, lr, time_budget=None, log=None):
    """Adam on the regression loss, cycling through the training gauge fields; returns losses."""
    import torch
    m, v, g = torch.zeros_like(W), torch.zeros_like(W), torch.empty_like(W)
    losses = []
    t0 = time.perf_counter()
    for step in range(1, steps + 1):
        ctx, x, y, nf = samples[(step - 1) % len(samples)]
        loss = dw.ptnet_loss_grad(ctx, W, nf, x, y, g)
        dw.ptnet_adam(W, g, m, v, step, lr)
        losses.append(loss)
        if log and (step % max(1, steps // 10) == 0 or step == 1):
            log(f"step {step}: loss {loss:.4f}")
        if time_budget is not None and time.perf_counter() - t0 > time_budget:
            break
    torch.cuda.synchronize()
    return losses


def deficit(dw, d, vlow, nv):
    """mean |(1 - P) v| / |v| over nv packed FP32 fields (P = Phi Phi^+, block projector)."""
    import torch
    fs = vlow.numel() // nv
    c = torch.empty(2 * d.Nb * d.Ns, dtype=torch.float32, device="cuda")
    pv = torch.empty(fs, dtype=torch.float32, device="cuda")
    out = []
    for k in range(nv):
        x = vlow[k * fs:(k + 1) * fs]
        dw.dfl_restrict(d, dw.DW_F32, x, c)
        dw.dfl_prolong(d, dw.DW_F32, c, pv)
        out.append(float(torch.linalg.norm((x - pv).double()) / torch.linalg.norm(x.double())))
    return float(np.mean(out))


def evaluate(dw, synth, W, L, seed, Ns, k0, n_inv, ncy, nmr, bs, m0, csw, nlow=6, low_steps=30, judge=0.95,
             solve=True):
    """Compare plain n_inv, plain k0 and learned subspaces on the gauge field of ``seed``."""
    import torch
    U = synth.random_gauge(L, seed, device="cuda").cpu()
    ctx = dw.dw_create(L, m0, csw, U, bs)
    start = synth.start_fields(L, Ns, seed + 100).cuda()
    # approximate low modes: many plain steps from independent start fields
    vlow = ctx.empty_field(dw.DW_F32, nlow)
    dw.dw_pack(ctx, dw.DW_F32, nlow, synth.start_fields(L, nlow, seed + 200).cuda(), vlow)
    dw.dfl_inverse_iteration(ctx, ncy, nmr, low_steps, nlow, vlow)
    eta = synth.gaussian_source(L, seed + 300).cuda()
    psi = torch.empty_like(eta)
    res = {}
    variants = (("plain_n_inv", dict(n_inv=n_inv)), ("plain_k0", dict(n_inv=k0)),
                ("learned", dict(n_inv=n_inv, net_weights=W, net_k0=k0, net_judge=judge)),
                ("learned_forced", dict(n_inv=n_inv, net_weights=W, net_k0=k0, net_judge=1e30)))
    for name, kw in variants:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = dw.deflation_build(ctx, bs, Ns, kw.pop("n_inv"), ncy, nmr, start, basis_prec=dw.DW_BF16,
                               iter_prec=dw.DW_F32, **kw)
        torch.cuda.synchronize()
        r = {"build_s": time.perf_counter() - t0, "deficit": deficit(dw, d, vlow, nlow)}
        if name.startswith("learned"):
            r.update(learned_used=int(d.info.learned_used), rho_in=d.info.rho_in, rho_out=d.info.rho_out)
        if solve:
            p = dw.sol_params(tol=1e-10, mixed=1)
            dw.gcr_solve(ctx, d, p, 1, eta, psi)      # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, inf = dw.gcr_solve(ctx, d, p, 1, eta, psi)
            torch.cuda.synchronize()
            r.update(solve_s=time.perf_counter() - t0, gcr_iterations=inf[0].iterations,
                     little_iterations=inf[0].little_iterations, relres=inf[0].relres, converged=rc == dw.DW_OK)
        res[name] = r
        del d
    return res


def main():
    import torch
    from paper_0706_2298_gb300 import dwsolve as dw
    from paper_0706_2298_gb300 import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--L", default="32,16,16,16")
    ap.add_argument("--Ns", type=int, default=20)
    ap.add_argument("--k0", type=int, default=2)
    ap.add_argument("--n-inv", type=int, default=11)
    ap.add_argument("--bs", default="4,4,4,4")
    ap.add_argument("--m0", type=float, default=0.0)
    ap.add_argument("--csw", type=float, default=1.0)
    ap.add_argument("--train-seeds", type=int, default=8)
    ap.add_argument("--eval-seeds", type=int, default=3)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--time-budget", type=float, default=240.0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    L = tuple(int(v) for v in args.L.split(","))
    bs = tuple(int(v) for v in args.bs.split(","))
    ncy = nmr = 4
    log = lambda m: print(m, file=sys.stderr, flush=True)
    samples = []
    t0 = time.perf_counter()
    for s in range(args.train_seeds):
        seed = 1001 + s
        U = synth.random_gauge(L, seed, device="cuda").cpu()
        ctx = dw.dw_create(L, args.m0, args.csw, U, bs)
        x, y = make_pairs(dw, synth, ctx, L, args.Ns, args.k0, args.n_inv, ncy, nmr, seed + 100)
        samples.append((ctx, x, y, args.Ns))
    t_data = time.perf_counter() - t0
    log(f"training data: {args.train_seeds} gauge fields x {args.Ns} fields in {t_data:.1f} s")
    W = init_weights(16, seed=7)
    t0 = time.perf_counter()
    losses = train(dw, samples, W, args.steps, args.lr, args.time_budget, log)
    t_train = time.perf_counter() - t0
    log(f"trained {len(losses)} steps in {t_train:.1f} s: loss {losses[0]:.4f} -> {losses[-1]:.4f}")
    del samples
    torch.cuda.empty_cache()
    evals = {}
    for s in range(args.eval_seeds):
        seed = 2001 + s
        evals[seed] = evaluate(dw, synth, W, L, seed, args.Ns, args.k0, args.n_inv, ncy, nmr, bs, args.m0, args.csw)
        log(json.dumps({seed: evals[seed]}))
    summary = {"L": L, "Ns": args.Ns, "k0": args.k0, "n_inv": args.n_inv, "m0": args.m0, "train_seeds": args.train_seeds,
               "steps": len(losses), "loss_first": losses[0], "loss_last": losses[-1], "train_s": t_train,
               "data_s": t_data, "eval": evals}
    for name in ("plain_n_inv", "plain_k0", "learned", "learned_forced"):
        summary[f"mean_{name}"] = {k: float(np.mean([e[name][k] for e in evals.values()]))
                                    for k in ("deficit", "build_s", "gcr_iterations", "little_iterations", "solve_s")}
    print(json.dumps(summary))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
