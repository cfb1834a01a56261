"""Training and evaluation driver of the learned path cost model.

The compute (MLP forward, backward, Adam, inference, plan execution) runs in
libtnq's kernels; this module only sequences calls through the C ABI:

  collect(): execute plans with per-kernel timing on, turn every step into a
             (features, ln microseconds) row;
  train():   fit the MLP on those rows on the GPU;
  evaluate(): for held-out circuits, build the flop-minimal plan and the
             learned plan over the same candidate set, time both, and report
             the regret t(learned) / t(flop-minimal) - 1 (negative = gain).

Run as a script it prints one JSON summary, e.g.
  python -m paper_2104_10523_gb300.costmodel --train 64 --eval 24
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import tnq


def circuit_flops(circ, n_candidates=8, seed=0, path_mode=tnq.TNQ_PATH_BEST):
    p = tnq.Plan(tnq.Circuit(circ), batch_log2=0, path_mode=path_mode, n_candidates=n_candidates, seed=seed)
    return p.info["flops_per_batch"]


def pick_circuits(seeds, max_flops, make, quick=False):
    """Circuits of the workload whose flop-minimal plan stays within max_flops
    (the rest are too expensive to time repeatedly).  quick: judge by one
    bisection candidate instead of eight (an upper bound, much faster)."""
    out = []
    for s in seeds:
        c = make(s)
        f = circuit_flops(c, 1, path_mode=tnq.TNQ_PATH_BISECT) if quick else circuit_flops(c)
        if f <= max_flops:
            out.append((s, c))
    return out


def time_batch(ctx, plan, bits, reps=3):
    """Best-of-reps device time (ms) of one amplitude batch (graph replay)."""
    import torch
    d = torch.from_numpy(np.ascontiguousarray(bits, dtype=np.int8)).cuda()
    out = torch.empty((bits.shape[0], 2), dtype=torch.float64, device="cuda")
    tnq.tnq_amplitudes(ctx.h, plan.h, d, out)  # warm (and capture)
    best = math.inf
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        tnq.tnq_amplitudes(ctx.h, plan.h, d, out)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def step_rows(ctx, plan, bits, precision):
    """(features, ln microseconds) of every step of one executed batch."""
    tnq.tnq_amplitudes(ctx.h, plan.h, bits, np.zeros((bits.shape[0], 2)))  # warm
    tnq.tnq_ctx_set_timing(ctx.h, True)
    tnq.tnq_amplitudes(ctx.h, plan.h, bits, np.zeros((bits.shape[0], 2)))
    rec = tnq.tnq_ctx_get_timings(ctx.h)
    tnq.tnq_ctx_set_timing(ctx.h, False)
    n_steps = plan.info["n_steps"]
    n_slices = 2 ** plan.info["n_sliced"]
    ms = np.zeros(n_steps)
    for r in rec:
        if r[1] >= 0:
            ms[int(r[1])] += r[8]
    # time of one run of a step: folded steps ran when the plan was bound (no
    # row), slice-invariant and slice-batched steps once, the others per slice
    st = plan.steps()
    runs = np.where(st[:, 7] & (4 | 16), 1, n_slices)
    keep = (st[:, 7] & 8) == 0
    us = np.maximum(ms / runs * 1e3, 1e-3)
    return plan.features(precision)[keep], np.log(us[keep]).astype(np.float32)


def collect(ctx, circuits, per_circuit, precision, seed=0):
    X, t = [], []
    for s, circ in circuits:
        bits = np.zeros((1, circ.n), dtype=np.int8)
        for j in range(per_circuit):
            plan = tnq.Plan(tnq.Circuit(circ), batch_log2=0, path_mode=tnq.TNQ_PATH_BISECT, n_candidates=1,
                            seed=seed * 100003 + s * 97 + j)
            ctx.bind(plan)
            f, y = step_rows(ctx, plan, bits, precision)
            X.append(f)
            t.append(y)
    return np.concatenate(X), np.concatenate(t)


def evaluate(ctx, model, circuits, n_candidates=16, seed=0):
    rows = []
    for s, circ in circuits:
        bits = np.zeros((1, circ.n), dtype=np.int8)
        tc = tnq.Circuit(circ)
        pf = tnq.Plan(tc, batch_log2=0, path_mode=tnq.TNQ_PATH_BEST, n_candidates=n_candidates, seed=seed + s)
        pl = model.plan(tc, batch_log2=0, path_mode=tnq.TNQ_PATH_BEST, n_candidates=n_candidates, seed=seed + s)
        cand = pl.candidates()
        ctx.bind(pf)
        tf = time_batch(ctx, pf, bits)
        ctx.bind(pl)
        tl = time_batch(ctx, pl, bits)
        rows.append({"seed": s, "n": circ.n, "t_flopmin_ms": tf, "t_learned_ms": tl, "regret": tl / tf - 1.0,
                     "same_pick": cand["chosen"] == cand["flopmin"],
                     "flops_flopmin": float(cand["flops"][cand["flopmin"]]),
                     "flops_learned": float(cand["flops"][cand["chosen"]])})
    return rows


def summarize(rows):
    r = np.array([x["regret"] for x in rows])
    return {"n": len(rows), "geomean_ratio": float(np.exp(np.mean(np.log1p(r)))) if len(r) else None,
            "mean_regret": float(r.mean()) if len(r) else None, "wins": int((r < -0.02).sum()),
            "losses": int((r > 0.02).sum()), "same_pick": int(sum(x["same_pick"] for x in rows))}


def run_config5(ctx, precision="tf32x3", max_flops=1e12, epochs=30, save=None):
    """The cost-model workload: training circuits from seeds 0-1999 and held-out
    circuits from seeds 2000-2199 whose flops stay within max_flops, one
    executed plan per training circuit, 32 candidate trees per held-out
    circuit.  Returns the summary (see main)."""
    from workloads import cost_model_circuit
    t0 = time.time()
    train_c = pick_circuits(range(0, 2000), max_flops, cost_model_circuit, quick=True)
    eval_c = pick_circuits(range(2000, 2200), max_flops, cost_model_circuit, quick=True)
    t_pick = time.time() - t0
    X, t = collect(ctx, train_c, 1, precision)
    t_collect = time.time() - t0 - t_pick
    model = tnq.CostModel(ctx, hidden=256, max_batch=4096, seed=1)
    loss = model.train(X, t, epochs=epochs, batch=1024, lr=1e-3)
    if save:
        np.save(save, model.get_params())
    rows = evaluate(ctx, model, eval_c, n_candidates=32)
    return {"train_circuits": len(train_c), "eval_circuits": len(eval_c), "train_rows": int(len(t)),
            "final_loss": loss, "target_variance": float(np.var(t)), "eval": summarize(rows),
            "seconds": {"pick": t_pick, "collect": t_collect, "total": time.time() - t0}, "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=64, help="training circuits (seeds 0..)")
    ap.add_argument("--eval", type=int, default=24, help="held-out circuits (seeds 2000..)")
    ap.add_argument("--per-circuit", type=int, default=6)
    ap.add_argument("--candidates", type=int, default=32)
    ap.add_argument("--max-flops", type=float, default=2e10)
    ap.add_argument("--precision", default="bf16x3")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--config5", action="store_true",
                    help="the cost-model workload: training seeds 0-1999, held-out seeds 2000-2199, 32 candidates "
                         "(circuits above --max-flops are left out)")
    ap.add_argument("--save", default=None, help="write the trained parameters (float32 .npy) here")
    a = ap.parse_args()
    from workloads import cost_model_circuit
    t0 = time.time()
    ctx = tnq.Context(0, a.precision)
    if a.config5:
        print(json.dumps(run_config5(ctx, a.precision, a.max_flops, a.epochs, a.save)))
        return
    else:
        train_c = pick_circuits(range(0, 4 * a.train), a.max_flops, cost_model_circuit)[: a.train]
        eval_c = pick_circuits(range(2000, 2000 + 4 * a.eval), a.max_flops, cost_model_circuit)[: a.eval]
    t_pick = time.time() - t0
    X, t = collect(ctx, train_c, a.per_circuit, a.precision)
    t_collect = time.time() - t0 - t_pick
    model = tnq.CostModel(ctx, hidden=256, max_batch=4096, seed=1)
    loss = model.train(X, t, epochs=a.epochs, batch=1024, lr=1e-3)
    if a.save:
        np.save(a.save, model.get_params())
    rows = evaluate(ctx, model, eval_c, n_candidates=a.candidates)
    out = {"train_circuits": len(train_c), "eval_circuits": len(eval_c), "train_rows": int(len(t)),
           "final_loss": loss, "target_variance": float(np.var(t)), "eval": summarize(rows),
           "seconds": {"pick": t_pick, "collect": t_collect, "total": time.time() - t0}, "rows": rows}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
