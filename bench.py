#!/usr/bin/env python3
"""Benchmark: bitstring amplitudes by full tensor-network contraction on GB300.

Workload (default): 6x6 grid random circuit, 14 cycles (sqrt-X/Y/W layers and
fSim(pi/2, pi/6) on the ABCDCDAB edge patterns), seed 2104; 1024 uniformly
random bitstrings (seed 10523); contraction path sliced so that no
intermediate exceeds 2^28 complex64 elements.  One step = one batch of
2^batch_log2 bitstrings through every slice of the plan (all pairwise
contractions, the FP64 cross-slice sum, the mapping to bitstring order).

Prints one JSON line (rank 0).  Under torchrun every rank contracts its own
bitstrings (weak scaling, no collective on the data path); the elapsed time is
the maximum over ranks.  The line also reports the relative L2 error of the
benched mode and of the plain FP32 arm against FP64 amplitudes stored by the
oracle for this workload (tests/golden/config3_amplitudes.txt).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

T_START = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - T_START:7.1f}s] {msg}", file=sys.stderr, flush=True)


METRIC = "amplitudes/s and contraction TFLOP/s, mixed vs plain FP32 at ≤1e-5 rel err"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32", "tf32x3", "bf16x3"],
                    help="default TF32x3: the tensor-core mode whose amplitudes meet the metric's 1e-5 "
                         "relative error against the FP64 oracle at this workload")
    ap.add_argument("--batch-log2", type=int, default=2)
    ap.add_argument("--candidates", type=int, default=2048)
    ap.add_argument("--cap", type=int, default=28)
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="circuit", choices=["circuit", "pair", "noisy"],
                    help="circuit: 6x6 amplitude workload; pair: one pairwise contraction (microbenchmark); "
                         "noisy: 4x5 noisy trajectory workload")
    ap.add_argument("--mnk", default="12,12,12", help="pair workload: log2 of M, N, K")
    ap.add_argument("--path", default="best", choices=["best", "learned"],
                    help="best: fewest sliced flops over the candidate trees; learned: least time predicted by "
                         "the cost model in --model")
    ap.add_argument("--model", default=os.path.join(ROOT, "paper_2104_10523_gb300", "data", "costmodel_tf32x3.npy"),
                    help="trained cost-model parameters (float32 .npy, hidden 256) for --path learned")
    ap.add_argument("--oracle-sample", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-min-slices", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--dump-amplitudes", default=None,
                    help="write the accuracy pass's amplitudes (every mode) to this JSON file")
    ap.add_argument("--dump-timings", default=None,
                    help="write the per-kernel records of the roofline pass (tnq_ctx_get_timings) to this JSON file")
    return ap.parse_args()


WORKLOAD = dict(rows=6, cols=6, cycles=14, seed=2104, n_bitstrings=1024, bits_seed=10523)


def workload_desc(a):
    return (f"{WORKLOAD['rows']}x{WORKLOAD['cols']} grid random circuit, {WORKLOAD['cycles']} cycles, "
            f"{WORKLOAD['n_bitstrings']} random bitstrings, max intermediate 2^{a.cap} complex64")


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------- CPU baseline (oracle)
ORDER_FILE = os.path.join(ROOT, "tests", "golden", "config3_order.txt")
GOLDEN_FILE = os.path.join(ROOT, "tests", "golden", "config3_amplitudes.txt")
ORACLE_CAP_LOG2 = 24


def oracle_slices(seconds, min_slices=1, bitstring=0):
    """The FP64 oracle (oracle.tn, O2) contracting one amplitude of the
    workload: its own network for bitstring `bitstring`, the stored contraction
    tree, its own slicing to <= 2^24-element tensors; slices are contracted one
    after the other until `seconds` have passed (at least `min_slices`).
    Returns (slices done, slices per amplitude, seconds)."""
    import itertools
    from oracle import golden, tn
    from workloads import grid_circuit, random_bitstrings
    circ = grid_circuit(WORKLOAD["rows"], WORKLOAD["cols"], WORKLOAD["cycles"], WORKLOAD["seed"])
    bits = random_bitstrings(circ.n, WORKLOAD["n_bitstrings"], WORKLOAD["bits_seed"])[bitstring]
    gw, pairs = golden.read_tree(ORDER_FILE)
    net, wires = tn.build_network_wires(circ, bits)
    order = tn.order_from_groups(net, wires, gw, pairs)
    sl = tn.choose_slices(net, order, ORACLE_CAP_LOG2)
    t0 = time.perf_counter()
    done = 0
    for vals in itertools.product((0, 1), repeat=len(sl)):
        tn.contract(tn.fix_labels(net, dict(zip(sl, vals))), order)
        done += 1
        if done >= min_slices and time.perf_counter() - t0 >= seconds:
            break
    return done, 2 ** len(sl), time.perf_counter() - t0


def oracle_sample_subprocess(threads, seconds, min_slices=1):
    """Run oracle_slices in a fresh interpreter whose BLAS uses `threads` threads."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(seconds), "--oracle-min-slices",
           str(min_slices)]
    res = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=3600)
    if res.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {res.stderr[-2000:]}")
    done, per_amp, dt = json.loads(res.stdout.strip().splitlines()[-1])
    return done, per_amp, dt


def cpu_baseline(seconds):
    """The oracle timed on the host cores: all cores, then one thread."""
    cores = os.cpu_count() or 1
    done, per_amp, dt = oracle_sample_subprocess(cores, seconds)
    d1, _, t1 = oracle_sample_subprocess(1, seconds)
    rate = done / per_amp / dt
    rate1 = d1 / per_amp / t1
    desc = (f"oracle O2 (FP64, np.tensordot) contracting amplitude 0 of the workload along the stored tree "
            f"(tests/golden/config3_order.txt), sliced by the oracle into {per_amp} slices of <= "
            f"2^{ORACLE_CAP_LOG2} elements: {done} slices in {dt:.1f} s on {cores} threads, scaled to "
            f"amplitudes/s; one thread: {d1} slices in {t1:.1f} s = {rate1:.3e} amplitudes/s")
    return {"value": rate, "unit": "amplitudes/s", "cores": cores, "kind": "oracle", "sample": desc,
            "single_thread_value": rate1}


def golden_amplitudes():
    """(indices, FP64 amplitudes) stored by the oracle for this workload, or (None, None)."""
    if not os.path.exists(GOLDEN_FILE):
        return None, None
    from oracle import golden
    return golden.read_amplitudes(GOLDEN_FILE)


# ---------------------------------------------------------------- main
def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if a.oracle_sample is not None:
        print(json.dumps(oracle_slices(a.oracle_sample, a.oracle_min_slices)), flush=True)
        return
    if a.impl == "reference":
        return run_reference(a, world, rank)
    if a.workload == "pair":
        return run_pair(a, local, rank)
    if a.workload == "noisy":
        return run_noisy(a, local, rank)

    import numpy as np
    import torch
    from paper_2104_10523_gb300 import build, tnq
    from workloads import grid_circuit, random_bitstrings

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    tnq.load()
    circ = grid_circuit(WORKLOAD["rows"], WORKLOAD["cols"], WORKLOAD["cycles"], WORKLOAD["seed"])
    bits_all = random_bitstrings(circ.n, WORKLOAD["n_bitstrings"], WORKLOAD["bits_seed"])
    B = 2 ** a.batch_log2
    t_plan = time.perf_counter()
    path_info = {"path": a.path}
    if a.path == "learned":
        import numpy as np
        mctx = tnq.Context(local, a.precision)
        model = tnq.CostModel(mctx, hidden=256, max_batch=4096, seed=1)
        model.set_params(np.load(a.model))
        plan = model.plan(tnq.Circuit(circ), max_intermediate_log2=a.cap, batch_log2=a.batch_log2,
                          path_mode=tnq.TNQ_PATH_BEST, n_candidates=a.candidates, seed=7)
        cand = plan.candidates()
        path_info.update({"chosen": int(cand["chosen"]), "flop_minimal": int(cand["flopmin"]),
                          "flops_ratio_vs_flop_minimal": float(cand["flops"][cand["chosen"]] /
                                                               cand["flops"][cand["flopmin"]])})
    else:
        plan = tnq.Plan(tnq.Circuit(circ), max_intermediate_log2=a.cap, batch_log2=a.batch_log2,
                        path_mode=tnq.TNQ_PATH_BEST, n_candidates=a.candidates, seed=7)
    t_plan = time.perf_counter() - t_plan
    log(f"plan: {plan.info['n_steps']} steps, 2^{plan.info['n_sliced']} slices, "
        f"{plan.info['flops_per_batch']:.3e} flops/step, search {t_plan:.1f} s")
    ctx = tnq.Context(local, a.precision)
    ctx.bind(plan)
    info = plan.info
    stream = ctx.stream
    t_tune = time.perf_counter()
    n_tc, n_cc = tnq.tnq_plan_autotune(ctx.h, plan.h, 3)
    t_tune = time.perf_counter() - t_tune
    log(f"autotune: {n_tc} steps on tensor cores, {n_cc} on CUDA cores, {t_tune:.1f} s")

    def batch(i):
        start = ((rank * (a.steps + a.warmup) + i) * B) % WORKLOAD["n_bitstrings"]
        idx = [(start + j) % WORKLOAD["n_bitstrings"] for j in range(B)]
        return bits_all[idx]

    dev_bits = [torch.from_numpy(batch(i)).to(f"cuda:{local}") for i in range(a.warmup + a.steps)]
    out = torch.empty((B, 2), dtype=torch.float64, device=f"cuda:{local}")

    def step(i):
        tnq.tnq_amplitudes(ctx.h, plan.h, dev_bits[i], out)

    for i in range(a.warmup):
        step(i)
        log(f"warmup step {i} done")
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    n0 = tnq.tnq_ctx_launch_count(ctx.h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(a.warmup, a.warmup + a.steps):
        step(i)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = tnq.tnq_ctx_launch_count(ctx.h) - n0
    clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    if world > 1:
        t = torch.tensor([elapsed], device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed = float(t.item())
        torch.distributed.barrier()
    amps = a.steps * B * world
    value = amps / elapsed
    flops_step = info["flops_per_batch"]
    tflops = flops_step * a.steps * world / elapsed / 1e12

    log(f"timed steps: {elapsed:.3f} s")
    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    host_bits = [torch.from_numpy(batch(i)).pin_memory() for i in range(a.warmup, a.warmup + a.steps)]
    host_out = torch.empty((B, 2), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for hb in host_bits:
        tnq.tnq_amplitudes(ctx.h, plan.h, hb, host_out)
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    e2e = {"value": a.steps * B * world / e2e_t if world == 1 else None, "unit": "amplitudes/s",
           "h2d_bytes_per_step": int(B * circ.n), "d2h_bytes_per_step": int(B * 16)}
    if world > 1:
        t = torch.tensor([e2e_t], device=f"cuda:{local}")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e["value"] = a.steps * B * world / float(t.item())

    log(f"e2e: {e2e_t:.3f} s")
    # ---- roofline of the dominant kernel: per-launch CUDA events over one more step
    tnq.tnq_ctx_set_timing(ctx.h, True)
    step(a.warmup + a.steps - 1)
    torch.cuda.synchronize()
    rec = tnq.tnq_ctx_get_timings(ctx.h)
    tnq.tnq_ctx_set_timing(ctx.h, False)
    roofline, kernel_share = roofline_of(rec, a.precision)
    if a.dump_timings and rank == 0:
        with open(a.dump_timings, "w") as f:
            json.dump({"fields": list(tnq.TIMING_FIELDS), "records": rec.tolist(),
                       "steps": plan.steps().tolist()}, f)

    log("roofline pass done")
    # ---- accuracy against the FP64 oracle on the stored bitstrings (same plan, same
    # kernels), and the plain FP32 arm: speed on the timed batches, accuracy on the stored ones
    gidx, gref = golden_amplitudes()
    if gidx is None:
        gidx = np.arange(4 * B)
    acc_bits = bits_all[gidx]
    dump = {"bitstring_indices": [int(i) for i in gidx]}

    def amps_of(c):
        o = np.empty((acc_bits.shape[0], 2))
        tnq.tnq_amplitudes(c.h, plan.h, np.ascontiguousarray(acc_bits), o)
        return o[:, 0] + 1j * o[:, 1]

    def err_of(amp):
        if gref is None:
            return None
        return float(np.linalg.norm(amp - gref) / np.linalg.norm(gref))

    mode_amp = amps_of(ctx)
    dump[a.precision] = [[z.real, z.imag] for z in mode_amp]
    accuracy = {"rel_l2_vs_fp64": err_of(mode_amp), "bitstrings": int(acc_bits.shape[0]),
                "reference": "FP64 oracle O2 amplitudes (tests/golden/config3_amplitudes.txt)"
                if gref is not None else "unavailable (no stored FP64 amplitudes)",
                "tolerance": 1e-5}
    compare = None
    if not a.skip_fp32:
        ctx32 = tnq.Context(local, "fp32")
        ctx32.bind(plan)
        last = a.warmup + a.steps - 1
        tnq.tnq_amplitudes(ctx32.h, plan.h, dev_bits[last], out)  # warm (captures the FP32 graph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            tnq.tnq_amplitudes(ctx32.h, plan.h, dev_bits[last], out)
        e1.record(stream)
        torch.cuda.synchronize()
        t32 = e0.elapsed_time(e1) / 1e3 / reps
        fp32_amp = amps_of(ctx32)
        dump["fp32"] = [[z.real, z.imag] for z in fp32_amp]
        compare = {"fp32_value": B / t32, "fp32_tflops": flops_step / t32 / 1e12,
                   "speedup_vs_fp32": value / world / (B / t32),
                   "fp32_rel_l2_vs_fp64": err_of(fp32_amp),
                   "rel_l2_vs_fp32": float(np.linalg.norm(mode_amp - fp32_amp) / np.linalg.norm(fp32_amp))}
        del ctx32
    accuracy["meets_tolerance"] = (accuracy["rel_l2_vs_fp64"] is not None and
                                   accuracy["rel_l2_vs_fp64"] <= accuracy["tolerance"])
    if a.dump_amplitudes and rank == 0:
        with open(a.dump_amplitudes, "w") as f:
            json.dump(dump, f)
    log("accuracy pass and fp32 arm done")

    line = {
        "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": elapsed / a.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": a.precision, "data": "synthetic",
        "config": {"workload": workload_desc(a), "bitstrings_per_step": B, "slices": 2 ** info["n_sliced"],
                   "max_intermediate_log2": info["max_log2"], "flops_per_step": flops_step,
                   "path_search_s": round(t_plan, 2), "autotune_s": round(t_tune, 2),
                   "autotuned_steps": {"tensor_core": n_tc, "cuda_core": n_cc}, "path": path_info,
                   "l2": "working set larger than L2 (intermediates up to "
                   f"2^{info['max_log2']} x 8 B)", "parallelism": f"dp{world} (independent bitstrings)"},
        "contraction_tflops": tflops,
        "accuracy": accuracy,
        "roofline": roofline,
        "kernel_share": kernel_share,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
        "compare": compare,
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(a.cpu_seconds)
        log("cpu baseline done")
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def roofline_of(rec, precision):
    """Dominant kernel by total time; its achieved rate against the measured peak."""
    import numpy as np
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        src = "measured"
    except OSError:
        peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
        src = "fallback"
    if len(rec) == 0:
        return None, None
    kinds = {0: "permute", 1: "cgemm_simt", 2: "cgemm_tc", 3: "other", 4: "cgemm_skinny", 5: "cgemm_tc_rows"}
    tot = {}
    for r in rec:
        k = int(r[0])
        t = tot.setdefault(k, [0.0, 0.0, 0.0, 0])
        t[0] += r[8]
        t[1] += r[6]
        t[2] += r[7]
        t[3] += 1
    all_ms = sum(v[0] for v in tot.values())
    share = {kinds[k]: round(v[0] / all_ms, 4) for k, v in tot.items()}
    k = max(tot, key=lambda x: tot[x][0])
    ms, flops, nbytes, n = tot[k]
    bf16_sus = float(peaks.get("bf16_tflops_sustained", 1720.9))
    traffic = load_traffic(kinds[k], nbytes / n)
    if k == 2:
        # tensor-pipe peak of the mode: TF32 runs at half the BF16 rate (nominal 1.1 vs 2.25 PF/s);
        # the split modes issue three products per useful product.
        per_mode = {"tf32": bf16_sus * 1.1 / 2.25, "tf32x3": bf16_sus * 1.1 / 2.25 / 3,
                    "bf16x3": bf16_sus / 3}
        peak = per_mode.get(precision, bf16_sus)
        ach = flops / (ms / 1e3) / 1e12
        return ({"kernel": "cgemm_tc", "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                 "frac": ach / peak, "traffic": traffic, "launches": n, "avg_launch_ms": ms / n,
                 "peak_source": f"{src} bf16 sustained, mode-adjusted"}, share)
    if k == 1:
        # FP32 FFMA roof: 152 SMs x 128 lanes x 2 flops x max SM clock
        peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        ach = flops / (ms / 1e3) / 1e12
        return ({"kernel": "cgemm_simt", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                 "frac": ach / peak, "traffic": traffic, "launches": n, "avg_launch_ms": ms / n,
                 "peak_source": "FFMA lanes x max clock"}, share)
    ach = nbytes / (ms / 1e3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    return ({"kernel": kinds[k], "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
             "traffic": traffic, "launches": n, "avg_launch_ms": ms / n, "peak_source": f"{src} copy"}, share)


def load_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None).  The summary holds the measured DRAM
    bytes over the algorithmic bytes of a captured small case; traffic scales in
    proportion to the units a launch processes, so that ratio times this
    workload's algorithmic bytes per launch is the traffic per launch here."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except OSError:
        return None
    ent = d.get(kernel)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2104_10523_gb300", "csrc", ent["source"])
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    if h != ent.get("source_sha256_16"):
        return None
    return ent["dram_over_algorithmic"] * alg_bytes_per_launch


def run_pair(a, local, rank):
    """Pairwise-contraction microbenchmark: all-dimension-2 complex64 operands of
    rank m+k and n+k with the shared indices scattered by a seeded permutation
    (entries complex normal / sqrt(2^k)); one step = one tnq_contract_pair call
    (operand permutes + complex GEMM + output permute).  Error against the FP64
    oracle on 16 sampled output rows."""
    import numpy as np
    import torch
    from oracle import contraction
    from paper_2104_10523_gb300 import build, tnq
    from workloads import microbench_case
    m, n, k = (int(x) for x in a.mnk.split(","))
    torch.cuda.set_device(local)
    build.build()
    tnq.load()
    al, bl, ol, A, B = microbench_case(m, n, k, seed=1)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty(2 ** (m + n), dtype=torch.complex64, device="cuda")
    ctx = tnq.Context(local, a.precision)
    nb = tnq.tnq_contract_workspace_bytes(tnq.PRECISIONS[a.precision], len(al), len(bl), len(ol))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")

    def step():
        tnq.tnq_contract_pair(ctx.h, At, al, Bt, bl, C, ol, ws, nb)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(a.steps):
        step()
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / a.steps
    tnq.tnq_ctx_set_timing(ctx.h, True)
    step()
    rec = tnq.tnq_ctx_get_timings(ctx.h)
    roofline, share = roofline_of(rec, a.precision)
    rows = np.random.default_rng(1).choice(2 ** m, size=min(16, 2 ** m), replace=False)
    ref = contraction.sampled_rows(A, al, B, bl, ol, rows, ol[:m])
    got = C.cpu().numpy().reshape(2 ** n, 2 ** m).T[rows]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    flops = 8.0 * 2.0 ** (m + n + k)
    line = {"metric": "contraction TFLOP/s", "value": flops / dt / 1e12, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": a.precision, "data": "synthetic",
            "config": {"workload": f"pairwise contraction M=2^{m} N=2^{n} K=2^{k}, complex64 all-dim-2 tensors"},
            "rel_l2_vs_fp64": err, "roofline": roofline, "kernel_share": share}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_noisy(a, local, rank):
    """Noisy workload: 4x5 grid random circuit, 10 cycles, depolarizing p = 1e-3
    on every qubit after every gate and amplitude damping gamma = 1e-3 per cycle
    (Kraus channels, Eq. kraus_sum); one step = the trajectory estimate of 256
    bitstring probabilities from 4096 trajectories (FP64 averaging), i.e.
    4096 x 256 trajectory amplitudes.  Checked against the exact probabilities
    of the doubled density-matrix network (Sec. 3.3) on the same GPU."""
    import numpy as np
    import torch
    from paper_2104_10523_gb300 import build, tnq
    from workloads import CONFIG_NOISY as cfg, noisy_grid_circuit, random_bitstrings
    torch.cuda.set_device(local)
    build.build()
    tnq.load()
    circ = noisy_grid_circuit(cfg["rows"], cfg["cols"], cfg["cycles"], cfg["seed"], cfg["p_depol"], cfg["gamma"])
    bits = random_bitstrings(circ.n, cfg["n_bitstrings"], cfg["bits_seed"])
    n_traj, nb = cfg["n_trajectories"], len(bits)
    plan = tnq.Plan(tnq.Circuit(circ), batch_log2=4, traj_log2=8, max_intermediate_log2=a.cap,
                    path_mode=tnq.TNQ_PATH_BEST, n_candidates=256, seed=1)
    ctx = tnq.Context(local, a.precision)
    ctx.bind(plan)
    tnq.tnq_plan_autotune(ctx.h, plan.h, 2)
    dbits = torch.from_numpy(bits).cuda()
    p_dev = torch.empty(nb, dtype=torch.float64, device="cuda")
    se_dev = torch.empty(nb, dtype=torch.float64, device="cuda")

    def step(seed):
        tnq.tnq_noisy_probabilities(ctx.h, plan.h, n_traj, seed, dbits, p_dev, se_dev)

    for i in range(a.warmup):
        step(cfg["traj_seed"])
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    n0 = tnq.tnq_ctx_launch_count(ctx.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for i in range(a.steps):
        step(cfg["traj_seed"])
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    clocks.stop()
    launches = tnq.tnq_ctx_launch_count(ctx.h) - n0
    dt = e0.elapsed_time(e1) / 1e3 / a.steps
    distinct = tnq.tnq_plan_get_info(plan.h)["distinct_trajectories"]
    p_est, se = p_dev.cpu().numpy(), se_dev.cpu().numpy()
    # end to end with host buffers
    hb = torch.from_numpy(bits).pin_memory()
    hp = torch.empty(nb, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(a.steps):
        tnq.tnq_noisy_probabilities(ctx.h, plan.h, n_traj, cfg["traj_seed"], hb, hp, None)
    torch.cuda.synchronize()
    e2e_dt = (time.perf_counter() - t0) / a.steps
    # exact probabilities from the doubled network, same bitstrings
    dplan = tnq.Plan(tnq.Circuit(circ), density=True, batch_log2=0, max_intermediate_log2=27, n_candidates=256,
                     seed=3)
    dctx = tnq.Context(local, "fp32")
    dctx.bind(dplan)
    t_ex = time.perf_counter()
    p_exact = dctx.density_probabilities(dplan, bits)
    t_ex = time.perf_counter() - t_ex
    z = np.abs(p_est - p_exact) / np.maximum(se, 1e-300)
    unit = "trajectory amplitudes/s"
    line = {"metric": "noisy bitstring probabilities by stochastic trajectories", "value": n_traj * nb / dt,
            "unit": unit, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": a.precision,
            "data": "synthetic",
            "config": {"workload": "4x5 grid random circuit, 10 cycles, depolarizing p=1e-3 after every gate, "
                       "amplitude damping gamma=1e-3 per cycle; 4096 trajectories x 256 bitstrings per step",
                       "bitstrings_per_pass": 16, "trajectories_per_pass": 256,
                       "distinct_trajectories": int(distinct), "slices": 2 ** plan.info["n_sliced"]},
            "accuracy": {"exact": "doubled density-matrix network (tnq_density_probabilities, FP32)",
                         "max_abs_z": float(z.max()), "mean_abs_z": float(z.mean()),
                         "within_4_se": bool(np.all(np.abs(p_est - p_exact) <= 4 * se + 1e-6 * p_exact)),
                         "exact_ms_per_bitstring": t_ex / nb * 1e3},
            "e2e": {"value": n_traj * nb / e2e_dt, "unit": unit, "h2d_bytes_per_step": int(bits.size),
                    "d2h_bytes_per_step": int(8 * nb)},
            "gpu_launches": int(launches), "clocks": clocks.summary()}
    if rank == 0:
        # the oracle on the host cores: statevector trajectories (O1) for a bounded sample
        from oracle import noise as onoise, statevector as osv
        tc = time.perf_counter()
        k = 0
        while k < 2 or time.perf_counter() - tc < a.cpu_seconds:
            onoise.noisy_probabilities(circ, bits, 1, cfg["traj_seed"] + k, osv.amplitudes)
            k += 1
        tc = time.perf_counter() - tc
        line["cpu_baseline"] = {"value": k * nb / tc, "unit": unit, "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": f"oracle O1 (FP64 statevector per trajectory, all 256 bitstrings) for "
                                          f"{k} trajectories in {tc:.1f} s"}
        print(json.dumps(line), flush=True)


def run_reference(a, world, rank):
    """The oracle on the host cores, same workload, metric and unit.  One step
    is one slice of one amplitude contracted by the FP64 oracle (O2) along the
    stored tree, sliced by the oracle itself; amplitudes/s = slices done /
    slices per amplitude / seconds."""
    if rank != 0:
        return
    for _ in range(a.warmup):
        oracle_slices(0.0, 1)
    times, per_amp = [], 1
    for i in range(a.steps):
        done, per_amp, dt = oracle_slices(0.0, 1)
        times.append(dt / done)
    t_slice = statistics.mean(times)
    value = 1.0 / per_amp / t_slice
    cores = os.cpu_count() or 1
    desc = (f"oracle O2 (FP64, np.tensordot, BLAS threads = {os.environ.get('OPENBLAS_NUM_THREADS', 'default')}) "
            f"contracting amplitude 0 of the workload along tests/golden/config3_order.txt, one of its {per_amp} "
            f"slices (<= 2^{ORACLE_CAP_LOG2} elements) per step, {t_slice:.2f} s per slice")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_slice * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(a), "step": f"one of the {per_amp} slices of one amplitude"},
            "cpu_baseline": {"value": value, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
