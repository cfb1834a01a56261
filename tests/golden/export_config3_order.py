#!/usr/bin/env python3
"""Write config3_order.txt: a contraction tree for the 6x6-grid, 14-cycle random
circuit (seed 2104), given over groups of circuit tensors.

The tree comes from the library's host-side path finder (tnq_plan_create with
one bitstring per pass, intermediates capped at 2^28 elements, the best of 2048
candidate trees by FLOPs, seed 7).  It is an input of the FP64 oracle, which
follows it with its own network, grouping check, slicing and contraction
(oracle.tn.order_from_groups, choose_slices, contract_sliced).  A contraction
order cannot change the exact value of a contraction (Sec. 3.1; pinned by the
oracle's order-independence tests), so the tree decides only the oracle's cost.

File format (one record per line, '#' starts a comment):
  group <i> <qubit> <position> [<qubit> <position> ...]   boundary wires of group i
  pair <a> <b>                                            one tree step
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2104_10523_gb300 import build, tnq  # noqa: E402
from workloads import grid_circuit  # noqa: E402

CONFIG = dict(rows=6, cols=6, cycles=14, seed=2104)


def main(path=os.path.join(HERE, "config3_order.txt")):
    build.build()
    tnq.load()
    circ = grid_circuit(CONFIG["rows"], CONFIG["cols"], CONFIG["cycles"], CONFIG["seed"])
    plan = tnq.Plan(tnq.Circuit(circ), max_intermediate_log2=28, batch_log2=0, path_mode=tnq.TNQ_PATH_BEST,
                    n_candidates=2048, seed=7)
    info = plan.info
    with open(path, "w") as f:
        f.write("# Contraction tree of the 6x6 grid random circuit, 14 cycles, seed 2104 (one bitstring per pass).\n")
        f.write(f"# Written by export_config3_order.py: {info['n_leaves']} groups, {info['n_steps']} steps, "
                f"{info['flops_per_pass']:.4e} flops per slice, {info['n_sliced']} indices sliced by the library.\n")
        for i, ws in enumerate(plan.leaf_wires()):
            f.write(f"group {i} " + " ".join(f"{q} {p}" for q, p in ws) + "\n")
        for a, b in plan.tree():
            f.write(f"pair {a} {b}\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
