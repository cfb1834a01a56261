#!/usr/bin/env python3
"""Write config3_amplitudes.txt: FP64 amplitudes <x|U|0...0> (Eq. ampl_calc) of
the first bitstrings of the 6x6-grid, 14-cycle random circuit (seed 2104;
bitstrings: 1024 uniform, seed 10523), computed by the oracle alone.

For each bitstring the oracle builds its own projected network
(oracle.tn.build_network_wires, Sec. 3.1 and 3.1.1), follows the contraction
tree of config3_order.txt (oracle.tn.order_from_groups), slices its own indices
until no tensor exceeds 2^24 elements (oracle.tn.choose_slices, Sec. 3.1) and
sums every slice's contraction in FP64 (oracle.tn.contract_sliced).
Bitstring 0 is also contracted with a different slicing (cap 2^21) as a
self-check; the relative difference is recorded in the header.

Usage: make_config3_amplitudes.py [n_bitstrings]   (default 16; about 3 min
each on 8 cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import golden, tn  # noqa: E402
from workloads import grid_circuit, random_bitstrings  # noqa: E402

CAP_LOG2 = 24


def amplitude(circ, bits, group_wires, pairs, cap_log2=CAP_LOG2):
    net, wires = tn.build_network_wires(circ, bits)
    order = tn.order_from_groups(net, wires, group_wires, pairs)
    sl = tn.choose_slices(net, order, cap_log2)
    val = tn.contract_sliced(net, sl, order) if sl else tn.contract(net, order)[0]
    return complex(np.asarray(val).reshape(())), len(sl)


def main(n=16, path=os.path.join(HERE, "config3_amplitudes.txt")):
    circ = grid_circuit(6, 6, 14, 2104)
    bits = random_bitstrings(circ.n, 1024, 10523)
    gw, pairs = golden.read_tree(os.path.join(HERE, "config3_order.txt"))
    rows = []
    t0 = time.time()
    for i in range(n):
        a, ns = amplitude(circ, bits[i], gw, pairs)
        rows.append((i, a))
        print(f"bitstring {i}: {a.real:.17e} {a.imag:.17e} ({ns} sliced indices, {time.time() - t0:.0f} s)",
              flush=True)
    check, ns2 = amplitude(circ, bits[0], gw, pairs, cap_log2=21)
    rel = abs(check - rows[0][1]) / abs(rows[0][1])
    with open(path, "w") as f:
        f.write("# FP64 amplitudes <x|U|0...0> (Eq. ampl_calc) of the 6x6 grid random circuit, 14 cycles,\n")
        f.write("# seed 2104; bitstring i = row i of random_bitstrings(36, 1024, 10523).\n")
        f.write(f"# Oracle O2 along config3_order.txt, sliced to <= 2^{CAP_LOG2} elements; written by\n")
        f.write("# make_config3_amplitudes.py.  Self-check: bitstring 0 with a different slicing\n")
        f.write(f"# ({ns2} indices, cap 2^21) differs by {rel:.2e} (relative).\n")
        f.write("# index re im\n")
        for i, a in rows:
            f.write(f"{i} {a.real:.17e} {a.imag:.17e}\n")
    print(f"wrote {path}; self-check {rel:.2e}")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 16)
