#!/usr/bin/env python3
"""Write grid5x5_amplitudes.txt: FP64 amplitudes <x|U|0...0> (Eq. ampl_calc) of
64 bitstrings of the 5x5-grid, 14-cycle random circuit (seed 55; bitstrings:
random_bitstrings(25, 64, 5505)), by brute-force statevector simulation
(oracle.statevector, O1) alone.  A 2^25-entry statevector is 512 MiB; the
script takes a few minutes.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import statevector as sv  # noqa: E402
from workloads import grid_circuit, random_bitstrings  # noqa: E402


def main(path=os.path.join(HERE, "grid5x5_amplitudes.txt")):
    circ = grid_circuit(5, 5, 14, 55)
    bits = random_bitstrings(circ.n, 64, 5505)
    psi = sv.final_state(circ)
    amp = np.array([psi[tuple(b)] for b in bits.astype(np.int64)])
    norm = float(np.vdot(psi, psi).real)
    with open(path, "w") as f:
        f.write("# FP64 amplitudes <x|U|0...0> (Eq. ampl_calc) of the 5x5 grid random circuit, 14 cycles,\n")
        f.write("# seed 55; bitstring i = row i of random_bitstrings(25, 64, 5505).  Oracle O1\n")
        f.write(f"# (statevector); written by make_grid5x5_amplitudes.py; state norm - 1 = {norm - 1:.1e}.\n")
        f.write("# index re im\n")
        for i, a in enumerate(amp):
            f.write(f"{i} {a.real:.17e} {a.imag:.17e}\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
