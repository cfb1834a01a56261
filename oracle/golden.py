"""Readers of the stored inputs and expected values under tests/golden.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A tree file lists, per group of circuit tensors, the circuit wires (qubit,
position) crossing its boundary, then the pairwise steps over group ids; see
oracle.tn.order_from_groups for how the oracle follows it.
"""
from __future__ import annotations


def read_tree(path):
    """(group_wires, pairs) from a tree file."""
    groups, pairs = {}, []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "group":
                v = [int(x) for x in line[2:]]
                groups[int(line[1])] = [(v[2 * j], v[2 * j + 1]) for j in range(len(v) // 2)]
            elif line[0] == "pair":
                pairs.append((int(line[1]), int(line[2])))
            else:
                raise ValueError(f"unknown record {line[0]!r} in {path}")
    return [groups[i] for i in range(len(groups))], pairs


def read_amplitudes(path):
    """(indices, complex128 amplitudes) from a golden amplitude file ("index re im" rows)."""
    idx, amp = [], []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                idx.append(int(line[0]))
                amp.append(float(line[1]) + 1j * float(line[2]))
    import numpy as np
    return np.array(idx, dtype=np.int64), np.array(amp, dtype=np.complex128)
