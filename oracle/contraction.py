"""One pairwise contraction of two all-dimension-2 complex tensors, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

This is the unit step of the sliced contraction sequence of Sec. 3.1: the two
operands are summed over every label they share (the contracted indices) and
the result carries the remaining labels in a caller-given order.

Layout convention (shared with the microbenchmark inputs): a tensor of rank r
is a flat array of 2^r entries and labels[p] names bit p of the flat index
(bit 0 has stride 1).
"""
from __future__ import annotations

import numpy as np


def _as_axes(flat: np.ndarray, labels):
    r = len(labels)
    # C-order reshape puts the most significant bit (bit r-1) on axis 0.
    return flat.reshape((2,) * r) if r else flat.reshape(()), list(reversed(labels))


def contract_labeled(A: np.ndarray, a_labels, B: np.ndarray, b_labels, out_labels) -> np.ndarray:
    """C[out] = sum over every label not in out_labels of A * B, as a flat
    complex128 array with out_labels[p] on bit p.  A label held by A, B and
    the output is a batch index (not summed)."""
    At, ax_a = _as_axes(np.asarray(A, np.complex128), a_labels)
    Bt, ax_b = _as_axes(np.asarray(B, np.complex128), b_labels)
    ids = {l: i for i, l in enumerate(sorted(set(ax_a) | set(ax_b)))}
    want = list(reversed(out_labels))
    C = np.einsum(At, [ids[l] for l in ax_a], Bt, [ids[l] for l in ax_b], [ids[l] for l in want])
    return np.ascontiguousarray(C).reshape(-1)


def sampled_rows(A, a_labels, B, b_labels, out_labels, rows, row_labels):
    """Exact FP64 values of a subset of output entries.

    row_labels: the output labels that select a "row"; rows: integer row ids
    (bit j of a row id = value of row_labels[j]).  Returns an array
    [len(rows)][2^(rank_out - len(row_labels))], columns ordered by the
    remaining out labels (in out_labels order, first = bit 0).
    """
    col_labels = [l for l in out_labels if l not in row_labels]
    res = []
    for r in rows:
        fix = {l: (int(r) >> j) & 1 for j, l in enumerate(row_labels)}
        Af, al = _fix(A, a_labels, fix)
        Bf, bl = _fix(B, b_labels, fix)
        res.append(contract_labeled(Af, al, Bf, bl, col_labels))
    return np.array(res)


def _fix(flat, labels, fix):
    T, axes = _as_axes(np.asarray(flat, np.complex128), labels)
    idx = tuple(fix[l] if l in fix else slice(None) for l in axes)
    keep = [l for l in labels if l not in fix]
    return np.ascontiguousarray(T[idx]).reshape(-1), keep
