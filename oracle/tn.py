"""O2: a plain FP64 tensor-network contractor for circuit amplitudes.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 3.1 of the paper step by step, without blocking or fusion:
  1. build (Sec. 3.1, Fig. 1): qubit = rank-1 tensor |0>, one-qubit gate =
     rank-2 tensor, two-qubit gate = rank-4 tensor; the circuit wiring gives
     the shared labels;
  2. project (Sec. 3.1.1, Fig. 2): close each open qubit leg with the basis
     tensor <x_q|, so the network evaluates to the scalar of Eq. ampl_calc;
  3. contract pairwise along an order (Sec. 3.1: a FLOP-reducing sequence; the
     order does not change the exact result, so any order is valid here);
  4. slicing (Sec. 3.1): fix chosen labels to each of their values, contract
     every resulting sub-network, and sum the scalars.

A tensor is (array, labels) with array.ndim == len(labels) and every dimension
2.  In a closed circuit network every label appears in exactly two tensors, so
a pairwise contraction sums over exactly the labels the pair shares.
"""
from __future__ import annotations

import itertools
from typing import List, Sequence, Tuple

import numpy as np

Tensor = Tuple[np.ndarray, List[int]]


def build_network(circ, bitstring=None, kraus_picks=None) -> List[Tensor]:
    """Tensors of <x| U |0...0>; with bitstring=None the final qubit legs stay
    open (their labels are returned by open_labels())."""
    n = circ.n
    counter = itertools.count()
    wire = []
    tensors: List[Tensor] = []
    for q in range(n):
        lab = next(counter)
        wire.append(lab)
        tensors.append((np.array([1.0, 0.0], dtype=np.complex128), [lab]))
    c = 0
    for op in circ.ops:
        if op.kind == "gate":
            M = op.mats[0]
        else:
            if kraus_picks is None:
                raise ValueError("noisy circuit needs kraus_picks")
            A = op.mats[int(kraus_picks[c])]
            q_k = np.real(np.trace(A.conj().T @ A)) / A.shape[0]
            M = A / np.sqrt(q_k)
            c += 1
        k = len(op.qubits)
        T = np.asarray(M, np.complex128).reshape((2,) * (2 * k))
        outs = [next(counter) for _ in op.qubits]
        tensors.append((T, outs + [wire[q] for q in op.qubits]))
        for q, lab in zip(op.qubits, outs):
            wire[q] = lab
    if bitstring is not None:
        for q in range(n):
            e = np.zeros(2, dtype=np.complex128)
            e[int(bitstring[q])] = 1.0
            tensors.append((e, [wire[q]]))
    build_network.last_open = list(wire)
    return tensors


def contract_pair(a: Tensor, b: Tensor) -> Tensor:
    """Sum over the labels a and b share; result labels: a's rest then b's rest."""
    A, la = a
    B, lb = b
    shared = [l for l in la if l in lb]
    ia = [la.index(l) for l in shared]
    ib = [lb.index(l) for l in shared]
    C = np.tensordot(A, B, axes=(ia, ib))
    lc = [l for l in la if l not in shared] + [l for l in lb if l not in shared]
    return C, lc


def _connected_pairs(tensors):
    where = {}
    for i, (_, labs) in enumerate(tensors):
        for l in labs:
            where.setdefault(l, []).append(i)
    pairs = set()
    for ids in where.values():
        for x in range(len(ids)):
            for y in range(x + 1, len(ids)):
                pairs.add((min(ids[x], ids[y]), max(ids[x], ids[y])))
    return pairs


def greedy_order(tensors: Sequence[Tensor]) -> List[Tuple[int, int]]:
    """A simple order: repeatedly contract the connected pair whose result has the
    fewest elements (ties: lowest ids).  Ids refer to a list where each
    contraction appends its result and retires its two inputs."""
    labs = {i: list(t[1]) for i, t in enumerate(tensors)}
    where = {}
    for i, ls in labs.items():
        for l in ls:
            where.setdefault(l, set()).add(i)
    nxt = len(tensors)
    order = []

    def out_rank(i, j):
        li, lj = labs[i], labs[j]
        return len(set(li) ^ set(lj))

    while len(labs) > 1:
        best = None
        for l, ids in where.items():
            if len(ids) < 2:
                continue
            s = sorted(ids)
            for x in range(len(s)):
                for y in range(x + 1, len(s)):
                    key = (out_rank(s[x], s[y]), s[x], s[y])
                    if best is None or key < best:
                        best = key
        if best is None:  # disconnected pieces: outer product of the two smallest
            s = sorted(labs, key=lambda i: (len(labs[i]), i))
            best = (0, min(s[0], s[1]), max(s[0], s[1]))
        _, i, j = best
        li, lj = labs.pop(i), labs.pop(j)
        lc = [l for l in li if l not in lj] + [l for l in lj if l not in li]
        for l in li + lj:
            where[l].discard(i)
            where[l].discard(j)
        for l in lc:
            where[l].add(nxt)
        for l in [l for l in li if l in lj]:
            if not where[l]:
                del where[l]
        labs[nxt] = lc
        order.append((i, j))
        nxt += 1
    return order


def random_order(tensors: Sequence[Tensor], seed: int) -> List[Tuple[int, int]]:
    """A seeded random order over connected pairs (any order is exact)."""
    rng = np.random.default_rng(seed)
    labs = {i: set(t[1]) for i, t in enumerate(tensors)}
    nxt = len(tensors)
    order = []
    while len(labs) > 1:
        ids = sorted(labs)
        pairs = [(i, j) for x, i in enumerate(ids) for j in ids[x + 1:] if labs[i] & labs[j]]
        if not pairs:
            pairs = [(ids[0], ids[1])]
        i, j = pairs[int(rng.integers(0, len(pairs)))]
        li, lj = labs.pop(i), labs.pop(j)
        labs[nxt] = li ^ lj
        order.append((i, j))
        nxt += 1
    return order


def contract(tensors: Sequence[Tensor], order=None) -> Tensor:
    """Contract the whole network along `order` (default: greedy_order)."""
    if order is None:
        order = greedy_order(tensors)
    pool = {i: t for i, t in enumerate(tensors)}
    nxt = len(tensors)
    for i, j in order:
        pool[nxt] = contract_pair(pool.pop(i), pool.pop(j))
        nxt += 1
    assert len(pool) == 1
    return next(iter(pool.values()))


def fix_labels(tensors: Sequence[Tensor], values: dict) -> List[Tensor]:
    """Slice: fix each label in `values` to its value in every tensor holding it."""
    out = []
    for T, labs in tensors:
        idx = tuple(values[l] if l in values else slice(None) for l in labs)
        out.append((T[idx], [l for l in labs if l not in values]))
    return out


def contract_sliced(tensors: Sequence[Tensor], slice_labels: Sequence[int], order=None):
    """Sec. 3.1 slicing: sum over all 2^s assignments of the sliced labels of the
    contraction of the fixed sub-network (each is a plain contraction)."""
    total = None
    for vals in itertools.product((0, 1), repeat=len(slice_labels)):
        sub = fix_labels(tensors, dict(zip(slice_labels, vals)))
        T, labs = contract(sub, order)
        total = T if total is None else total + T
    return total


def amplitude(circ, bitstring, order: str = "greedy", seed: int = 0,
              slice_labels: Sequence[int] = (), kraus_picks=None) -> complex:
    """<x|U|0...0> by full contraction of the projected network."""
    net = build_network(circ, bitstring, kraus_picks)
    if order == "greedy":
        o = greedy_order(net)
    elif order == "random":
        o = random_order(net, seed)
    else:
        raise ValueError(order)
    if slice_labels:
        val = contract_sliced(net, list(slice_labels), o)
    else:
        val = contract(net, o)[0]
    return complex(np.asarray(val).reshape(()))


def amplitudes(circ, bitstrings, **kw) -> np.ndarray:
    return np.array([amplitude(circ, b, **kw) for b in np.asarray(bitstrings)],
                    dtype=np.complex128)


def order_cost(tensors: Sequence[Tensor], order) -> Tuple[float, int]:
    """(total flops at 8 real flops per complex multiply-add, max log2 size)
    of a pairwise order."""
    labs = {i: set(t[1]) for i, t in enumerate(tensors)}
    nxt = len(tensors)
    flops = 0.0
    mx = max(len(l) for l in labs.values())
    for i, j in order:
        li, lj = labs.pop(i), labs.pop(j)
        flops += 8.0 * 2.0 ** len(li | lj)
        labs[nxt] = li ^ lj
        mx = max(mx, len(labs[nxt]))
        nxt += 1
    return flops, mx
