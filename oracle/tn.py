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
    return build_network_wires(circ, bitstring, kraus_picks)[0]


def build_network_wires(circ, bitstring=None, kraus_picks=None):
    """(tensors, wires): the network of build_network and the label of every
    circuit wire, wires[(q, k)] = label of qubit q's wire after the k-th op
    acting on q (k = 0: the |0> input)."""
    n = circ.n
    counter = itertools.count()
    wire = []
    pos = [0] * n
    wires = {}
    tensors: List[Tensor] = []
    for q in range(n):
        lab = next(counter)
        wire.append(lab)
        wires[(q, 0)] = lab
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
            pos[q] += 1
            wires[(q, pos[q])] = lab
    if bitstring is not None:
        for q in range(n):
            if int(bitstring[q]) == -1:   # open qubit (Sec. 4.4): no projection
                continue
            e = np.zeros(2, dtype=np.complex128)
            e[int(bitstring[q])] = 1.0
            tensors.append((e, [wire[q]]))
    build_network.last_open = list(wire)
    return tensors, wires


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


def wavefunction_slice(circ, bitstring, order: str = "greedy", seed: int = 0) -> np.ndarray:
    """Sec. 4.4: the network with the qubits marked -1 left open, contracted
    to a tensor over their final wires; returned as a 2^k vector with the open
    qubit of lowest index as the most significant bit."""
    net = build_network(circ, bitstring)
    open_labels = [build_network.last_open[q] for q in range(circ.n) if int(bitstring[q]) == -1]
    o = greedy_order(net) if order == "greedy" else random_order(net, seed)
    T, labs = contract(net, o)
    T = np.asarray(T).reshape((2,) * len(labs)) if labs else np.asarray(T)
    return np.ascontiguousarray(np.transpose(T, [labs.index(l) for l in open_labels])).reshape(-1)


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


def order_from_groups(tensors: Sequence[Tensor], wires: dict, group_wires, pairs) -> List[Tuple[int, int]]:
    """A pairwise order over this module's own network that follows a
    contraction tree given over groups of circuit tensors (the grouping of
    small gate tensors into larger ones of Sec. 3.1.1, then the pairwise
    sequence of Sec. 3.1).

    group_wires[i]: the circuit wires (qubit, position) that cross the boundary
    of group i ((-1, -1) entries, batch indices, are ignored); pairs: the
    tree's steps over group ids (groups 0..G-1, then the result of step j as
    G + j).  The network is cut at every listed wire; each connected piece must
    have exactly the listed boundary of one group.  Each piece is contracted
    internally first (greedy_order), then the tree is followed.  The order does
    not change the exact value of the contraction, only its cost.
    """
    cut = {wires[tuple(w)] for g in group_wires for w in g if w[0] >= 0}
    parent = list(range(len(tensors)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    holders = {}
    for i, (_, labs) in enumerate(tensors):
        for l in labs:
            holders.setdefault(l, []).append(i)
    for l, ids in holders.items():
        if l not in cut:
            for j in ids[1:]:
                parent[find(j)] = find(ids[0])
    pieces = {}
    for i in range(len(tensors)):
        pieces.setdefault(find(i), []).append(i)
    by_boundary = {}
    for members in pieces.values():
        bnd = frozenset(l for i in members for l in tensors[i][1] if l in cut)
        by_boundary.setdefault(bnd, []).append(members)
    order: List[Tuple[int, int]] = []
    nxt = len(tensors)
    group_id = []
    for g in group_wires:
        key = frozenset(wires[tuple(w)] for w in g if w[0] >= 0)
        if not by_boundary.get(key):
            raise ValueError(f"no piece of the network has the boundary of group {len(group_id)}")
        members = by_boundary[key].pop()
        if len(members) == 1:
            group_id.append(members[0])
            continue
        sub = [tensors[i] for i in members]
        ids = list(members)
        for a, b in greedy_order(sub):
            order.append((ids[a], ids[b]))
            ids.append(nxt)
            nxt += 1
        group_id.append(ids[-1])
    if any(v for v in by_boundary.values()):
        raise ValueError("network pieces left over that no group covers")
    ids = list(group_id)
    for a, b in pairs:
        order.append((ids[int(a)], ids[int(b)]))
        ids.append(nxt)
        nxt += 1
    return order


def choose_slices(tensors: Sequence[Tensor], order, cap_log2: int) -> List[int]:
    """Slicing (Sec. 3.1): pick indices to fix until no tensor met along
    `order` has more than 2^cap_log2 elements.  Each round slices the label
    held by the most tensors of the current largest rank (ties: lowest label)."""
    sliced: List[int] = []
    while True:
        labs = {i: set(t[1]) - set(sliced) for i, t in enumerate(tensors)}
        seen = list(labs.values())
        nxt = len(tensors)
        for i, j in order:
            li, lj = labs.pop(i), labs.pop(j)
            labs[nxt] = li ^ lj
            seen.append(labs[nxt])
            nxt += 1
        top = max(len(x) for x in seen)
        if top <= cap_log2:
            return sliced
        count = {}
        for x in seen:
            if len(x) == top:
                for l in x:
                    count[l] = count.get(l, 0) + 1
        sliced.append(min(count, key=lambda l: (-count[l], l)))


def build_density_network_wires(circ, bitstring):
    """(tensors, wires): the doubled network of Sec. 3.3 whose value is
    p(x) = <x|rho|x>.  Every qubit has a ket wire and a bra wire, both starting
    in |0>; a gate U is the tensor U on the ket wires and its complex conjugate
    on the bra wires; a one-qubit channel {A_k} (Eq. kraus_sum) is one rank-4
    tensor joining the qubit's ket and bra wires, S[i, i', j, j'] =
    sum_k A_k[i, j] conj(A_k[i', j']) (outputs i, i'; inputs j, j'); both wires
    of qubit q end in <x_q|.  wires[(q, k)] / wires[(q + n, k)] name the ket /
    bra wire of qubit q after the k-th op acting on it."""
    n = circ.n
    counter = itertools.count()
    ket, bra, pos = [], [], [0] * n
    wires = {}
    tensors: List[Tensor] = []
    for side, lst in ((0, ket), (n, bra)):
        for q in range(n):
            lab = next(counter)
            lst.append(lab)
            wires[(q + side, 0)] = lab
            tensors.append((np.array([1.0, 0.0], dtype=np.complex128), [lab]))
    for op in circ.ops:
        k = len(op.qubits)
        if op.kind == "gate":
            U = np.asarray(op.mats[0], np.complex128)
            for lst, M in ((ket, U), (bra, U.conj())):
                outs = [next(counter) for _ in op.qubits]
                tensors.append((M.reshape((2,) * (2 * k)), outs + [lst[q] for q in op.qubits]))
                for q, lab in zip(op.qubits, outs):
                    lst[q] = lab
        else:
            if k != 1:
                raise ValueError("the doubled network takes one-qubit channels only")
            q = op.qubits[0]
            S = sum(np.einsum("ij,kl->ikjl", A, np.conj(A)) for A in op.mats)
            o_ket, o_bra = next(counter), next(counter)
            tensors.append((S, [o_ket, o_bra, ket[q], bra[q]]))
            ket[q], bra[q] = o_ket, o_bra
        for q in op.qubits:
            pos[q] += 1
            wires[(q, pos[q])] = ket[q]
            wires[(q + n, pos[q])] = bra[q]
    for lst in (ket, bra):
        for q in range(n):
            e = np.zeros(2, dtype=np.complex128)
            e[int(bitstring[q])] = 1.0
            tensors.append((e, [lst[q]]))
    return tensors, wires


def density_probability(circ, bitstring, order=None) -> float:
    """<x|rho|x> by contracting the doubled network (real part; the imaginary
    part is rounding)."""
    net, _ = build_density_network_wires(circ, bitstring)
    val = contract(net, order)[0]
    return float(np.real(np.asarray(val).reshape(())))


_PAULI = {"I": np.eye(2, dtype=np.complex128),
          "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
          "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128)}


def build_expectation_network(circ, pauli_string) -> List[Tensor]:
    """The double-depth network of Fig. 3 for <psi|P|psi>: the circuit's
    network U|0...0> with its final legs open, one Pauli tensor per qubit on
    them, then the conjugate network (every tensor of U|0...0> complex
    conjugated, its output legs joined to the Pauli tensors)."""
    ket = build_network(circ)
    ket_open = list(build_network.last_open)
    shift = 1 + max(l for _, ls in ket for l in ls)
    bra = [(np.conj(T), [l + shift for l in ls]) for T, ls in ket]
    tensors = list(ket) + bra
    for q, ch in enumerate(pauli_string):
        # P[out, in]: in = the ket's final leg, out = the bra's final leg
        tensors.append((_PAULI[ch], [ket_open[q] + shift, ket_open[q]]))
    return tensors


def expectation(circ, paulis, coeffs, order: str = "greedy", seed: int = 0):
    """(value, per-term values) of <psi|H|psi> through the double-depth network."""
    vals = []
    for ps in paulis:
        net = build_expectation_network(circ, ps)
        o = greedy_order(net) if order == "greedy" else random_order(net, seed)
        vals.append(complex(np.asarray(contract(net, o)[0]).reshape(())))
    vals = np.array(vals)
    return complex(np.dot(coeffs, vals)), vals
