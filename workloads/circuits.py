"""Grid random circuits, closed-form test circuits, noise channels and bitstrings.

Conventions (shared by every consumer):
  * qubit q of an R x C grid sits at row q // C, column q % C;
  * a k-qubit gate matrix acts on the basis |q_0 ... q_{k-1}> of its listed
    qubits, with the first listed qubit as the most significant bit;
  * bitstring entry bits[q] is the value of qubit q; as a statevector index the
    string reads sum_q bits[q] * 2**(n-1-q) (qubit 0 is the most significant bit),
    matching a length-n bit-string vector as used for the amplitude request of the
    paper's Sec. 4.3.

The random-circuit recipe stands in for the Sycamore circuits of the paper's
Sec. 4.3 (53 qubits, depth 14), which are not available here: each cycle applies a
random single-qubit gate from {sqrt-X, sqrt-Y, sqrt-W} to every qubit, then
fSim(pi/2, pi/6) on one of four alternating grid-edge patterns in the order
ABCDCDAB.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

_S2 = 1.0 / np.sqrt(2.0)

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = _S2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
# sqrt-X = exp(-i pi X / 4), sqrt-Y = exp(-i pi Y / 4), sqrt-W = exp(-i pi W / 4)
# with W = (X + Y) / sqrt(2).
SQRT_X = _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)
SQRT_Y = _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)
SQRT_W = _S2 * np.array([[1, np.exp(-0.75j * np.pi)], [np.exp(-0.25j * np.pi), 1]],
                        dtype=np.complex128)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)

SINGLE_QUBIT_SET = (SQRT_X, SQRT_Y, SQRT_W)


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) on |q_a q_b>: iSWAP-like rotation by theta plus a
    controlled phase exp(-i phi) on |11>."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


FSIM_SYC = fsim(np.pi / 2, np.pi / 6)


@dataclass
class Op:
    """One circuit element.

    kind == "gate":    mats = [U] with U a 2^k x 2^k unitary;
    kind == "channel": mats = [A_0, A_1, ...], Kraus operators with
                       sum_k A_k^dagger A_k = I (Eq. kraus_sum of Sec. 3.3).
    """
    kind: str
    qubits: Tuple[int, ...]
    mats: List[np.ndarray]


@dataclass
class Circuit:
    n: int
    ops: List[Op] = field(default_factory=list)

    def gate(self, U, *qubits):
        self.ops.append(Op("gate", tuple(int(q) for q in qubits), [np.asarray(U, np.complex128)]))
        return self

    def channel(self, kraus, *qubits):
        self.ops.append(Op("channel", tuple(int(q) for q in qubits),
                           [np.asarray(A, np.complex128) for A in kraus]))
        return self

    @property
    def n_gates(self):
        return sum(1 for o in self.ops if o.kind == "gate")

    @property
    def n_channels(self):
        return sum(1 for o in self.ops if o.kind == "channel")


def grid_edges(rows: int, cols: int, letter: str) -> List[Tuple[int, int]]:
    """Couplers of one edge pattern on a rows x cols grid (qubit = r*cols + c).

    A: horizontal (r,c)-(r,c+1), c even;  B: horizontal, c odd;
    C: vertical (r,c)-(r+1,c), r even;    D: vertical, r odd.
    """
    out = []
    if letter in "AB":
        par = 0 if letter == "A" else 1
        for r in range(rows):
            for c in range(par, cols - 1, 2):
                out.append((r * cols + c, r * cols + c + 1))
    elif letter in "CD":
        par = 0 if letter == "C" else 1
        for r in range(par, rows - 1, 2):
            for c in range(cols):
                out.append((r * cols + c, (r + 1) * cols + c))
    else:
        raise ValueError(letter)
    return out


def grid_circuit(rows: int, cols: int, cycles: int, seed: int,
                 pattern: str = "ABCDCDAB", no_repeat: bool = True,
                 two_qubit=None) -> Circuit:
    """Seeded grid random circuit (the synthetic stand-in for Sec. 4.3's circuits).

    Per cycle i: a single-qubit gate on every qubit, drawn uniformly from
    {sqrt-X, sqrt-Y, sqrt-W} (excluding the one the same qubit got in cycle i-1
    when no_repeat is set), then fSim(pi/2, pi/6) on every coupler of edge
    pattern pattern[i mod len(pattern)].  Initial state |0...0>; no trailing
    single-qubit layer.
    """
    rng = np.random.default_rng(seed)
    n = rows * cols
    two = FSIM_SYC if two_qubit is None else two_qubit
    circ = Circuit(n)
    prev = [-1] * n
    for cyc in range(cycles):
        for q in range(n):
            if no_repeat and prev[q] >= 0:
                choices = [g for g in range(3) if g != prev[q]]
                g = choices[int(rng.integers(0, 2))]
            else:
                g = int(rng.integers(0, 3))
            prev[q] = g
            circ.gate(SINGLE_QUBIT_SET[g], q)
        for (a, b) in grid_edges(rows, cols, pattern[cyc % len(pattern)]):
            circ.gate(two, a, b)
    return circ


def depolarizing(p: float) -> List[np.ndarray]:
    """Single-qubit depolarizing channel: sqrt(1-p) I and sqrt(p/3) X, Y, Z."""
    return [np.sqrt(1 - p) * I2, np.sqrt(p / 3) * X, np.sqrt(p / 3) * Y, np.sqrt(p / 3) * Z]


def amplitude_damping(gamma: float) -> List[np.ndarray]:
    """Amplitude damping: A0 = diag(1, sqrt(1-gamma)), A1 = sqrt(gamma)|0><1|."""
    return [np.array([[1, 0], [0, np.sqrt(1 - gamma)]], dtype=np.complex128),
            np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)]


def noisy_grid_circuit(rows: int, cols: int, cycles: int, seed: int,
                       p_depol: float, gamma: float, pattern: str = "ABCDCDAB") -> Circuit:
    """Grid random circuit with a depolarizing channel on every qubit a gate acted
    on (right after that gate) and amplitude damping on every qubit at the end of
    each cycle."""
    base = grid_circuit(rows, cols, cycles, seed, pattern)
    n = rows * cols
    circ = Circuit(n)
    i = 0
    for cyc in range(cycles):
        n2 = len(grid_edges(rows, cols, pattern[cyc % len(pattern)]))
        for op in base.ops[i:i + n + n2]:
            circ.ops.append(op)
            if p_depol > 0:
                for q in op.qubits:
                    circ.channel(depolarizing(p_depol), q)
        i += n + n2
        if gamma > 0:
            for q in range(n):
                circ.channel(amplitude_damping(gamma), q)
    return circ


def bell_circuit() -> Circuit:
    """H on qubit 0 then CNOT(0 -> 1): the Bell pair of the paper's Sec. 4.1 example."""
    return Circuit(2).gate(H, 0).gate(CNOT, 0, 1)


def ghz_circuit(n: int) -> Circuit:
    """Cat state of Sec. 4.4: H on qubit 0 then CNOT(0 -> i) for i = 1..n-1."""
    c = Circuit(n).gate(H, 0)
    for i in range(1, n):
        c.gate(CNOT, 0, i)
    return c


def inverse_circuit(circ: Circuit) -> Circuit:
    """U followed by U^dagger (gates reversed and conjugate-transposed)."""
    out = Circuit(circ.n, list(circ.ops))
    for op in reversed(circ.ops):
        assert op.kind == "gate"
        out.gate(op.mats[0].conj().T, *op.qubits)
    return out


def random_bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """count bitstrings uniform over {0,1}^n, int8 array [count][n]."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(count, n), dtype=np.int8)


# The three circuit workloads (rows, cols, cycles, circuit seed, n bitstrings,
# bitstring seed, ...).
CONFIG_SMALL = dict(rows=3, cols=4, cycles=8, seed=1234, n_bitstrings=64, bits_seed=99)
CONFIG_LARGE = dict(rows=6, cols=6, cycles=14, seed=2104, n_bitstrings=1024, bits_seed=10523,
                    max_intermediate_log2=28)
CONFIG_NOISY = dict(rows=4, cols=5, cycles=10, seed=2021, p_depol=1e-3, gamma=1e-3,
                    n_trajectories=4096, traj_seed=7, n_bitstrings=256, bits_seed=77)


def cost_model_circuit(seed: int) -> Circuit:
    """Circuit `seed` of the path-cost-model workload: grid rows uniform in
    {4,5,6}, columns in {4..7}, cycles in {8..16} (drawn from `seed`), then the
    grid random circuit of that shape with the same seed."""
    rng = np.random.default_rng(1_000_003 + seed)
    rows = int(rng.integers(4, 7))
    cols = int(rng.integers(4, 8))
    cycles = int(rng.integers(8, 17))
    return grid_circuit(rows, cols, cycles, seed)
