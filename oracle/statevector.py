"""O1: brute-force statevector and density-matrix simulation in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The amplitude of bitstring x is the plain definition <x| U_circuit |0...0> of
Eq. ampl_calc (Sec. 3.1.1); a noisy circuit evolves a density matrix by the
Kraus sum rho -> sum_k A_k rho A_k^dagger of Eq. kraus_sum (Sec. 3.3).

Qubit q is array axis q of the (2,)*n state (C order, so qubit 0 is the most
significant bit of the flat index); a k-qubit matrix acts on the basis of its
listed qubits with the first listed qubit most significant.
"""
from __future__ import annotations

import numpy as np


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    return psi


def apply_matrix(psi: np.ndarray, U: np.ndarray, qubits) -> np.ndarray:
    """psi <- (U on `qubits`) psi, for a state tensor of shape (2,)*n."""
    k = len(qubits)
    Ut = np.asarray(U, np.complex128).reshape((2,) * (2 * k))
    out = np.tensordot(Ut, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    return np.moveaxis(out, list(range(k)), list(qubits))


def final_state(circ, kraus_picks=None) -> np.ndarray:
    """U|0...0> for a gate-only circuit.

    With kraus_picks (one Kraus index per channel, in circuit order) every
    channel is replaced by its picked operator rescaled to A_k / sqrt(q_k),
    q_k = Tr(A_k^dagger A_k) / d: one stochastic trajectory.
    """
    psi = zero_state(circ.n)
    c = 0
    for op in circ.ops:
        if op.kind == "gate":
            psi = apply_matrix(psi, op.mats[0], op.qubits)
        else:
            if kraus_picks is None:
                raise ValueError("circuit has channels; pass kraus_picks or use density_matrix")
            A = op.mats[int(kraus_picks[c])]
            d = A.shape[0]
            q = np.real(np.trace(A.conj().T @ A)) / d
            psi = apply_matrix(psi, A / np.sqrt(q), op.qubits)
            c += 1
    return psi


def amplitudes(circ, bitstrings, kraus_picks=None) -> np.ndarray:
    """complex128 amplitudes <x|U|0> for each row x of bitstrings [B][n]."""
    psi = final_state(circ, kraus_picks)
    bits = np.asarray(bitstrings, dtype=np.int64)
    return np.array([psi[tuple(b)] for b in bits], dtype=np.complex128)


def density_matrix(circ) -> np.ndarray:
    """rho after the circuit, as a (2,)*(2n) tensor: ket axes 0..n-1, bra axes n..2n-1.

    Gates act as U rho U^dagger, channels as sum_k A_k rho A_k^dagger (Eq. kraus_sum).
    """
    n = circ.n
    rho = np.zeros((2,) * (2 * n), dtype=np.complex128)
    rho[(0,) * (2 * n)] = 1.0
    for op in circ.ops:
        ket = list(op.qubits)
        bra = [q + n for q in op.qubits]
        if op.kind == "gate":
            U = op.mats[0]
            rho = apply_matrix(apply_matrix(rho, U, ket), U.conj(), bra)
        else:
            acc = np.zeros_like(rho)
            for A in op.mats:
                acc += apply_matrix(apply_matrix(rho, A, ket), A.conj(), bra)
            rho = acc
    return rho


def probabilities_dm(circ, bitstrings) -> np.ndarray:
    """p(x) = <x| rho |x> from the exact density matrix."""
    rho = density_matrix(circ)
    bits = np.asarray(bitstrings, dtype=np.int64)
    return np.array([np.real(rho[tuple(b) + tuple(b)]) for b in bits])


def wavefunction_slice(circ, bitstrings) -> np.ndarray:
    """Marginal wave-function slices (Sec. 4.4): for each row x of bitstrings
    [B][n] with -1 at the open qubits (the same ones in every row), the
    amplitudes <x_fixed, y|U|0...0> for every value y of the open qubits, as
    [B][2^k]; the open qubit with the lowest index is the most significant bit
    of y."""
    psi = final_state(circ)
    rows = []
    for b in np.asarray(bitstrings, dtype=np.int64):
        idx = tuple(slice(None) if v == -1 else int(v) for v in b)
        rows.append(np.ascontiguousarray(psi[idx]).reshape(-1))
    return np.array(rows, dtype=np.complex128)


PAULI = {"I": np.eye(2, dtype=np.complex128),
         "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
         "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
         "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128)}


def expectation(circ, paulis, coeffs):
    """<psi|H|psi> (Eq. exp_val) for |psi> = U|0...0> and H = sum_t c_t P_t,
    P_t given as a string over IXYZ (character q acts on qubit q).  Returns
    (value, per-term <psi|P_t|psi>)."""
    psi = final_state(circ)
    vals = []
    for ps in paulis:
        phi = psi
        for q, ch in enumerate(ps):
            if ch != "I":
                phi = apply_matrix(phi, PAULI[ch], [q])
        vals.append(np.vdot(psi, phi))
    vals = np.array(vals)
    return complex(np.dot(coeffs, vals)), vals
