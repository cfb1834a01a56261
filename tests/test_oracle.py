"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test pins the oracle to something other than itself: brute-force
operators built entry by entry, closed forms, invariants, a second independent
formulation, or printed test vectors.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import contraction, noise, statevector as sv, tn
from workloads import (CNOT, H, SQRT_W, SQRT_X, SQRT_Y, X, Y, Z, Circuit, bell_circuit, fsim,
                       ghz_circuit, grid_circuit, grid_edges, inverse_circuit, noisy_grid_circuit,
                       random_bitstrings, depolarizing, amplitude_damping)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- gate table
def test_gate_table_unitary():
    for U in (SQRT_X, SQRT_Y, SQRT_W, H, CNOT, fsim(np.pi / 2, np.pi / 6), fsim(0.3, 1.1)):
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-15)


def test_sqrt_gates_square_to_rotations():
    W = (X + Y) / np.sqrt(2)
    # exp(-i pi P / 4)^2 = exp(-i pi P / 2) = -i P for a Pauli-like P with P^2 = I
    assert np.allclose(SQRT_X @ SQRT_X, -1j * X, atol=1e-15)
    assert np.allclose(SQRT_Y @ SQRT_Y, -1j * Y, atol=1e-15)
    assert np.allclose(SQRT_W @ SQRT_W, -1j * W, atol=1e-15)


def test_fsim_special_cases():
    iswap_dag = np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]])
    assert np.allclose(fsim(np.pi / 2, 0.0), iswap_dag)
    assert np.allclose(fsim(0.0, np.pi), np.diag([1, 1, 1, -1]))


# ---------------------------------------------------------------- circuits
@pytest.mark.parametrize("rows,cols,cycles,n1,n2", [(3, 4, 8, 96, 34), (6, 6, 14, 504, 210),
                                                    (4, 5, 10, 200, 78)])
def test_grid_circuit_gate_counts(rows, cols, cycles, n1, n2):
    c = grid_circuit(rows, cols, cycles, seed=1)
    assert sum(len(o.qubits) == 1 for o in c.ops) == n1
    assert sum(len(o.qubits) == 2 for o in c.ops) == n2


def test_grid_patterns_partition_edges():
    rows, cols = 5, 6
    all_edges = set()
    for L in "ABCD":
        e = grid_edges(rows, cols, L)
        qs = [q for ab in e for q in ab]
        assert len(qs) == len(set(qs)), "a pattern is a matching"
        for a, b in e:
            ra, ca, rb, cb = a // cols, a % cols, b // cols, b % cols
            assert abs(ra - rb) + abs(ca - cb) == 1
        all_edges |= set(e)
    assert len(all_edges) == rows * (cols - 1) + (rows - 1) * cols


def test_no_repeat_rule():
    c = grid_circuit(3, 3, 12, seed=5)
    last = {}
    for o in c.ops:
        if len(o.qubits) == 1:
            q = o.qubits[0]
            key = o.mats[0].tobytes()
            assert last.get(q) != key
            last[q] = key


# ---------------------------------------------------------------- O1
def _brute_operator(U, qubits, n):
    """Full 2^n x 2^n matrix of U on `qubits`, entry by entry (qubit 0 = MSB)."""
    D = 1 << n
    M = np.zeros((D, D), dtype=np.complex128)
    for x in range(D):
        xb = [(x >> (n - 1 - q)) & 1 for q in range(n)]
        for y in range(D):
            yb = [(y >> (n - 1 - q)) & 1 for q in range(n)]
            if any(xb[q] != yb[q] for q in range(n) if q not in qubits):
                continue
            r = 0
            c = 0
            for q in qubits:
                r = 2 * r + yb[q]
                c = 2 * c + xb[q]
            M[y, x] = U[r, c]
    return M


def _random_unitary(rng, d):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_statevector_matches_brute_force_operator():
    rng = np.random.default_rng(3)
    n = 4
    c = Circuit(n)
    for qs in [(0,), (2,), (3, 1), (0, 2), (1,), (2, 3), (3, 0), (1, 2)]:
        c.gate(_random_unitary(rng, 1 << len(qs)), *qs)
    psi0 = np.zeros(1 << n, dtype=np.complex128)
    psi0[0] = 1
    for op in c.ops:
        psi0 = _brute_operator(op.mats[0], op.qubits, n) @ psi0
    allbits = np.array(list(itertools.product((0, 1), repeat=n)))
    assert np.allclose(sv.amplitudes(c, allbits), psi0, atol=1e-14)


def test_density_matrix_matches_brute_force_kraus_sum():
    rng = np.random.default_rng(4)
    n = 3
    c = Circuit(n)
    c.gate(_random_unitary(rng, 4), 2, 0)
    c.channel(depolarizing(0.2), 1)
    c.gate(_random_unitary(rng, 2), 1)
    c.channel(amplitude_damping(0.3), 0)
    c.gate(_random_unitary(rng, 4), 1, 2)
    D = 1 << n
    rho = np.zeros((D, D), dtype=np.complex128)
    rho[0, 0] = 1
    for op in c.ops:
        mats = [_brute_operator(A, op.qubits, n) for A in op.mats]
        rho = sum(M @ rho @ M.conj().T for M in mats)
    allbits = np.array(list(itertools.product((0, 1), repeat=n)))
    assert np.allclose(sv.probabilities_dm(c, allbits), np.real(np.diag(rho)), atol=1e-14)


def _golden_closed_forms():
    rows = {}
    with open(os.path.join(GOLDEN, "closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, key, re, im = line.split()
            rows[(name, key)] = complex(float(re), float(im))
    return rows


def test_bell_closed_form_both_oracles():
    g = _golden_closed_forms()
    c = bell_circuit()
    for key in ("00", "11", "01", "10"):
        bits = [int(ch) for ch in key]
        assert abs(sv.amplitudes(c, [bits])[0] - g[("bell", key)]) < 1e-15
        assert abs(tn.amplitude(c, bits) - g[("bell", key)]) < 1e-15


@pytest.mark.parametrize("n", [12, 36, 60])
def test_ghz_closed_form_tn(n):
    g = _golden_closed_forms()
    c = ghz_circuit(n)
    assert abs(tn.amplitude(c, [0] * n) - g[("ghz", "all0")]) < 1e-14
    assert abs(tn.amplitude(c, [1] * n) - g[("ghz", "all1")]) < 1e-14
    rng = np.random.default_rng(n)
    x = rng.integers(0, 2, n)
    x[0], x[1] = 0, 1
    assert abs(tn.amplitude(c, x)) < 1e-15
    if n <= 12:
        assert abs(sv.amplitudes(c, [[1] * n])[0] - g[("ghz", "all1")]) < 1e-14


@pytest.mark.parametrize("n", [8, 60])
def test_wavefunction_slice_cat_state_closed_form(n):
    """Sec. 4.4, Fig. 9: the cat state (H then CX chain) with qubits 2 and
    min(47, n-1) open.  Other qubits all 0 -> (1/sqrt2) [1,0,0,0], all 1 ->
    (1/sqrt2) [0,0,0,1] (the paper prints the normalised vectors [1,0,0,0] and
    [0,0,0,1]); any mixed assignment -> 0."""
    c = ghz_circuit(n)
    o2 = min(47, n - 1)
    s = 1 / np.sqrt(2)
    for fill, want in ((0, [s, 0, 0, 0]), (1, [0, 0, 0, s])):
        bits = [fill] * n
        bits[2] = bits[o2] = -1
        got = tn.wavefunction_slice(c, bits)
        assert np.allclose(got, want, atol=1e-15)
        assert np.allclose(got / np.linalg.norm(got), np.array(want) / s, atol=1e-15)
        if n <= 12:
            assert np.allclose(sv.wavefunction_slice(c, [bits])[0], want, atol=1e-15)
    bits = [0] * n
    bits[2] = bits[o2] = -1
    bits[n - 2 if n - 2 not in (2, o2) else 1] = 1
    assert np.allclose(tn.wavefunction_slice(c, bits), 0, atol=1e-15)


def test_wavefunction_slice_both_oracles_and_norm():
    """O1's slice (statevector indexing) and O2's (network with open legs)
    agree on a random grid circuit, and the slices over every assignment of
    the fixed qubits hold the whole normalised state."""
    c = grid_circuit(3, 3, 6, 31)
    open_q = [1, 4, 8]
    rows = []
    for vals in itertools.product((0, 1), repeat=6):
        b = [-1] * 9
        for q, v in zip([q for q in range(9) if q not in open_q], vals):
            b[q] = v
        rows.append(b)
    s1 = sv.wavefunction_slice(c, rows)
    assert s1.shape == (64, 8)
    assert abs(np.sum(np.abs(s1) ** 2) - 1.0) < 1e-13
    for i in (0, 17, 63):
        s2 = tn.wavefunction_slice(c, rows[i], order="random", seed=i)
        assert np.allclose(s2, s1[i], atol=1e-14)
    # entry y of the slice is the amplitude of the completed bitstring
    full = np.array(rows[17])
    y = 5
    for k, q in enumerate(open_q):
        full[q] = (y >> (len(open_q) - 1 - k)) & 1
    assert abs(s1[17][y] - sv.amplitudes(c, [full])[0]) < 1e-15


def test_expectation_closed_forms():
    """Sec. 3.1.2, Eq. exp_val.  Cat state (H then CX chain): <Z_0 Z_k> = 1,
    <X...X> = 1, <Z_0> = 0, <Y_0 Y_1 X_2...X_{n-1}> = -1 (two Y's on a cat
    state give i*i = -1); X on qubit 0 of |0>: <Z_0> = -1.  Both oracles."""
    n = 6
    c = ghz_circuit(n)
    terms = ["ZIIIIZ", "XXXXXX", "ZIIIII", "YYXXXX", "IIIIII"]
    want = np.array([1.0, 1.0, 0.0, -1.0, 1.0])
    coeffs = np.array([0.5, -2.0, 3.0, 1.5, 0.25])
    for fn in (sv.expectation, tn.expectation):
        v, per = fn(c, terms, coeffs)
        assert np.allclose(per, want, atol=1e-14)
        assert abs(v - np.dot(coeffs, want)) < 1e-13
    v, per = tn.expectation(Circuit(2).gate(X, 0), ["ZI", "IZ"], [1.0, 1.0])
    assert np.allclose(per, [-1.0, 1.0], atol=1e-15)


def test_expectation_both_oracles_random_circuit():
    """O1 (Pauli strings applied to the statevector) and O2 (the double-depth
    network of Fig. 3, random order) agree; every term is real (P Hermitian),
    and the sum over all 4^n Pauli strings of <P>^2 equals 2^n for a pure
    state (purity)."""
    c = grid_circuit(2, 2, 4, 17)
    rng = np.random.default_rng(3)
    terms = ["".join(rng.choice(list("IXYZ"), size=4)) for _ in range(12)]
    coeffs = rng.standard_normal(12)
    v1, p1 = sv.expectation(c, terms, coeffs)
    v2, p2 = tn.expectation(c, terms, coeffs, order="random", seed=5)
    assert np.allclose(p1, p2, atol=1e-14)
    assert np.allclose(np.imag(p1), 0, atol=1e-15)
    allp = ["".join(t) for t in itertools.product("IXYZ", repeat=4)]
    _, pa = sv.expectation(c, allp, np.zeros(len(allp)))
    assert abs(np.sum(np.abs(pa) ** 2) - 16.0) < 1e-12


def test_norm_statevector_config_small():
    c = grid_circuit(3, 4, 8, 1234)
    psi = sv.final_state(c)
    assert abs(np.sum(np.abs(psi) ** 2) - 1.0) < 1e-13


# ---------------------------------------------------------------- O2
def test_tn_matches_statevector_config_small():
    c = grid_circuit(3, 4, 8, 1234)
    bits = random_bitstrings(12, 64, 99)
    a1 = sv.amplitudes(c, bits)
    a2 = tn.amplitudes(c, bits)
    assert np.linalg.norm(a2 - a1) / np.linalg.norm(a1) < 1e-12


def test_tn_norm_small_grid():
    c = grid_circuit(2, 3, 6, 11)
    allbits = np.array(list(itertools.product((0, 1), repeat=6)))
    a = tn.amplitudes(c, allbits)
    assert abs(np.sum(np.abs(a) ** 2) - 1.0) < 1e-13


def test_tn_order_and_slicing_independence():
    # random orders on a small grid (their intermediates can be large), slicings on config-1 size
    small = grid_circuit(2, 3, 5, 21)
    sbits = random_bitstrings(6, 1, 2)[0]
    snet = tn.build_network(small, sbits)
    sref = complex(tn.contract(snet)[0])
    assert abs(sref - sv.amplitudes(small, [sbits])[0]) < 1e-14
    for s in range(3):
        v = complex(tn.contract(snet, tn.random_order(snet, s))[0])
        assert abs(v - sref) <= 1e-12 * abs(sref)
    c = grid_circuit(3, 4, 8, 1234)
    bits = random_bitstrings(12, 3, 5)
    net = tn.build_network(c, bits[0])
    ref = tn.contract(net)[0]
    vals = []
    labels = sorted({l for _, ls in net for l in ls})
    rng = np.random.default_rng(0)
    for k in (2, 4):
        sl = list(rng.choice(labels, size=k, replace=False))
        vals.append(tn.contract_sliced(net, sl))
    for v in vals:
        assert abs(complex(v) - complex(ref)) <= 1e-12 * abs(complex(ref))


def test_tn_identity_circuit():
    c = inverse_circuit(grid_circuit(3, 4, 8, 77))
    assert abs(tn.amplitude(c, [0] * 12) - 1.0) < 1e-12
    x = [0] * 12
    x[5] = 1
    assert abs(tn.amplitude(c, x)) < 1e-12


# ---------------------------------------------------------------- pairwise contraction
def test_contraction_matches_loop_brute_force():
    rng = np.random.default_rng(9)
    a_labels = [3, 0, 4, 1]      # bit p of A's index carries label a_labels[p]
    b_labels = [2, 4, 3]
    out_labels = [1, 2, 0]       # shared labels 3 and 4 are summed
    A = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    B = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    C = contraction.contract_labeled(A, a_labels, B, b_labels, out_labels)

    def idx(labels, val):
        return sum(val[l] << p for p, l in enumerate(labels))

    ref = np.zeros(8, dtype=np.complex128)
    for v in itertools.product((0, 1), repeat=5):
        val = dict(enumerate(v))
        ref[idx(out_labels, val)] += A[idx(a_labels, val)] * B[idx(b_labels, val)]
    assert np.allclose(C, ref, atol=1e-14)
    # a label held by A, B and the output is a batch index
    a2, b2, o2 = [3, 0, 5, 1], [5, 2, 3], [1, 5, 2, 0]
    C2 = contraction.contract_labeled(A, a2, B, b2, o2)
    ref2 = np.zeros(16, dtype=np.complex128)
    for v in itertools.product((0, 1), repeat=5):
        val = dict(zip([0, 1, 2, 3, 5], v))
        ref2[idx(o2, val)] += A[idx(a2, val)] * B[idx(b2, val)]
    assert np.allclose(C2, ref2, atol=1e-14)
    rows = contraction.sampled_rows(A, a_labels, B, b_labels, out_labels, rows=[0, 3],
                                    row_labels=[0, 1])
    for i, r in enumerate([0, 3]):
        for cidx in range(2):  # remaining label 2
            val = {0: r & 1, 1: (r >> 1) & 1, 2: cidx}
            assert abs(rows[i, cidx] - ref[idx(out_labels, val)]) < 1e-14


# ---------------------------------------------------------------- noise
def _splitmix_golden():
    out = []
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            vals = [int(v) for v in line.split()]
            out.append((vals[0], vals[1:]))
    return out


def test_splitmix64_published_vectors():
    for seed, outs in _splitmix_golden():
        assert noise.splitmix64_stream(seed, len(outs)) == outs


def test_counter_based_uniform_is_stream_element():
    s = noise.splitmix64_stream(42, 5)
    for c in range(5):
        assert noise.uniform(42, 0, c) == (s[c] >> 11) / 2.0 ** 53


def test_kraus_completeness_and_probabilities():
    for kr in (depolarizing(1e-3), amplitude_damping(1e-3), depolarizing(0.3)):
        S = sum(A.conj().T @ A for A in kr)
        assert np.allclose(S, np.eye(2), atol=1e-15)
        assert abs(noise.kraus_probabilities(kr).sum() - 1) < 1e-15
    assert np.allclose(noise.kraus_probabilities(amplitude_damping(0.2)), [0.9, 0.1])
    assert np.allclose(noise.kraus_probabilities(depolarizing(0.3)), [0.7, 0.1, 0.1, 0.1])


def test_amplitude_damping_closed_form():
    gamma, m = 0.07, 9
    c = Circuit(1).gate(X, 0)
    for _ in range(m):
        c.channel(amplitude_damping(gamma), 0)
    p1 = sv.probabilities_dm(c, [[1]])[0]
    assert abs(p1 - (1 - gamma) ** m) < 1e-14


def test_depolarizing_hh_closed_form():
    # H-H cycles with depolarizing noise after every gate (the shape of Fig. 8):
    # each channel shrinks the Bloch vector by (1 - 4p/3), so <Z> = (1 - 4p/3)^(2m).
    p, m = 0.01, 7
    c = Circuit(1)
    for _ in range(m):
        c.gate(H, 0).channel(depolarizing(p), 0).gate(H, 0).channel(depolarizing(p), 0)
    pz = sv.probabilities_dm(c, [[0], [1]])
    assert abs((pz[0] - pz[1]) - (1 - 4 * p / 3) ** (2 * m)) < 1e-14


def test_density_network_matches_density_matrix():
    """O2's doubled network (Sec. 3.3) against O1's Kraus-sum density matrix
    on a noisy grid circuit, plus the trace: the probabilities of all 2^n
    bitstrings sum to 1."""
    c = noisy_grid_circuit(2, 3, 4, seed=5, p_depol=0.05, gamma=0.08)
    allbits = np.array(list(itertools.product((0, 1), repeat=6)))
    exact = sv.probabilities_dm(c, allbits)
    got = np.array([tn.density_probability(c, b) for b in allbits])
    assert np.allclose(got, exact, atol=1e-14)
    assert abs(got.sum() - 1.0) < 1e-13
    net, _ = tn.build_density_network_wires(c, allbits[5])
    v = tn.contract(net, tn.random_order(net, 3))[0]
    assert abs(complex(np.asarray(v).reshape(())) - exact[5]) < 1e-14


def test_density_network_closed_forms():
    """Amplitude damping on |1> for m rounds: P(1) = (1 - gamma)^m; depolarizing
    H-H (the shape of Fig. 8): <Z> = (1 - 4p/3)^(2m) -- through the doubled network."""
    gamma, m = 0.07, 9
    c = Circuit(1).gate(X, 0)
    for _ in range(m):
        c.channel(amplitude_damping(gamma), 0)
    assert abs(tn.density_probability(c, [1]) - (1 - gamma) ** m) < 1e-14
    p, m = 0.01, 7
    c = Circuit(1)
    for _ in range(m):
        c.gate(H, 0).channel(depolarizing(p), 0).gate(H, 0).channel(depolarizing(p), 0)
    z = tn.density_probability(c, [0]) - tn.density_probability(c, [1])
    assert abs(z - (1 - 4 * p / 3) ** (2 * m)) < 1e-14


def test_trajectory_estimator_exactly_unbiased():
    """Summing q-weighted |amp|^2 over every pick sequence gives <x|rho|x> exactly."""
    rng = np.random.default_rng(8)
    c = Circuit(2)
    c.gate(_random_unitary(rng, 4), 0, 1)
    c.channel(depolarizing(0.2), 0)
    c.gate(_random_unitary(rng, 2), 1)
    c.channel(amplitude_damping(0.3), 1)
    c.gate(_random_unitary(rng, 4), 1, 0)
    chans = [o for o in c.ops if o.kind == "channel"]
    allbits = np.array(list(itertools.product((0, 1), repeat=2)))
    exact = sv.probabilities_dm(c, allbits)
    acc = np.zeros(4)
    for picks in itertools.product(*[range(len(o.mats)) for o in chans]):
        w = np.prod([noise.kraus_probabilities(o.mats)[k] for o, k in zip(chans, picks)])
        acc += w * np.abs(sv.amplitudes(c, allbits, kraus_picks=picks)) ** 2
        # the same trajectory amplitude through the tensor network
        a_tn = tn.amplitudes(c, allbits, kraus_picks=picks)
        assert np.allclose(a_tn, sv.amplitudes(c, allbits, kraus_picks=picks), atol=1e-14)
    assert np.allclose(acc, exact, atol=1e-14)


def test_trajectory_standard_error_closed_form():
    """X then one amplitude-damping channel on one qubit: a trajectory picks
    A_0 (probability 1 - gamma/2) and gives |amp(1)|^2 = v = (1-gamma)/(1-gamma/2),
    or A_1 and gives 0.  With j jumps among n trajectories (counted from the
    pinned counter-based uniforms: a jump is u >= 1 - gamma/2) the estimate is
    m = (n-j) v / n and the standard error sqrt((m v - m^2) / (n - 1)), since
    the mean of |amp|^4 is (n-j) v^2 / n.  For bitstring 0 the values are 0 or
    2: m0 = 2 j / n."""
    gamma, n, seed = 0.3, 200, 12345
    c = Circuit(1).gate(X, 0).channel(amplitude_damping(gamma), 0)
    j = sum(1 for t in range(n) if noise.uniform(seed, t, 0) >= 1 - gamma / 2)
    assert 10 < j < 60   # the sample holds both outcomes
    v = (1 - gamma) / (1 - gamma / 2)
    m1 = (n - j) * v / n
    se1 = np.sqrt((m1 * v - m1 * m1) / (n - 1))
    m0 = 2.0 * j / n
    se0 = np.sqrt((m0 * 2.0 - m0 * m0) / (n - 1))
    mean, se = noise.noisy_probabilities(c, [[1], [0]], n, seed, sv.amplitudes)
    assert abs(mean[0] - m1) < 1e-14 and abs(se[0] - se1) < 1e-14
    assert abs(mean[1] - m0) < 1e-14 and abs(se[1] - se0) < 1e-14


def test_trajectory_mean_within_stderr_of_density_matrix():
    c = noisy_grid_circuit(2, 2, 4, seed=3, p_depol=0.05, gamma=0.05)
    bits = random_bitstrings(4, 6, 1)
    exact = sv.probabilities_dm(c, bits)
    mean, se = noise.noisy_probabilities(c, bits, 3000, seed=11,
                                         amplitude_fn=lambda cc, b, p: sv.amplitudes(cc, b, p))
    assert np.all(np.abs(mean - exact) <= 4 * se + 1e-12)


# ---------------------------------------------------------------- cost-model MLP
def test_mlp_gradients_match_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    P = mlp.init_params(5, 7, seed=1)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.standard_normal(P[k].shape) * 0.1   # non-zero biases exercise every path
    X = rng.standard_normal((9, 5))
    t = rng.standard_normal(9)
    G = mlp.gradients(P, X, t)
    h = 1e-6
    for k in mlp.PARAMS:
        num = np.zeros_like(P[k])
        for idx in np.ndindex(P[k].shape):
            Pp = {q: v.copy() for q, v in P.items()}
            Pm = {q: v.copy() for q, v in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            num[idx] = (mlp.loss(Pp, X, t) - mlp.loss(Pm, X, t)) / (2 * h)
        assert np.allclose(G[k], num, rtol=1e-5, atol=1e-8), k


def test_mlp_linear_regime_is_least_squares_gradient():
    """With every hidden unit active and W2 = I, the model is linear in x and the
    gradient of the last layer equals the textbook least-squares gradient."""
    from oracle import mlp
    rng = np.random.default_rng(2)
    d, h, B = 3, 4, 6
    P = {"W1": np.abs(rng.standard_normal((d, h))), "b1": np.full(h, 10.0),
         "W2": np.eye(h), "b2": np.zeros(h), "W3": rng.standard_normal((h, 1)), "b3": np.zeros(1)}
    X = np.abs(rng.standard_normal((B, d)))
    t = rng.standard_normal(B)
    A = X @ P["W1"] + P["b1"]                       # all positive, so relu is the identity
    y = A @ P["W3"][:, 0]
    g_ls = 2.0 / B * A.T @ (y - t)
    assert np.allclose(mlp.gradients(P, X, t)["W3"][:, 0], g_ls, atol=1e-12)


def test_adam_first_step_moves_by_lr_sign():
    """Adam's first bias-corrected step is lr * g / (|g| + eps): magnitude lr."""
    from oracle import mlp
    P = {k: np.zeros((2, 2)) for k in mlp.PARAMS}
    G = {k: np.array([[1.0, -2.0], [0.5, 0.0]]) for k in mlp.PARAMS}
    st = {}
    mlp.adam_step(P, G, st, lr=0.01, step=1)
    want = -0.01 * np.array([[1.0, -1.0], [1.0, 0.0]])
    assert np.allclose(P["W1"], want, atol=1e-9)


def test_bf16_rounding_known_values():
    from oracle import mlp
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to even (1.0);
    # 1 + 3*2^-9 rounds up to 1 + 2^-7; powers of two are exact.
    x = np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 0.75, -3.0, 2.0 ** -20])
    assert np.array_equal(mlp.bf16_round(x), [1.0, 1.0 + 2 ** -7, 0.75, -3.0, 2.0 ** -20])
