"""GPU parity of expectation values <psi|H|psi> (Sec. 3.1.2, Eq. exp_val)
through the conjugate (double-depth) network of Fig. 3, against the FP64
oracle, and the cat-state closed forms at 36 and 60 qubits.  Terms are real
numbers in [-1, 1]; bound on each term's absolute error: FP32 and TF32x3 1e-5,
BF16x3 2e-5."""
import numpy as np
import pytest

from oracle import statevector as sv
from workloads import ghz_circuit, grid_circuit

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5}


@pytest.fixture(scope="module")
def T():
    from paper_2104_10523_gb300 import build, tnq
    build.build()
    tnq.load()
    return tnq


def random_terms(n, count, weight, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        s = ["I"] * n
        for q in rng.choice(n, size=weight, replace=False):
            s[q] = "XYZ"[rng.integers(0, 3)]
        out.append("".join(s))
    return out


@pytest.mark.parametrize("t", [0, 3, 6])
def test_grid_3x4_random_observable(T, t):
    c = grid_circuit(3, 4, 8, 1234)
    terms = random_terms(12, 40, 3, 7) + ["I" * 12]
    coeffs = np.random.default_rng(1).standard_normal(len(terms))
    ref, ref_terms = sv.expectation(c, terms, coeffs)
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(c), paulis=terms, traj_log2=t, n_candidates=8, seed=2)
    ctx.bind(plan)
    v, per = ctx.expectation(plan, coeffs)
    assert np.max(np.abs(per - ref_terms.real)) <= TOL["fp32"]
    assert abs(v - ref.real) <= TOL["fp32"] * np.sum(np.abs(coeffs))
    assert abs(per[-1] - 1.0) <= 1e-6


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_grid_4x5_local_observable(T, prec):
    """A nearest-neighbour ZZ + transverse X observable on the 4x5 grid, 10
    cycles: every qubit is in the light cone after 10 cycles."""
    c = grid_circuit(4, 5, 10, 2021)
    n = 20
    terms = []
    for q in range(n):
        r, col = divmod(q, 5)
        if col + 1 < 5:
            s = ["I"] * n
            s[q] = s[q + 1] = "Z"
            terms.append("".join(s))
        if r + 1 < 4:
            s = ["I"] * n
            s[q] = s[q + 5] = "Z"
            terms.append("".join(s))
        s = ["I"] * n
        s[q] = "X"
        terms.append("".join(s))
    coeffs = np.where([t.count("Z") == 2 for t in terms], -1.0, -0.5)
    ref, ref_terms = sv.expectation(c, terms, coeffs)
    ctx = T.Context(0, prec)
    plan = T.Plan(T.Circuit(c), paulis=terms, traj_log2=5, n_candidates=32, seed=4)
    ctx.bind(plan)
    if prec != "fp32":
        T.tnq_ctx_set_kernel_policy(ctx.h, T.TNQ_KERNELS_TENSOR_CORES)
    v, per = ctx.expectation(plan, coeffs)
    err = np.max(np.abs(per - ref_terms.real))
    print(f"4x5 observable {prec}: max term error {err:.2e}, value {v:.6f} (oracle {ref.real:.6f})")
    assert err <= TOL[prec]


def test_light_cone_of_a_shallow_circuit(T):
    """Z on qubit 0 after two cycles of the 6x6 grid: its backward light cone
    holds few gates, so the plan's network is small (most of U cancels against
    U^dagger); the oracle contracts the whole double-depth network."""
    from oracle import tn as otn
    c = grid_circuit(6, 6, 2, 9)
    terms = ["Z" + "I" * 35, "I" * 20 + "X" + "I" * 15]
    ref, ref_terms = otn.expectation(c, terms, [1.0, 1.0])
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(c), paulis=terms)
    ctx.bind(plan)
    assert plan.info["n_leaves"] < 30
    v, per = ctx.expectation(plan, [1.0, 1.0])
    assert np.allclose(per, ref_terms.real, atol=1e-6)


@pytest.mark.parametrize("n", [36, 60])
def test_cat_state_closed_forms(T, n):
    c = ghz_circuit(n)
    z0zk = ["Z" + "I" * (n - 2) + "Z"]
    xall = ["X" * n]
    yy = ["YY" + "X" * (n - 2)]
    z0 = ["Z" + "I" * (n - 1)]
    terms = z0zk + xall + yy + z0
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(c), paulis=terms, traj_log2=2)
    ctx.bind(plan)
    v, per = ctx.expectation(plan, [1.0, 1.0, 1.0, 1.0])
    assert np.allclose(per, [1.0, 1.0, -1.0, 0.0], atol=1e-6)
    assert abs(v - 1.0) <= 1e-5
