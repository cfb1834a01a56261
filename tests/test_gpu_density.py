"""GPU parity of exact noisy probabilities through the doubled density-matrix
network (Sec. 3.3, Fig. 7): ket and bra wires, channels as rank-4
superoperator tensors, both wires projected on the bitstring.

* against the FP64 Kraus-sum density matrix (oracle O1) on small noisy grids,
  in every precision mode, with the trace (all probabilities sum to 1);
* the closed forms of amplitude damping and depolarizing noise;
* at the full noisy workload (4x5 grid, 10 cycles, p = gamma = 1e-3) the
  stochastic-trajectory estimates of the same library agree with the exact
  probabilities within 4 standard errors.
Tolerance: relative L2 error of the probabilities, FP32 and TF32x3 <= 1e-5,
BF16x3 <= 2e-5.
"""
import itertools

import numpy as np
import pytest

from oracle import statevector as sv
from workloads import (CONFIG_NOISY, Circuit, H, X, amplitude_damping, depolarizing, noisy_grid_circuit,
                       random_bitstrings)

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5}


@pytest.fixture(scope="module")
def T():
    from paper_2104_10523_gb300 import build, tnq
    build.build()
    tnq.load()
    return tnq


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def exact(T, circ, bits, prec="fp32", force_tc=False, **opts):
    ctx = T.Context(0, prec)
    plan = T.Plan(T.Circuit(circ), density=True, **opts)
    ctx.bind(plan)
    if force_tc:
        T.tnq_ctx_set_kernel_policy(ctx.h, T.TNQ_KERNELS_TENSOR_CORES)
    return ctx.density_probabilities(plan, bits), plan


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_small_grid_all_bitstrings(T, prec):
    c = noisy_grid_circuit(2, 3, 4, seed=5, p_depol=0.05, gamma=0.08)
    allbits = np.array(list(itertools.product((0, 1), repeat=6)), dtype=np.int8)
    ref = sv.probabilities_dm(c, allbits)
    got, _ = exact(T, c, allbits, prec, force_tc=prec != "fp32", batch_log2=3)
    assert rel_l2(got, ref) <= TOL[prec]
    assert abs(got.sum() - 1.0) <= 1e-5


@pytest.mark.parametrize("cap", [28, 8])
def test_grid_3x3_against_density_matrix(T, cap):
    c = noisy_grid_circuit(3, 3, 6, seed=4, p_depol=0.02, gamma=0.03)
    bits = random_bitstrings(9, 40, 6)   # 5 batches of 8
    ref = sv.probabilities_dm(c, bits)
    got, plan = exact(T, c, bits, "fp32", batch_log2=3, max_intermediate_log2=cap, path_mode=0)
    if cap == 8:
        assert plan.info["n_sliced"] >= 1
    assert rel_l2(got, ref) <= TOL["fp32"]


def test_closed_forms(T):
    gamma, m = 0.07, 9
    c = Circuit(1).gate(X, 0)
    for _ in range(m):
        c.channel(amplitude_damping(gamma), 0)
    p, _ = exact(T, c, np.array([[1]], dtype=np.int8))
    assert abs(p[0] - (1 - gamma) ** m) < 1e-6
    pd, m2 = 0.01, 7
    c = Circuit(1)
    for _ in range(m2):
        c.gate(H, 0).channel(depolarizing(pd), 0).gate(H, 0).channel(depolarizing(pd), 0)
    p, _ = exact(T, c, np.array([[0], [1]], dtype=np.int8), batch_log2=1)
    assert abs((p[0] - p[1]) - (1 - 4 * pd / 3) ** (2 * m2)) < 1e-6


def test_two_qubit_channel_rejected(T):
    c = Circuit(2).gate(np.eye(4), 0, 1)
    c.channel([np.eye(4)], 0, 1)
    with pytest.raises(T.TnqError) as e:
        T.Plan(T.Circuit(c), density=True)
    assert e.value.status == T.TNQ_ERR_NOT_SUPPORTED


def test_amplitude_calls_refuse_density_plans(T):
    c = noisy_grid_circuit(2, 2, 2, seed=1, p_depol=0.01, gamma=0.01)
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(c), density=True)
    ctx.bind(plan)
    with pytest.raises(T.TnqError):
        ctx.amplitudes(plan, np.zeros((1, 4), dtype=np.int8))


def test_config4_trajectories_agree_with_exact(T):
    """The full noisy workload: exact p(x) from the doubled network, and the
    trajectory estimate from 4096 trajectories, for 16 of its bitstrings."""
    cfg = CONFIG_NOISY
    c = noisy_grid_circuit(cfg["rows"], cfg["cols"], cfg["cycles"], cfg["seed"], cfg["p_depol"], cfg["gamma"])
    bits = random_bitstrings(c.n, cfg["n_bitstrings"], cfg["bits_seed"])[:16]
    p_exact, plan = exact(T, c, bits, "fp32", batch_log2=0, max_intermediate_log2=27, n_candidates=256, seed=3)
    ctx = T.Context(0, "fp32")
    tplan = T.Plan(T.Circuit(c), batch_log2=4, traj_log2=8, n_candidates=64, seed=1)
    ctx.bind(tplan)
    p_traj, se = ctx.noisy_probabilities(tplan, bits, cfg["n_trajectories"], cfg["traj_seed"])
    z = np.abs(p_traj - p_exact) / np.maximum(se, 1e-30)
    print(f"config4 exact vs trajectories: max |z| {z.max():.2f}, mean p {p_exact.mean():.3e}")
    assert np.all(np.abs(p_traj - p_exact) <= 4 * se + 1e-6 * p_exact)
    assert np.all(p_exact > 0)
