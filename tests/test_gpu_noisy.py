"""GPU parity of the Kraus-trajectory path (stochastic noise, Sec. 3.3).

* Per trajectory, the GPU amplitude equals the oracle's amplitude for the same
  Kraus draws (counter-based SplitMix64 on both sides), within the FP32 bound.
* The GPU trajectory mean equals the oracle's mean over the same trajectories.
* The estimate agrees with the exact density matrix within 4 standard errors.
* At the full noisy workload (4x5 grid, 10 cycles, p = gamma = 1e-3, 2^8
  trajectories per pass, 256 bitstrings) sampled trajectories match the
  tensor-network oracle one by one.
"""
import itertools

import numpy as np
import pytest

from oracle import noise as onoise
from oracle import statevector as sv
from oracle import tn as otn
from workloads import CONFIG_NOISY, noisy_grid_circuit, random_bitstrings

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2104_10523_gb300 import build, tnq
    build.build()
    tnq.load()
    return tnq


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def setup(T, circ, w, t, prec="fp32", **kw):
    ctx = T.Context(0, prec)
    plan = T.Plan(T.Circuit(circ), batch_log2=w, traj_log2=t, **kw)
    ctx.bind(plan)
    return ctx, plan


@pytest.mark.parametrize("t", [0, 3])
def test_trajectory_amplitudes_match_oracle(T, t):
    circ = noisy_grid_circuit(3, 3, 6, seed=4, p_depol=0.05, gamma=0.05)
    bits = random_bitstrings(9, 8, 2)
    ctx, plan = setup(T, circ, 3, t, path_mode=0)
    seed, first, n = 123, 5, 12
    amps = ctx.trajectory_amplitudes(plan, bits, seed, first, n)
    jumps = 0
    for j in range(n):
        picks = onoise.trajectory_picks(circ, seed, first + j)
        jumps += int(np.any(picks != 0))
        ref = sv.amplitudes(circ, bits, kraus_picks=picks)
        assert rel(amps[j], ref) <= 1e-5, (j, rel(amps[j], ref))
    assert jumps >= 3  # the sample exercises non-identity draws


def test_trajectory_mean_matches_oracle_mean(T):
    circ = noisy_grid_circuit(2, 3, 5, seed=9, p_depol=0.08, gamma=0.08)
    bits = np.array(list(itertools.product((0, 1), repeat=6)), dtype=np.int8)
    ctx, plan = setup(T, circ, 6, 4, path_mode=0)
    p, se = ctx.noisy_probabilities(plan, bits, 40, 7)
    ref_mean, ref_se = onoise.noisy_probabilities(circ, bits, 40, 7,
                                                  lambda c, b, pk: sv.amplitudes(c, b, kraus_picks=pk))
    assert rel(p, ref_mean) <= 1e-5
    assert rel(se, ref_se) <= 1e-4


def test_estimate_within_stderr_of_density_matrix(T):
    circ = noisy_grid_circuit(2, 3, 4, seed=3, p_depol=0.05, gamma=0.05)
    bits = np.array(list(itertools.product((0, 1), repeat=6)), dtype=np.int8)
    ctx, plan = setup(T, circ, 6, 8, path_mode=0)
    p, se = ctx.noisy_probabilities(plan, bits, 4096, 11)
    exact = sv.probabilities_dm(circ, bits)
    assert np.all(np.abs(p - exact) <= 4 * se + 1e-9)
    assert abs(p.sum() - 1.0) <= 4 * np.sqrt((se ** 2).sum()) + 1e-6  # total probability


def test_mixed_precision_trajectories(T):
    circ = noisy_grid_circuit(3, 3, 6, seed=4, p_depol=0.05, gamma=0.05)
    bits = random_bitstrings(9, 8, 2)
    ref_ctx, plan = setup(T, circ, 3, 3, path_mode=0)
    ref = ref_ctx.trajectory_amplitudes(plan, bits, 5, 0, 8)
    ctx = T.Context(0, "bf16x3")
    ctx.bind(plan)
    got = ctx.trajectory_amplitudes(plan, bits, 5, 0, 8)
    assert rel(got, ref) <= 2e-5


def test_noisy_rejections(T):
    circ = noisy_grid_circuit(2, 2, 2, seed=1, p_depol=0.1, gamma=0.1)
    ctx, plan = setup(T, circ, 1, 1, path_mode=0)
    with pytest.raises(T.TnqError) as e:
        ctx.noisy_probabilities(plan, np.zeros((2, 4), np.int8), 0, 1)
    assert e.value.status == T.TNQ_ERR_INVALID_ARG
    with pytest.raises(T.TnqError) as e:
        ctx.amplitudes(plan, np.zeros((2, 4), np.int8))
    assert e.value.status == T.TNQ_ERR_INVALID_ARG


def test_full_noisy_workload_sampled_trajectories(T):
    c = CONFIG_NOISY
    circ = noisy_grid_circuit(c["rows"], c["cols"], c["cycles"], c["seed"], c["p_depol"], c["gamma"])
    bits = random_bitstrings(20, c["n_bitstrings"], c["bits_seed"])
    ctx, plan = setup(T, circ, 8, 8, path_mode=2, n_candidates=16, seed=1)
    # a trajectory with at least one non-identity draw, plus the first two
    seed = c["traj_seed"]
    jumpy = next(t for t in range(2, 400) if np.any(onoise.trajectory_picks(circ, seed, t) != 0))
    sample_bits = bits[:6]
    for t in (0, 1, jumpy):
        got = ctx.trajectory_amplitudes(plan, sample_bits, seed, t, 1)[0]
        picks = onoise.trajectory_picks(circ, seed, t)
        ref = np.array([otn.amplitude(circ, b, kraus_picks=picks) for b in sample_bits])
        assert rel(got, ref) <= 1e-5, (t, rel(got, ref))
    # whole workload: 4096 trajectories x 256 bitstrings, probabilities valid
    p, se = ctx.noisy_probabilities(plan, bits, c["n_trajectories"], seed)
    assert np.all(p >= 0) and np.all(np.isfinite(se))
    # mean of 2^n p over uniform bitstrings is ~1 for a scrambling circuit (loose sanity)
    assert 0.5 < p.mean() * 2 ** 20 < 1.5


def test_distinct_trajectories_counted_once(T):
    """Most trajectories of a weakly noisy circuit draw A_0 on every channel;
    the estimate contracts each distinct pick sequence once with its
    multiplicity, which leaves the estimate equal (to rounding) to the mean
    over the individual trajectories."""
    circ = noisy_grid_circuit(2, 3, 4, seed=2, p_depol=0.01, gamma=0.01)
    bits = random_bitstrings(6, 8, 4)
    ctx, plan = setup(T, circ, 3, 4, path_mode=0)
    n_traj, seed = 256, 77
    p, se = ctx.noisy_probabilities(plan, bits, n_traj, seed)
    distinct = T.tnq_plan_get_info(plan.h)["distinct_trajectories"]
    picks = [tuple(onoise.trajectory_picks(circ, seed, t)) for t in range(n_traj)]
    assert distinct == len(set(picks)) and distinct < n_traj // 2
    amps = ctx.trajectory_amplitudes(plan, bits, seed, 0, n_traj)
    mean = np.mean(np.abs(amps) ** 2, axis=0)
    assert np.allclose(p, mean, rtol=1e-10, atol=1e-14)
    m2 = np.mean(np.abs(amps) ** 4, axis=0)
    se_ref = np.sqrt(np.maximum(m2 - mean ** 2, 0) / (n_traj - 1))
    assert np.allclose(se, se_ref, rtol=1e-6, atol=1e-14)

