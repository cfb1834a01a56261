"""Stochastic Kraus-trajectory estimator of noisy bitstring probabilities.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper models noise with Kraus operators {A_k}, sum_k A_k^dagger A_k = I
(Eq. kraus_sum, Sec. 3.3) and states that noise enters "stochastically"
(abstract, Sec. 3) without giving the sampler.  The reading used here:

  * at each channel draw k with probability q_k = Tr(A_k^dagger A_k) / d
    (these sum to 1 by completeness) and apply A_k / sqrt(q_k);
  * then E[ |<x| psi_traj>|^2 ] = sum over all pick sequences of
    |<x| prod A_k |0>|^2 = <x| rho |x>, exactly, so each trajectory is a plain
    (unnormalised) amplitude contraction and the estimate is the FP64 mean of
    |amp|^2 over trajectories, with its standard error.

Draws are counter based: the uniform for (trajectory t, channel c) is the
(t * 2^32 + c + 1)-th output of a SplitMix64 generator started at `seed`
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), i.e. mix(seed + i * 0x9E3779B97F4A7C15) with i = t * 2^32 + c + 1,
turned into a double in [0, 1) from its top 53 bits.  Pick = the first k with
u < q_0 + ... + q_k (cumulative sum in FP64, in index order).
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    """The SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, count: int):
    """First `count` outputs of SplitMix64 started at state `seed`."""
    out = []
    s = seed & MASK64
    for _ in range(count):
        s = (s + GOLDEN_GAMMA) & MASK64
        out.append(splitmix64_mix(s))
    return out


def uniform(seed: int, traj: int, channel: int) -> float:
    i = (traj << 32) + channel + 1
    z = splitmix64_mix((seed + i * GOLDEN_GAMMA) & MASK64)
    return (z >> 11) * (1.0 / 9007199254740992.0)


def kraus_probabilities(kraus) -> np.ndarray:
    d = kraus[0].shape[0]
    return np.array([np.real(np.trace(A.conj().T @ A)) / d for A in kraus])


def pick(kraus, u: float) -> int:
    q = kraus_probabilities(kraus)
    acc = 0.0
    for k, qk in enumerate(q):
        acc += qk
        if u < acc:
            return k
    return len(q) - 1


def trajectory_picks(circ, seed: int, traj: int) -> np.ndarray:
    """Kraus index for every channel of circ (circuit order) in trajectory traj."""
    picks = []
    c = 0
    for op in circ.ops:
        if op.kind == "channel":
            picks.append(pick(op.mats, uniform(seed, traj, c)))
            c += 1
    return np.array(picks, dtype=np.int64)


def noisy_probabilities(circ, bitstrings, n_traj: int, seed: int, amplitude_fn):
    """Trajectory estimate of p(x) = <x|rho|x> and its standard error.

    amplitude_fn(circ, bitstrings, picks) -> complex amplitudes of one
    trajectory (e.g. statevector.amplitudes or a tn-based routine).
    """
    bits = np.asarray(bitstrings)
    acc = np.zeros(len(bits))
    acc2 = np.zeros(len(bits))
    for t in range(n_traj):
        picks = trajectory_picks(circ, seed, t)
        p = np.abs(amplitude_fn(circ, bits, picks)) ** 2
        acc += p
        acc2 += p * p
    mean = acc / n_traj
    var = np.maximum(acc2 / n_traj - mean * mean, 0.0)
    stderr = np.sqrt(var / max(n_traj - 1, 1))
    return mean, stderr
