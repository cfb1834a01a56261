"""Seeded synthetic workloads shared by the CUDA path and the CPU oracle.

This package holds input data only: the gate and channel matrices that define a
circuit, the seeded choices that pick gates and edge patterns, random bitstrings
and random operand tensors.  It contains none of the method's arithmetic (no
network building, no contraction, no sampling of Kraus operators), so that both
sides can consume the same inputs without sharing any computation.
"""
from .circuits import (  # noqa: F401
    Op, Circuit, SQRT_X, SQRT_Y, SQRT_W, H, X, Y, Z, I2, CNOT, CZ, fsim,
    grid_edges, grid_circuit, noisy_grid_circuit, depolarizing, amplitude_damping,
    bell_circuit, ghz_circuit, inverse_circuit, random_bitstrings, cost_model_circuit,
    CONFIG_SMALL, CONFIG_LARGE, CONFIG_NOISY,
)
from .tensors import microbench_case, MICROBENCH_SHAPES  # noqa: F401
