"""GPU parity at full size against stored FP64 oracle amplitudes.

* 6x6 grid, 14 cycles (seed 2104), intermediates capped at 2^28 elements: the
  benchmark workload, in the benchmark's launch configuration (4 bitstrings
  per pass, best of 2048 candidate trees, seed 7, autotuned kernels), against
  tests/golden/config3_amplitudes.txt (the FP64 tensor-network oracle O2).
* 5x5 grid, 14 cycles (seed 55): a deep circuit below full size, against
  tests/golden/grid5x5_amplitudes.txt (the FP64 statevector oracle O1).

Tolerance: relative L2 error over the stored bitstrings, per precision mode:
FP32 and TF32x3 <= 1e-5, TF32 <= 5e-3, and BF16x3 <= 5e-5 for these deep
networks.  The BF16x3 bound follows from its arithmetic: splitting an FP32
value into two BF16 parts leaves a relative representation error of about
2^-17, so one contraction carries an error of a few 1e-6 (4.4e-6 measured on
the tall-skinny steps of this workload); independent errors of the steps on a
chain of the contraction tree add in quadrature, and the chains here are up to
about a hundred steps long.
"""
import os

import numpy as np
import pytest

from oracle import golden
from workloads import grid_circuit, random_bitstrings

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 5e-5, "tf32": 5e-3}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def T():
    from paper_2104_10523_gb300 import build, tnq
    build.build()
    tnq.load()
    return tnq


@pytest.fixture(scope="module")
def config3(T):
    circ = grid_circuit(6, 6, 14, 2104)
    idx, ref = golden.read_amplitudes(os.path.join(HERE, "golden", "config3_amplitudes.txt"))
    bits = random_bitstrings(circ.n, 1024, 10523)[idx]
    circuit = T.Circuit(circ)
    plan = T.Plan(circuit, max_intermediate_log2=28, batch_log2=2, path_mode=T.TNQ_PATH_BEST,
                  n_candidates=2048, seed=7)
    assert plan.info["max_log2"] <= 28
    return circuit, plan, bits, ref


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "tf32"])
def test_config3_against_fp64_oracle(T, config3, prec):
    _, plan, bits, ref = config3
    ctx = T.Context(0, prec)
    ctx.bind(plan)
    amp = ctx.amplitudes(plan, bits)
    err = rel_l2(amp, ref)
    print(f"config3 {prec} default kernels: rel L2 vs FP64 {err:.3e}")
    assert err <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_config3_autotuned_against_fp64_oracle(T, config3, prec):
    """The benchmark's own launch configuration: kernels chosen by the autotuner."""
    _, plan, bits, ref = config3
    ctx = T.Context(0, prec)
    ctx.bind(plan)
    n_tc, n_cc = T.tnq_plan_autotune(ctx.h, plan.h, 2)
    amp = ctx.amplitudes(plan, bits)
    err = rel_l2(amp, ref)
    print(f"config3 {prec} autotuned ({n_tc} tensor-core, {n_cc} CUDA-core steps): rel L2 vs FP64 {err:.3e}")
    assert err <= TOL[prec]


def test_config3_golden_porter_thomas(config3):
    """Sanity of the stored values: for a random circuit, 2^n |amp|^2 averages
    to about 1 (Porter-Thomas); 16 samples give a loose window."""
    _, _, _, ref = config3
    m = float(np.mean(2.0 ** 36 * np.abs(ref) ** 2))
    assert 0.3 < m < 3.0, m


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3", "tf32"])
def test_grid5x5_deep_against_statevector(T, prec):
    circ = grid_circuit(5, 5, 14, 55)
    idx, ref = golden.read_amplitudes(os.path.join(HERE, "golden", "grid5x5_amplitudes.txt"))
    bits = random_bitstrings(circ.n, 64, 5505)[idx]
    ctx = T.Context(0, prec)
    plan = T.Plan(T.Circuit(circ), max_intermediate_log2=26, batch_log2=4, path_mode=T.TNQ_PATH_BEST,
                  n_candidates=64, seed=5)
    ctx.bind(plan)
    amp = ctx.amplitudes(plan, bits)
    err = rel_l2(amp, ref)
    if prec != "fp32":
        T.tnq_ctx_set_kernel_policy(ctx.h, T.TNQ_KERNELS_TENSOR_CORES)
        forced = ctx.amplitudes(plan, bits)
        err_forced = rel_l2(forced, ref)
        print(f"grid5x5 {prec}: rel L2 vs FP64 {err:.3e} (default kernels), {err_forced:.3e} (tensor cores forced)")
        assert err_forced <= TOL[prec]
    else:
        print(f"grid5x5 {prec}: rel L2 vs FP64 {err:.3e}")
    assert err <= TOL[prec]
