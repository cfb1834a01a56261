"""Host-side checks of libtnq: it loads, exports every symbol of include/tnq.h,
validates its inputs, and plans consistently.  No GPU compute is called."""
import math
import os
import re

import numpy as np
import pytest

from paper_2104_10523_gb300 import build as tnq_build
from paper_2104_10523_gb300 import tnq
from workloads import (amplitude_damping, depolarizing, ghz_circuit, grid_circuit,
                       noisy_grid_circuit)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    tnq_build.build()
    return tnq.load()


def test_exports_match_header():
    hdr = open(os.path.join(ROOT, "include", "tnq.h")).read()
    declared = set(re.findall(r"\b(tnq_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(tnq.EXPORTS)
    L = tnq.load()
    for name in declared:
        assert hasattr(L, name), name
    assert "sm_103a" in tnq.tnq_version()


def test_circuit_validation():
    h = tnq.tnq_circuit_create(3)
    with pytest.raises(tnq.TnqError) as e:
        tnq.tnq_circuit_gate(h, [0], np.array([[1, 1], [0, 1]]))
    assert e.value.status == tnq.TNQ_ERR_INVALID_ARG
    with pytest.raises(tnq.TnqError):
        tnq.tnq_circuit_gate(h, [0, 3], np.eye(4))
    with pytest.raises(tnq.TnqError):
        tnq.tnq_circuit_gate(h, [1, 1], np.eye(4))
    with pytest.raises(tnq.TnqError):
        tnq.tnq_circuit_channel(h, [0], [0.5 * np.eye(2)])  # incomplete Kraus set
    tnq.tnq_circuit_channel(h, [0], depolarizing(0.1))
    tnq.tnq_circuit_channel(h, [2], amplitude_damping(0.2))
    with pytest.raises(tnq.TnqError):
        tnq.tnq_circuit_create(0)
    tnq.tnq_circuit_destroy(h)


def _plan(circ, **kw):
    return tnq.Plan(tnq.Circuit(circ), **kw)


@pytest.mark.parametrize("mode", [tnq.TNQ_PATH_GREEDY, tnq.TNQ_PATH_BISECT, tnq.TNQ_PATH_BEST])
@pytest.mark.parametrize("w", [0, 3, 6])
def test_plan_step_accounting(mode, w):
    p = _plan(grid_circuit(3, 4, 8, 1234), batch_log2=w, path_mode=mode, n_candidates=8, seed=3)
    info = p.info
    st = p.steps()
    assert info["n_steps"] == info["n_leaves"] - 1
    flops = sum(8.0 * 2.0 ** (r[3] + r[4] + r[5] + r[6]) for r in st)
    assert math.isclose(flops, info["flops_per_pass"], rel_tol=1e-12)
    # slice-invariant steps run once per batch, the rest once per slice
    inv = [bool(r[7] & 4) for r in st]
    per = [8.0 * 2.0 ** (r[3] + r[4] + r[5] + r[6]) for r in st]
    want = sum(f if i else f * 2 ** info["n_sliced"] for f, i in zip(per, inv))
    assert math.isclose(info["flops_per_batch"], want, rel_tol=1e-12)
    if info["n_sliced"] == 0:
        assert all(inv)
    else:
        assert not inv[-1]  # the root holds every leaf, sliced ones included

    # GEMM shape consistency: a = K+M+H bits, b = K+N+H bits, out = N+M+H bits
    for r in st:
        assert r[0] == r[6] + r[4] + r[3]
        assert r[1] == r[6] + r[5] + r[3]
        assert r[2] == r[5] + r[4] + r[3]
    # the root holds exactly the batch bits
    assert st[-1][2] == w


def test_slicing_meets_cap():
    c = grid_circuit(4, 4, 10, 5)
    full = _plan(c, max_intermediate_log2=30, path_mode=tnq.TNQ_PATH_GREEDY)
    cap = max(full.info["max_log2"] - 4, 6)
    p = _plan(c, max_intermediate_log2=cap, path_mode=tnq.TNQ_PATH_GREEDY)
    assert p.info["max_log2"] <= cap
    assert p.info["n_sliced"] >= 1
    assert all(max(r[0], r[1], r[2]) <= cap for r in p.steps())


def test_plan_infeasible_when_batch_exceeds_cap():
    with pytest.raises(tnq.TnqError) as e:
        _plan(grid_circuit(2, 2, 4, 1), batch_log2=10, max_intermediate_log2=8)
    assert e.value.status == tnq.TNQ_ERR_PLAN_INFEASIBLE


def test_plan_deterministic():
    a = _plan(grid_circuit(3, 3, 6, 9), path_mode=tnq.TNQ_PATH_BEST, n_candidates=6, seed=11)
    b = _plan(grid_circuit(3, 3, 6, 9), path_mode=tnq.TNQ_PATH_BEST, n_candidates=6, seed=11)
    assert np.array_equal(a.steps(), b.steps())
    assert a.info["flops_per_batch"] == b.info["flops_per_batch"]


def test_plan_ghz_60_is_cheap():
    p = _plan(ghz_circuit(60), batch_log2=2, path_mode=tnq.TNQ_PATH_GREEDY)
    assert p.info["max_log2"] <= 8


def test_noisy_plan_carries_trajectory_bits():
    c = noisy_grid_circuit(2, 3, 4, seed=1, p_depol=1e-3, gamma=1e-3)
    p = _plan(c, batch_log2=2, traj_log2=3, path_mode=tnq.TNQ_PATH_GREEDY)
    assert p.info["traj_log2"] == 3
    assert p.steps()[-1][2] == 5  # root = batch bits + trajectory bits


def test_ctx_create_without_gpu_reports_no_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tnq.TnqError) as e:
        tnq.tnq_ctx_create(0, None, tnq.TNQ_PREC_FP32)
    assert e.value.status == tnq.TNQ_ERR_NO_DEVICE
