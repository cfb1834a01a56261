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
    per = [8.0 * 2.0 ** (r[3] + r[4] + r[5] + r[6]) for r in st]
    inv = [bool(r[7] & 4) for r in st]
    fold = [bool(r[7] & 8) for r in st]
    batched = [bool(r[7] & 16) for r in st]
    # a slice-batched step keeps its sliced indices, so only the others add
    # up to the per-slice flops of the tree
    plain = sum(f for f, b in zip(per, batched) if not b)
    if not any(batched):
        assert math.isclose(plain, info["flops_per_pass"], rel_tol=1e-12)
    else:
        assert plain < info["flops_per_pass"]
    # folded steps run when the plan is bound, slice-invariant and slice-batched
    # steps once per batch, the rest once per slice
    want = sum(0.0 if fo else f if (i or b) else f * 2 ** info["n_sliced"]
               for f, i, fo, b in zip(per, inv, fold, batched))
    assert math.isclose(info["flops_per_batch"], want, rel_tol=1e-12)
    assert not any(fo and b for fo, b in zip(fold, batched))
    assert all(i for fo, i in zip(fold, inv) if fo)      # a constant subtree holds no sliced index
    assert not any(i for b, i in zip(batched, inv) if b)  # a slice-batched one does
    if info["n_sliced"] == 0:
        assert all(inv) and not any(batched)
    else:
        assert not inv[-1] and not batched[-1]  # the root holds every leaf and adds into the slice sum
    # with batch indices every projection leaf depends on the bitstrings, so
    # the root never folds
    assert not fold[-1]

    # GEMM shape consistency: a = K+M+H bits, b = K+N+H bits, out = N+M+H bits
    for r in st:
        assert r[0] == r[6] + r[4] + r[3]
        assert r[1] == r[6] + r[5] + r[3]
        assert r[2] == r[5] + r[4] + r[3]
    # the root holds exactly the batch bits
    assert st[-1][2] == w


def test_folded_and_slice_batched_steps():
    """A sliced plan of a deep circuit has constant subtrees (folded at bind)
    and small slice-dependent subtrees that keep their sliced indices."""
    p = _plan(grid_circuit(4, 4, 10, 5), max_intermediate_log2=9, batch_log2=2, path_mode=tnq.TNQ_PATH_GREEDY)
    st = p.steps()
    assert p.info["n_sliced"] >= 2
    assert any(r[7] & 8 for r in st)
    assert any(r[7] & 16 for r in st)
    assert all(max(r[0], r[1], r[2]) <= 16 for r in st if r[7] & 16)


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


@pytest.mark.parametrize("rows,cols,cycles,w", [(3, 4, 8, 0), (3, 4, 8, 2), (4, 4, 10, 0)])
def test_exported_tree_followed_by_oracle(rows, cols, cycles, w):
    """tnq_plan_get_tree / tnq_plan_get_leaf_wires describe a valid contraction
    of the circuit network: the oracle cuts its own network at the exported
    wires into exactly the plan's groups, follows the tree with its own
    slicing, and gets the statevector amplitudes."""
    from oracle import statevector as sv
    from oracle import tn as otn
    from workloads import random_bitstrings
    circ = grid_circuit(rows, cols, cycles, 7)
    p = _plan(circ, max_intermediate_log2=12, batch_log2=w, path_mode=tnq.TNQ_PATH_BEST, n_candidates=8, seed=2)
    pairs, gw = p.tree(), p.leaf_wires()
    assert pairs.shape == (p.info["n_steps"], 2) and len(gw) == p.info["n_leaves"]
    # every id is used once as an operand; results only after they exist
    used = sorted(int(x) for x in pairs.ravel())
    assert used == list(range(p.info["n_leaves"] + p.info["n_steps"] - 1))
    assert all(max(a, b) < p.info["n_leaves"] + j for j, (a, b) in enumerate(pairs))
    # batch labels appear as (-1, -1) on projection leaves only
    assert sum(1 for g in gw for q, _ in g if q < 0) == circ.n * w
    bits = random_bitstrings(circ.n, 3, 11)
    ref = sv.amplitudes(circ, bits)
    for b, want in zip(bits, ref):
        net, wires = otn.build_network_wires(circ, b)
        order = otn.order_from_groups(net, wires, gw, pairs)
        sl = otn.choose_slices(net, order, 7)
        got = complex(np.asarray(otn.contract_sliced(net, sl, order)).reshape(()))
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def test_leaf_wires_rejects_bad_leaf():
    p = _plan(grid_circuit(2, 2, 2, 1))
    with pytest.raises(tnq.TnqError):
        tnq.tnq_plan_get_leaf_wires(p.h, p.info["n_leaves"])


def test_stored_config3_tree_matches_oracle_network():
    """The stored tree of the benchmark circuit partitions the oracle's own
    network (every group found, nothing left over) for a few bitstrings."""
    from oracle import golden
    from oracle import tn as otn
    from workloads import random_bitstrings
    circ = grid_circuit(6, 6, 14, 2104)
    gw, pairs = golden.read_tree(os.path.join(ROOT, "tests", "golden", "config3_order.txt"))
    for b in random_bitstrings(36, 1024, 10523)[:3]:
        net, wires = otn.build_network_wires(circ, b)
        order = otn.order_from_groups(net, wires, gw, pairs)
        assert len(order) == len(net) - 1
        flops, mx = otn.order_cost(otn.fix_labels(net, {l: 0 for l in otn.choose_slices(net, order, 24)}), order)
        assert mx <= 24 and flops < 1e11


def test_kernel_policy_validation():
    """Only the two documented kernel policies are accepted (checked before any
    device work, so this runs without a GPU)."""
    L = tnq.load()
    assert L.tnq_ctx_set_kernel_policy(None, 1) == tnq.TNQ_ERR_INVALID_ARG


def test_open_plan_validation():
    c = tnq.Circuit(grid_circuit(3, 4, 8, 1))
    for bad in ([12], [3, 3], [-1]):
        with pytest.raises(tnq.TnqError) as e:
            tnq.Plan(c, open_qubits=bad)
        assert e.value.status == tnq.TNQ_ERR_INVALID_ARG
    with pytest.raises(tnq.TnqError) as e:
        tnq.Plan(c, open_qubits=list(range(6)), max_intermediate_log2=5)
    assert e.value.status == tnq.TNQ_ERR_PLAN_INFEASIBLE
    p = tnq.Plan(c, open_qubits=[1, 6], batch_log2=2)
    assert p.info["n_open"] == 2
    # the root keeps the batch and open indices; no projection leaf for open qubits
    assert p.steps()[-1][2] == 4
    assert sum(1 for g in p.leaf_wires() if len(g) == 3 and g[1] == (-1, -1)) == 10
    noisy = tnq.Circuit(noisy_grid_circuit(2, 2, 2, 1, 1e-3, 1e-3))
    with pytest.raises(tnq.TnqError) as e:
        tnq.Plan(noisy, open_qubits=[0])
    assert e.value.status == tnq.TNQ_ERR_NOT_SUPPORTED


def test_expectation_plan_validation():
    c = tnq.Circuit(grid_circuit(2, 2, 2, 1))
    with pytest.raises(tnq.TnqError) as e:
        tnq.Plan(c, paulis=["XQII"])
    assert e.value.status == tnq.TNQ_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        tnq.Plan(c, paulis=["XI"])
    p = tnq.Plan(c, paulis=["ZIII", "IXII", "IIYZ"], traj_log2=6)
    # the terms share one contraction per pass: 2 term bits are enough for 3 terms
    assert p.info["traj_log2"] == 2
    noisy = tnq.Circuit(noisy_grid_circuit(2, 2, 2, 1, 1e-3, 1e-3))
    with pytest.raises(tnq.TnqError) as e:
        tnq.Plan(noisy, paulis=["ZIII"])
    assert e.value.status == tnq.TNQ_ERR_NOT_SUPPORTED
