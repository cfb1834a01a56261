"""GPU parity of marginal wave-function slices (Sec. 4.4) against the FP64
oracle: qubits marked -1 stay open and each bitstring of the other qubits
yields 2^n_open amplitudes.  Tolerance as for amplitudes (relative L2 error
over all returned entries): FP32 and TF32x3 <= 1e-5, BF16x3 <= 2e-5."""
import numpy as np
import pytest

from oracle import statevector as sv
from workloads import ghz_circuit, grid_circuit, random_bitstrings

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


def marked(bits, open_q):
    b = np.array(bits, dtype=np.int8, copy=True)
    b[:, open_q] = -1
    return b


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("w,cap", [(2, 28), (0, 6)])
def test_slice_grid_3x4(T, prec, w, cap):
    c = grid_circuit(3, 4, 8, 1234)
    open_q = [2, 7]
    bits = marked(random_bitstrings(12, 13, 41), open_q)   # 13: three full batches of 4 and a ragged one
    ref = sv.wavefunction_slice(c, bits)
    ctx = T.Context(0, prec)
    plan = T.Plan(T.Circuit(c), open_qubits=open_q, batch_log2=w, max_intermediate_log2=cap,
                  path_mode=T.TNQ_PATH_BEST, n_candidates=8, seed=1)
    assert plan.info["n_open"] == 2
    if cap == 6:
        assert plan.info["n_sliced"] >= 1
    ctx.bind(plan)
    if prec != "fp32":
        T.tnq_ctx_set_kernel_policy(ctx.h, T.TNQ_KERNELS_TENSOR_CORES)
    got = ctx.amplitudes(plan, bits)
    assert got.shape == (13, 4)
    assert rel_l2(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16x3"])
def test_slice_grid_4x5_six_open(T, prec):
    c = grid_circuit(4, 5, 10, 2021)
    open_q = [0, 3, 7, 12, 15, 19]
    bits = marked(random_bitstrings(20, 16, 9), open_q)
    ref = sv.wavefunction_slice(c, bits)
    ctx = T.Context(0, prec)
    plan = T.Plan(T.Circuit(c), open_qubits=open_q, batch_log2=4, path_mode=T.TNQ_PATH_BEST, n_candidates=32,
                  seed=2)
    ctx.bind(plan)
    got = ctx.amplitudes(plan, bits)
    assert got.shape == (16, 64)
    assert rel_l2(got, ref) <= TOL[prec]


def test_cat_state_60_qubits(T):
    """The paper's Fig. 9 example: cat state on 60 qubits, qubits 2 and 47
    open.  Others all 0 -> [1,0,0,0]/sqrt2, all 1 -> [0,0,0,1]/sqrt2, mixed -> 0."""
    n = 60
    bits = np.zeros((4, n), dtype=np.int8)
    bits[1] = 1
    bits[2, 10] = 1
    bits[3, ::2] = 1
    bits[:, [2, 47]] = -1
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(ghz_circuit(n)), open_qubits=[47, 2], batch_log2=2)
    ctx.bind(plan)
    got = ctx.amplitudes(plan, bits)
    s = 1 / np.sqrt(2)
    want = np.array([[s, 0, 0, 0], [0, 0, 0, s], [0, 0, 0, 0], [0, 0, 0, 0]])
    assert np.allclose(got, want, atol=1e-7)


def test_device_buffers_and_graph_replay(T):
    import torch
    c = grid_circuit(3, 4, 8, 5)
    open_q = [0, 5, 11]
    bits = marked(random_bitstrings(12, 8, 3), open_q)
    ref = sv.wavefunction_slice(c, bits)
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(c), open_qubits=open_q, batch_log2=2)
    ctx.bind(plan)
    T.tnq_ctx_set_graphs(ctx.h, False)
    direct = ctx.amplitudes(plan, bits)
    T.tnq_ctx_set_graphs(ctx.h, True)
    out = ctx.amplitudes(plan, torch.from_numpy(bits).cuda()).cpu().numpy()
    dev = (out[:, 0] + 1j * out[:, 1]).reshape(8, 8)
    assert np.array_equal(dev, direct)
    assert rel_l2(direct, ref) <= TOL["fp32"]


def test_open_marker_required(T):
    import torch
    c = grid_circuit(3, 4, 8, 5)
    ctx = T.Context(0, "fp32")
    plan = T.Plan(T.Circuit(c), open_qubits=[3], batch_log2=1)
    ctx.bind(plan)
    bits = random_bitstrings(12, 2, 1)   # no -1 at qubit 3
    for b in (bits, torch.from_numpy(bits).cuda()):
        with pytest.raises(T.TnqError) as e:
            ctx.amplitudes(plan, b)
        assert e.value.status == T.TNQ_ERR_INVALID_ARG
    bad = marked(bits, [3])
    bad[0, 5] = -1   # -1 on a projected qubit
    with pytest.raises(T.TnqError):
        ctx.amplitudes(plan, bad)
