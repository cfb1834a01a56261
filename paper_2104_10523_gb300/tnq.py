"""ctypes binding of libtnq (include/tnq.h): same names, argument marshalling only.

Every step of the contraction runs inside libtnq's own CUDA kernels; this
module only converts Python/NumPy/torch arguments to the C ABI.  Loading fails
loudly when the library has not been built (``paper_2104_10523_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TNQ_OK = 0
TNQ_ERR_INVALID_ARG = 1
TNQ_ERR_PLAN_INFEASIBLE = 2
TNQ_ERR_WORKSPACE = 3
TNQ_ERR_CUDA = 4
TNQ_ERR_TIMEOUT = 5
TNQ_ERR_NOT_SUPPORTED = 6
TNQ_ERR_NO_DEVICE = 7

TNQ_PREC_FP32, TNQ_PREC_TF32, TNQ_PREC_TF32X3, TNQ_PREC_BF16X3 = 0, 1, 2, 3
PRECISIONS = {"fp32": 0, "tf32": 1, "tf32x3": 2, "bf16x3": 3}
TNQ_PATH_GREEDY, TNQ_PATH_BISECT, TNQ_PATH_BEST, TNQ_PATH_LEARNED = 0, 1, 2, 3
TNQ_KERNELS_DEFAULT, TNQ_KERNELS_TENSOR_CORES = 0, 1

# Every exported symbol of include/tnq.h (checked by the CPU tests).
EXPORTS = (
    "tnq_version", "tnq_status_string", "tnq_last_error",
    "tnq_circuit_create", "tnq_circuit_destroy", "tnq_circuit_gate", "tnq_circuit_channel",
    "tnq_circuit_n_qubits", "tnq_plan_create", "tnq_plan_destroy", "tnq_plan_get_info",
    "tnq_plan_get_steps", "tnq_ctx_create", "tnq_ctx_destroy", "tnq_ctx_set_precision",
    "tnq_plan_bind", "tnq_amplitudes", "tnq_noisy_probabilities",
    "tnq_contract_workspace_bytes", "tnq_contract_pair",
    "tnq_ctx_launch_count", "tnq_ctx_set_timing", "tnq_ctx_get_timings",
    "tnq_contract_pair_noalloc", "tnq_trajectory_amplitudes", "tnq_ctx_set_graphs",
    "tnq_step_feature_count", "tnq_cost_model_create", "tnq_cost_model_destroy", "tnq_cost_model_workspace_bytes",
    "tnq_cost_model_n_params", "tnq_cost_model_bind", "tnq_cost_model_set_params", "tnq_cost_model_get_params",
    "tnq_cost_model_gradients", "tnq_cost_model_train", "tnq_cost_model_predict", "tnq_plan_step_features",
    "tnq_plan_create_learned", "tnq_plan_get_candidates", "tnq_plan_autotune", "tnq_amplitudes_slices",
    "tnq_plan_get_tree", "tnq_plan_get_leaf_wires", "tnq_ctx_set_kernel_policy", "tnq_plan_create_open",
    "tnq_plan_create_density", "tnq_density_probabilities", "tnq_plan_create_expectation", "tnq_expectation",
)


class TnqOptions(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p), ("precision", C.c_int)]


class TnqPlanOpts(C.Structure):
    _fields_ = [("max_intermediate_log2", C.c_int), ("batch_log2", C.c_int), ("traj_log2", C.c_int),
                ("path_mode", C.c_int), ("n_candidates", C.c_int), ("seed", C.c_uint64)]


class TnqPlanInfo(C.Structure):
    _fields_ = [("n_leaves", C.c_int), ("n_steps", C.c_int), ("n_sliced", C.c_int), ("max_log2", C.c_int),
                ("batch_log2", C.c_int), ("traj_log2", C.c_int), ("flops_per_pass", C.c_double),
                ("flops_per_batch", C.c_double), ("bytes_per_pass", C.c_double), ("search_ms", C.c_double),
                ("workspace_bytes", C.c_size_t), ("n_open", C.c_int), ("distinct_trajectories", C.c_int64)]


class TnqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tnq status {status}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libtnq is not built ({path} missing); run paper_2104_10523_gb300.build.build()")
    L = C.CDLL(path)
    vp, ip, i32, i64, u64, dp, sz = C.c_void_p, C.POINTER(C.c_int), C.c_int, C.c_int64, C.c_uint64, \
        C.POINTER(C.c_double), C.c_size_t
    fp = C.POINTER(C.c_float)
    sig = {
        "tnq_version": ([], C.c_char_p),
        "tnq_status_string": ([i32], C.c_char_p),
        "tnq_last_error": ([], C.c_char_p),
        "tnq_circuit_create": ([i32, C.POINTER(vp)], i32),
        "tnq_circuit_destroy": ([vp], None),
        "tnq_circuit_gate": ([vp, i32, ip, dp], i32),
        "tnq_circuit_channel": ([vp, i32, ip, i32, dp], i32),
        "tnq_circuit_n_qubits": ([vp], i32),
        "tnq_plan_create": ([vp, C.POINTER(TnqPlanOpts), C.POINTER(vp)], i32),
        "tnq_plan_destroy": ([vp], None),
        "tnq_plan_get_info": ([vp, C.POINTER(TnqPlanInfo)], i32),
        "tnq_plan_get_steps": ([vp, ip], i32),
        "tnq_ctx_create": ([C.POINTER(TnqOptions), C.POINTER(vp)], i32),
        "tnq_ctx_destroy": ([vp], None),
        "tnq_ctx_set_precision": ([vp, i32], i32),
        "tnq_plan_bind": ([vp, vp, vp, sz], i32),
        "tnq_amplitudes": ([vp, vp, i64, vp, vp], i32),
        "tnq_noisy_probabilities": ([vp, vp, i64, u64, i64, vp, vp, vp], i32),
        "tnq_contract_workspace_bytes": ([i32, i32, i32, i32], sz),
        "tnq_contract_pair": ([vp, vp, i32, ip, vp, i32, ip, vp, i32, ip, vp, sz], i32),
        "tnq_ctx_launch_count": ([vp, C.POINTER(C.c_uint64)], i32),
        "tnq_ctx_set_timing": ([vp, i32], i32),
        "tnq_ctx_get_timings": ([vp, dp, i32, ip], i32),
        "tnq_contract_pair_noalloc": ([vp, vp, i32, ip, vp, i32, ip, vp, i32, ip], i32),
        "tnq_trajectory_amplitudes": ([vp, vp, u64, i64, i64, i64, vp, vp], i32),
        "tnq_ctx_set_graphs": ([vp, i32], i32),
        "tnq_step_feature_count": ([], i32),
        "tnq_cost_model_create": ([i32, i32, i32, u64, C.POINTER(vp)], i32),
        "tnq_cost_model_destroy": ([vp], None),
        "tnq_cost_model_workspace_bytes": ([vp], sz),
        "tnq_cost_model_n_params": ([vp], i64),
        "tnq_cost_model_bind": ([vp, vp, vp, sz], i32),
        "tnq_cost_model_set_params": ([vp, vp, fp], i32),
        "tnq_cost_model_get_params": ([vp, vp, fp], i32),
        "tnq_cost_model_gradients": ([vp, vp, fp, fp, i64, fp, fp], i32),
        "tnq_cost_model_train": ([vp, vp, fp, fp, i64, i32, i32, C.c_float, fp], i32),
        "tnq_cost_model_predict": ([vp, vp, fp, i64, fp], i32),
        "tnq_plan_step_features": ([vp, i32, fp], i32),
        "tnq_plan_create_learned": ([vp, vp, vp, C.POINTER(TnqPlanOpts), C.POINTER(vp)], i32),
        "tnq_plan_get_candidates": ([vp, dp, dp, i32, ip, ip, ip], i32),
        "tnq_plan_autotune": ([vp, vp, i32, ip, ip], i32),
        "tnq_amplitudes_slices": ([vp, vp, i64, vp, i64, i64, vp], i32),
        "tnq_plan_get_tree": ([vp, ip], i32),
        "tnq_plan_get_leaf_wires": ([vp, i32, i32, ip, ip], i32),
        "tnq_ctx_set_kernel_policy": ([vp, i32], i32),
        "tnq_plan_create_open": ([vp, C.POINTER(TnqPlanOpts), i32, ip, C.POINTER(vp)], i32),
        "tnq_plan_create_density": ([vp, C.POINTER(TnqPlanOpts), C.POINTER(vp)], i32),
        "tnq_density_probabilities": ([vp, vp, i64, vp, vp], i32),
        "tnq_plan_create_expectation": ([vp, C.POINTER(TnqPlanOpts), i64, C.c_char_p, C.POINTER(vp)], i32),
        "tnq_expectation": ([vp, vp, dp, dp, dp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def check(status: int):
    if status != TNQ_OK:
        raise TnqError(status, load().tnq_last_error().decode())


def _int_array(v):
    return (C.c_int * len(v))(*[int(x) for x in v])


def _ptr(x):
    """Data pointer of a torch tensor or a NumPy array (host or device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


# ---------------------------------------------------------------- thin wrappers
def tnq_version() -> str:
    return load().tnq_version().decode()


def tnq_circuit_create(n_qubits: int):
    h = C.c_void_p()
    check(load().tnq_circuit_create(int(n_qubits), C.byref(h)))
    return h


def tnq_circuit_destroy(h):
    load().tnq_circuit_destroy(h)


def tnq_circuit_gate(h, qubits, matrix):
    m = np.ascontiguousarray(np.asarray(matrix, np.complex128)).view(np.float64)
    check(load().tnq_circuit_gate(h, len(qubits), _int_array(qubits),
                                  m.ctypes.data_as(C.POINTER(C.c_double))))


def tnq_circuit_channel(h, qubits, kraus):
    k = np.ascontiguousarray(np.asarray(kraus, np.complex128)).view(np.float64)
    check(load().tnq_circuit_channel(h, len(qubits), _int_array(qubits), len(kraus),
                                     k.ctypes.data_as(C.POINTER(C.c_double))))


def tnq_plan_create(circ_h, max_intermediate_log2=28, batch_log2=0, traj_log2=0,
                    path_mode=TNQ_PATH_BEST, n_candidates=16, seed=0):
    o = TnqPlanOpts(max_intermediate_log2, batch_log2, traj_log2, path_mode, n_candidates, seed)
    h = C.c_void_p()
    check(load().tnq_plan_create(circ_h, C.byref(o), C.byref(h)))
    return h


def tnq_plan_create_open(circ_h, open_qubits, max_intermediate_log2=28, batch_log2=0, traj_log2=0,
                         path_mode=TNQ_PATH_BEST, n_candidates=16, seed=0):
    o = TnqPlanOpts(max_intermediate_log2, batch_log2, traj_log2, path_mode, n_candidates, seed)
    h = C.c_void_p()
    check(load().tnq_plan_create_open(circ_h, C.byref(o), len(open_qubits), _int_array(open_qubits), C.byref(h)))
    return h


def tnq_plan_create_density(circ_h, max_intermediate_log2=28, batch_log2=0, path_mode=TNQ_PATH_BEST,
                            n_candidates=16, seed=0):
    o = TnqPlanOpts(max_intermediate_log2, batch_log2, 0, path_mode, n_candidates, seed)
    h = C.c_void_p()
    check(load().tnq_plan_create_density(circ_h, C.byref(o), C.byref(h)))
    return h


def tnq_density_probabilities(ctx, plan, bits, p_out):
    """bits: int8 [n_bs][n] (host or device); p_out: float64 [n_bs] (same choices)."""
    check(load().tnq_density_probabilities(ctx, plan, int(bits.shape[0]), _ptr(bits), _ptr(p_out)))


def tnq_plan_create_expectation(circ_h, paulis, max_intermediate_log2=28, traj_log2=6, path_mode=TNQ_PATH_BEST,
                                n_candidates=16, seed=0):
    """paulis: list of strings over "IXYZ", one per term, each of length n_qubits."""
    n = load().tnq_circuit_n_qubits(circ_h)
    if any(len(ps) != n for ps in paulis):
        raise ValueError("every Pauli string must have one character per qubit")
    o = TnqPlanOpts(max_intermediate_log2, 0, traj_log2, path_mode, n_candidates, seed)
    h = C.c_void_p()
    check(load().tnq_plan_create_expectation(circ_h, C.byref(o), len(paulis), "".join(paulis).encode(), C.byref(h)))
    return h


def tnq_expectation(ctx, plan, coeffs):
    """(value, per-term values) for real coefficients [n_terms]."""
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    v = C.c_double()
    tv = np.zeros(c.shape[0])
    check(load().tnq_expectation(ctx, plan, c.ctypes.data_as(dp_t()), C.byref(v), tv.ctypes.data_as(dp_t())))
    return float(v.value), tv


def dp_t():
    return C.POINTER(C.c_double)


def tnq_plan_destroy(h):
    load().tnq_plan_destroy(h)


def tnq_plan_get_info(h) -> dict:
    info = TnqPlanInfo()
    check(load().tnq_plan_get_info(h, C.byref(info)))
    return {f: getattr(info, f) for f, _ in TnqPlanInfo._fields_}


def tnq_plan_get_steps(h, n_steps) -> np.ndarray:
    rec = np.zeros(8 * n_steps, dtype=np.int32)
    check(load().tnq_plan_get_steps(h, rec.ctypes.data_as(C.POINTER(C.c_int))))
    return rec.reshape(n_steps, 8)


def tnq_plan_get_tree(h, n_steps) -> np.ndarray:
    """[n_steps][2] tensor ids contracted by each step (leaves first, then step results)."""
    pairs = np.zeros(2 * max(n_steps, 1), dtype=np.int32)
    check(load().tnq_plan_get_tree(h, pairs.ctypes.data_as(C.POINTER(C.c_int))))
    return pairs[:2 * n_steps].reshape(n_steps, 2)


def tnq_plan_get_leaf_wires(h, leaf) -> list:
    """[(qubit, position), ...] of the leaf's indices ((-1, -1) = batch/trajectory index)."""
    n = C.c_int()
    check(load().tnq_plan_get_leaf_wires(h, int(leaf), 0, None, C.byref(n)))
    w = np.zeros(2 * max(n.value, 1), dtype=np.int32)
    check(load().tnq_plan_get_leaf_wires(h, int(leaf), n.value, w.ctypes.data_as(C.POINTER(C.c_int)), C.byref(n)))
    return [(int(w[2 * j]), int(w[2 * j + 1])) for j in range(n.value)]


def tnq_ctx_create(device=0, stream=None, precision=TNQ_PREC_FP32):
    o = TnqOptions(int(device), C.c_void_p(stream or 0), int(precision))
    h = C.c_void_p()
    check(load().tnq_ctx_create(C.byref(o), C.byref(h)))
    return h


def tnq_ctx_destroy(h):
    load().tnq_ctx_destroy(h)


def tnq_ctx_set_precision(h, precision):
    check(load().tnq_ctx_set_precision(h, int(precision)))


def tnq_plan_bind(ctx, plan, workspace, nbytes):
    check(load().tnq_plan_bind(ctx, plan, _ptr(workspace), int(nbytes)))


def tnq_amplitudes(ctx, plan, bits, out):
    """bits: int8 [n_bs][n] (NumPy host or torch device); out: float64 [n_bs][2] (same choices)."""
    n_bs = int(bits.shape[0])
    check(load().tnq_amplitudes(ctx, plan, n_bs, _ptr(bits), _ptr(out)))


def tnq_amplitudes_slices(ctx, plan, bits, slice_begin, slice_count, out):
    check(load().tnq_amplitudes_slices(ctx, plan, int(bits.shape[0]), _ptr(bits), int(slice_begin),
                                       int(slice_count), _ptr(out)))


def tnq_noisy_probabilities(ctx, plan, n_traj, seed, bits, p_out, se_out=None):
    check(load().tnq_noisy_probabilities(ctx, plan, int(n_traj), int(seed), int(bits.shape[0]), _ptr(bits),
                                         _ptr(p_out), _ptr(se_out)))


def tnq_trajectory_amplitudes(ctx, plan, seed, traj_begin, n_traj, bits, out):
    """out: float64 [n_traj][n_bs][2] (NumPy host or torch device)."""
    check(load().tnq_trajectory_amplitudes(ctx, plan, int(seed), int(traj_begin), int(n_traj), int(bits.shape[0]),
                                           _ptr(bits), _ptr(out)))


def tnq_contract_workspace_bytes(precision, ra, rb, rc) -> int:
    return int(load().tnq_contract_workspace_bytes(int(precision), int(ra), int(rb), int(rc)))


def tnq_contract_pair(ctx, A, a_labels, B, b_labels, Cout, c_labels, workspace, nbytes):
    check(load().tnq_contract_pair(ctx, _ptr(A), len(a_labels), _int_array(a_labels), _ptr(B), len(b_labels),
                                   _int_array(b_labels), _ptr(Cout), len(c_labels), _int_array(c_labels),
                                   _ptr(workspace), int(nbytes)))


def tnq_contract_pair_noalloc(ctx, A, a_labels, B, b_labels, Cout, c_labels):
    """tnq_contract_pair without a workspace argument (scratch is static in the library)."""
    check(load().tnq_contract_pair_noalloc(ctx, _ptr(A), len(a_labels), _int_array(a_labels), _ptr(B),
                                           len(b_labels), _int_array(b_labels), _ptr(Cout), len(c_labels),
                                           _int_array(c_labels)))


def tnq_plan_autotune(ctx, plan, reps=3):
    """Returns (steps on tensor cores, steps on CUDA cores) among the tuned steps."""
    a, b = C.c_int(), C.c_int()
    check(load().tnq_plan_autotune(ctx, plan, int(reps), C.byref(a), C.byref(b)))
    return a.value, b.value


def tnq_ctx_set_graphs(ctx, enable: bool):
    check(load().tnq_ctx_set_graphs(ctx, 1 if enable else 0))


def tnq_ctx_set_kernel_policy(ctx, policy: int):
    check(load().tnq_ctx_set_kernel_policy(ctx, int(policy)))


def tnq_ctx_launch_count(ctx) -> int:
    v = C.c_uint64()
    check(load().tnq_ctx_launch_count(ctx, C.byref(v)))
    return int(v.value)


def tnq_ctx_set_timing(ctx, enable: bool):
    check(load().tnq_ctx_set_timing(ctx, 1 if enable else 0))


TIMING_FIELDS = ("kind", "step", "log2_h", "log2_m", "log2_n", "log2_k", "flops", "bytes", "ms", "pad")


def tnq_ctx_get_timings(ctx) -> np.ndarray:
    """Per-kernel records [n][10] (see TIMING_FIELDS)."""
    n = C.c_int()
    check(load().tnq_ctx_get_timings(ctx, None, 0, C.byref(n)))
    rec = np.zeros((max(n.value, 1), 10), dtype=np.float64)
    check(load().tnq_ctx_get_timings(ctx, rec.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)))
    return rec[:n.value]


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def tnq_plan_step_features(plan_h, precision, n_steps) -> np.ndarray:
    d = load().tnq_step_feature_count()
    out = np.zeros((n_steps, d), dtype=np.float32)
    check(load().tnq_plan_step_features(plan_h, int(precision), _fptr(out)))
    return out


def tnq_plan_get_candidates(plan_h) -> dict:
    n, fm, ch = C.c_int(), C.c_int(), C.c_int()
    check(load().tnq_plan_get_candidates(plan_h, None, None, 0, C.byref(n), C.byref(fm), C.byref(ch)))
    fl = np.zeros(max(n.value, 1))
    pr = np.zeros(max(n.value, 1))
    check(load().tnq_plan_get_candidates(plan_h, fl.ctypes.data_as(C.POINTER(C.c_double)),
                                         pr.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n),
                                         C.byref(fm), C.byref(ch)))
    return {"flops": fl[:n.value], "predicted_ms": pr[:n.value], "flopmin": fm.value, "chosen": ch.value}


class CostModel:
    """Owns a tnq_cost_model and its device workspace (a torch tensor)."""

    def __init__(self, ctx, hidden=256, max_batch=4096, seed=0):
        import torch
        L = load()
        self.ctx = ctx
        self.d_in = L.tnq_step_feature_count()
        self.h = C.c_void_p()
        check(L.tnq_cost_model_create(self.d_in, hidden, max_batch, seed, C.byref(self.h)))
        nb = int(L.tnq_cost_model_workspace_bytes(self.h))
        self.ws = torch.empty(nb, dtype=torch.uint8, device=f"cuda:{ctx.device}")
        check(L.tnq_cost_model_bind(ctx.h, self.h, C.c_void_p(self.ws.data_ptr()), nb))
        self.n_params = int(L.tnq_cost_model_n_params(self.h))

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(load().tnq_cost_model_set_params(self.ctx.h, self.h, _fptr(p)))

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        check(load().tnq_cost_model_get_params(self.ctx.h, self.h, _fptr(p)))
        return p

    def gradients(self, X, t):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        check(load().tnq_cost_model_gradients(self.ctx.h, self.h, _fptr(X), _fptr(t), X.shape[0], _fptr(g),
                                              _fptr(loss)))
        return g, float(loss[0])

    def train(self, X, t, epochs=20, batch=1024, lr=1e-3):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        check(load().tnq_cost_model_train(self.ctx.h, self.h, _fptr(X), _fptr(t), X.shape[0], epochs, batch,
                                          C.c_float(lr), _fptr(loss)))
        return float(loss[0])

    def predict(self, X):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.zeros(X.shape[0], dtype=np.float32)
        check(load().tnq_cost_model_predict(self.ctx.h, self.h, _fptr(X), X.shape[0], _fptr(y)))
        return y

    def plan(self, circuit, **opts):
        """A Plan whose candidate tree is chosen by predicted time."""
        o = TnqPlanOpts(opts.get("max_intermediate_log2", 28), opts.get("batch_log2", 0), opts.get("traj_log2", 0),
                        opts.get("path_mode", TNQ_PATH_BEST), opts.get("n_candidates", 16), opts.get("seed", 0))
        h = C.c_void_p()
        check(load().tnq_plan_create_learned(self.ctx.h, self.h, circuit.h, C.byref(o), C.byref(h)))
        return Plan.from_handle(circuit, h)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tnq_cost_model_destroy(self.h)
            self.h = None


# ---------------------------------------------------------------- owning helpers
class Circuit:
    """Owns a tnq_circuit built from a workloads.Circuit (gates and channels in order)."""

    def __init__(self, circ):
        self.n = circ.n
        self.h = tnq_circuit_create(circ.n)
        for op in circ.ops:
            if op.kind == "gate":
                tnq_circuit_gate(self.h, op.qubits, op.mats[0])
            else:
                tnq_circuit_channel(self.h, op.qubits, np.stack(op.mats))

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tnq_circuit_destroy(self.h)
            self.h = None


class Plan:
    """Owns a tnq_plan; info() and steps() describe it."""

    def __init__(self, circuit: Circuit, open_qubits=None, density=False, paulis=None, **opts):
        self.circuit = circuit
        if paulis is not None:
            self.h = tnq_plan_create_expectation(circuit.h, list(paulis), **opts)
        elif density:
            self.h = tnq_plan_create_density(circuit.h, **opts)
        elif open_qubits:
            self.h = tnq_plan_create_open(circuit.h, list(open_qubits), **opts)
        else:
            self.h = tnq_plan_create(circuit.h, **opts)
        self.info = tnq_plan_get_info(self.h)
        self.workspace = None

    @classmethod
    def from_handle(cls, circuit, h):
        self = cls.__new__(cls)
        self.circuit = circuit
        self.h = h
        self.info = tnq_plan_get_info(h)
        self.workspace = None
        return self

    def steps(self):
        return tnq_plan_get_steps(self.h, self.info["n_steps"])

    def features(self, precision):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        return tnq_plan_step_features(self.h, prec, self.info["n_steps"])

    def candidates(self):
        return tnq_plan_get_candidates(self.h)

    def tree(self):
        return tnq_plan_get_tree(self.h, self.info["n_steps"])

    def leaf_wires(self):
        return [tnq_plan_get_leaf_wires(self.h, i) for i in range(self.info["n_leaves"])]

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tnq_plan_destroy(self.h)
            self.h = None


class Context:
    """Owns a tnq_ctx on a device and the torch stream it orders work on."""

    def __init__(self, device=0, precision="fp32", stream=None):
        import torch
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.h = tnq_ctx_create(device, self.stream.cuda_stream, prec)

    def set_precision(self, precision):
        tnq_ctx_set_precision(self.h, PRECISIONS[precision] if isinstance(precision, str) else int(precision))

    def bind(self, plan: Plan):
        import torch
        nbytes = int(plan.info["workspace_bytes"])
        plan.workspace = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        tnq_plan_bind(self.h, plan.h, plan.workspace, nbytes)

    def amplitudes(self, plan: Plan, bits):
        """complex128 amplitudes; bits: int8 NumPy [n_bs][n] (host) or a torch cuda int8 tensor.
        For a plan with open qubits the result is [n_bs][2^n_open]."""
        k = plan.info["n_open"]
        if hasattr(bits, "is_cuda") and bits.is_cuda:
            import torch
            out = torch.empty((bits.shape[0] << k, 2), dtype=torch.float64, device=bits.device)
            tnq_amplitudes(self.h, plan.h, bits, out)
            return out
        b = np.ascontiguousarray(bits, dtype=np.int8)
        out = np.empty((b.shape[0] << k, 2), dtype=np.float64)
        tnq_amplitudes(self.h, plan.h, b, out)
        amp = out[:, 0] + 1j * out[:, 1]
        return amp.reshape(b.shape[0], 2 ** k) if k else amp

    def density_probabilities(self, plan: Plan, bits):
        """Exact p(x) (float64 [n_bs]) of a density-matrix plan for host int8 bits [n_bs][n]."""
        b = np.ascontiguousarray(bits, dtype=np.int8)
        p = np.empty(b.shape[0], dtype=np.float64)
        tnq_density_probabilities(self.h, plan.h, b, p)
        return p

    def expectation(self, plan: Plan, coeffs):
        """(<psi|H|psi>, per-term <psi|P_t|psi>) for an expectation-value plan."""
        return tnq_expectation(self.h, plan.h, coeffs)

    def noisy_probabilities(self, plan: Plan, bits, n_traj, seed):
        """(p, stderr) as float64 arrays for host int8 bits [n_bs][n]."""
        b = np.ascontiguousarray(bits, dtype=np.int8)
        p = np.empty(b.shape[0], dtype=np.float64)
        se = np.empty(b.shape[0], dtype=np.float64)
        tnq_noisy_probabilities(self.h, plan.h, n_traj, seed, b, p, se)
        return p, se

    def trajectory_amplitudes(self, plan: Plan, bits, seed, traj_begin, n_traj):
        """complex128 [n_traj][n_bs] amplitudes of individual trajectories."""
        b = np.ascontiguousarray(bits, dtype=np.int8)
        out = np.empty((n_traj, b.shape[0], 2), dtype=np.float64)
        tnq_trajectory_amplitudes(self.h, plan.h, seed, traj_begin, n_traj, b, out)
        return out[..., 0] + 1j * out[..., 1]

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.tnq_ctx_destroy(self.h)
            self.h = None
