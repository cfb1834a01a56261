"""Slice sharding end to end: two gloo ranks (separate processes sharing this
GPU; their kernels never wait on one another, only the FP64 all-reduce on the
host joins them) each contract their block of the slices of a sliced plan
with parallel.amplitudes_slice_sharded, and every rank gets the amplitudes of
the whole sliced sum, checked against the statevector oracle."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2104_10523_gb300 import parallel, tnq
    from workloads import grid_circuit, random_bitstrings
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tnq.load()
        circ = grid_circuit(3, 4, 8, 1234)
        bits = random_bitstrings(12, 16, 99)
        ctx = tnq.Context(0, "tf32x3")
        plan = tnq.Plan(tnq.Circuit(circ), batch_log2=3, max_intermediate_log2=7, path_mode=0)
        ctx.bind(plan)
        amp = parallel.amplitudes_slice_sharded(ctx, plan, bits)
        q.put((rank, plan.info["n_sliced"], [[z.real, z.imag] for z in amp]))
    finally:
        dist.destroy_process_group()


def test_slice_sharded_amplitudes_two_ranks():
    import multiprocessing as mp
    from oracle import statevector as sv
    from workloads import grid_circuit, random_bitstrings
    from paper_2104_10523_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        r, n_sliced, amp = q.get(timeout=300)
        out[r] = (n_sliced, np.array(amp))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = sv.amplitudes(grid_circuit(3, 4, 8, 1234), random_bitstrings(12, 16, 99))
    for r in (0, 1):
        n_sliced, a = out[r]
        assert n_sliced >= 2
        got = a[:, 0] + 1j * a[:, 1]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    assert np.array_equal(out[0][1], out[1][1])
