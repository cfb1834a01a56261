"""Multi-rank logic on CPU: 2 gloo ranks shard the slices of a sliced
contraction and all-reduce the FP64 partial amplitudes; the result equals the
unsliced amplitude.  Partial sums per slice block come from the oracle's
sliced contraction (test side); the partition and the reduction are the
package's."""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_2104_10523_gb300 import parallel


def test_block_range_partitions():
    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            covered = []
            for r in range(world):
                b, c = parallel.block_range(r, world, n)
                covered.extend(range(b, b + c))
            assert covered == list(range(n))
    with pytest.raises(ValueError):
        parallel.block_range(2, 2, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from oracle import tn
    from workloads import grid_circuit, random_bitstrings
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        circ = grid_circuit(3, 3, 6, 17)
        bits = random_bitstrings(9, 3, 4)
        results = []
        for x in bits:
            net = tn.build_network(circ, x)
            labels = sorted({l for _, ls in net for l in ls})[:4]   # 2^4 = 16 slices
            assigns = list(itertools.product((0, 1), repeat=len(labels)))
            b, c = parallel.block_range(rank, world, len(assigns))
            part = 0j
            order = tn.greedy_order(net)
            for vals in assigns[b:b + c]:
                part += complex(tn.contract(tn.fix_labels(net, dict(zip(labels, vals))), order)[0])
            results.append([part.real, part.imag])
        total = parallel.allreduce_partials(np.array(results))
        q.put((rank, total.tolist()))
    finally:
        dist.destroy_process_group()


def test_slice_sharding_two_gloo_ranks():
    import multiprocessing as mp
    from oracle import statevector as sv
    from workloads import grid_circuit, random_bitstrings
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circ = grid_circuit(3, 3, 6, 17)
    ref = sv.amplitudes(circ, random_bitstrings(9, 3, 4))
    for r in (0, 1):
        got = np.array(out[r])
        assert np.allclose(got[:, 0] + 1j * got[:, 1], ref, atol=1e-13)
