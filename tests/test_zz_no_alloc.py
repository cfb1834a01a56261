"""The allocation-free pairwise contraction (tnq_contract_pair_noalloc).

It serves callers that may not allocate device memory while running (a program
whose own pool owns the device memory, a loop that cannot take the
synchronisation of freeing memory); its scratch is a fixed static array inside
the library.  Each case calls it twice in a row on different operands (the
second call runs on the scratch the first one left behind) and checks that:
  * the result is bitwise the one of the workspace-taking tnq_contract_pair
    (same kernels, same split of the work), and within the contraction tests'
    tolerance of the FP64 oracle (oracle.contraction);
  * the second call leaves the device's free memory unchanged (the first call
    on a device may commit the library module that holds the array).
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from oracle import contraction
from workloads import microbench_case

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 2e-5, "tf32": 5e-3}


@pytest.fixture(scope="module")
def T():
    from paper_2104_10523_gb300 import build, tnq
    build.build()
    tnq.load()
    return tnq


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("mnk", [(6, 6, 6), (2, 2, 16), (3, 9, 8), (7, 5, 6)])
def test_noalloc_matches_workspace_entry_point(T, prec, mnk):
    import torch
    m, n, k = mnk
    ctx = T.Context(0, prec)
    for rep in range(2):
        al, bl, ol, A, B = microbench_case(m, n, k, seed=31 * rep + m + n + k)
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        want = torch.full((2 ** len(ol),), float("nan"), dtype=torch.complex64, device="cuda")
        got = torch.full((2 ** len(ol),), float("nan"), dtype=torch.complex64, device="cuda")
        nb = T.tnq_contract_workspace_bytes(T.PRECISIONS[prec], len(al), len(bl), len(ol))
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        T.tnq_contract_pair(ctx.h, At, al, Bt, bl, want, ol, ws, nb)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        T.tnq_contract_pair_noalloc(ctx.h, At, al, Bt, bl, got, ol)
        torch.cuda.synchronize()
        if rep == 1:
            assert torch.cuda.mem_get_info()[0] == free_before, "the call changed the device's free memory"
        w, g = want.cpu().numpy(), got.cpu().numpy()
        assert np.array_equal(g, w), (prec, mnk, rep)
        ref = contraction.contract_labeled(A, al, B, bl, ol)
        assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= TOL[prec], (prec, mnk, rep)


def test_noalloc_rejects_oversized(T):
    import torch
    ctx = T.Context(0, "fp32")
    A = torch.zeros(4, dtype=torch.complex64, device="cuda")
    al, bl, ol = list(range(22)), list(range(22)), []   # needs far more than the static scratch
    with pytest.raises(T.TnqError) as e:
        T.tnq_contract_pair_noalloc(ctx.h, A, al, A, bl, A, ol)
    assert e.value.status == T.TNQ_ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
