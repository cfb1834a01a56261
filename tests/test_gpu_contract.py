"""GPU parity of one pairwise contraction (permute + complex GEMM) in every
precision mode against the FP64 oracle (oracle.contraction).

Operands are the seeded microbenchmark pairs (all index dimensions 2, shared
indices scattered by a seeded permutation, entries complex normal / sqrt(K)).
Small cases compare every output entry; large ones compare sampled output rows
that the oracle computes one by one.  Shapes with a tiny output and a long
contracted dimension exercise the split-K path (FP32 partials, ordered sum).  Bound on the relative L2 error per mode
for a single contraction: FP32 and TF32x3 1e-5, BF16x3 2e-5, TF32 5e-3.
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


def _run(T, prec, A, al, B, bl, ol):
    import torch
    ctx = T.Context(0, prec)
    At = torch.from_numpy(A).cuda()
    Bt = torch.from_numpy(B).cuda()
    Ct = torch.full((2 ** len(ol),), float("nan"), dtype=torch.complex64, device="cuda")
    nb = T.tnq_contract_workspace_bytes(T.PRECISIONS[prec], len(al), len(bl), len(ol))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    T.tnq_contract_pair(ctx.h, At, al, Bt, bl, Ct, ol, ws, nb)
    torch.cuda.synchronize()
    return Ct.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("mnk", [(2, 3, 4), (6, 6, 6), (7, 5, 8), (3, 9, 10), (8, 8, 2), (6, 8, 10),
                                 (2, 2, 18), (0, 1, 16), (5, 6, 14), (9, 4, 12), (3, 3, 14), (3, 2, 12),
                                 (4, 10, 5), (2, 12, 0), (12, 3, 3), (5, 12, 5), (12, 5, 4), (1, 13, 3),
                                 (3, 18, 3), (17, 4, 4), (5, 16, 5), (0, 15, 2), (6, 14, 6), (15, 6, 5),
                                 (6, 13, 3), (7, 14, 4), (13, 7, 5)])
def test_full_output(T, prec, mnk):
    m, n, k = mnk
    al, bl, ol, A, B = microbench_case(m, n, k, seed=m * 100 + n * 10 + k)
    C = _run(T, prec, A, al, B, bl, ol)
    ref = contraction.contract_labeled(A, al, B, bl, ol)
    assert np.all(np.isfinite(C))
    assert rel(C, ref) <= TOL[prec], (prec, mnk, rel(C, ref))


@pytest.mark.parametrize("prec", ["fp32", "tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("mnk", [(10, 10, 12), (12, 8, 14), (8, 14, 8)])
def test_sampled_rows(T, prec, mnk):
    m, n, k = mnk
    al, bl, ol, A, B = microbench_case(m, n, k, seed=7 + m + n + k)
    C = _run(T, prec, A, al, B, bl, ol)
    rows = np.random.default_rng(1).choice(2 ** m, size=16, replace=False)
    ref = contraction.sampled_rows(A, al, B, bl, ol, rows, ol[:m])
    got = C.reshape(2 ** n, 2 ** m).T[rows]
    assert rel(got, ref) <= TOL[prec], (prec, mnk, rel(got, ref))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_batch_labels(T, prec):
    """Labels held by A, B and C are batch indices (the batched-GEMM case)."""
    rng = np.random.default_rng(5)
    al = [0, 1, 2, 3, 4, 5, 6, 7, 20, 21]         # 20, 21: batch; 4..7 contracted
    bl = [21, 4, 5, 6, 7, 8, 9, 10, 11, 20]
    ol = [8, 0, 9, 1, 20, 2, 10, 3, 11, 21]
    A = (rng.standard_normal(2 ** 10) + 1j * rng.standard_normal(2 ** 10)).astype(np.complex64)
    B = (rng.standard_normal(2 ** 10) + 1j * rng.standard_normal(2 ** 10)).astype(np.complex64)
    C = _run(T, prec, A, al, B, bl, ol)
    ref = contraction.contract_labeled(A, al, B, bl, ol)
    assert rel(C, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("shape", [(3, 14, 3), (7, 12, 5)])
def test_tall_skinny_batch(T, prec, shape):
    """A tall-skinny step with batch labels (2^s x 2^g output per batch entry,
    K = 2^k, 2^2 batch entries, every operand's bits scattered): the large
    operand is gathered in place and the small one expanded per batch entry
    (with 2^7 small rows, one launch per batch entry)."""
    ns, ng, nk = shape
    rng = np.random.default_rng(11 + ns)
    small, big = list(range(40, 40 + ns)), list(range(60, 60 + ng))
    kl, hl = list(range(nk)), [100, 101]
    al = list(rng.permutation(small + kl + hl))
    bl = list(rng.permutation(big + kl + hl))
    ol = list(rng.permutation(small + big + hl))
    A = (rng.standard_normal(2 ** len(al)) + 1j * rng.standard_normal(2 ** len(al))).astype(np.complex64)
    B = (rng.standard_normal(2 ** len(bl)) + 1j * rng.standard_normal(2 ** len(bl))).astype(np.complex64)
    C = _run(T, prec, A, al, B, bl, ol)
    ref = contraction.contract_labeled(A, al, B, bl, ol)
    assert np.all(np.isfinite(C))
    assert rel(C, ref) <= TOL[prec], (prec, rel(C, ref))


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("both", [False, True])
def test_dot_in_place(T, prec, both):
    """A dot-shaped contraction (2^3 x 2^3 outputs, K = 2^14, 2^2 batch
    entries) whose larger operand stores seven K labels lowest: the dot kernel
    reads it in place, K ordered by it; with `both` the other operand stores
    its K labels in the same order (other labels between them) and neither is
    permuted."""
    rng = np.random.default_rng(23)
    kl, ml, nl, hl = list(range(14)), [20, 21, 22], [30, 31, 32], [40, 41]
    bl = kl[:7] + [30, 40] + kl[7:] + [31, 41, 32]
    if both:
        al = kl[:7] + [20, 40] + kl[7:11] + [21] + kl[11:] + [41, 22]
    else:
        al = list(rng.permutation(kl + ml + hl))
    ol = list(rng.permutation(ml + nl + hl))
    A = (rng.standard_normal(2 ** 19) + 1j * rng.standard_normal(2 ** 19)).astype(np.complex64)
    B = (rng.standard_normal(2 ** 19) + 1j * rng.standard_normal(2 ** 19)).astype(np.complex64)
    C = _run(T, prec, A, al, B, bl, ol)
    ref = contraction.contract_labeled(A, al, B, bl, ol)
    assert np.all(np.isfinite(C))
    assert rel(C, ref) <= TOL[prec], (prec, rel(C, ref))


def test_invalid_labels_rejected(T):
    import torch
    ctx = T.Context(0, "fp32")
    A = torch.zeros(4, dtype=torch.complex64, device="cuda")
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TnqError) as e:
        T.tnq_contract_pair(ctx.h, A, [0, 1], A, [1, 2], A, [0, 5], ws, 1 << 16)
    assert e.value.status == T.TNQ_ERR_INVALID_ARG


@pytest.mark.parametrize("prec", ["tf32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("shape", [(6, 16, 6), (5, 16, 6), (6, 15, 5), (4, 17, 6), (6, 14, 3),
                                   (6, 14, 8), (4, 15, 7), (2, 16, 8)])
def test_tall_skinny_long_k(T, prec, shape):
    """Tall-skinny steps of the benchmark's shape class (2^s <= 64 small rows,
    2^g large rows, K = 2^k up to 64, operand bits scattered) run on the
    tall-skinny tcgen05 kernel (timing kind 5) in every tensor-core mode; in
    TF32 with K = 64 a 128-row tile passes through shared memory in four
    K-parts; with K = 128 or 256 the expanded small operand is streamed from a
    global copy into each stage beside its K-part.  TF32x3 keeps the correction products in their own TMEM
    accumulator, so TF32x3 stays within a few FP32 roundings of the FP64
    result."""
    import torch
    ns, ng, nk = shape
    rng = np.random.default_rng(100 + ns + ng + nk)
    small, big, kl = list(range(40, 40 + ns)), list(range(60, 60 + ng)), list(range(nk))
    al = list(rng.permutation(small + kl))
    bl = list(rng.permutation(big + kl))
    ol = list(rng.permutation(small + big))
    A = ((rng.standard_normal(2 ** len(al)) + 1j * rng.standard_normal(2 ** len(al))) / 2 ** (nk / 2)).astype(np.complex64)
    B = (rng.standard_normal(2 ** len(bl)) + 1j * rng.standard_normal(2 ** len(bl))).astype(np.complex64)
    ctx = T.Context(0, prec)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Ct = torch.full((2 ** len(ol),), float("nan"), dtype=torch.complex64, device="cuda")
    nb = T.tnq_contract_workspace_bytes(T.PRECISIONS[prec], len(al), len(bl), len(ol))
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    T.tnq_ctx_set_timing(ctx.h, True)
    T.tnq_contract_pair(ctx.h, At, al, Bt, bl, Ct, ol, ws, nb)
    kinds = T.tnq_ctx_get_timings(ctx.h)[:, 0].astype(int)
    assert 5 in kinds, kinds
    C = Ct.cpu().numpy()
    rows = rng.choice(2 ** ns, size=min(8, 2 ** ns), replace=False)
    # sampled output rows of the small operand's index, exact in FP64
    ref = contraction.sampled_rows(A, al, B, bl, ol, rows, small)
    lab_rest = [l for l in ol if l not in small]
    got = np.empty_like(ref)
    for i, r in enumerate(rows):
        fix = {l: (int(r) >> j) & 1 for j, l in enumerate(small)}
        sub = C.reshape((2,) * len(ol))[tuple(fix[l] if l in fix else slice(None) for l in reversed(ol))]
        axes = [l for l in reversed(ol) if l not in fix]
        got[i] = np.transpose(sub, [axes.index(l) for l in reversed(lab_rest)]).reshape(-1)
    err = rel(got, ref)
    bound = {"tf32x3": 2e-6, "bf16x3": 2e-5, "tf32": 5e-3}[prec]
    print(f"tall-skinny {shape} {prec}: rel L2 vs FP64 {err:.2e}")
    assert err <= bound, (prec, shape, err)
