"""Seeded operand pairs for the pairwise-contraction microbenchmark.

Every index has dimension 2.  Operand A has rank m+k, operand B rank n+k; the k
shared (contracted) indices are scattered among the free ones by a seeded
permutation, so the contraction needs real index permutations.  Entries are
i.i.d. complex normal with Re, Im ~ N(0, 1/2), scaled by 1/sqrt(2^k) so that
output entries have unit variance.

Label convention: labels[p] is the label of bit p of the flat element index
(bit 0 = stride-1).  Free labels of A are 0..m-1, free labels of B are
m..m+n-1, shared labels are m+n..m+n+k-1.
"""
from __future__ import annotations

import numpy as np

_EXPS = (6, 8, 10, 12, 14)

# (m, n, k) exponents of the GEMM-equivalent sizes M = 2^m, N = 2^n, K = 2^k.
MICROBENCH_SHAPES = tuple(
    (m, n, k) for m in _EXPS for n in _EXPS for k in _EXPS
    if 16 <= m + k <= 30 and 16 <= n + k <= 30 and m + n <= 28
)


def microbench_case(m: int, n: int, k: int, seed: int, generate_data: bool = True):
    """Return (a_labels, b_labels, out_labels, A, B).

    A, B are complex64 flat arrays of 2^(m+k), 2^(n+k) elements (None when
    generate_data is False, e.g. when a caller generates them elsewhere from
    the same seed).  out_labels lists the output's labels, free A labels first
    (low bits) then free B labels, a layout callers may permute freely.
    """
    rng = np.random.default_rng(seed)
    shared = list(range(m + n, m + n + k))
    a_labels = list(range(m)) + shared
    b_labels = list(range(m, m + n)) + shared
    a_labels = [a_labels[i] for i in rng.permutation(len(a_labels))]
    b_labels = [b_labels[i] for i in rng.permutation(len(b_labels))]
    out_labels = list(range(m)) + list(range(m, m + n))
    if not generate_data:
        return a_labels, b_labels, out_labels, None, None
    scale = np.float32(np.sqrt(0.5) / np.sqrt(2.0 ** k))

    def draw(r):
        z = np.empty(1 << r, dtype=np.complex64)
        z.real = rng.standard_normal(1 << r, dtype=np.float32) * scale
        z.imag = rng.standard_normal(1 << r, dtype=np.float32) * scale
        return z

    A = draw(m + k)
    B = draw(n + k)
    return a_labels, b_labels, out_labels, A, B
