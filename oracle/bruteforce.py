"""Exhaustive ground state of the QUBO of Eq. 13 for small N (oracle side).
Test infrastructure only.

Every state T in {0,1}^N is enumerated (in chunks of the 2^N integers) and
O(T) = T.a + sum_{j<i} b_ij T_i T_j is evaluated from a dense lower triangle.
"""
import numpy as np


def dense_lower(q):
    B = np.zeros((q.n, q.n))
    for i in range(q.n):
        for p in range(q.rowptr[i], q.rowptr[i + 1]):
            j = q.col[p]
            if j < i:
                B[i, j] = q.val[p]
    return B


def ground_state(q, chunk_bits=16):
    """Return (E_min, list of minimising 0/1 vectors as int arrays)."""
    n = q.n
    assert n <= 22, "exhaustive search is for N <= 22"
    B = dense_lower(q)
    bits = np.arange(n, dtype=np.int64)
    best = np.inf
    arg = []
    total = 1 << n
    step = 1 << min(chunk_bits, n)
    for start in range(0, total, step):
        ids = np.arange(start, min(start + step, total), dtype=np.int64)
        T = ((ids[:, None] >> bits[None, :]) & 1).astype(np.float64)
        E = T @ q.lin + np.einsum("si,ij,sj->s", T, B, T)
        m = E.min()
        if m < best - 1e-12:
            best = m
            arg = []
        if m <= best + 1e-12:
            for k in np.nonzero(E <= best + 1e-12)[0]:
                arg.append(T[k].astype(np.int8))
    return float(best), arg
