"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds no arithmetic of the method: it only draws random sparse structures and
values (numpy's PCG64 generator) and packs them as CSR arrays.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class QuboArrays:
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    lin: np.ndarray
    trip: np.ndarray = None


def random_qubo(n, avg_degree, seed, values=(-1.0, 1.0), lin_low=0.0, lin_high=1.0):
    """Symmetric sparse QUBO: each unordered pair is present with probability
    avg_degree / (n - 1); b drawn from ``values``; a ~ U[lin_low, lin_high)."""
    rng = np.random.default_rng(seed)
    p = min(1.0, avg_degree / max(n - 1, 1))
    rows = [[] for _ in range(n)]
    for i in range(n):
        for j in range(i):
            if rng.random() < p:
                v = float(rng.choice(values))
                rows[i].append((j, v))
                rows[j].append((i, v))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    col, val = [], []
    for i in range(n):
        rows[i].sort()
        col += [c for c, _ in rows[i]]
        val += [v for _, v in rows[i]]
        rowptr[i + 1] = len(col)
    lin = rng.uniform(lin_low, lin_high, size=n)
    return QuboArrays(n, rowptr, np.asarray(col, np.int32), np.asarray(val, np.float64), lin)


def grouped_qubo(n, K, n_ids, couple, w, extra_degree, seed):
    """QUBO whose couplings are mostly one weight shared by whole groups: row i
    belongs to group member[i, s] in slot s (ids drawn uniformly, a slot empty
    with probability 0.1), and b_ij = w * sum_{s, s'} couple[s][s'] [member[i, s]
    == member[j, s']] for i != j, plus a sparse symmetric perturbation of +-1
    (about extra_degree per row). Returns (QuboArrays, member)."""
    rng = np.random.default_rng(seed)
    member = rng.integers(0, n_ids, size=(n, K)).astype(np.int32)
    member[rng.random((n, K)) < 0.1] = -1
    B = np.zeros((n, n))
    for s in range(K):
        for s2 in range(K):
            if couple[s][s2]:
                a, b = member[:, s], member[:, s2]
                B += w * ((a[:, None] == b[None, :]) & (a[:, None] >= 0))
    P = np.triu(rng.random((n, n)) < extra_degree / max(n - 1, 1), 1)
    V = np.triu(rng.choice([-1.0, 1.0], size=(n, n)), 1) * P
    B += V + V.T
    np.fill_diagonal(B, 0.0)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(B[i])[0]
        cols.append(nz.astype(np.int32))
        vals.append(B[i, nz])
        rowptr[i + 1] = rowptr[i] + len(nz)
    lin = rng.uniform(0.0, 1.0, size=n)
    return QuboArrays(n, rowptr, np.concatenate(cols), np.concatenate(vals), lin), member


def random_state(n, R, seed, scale=1.0):
    """(x, y) uniform in [-scale, scale], float32 values."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-scale, scale, size=(n, R)).astype(np.float32)
    y = rng.uniform(-scale, scale, size=(n, R)).astype(np.float32)
    return x, y


def random_spins(n, R, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(n, R)).astype(np.int8)
