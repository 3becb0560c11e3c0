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


def random_state(n, R, seed, scale=1.0):
    """(x, y) uniform in [-scale, scale], float32 values."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-scale, scale, size=(n, R)).astype(np.float32)
    y = rng.uniform(-scale, scale, size=(n, R)).astype(np.float32)
    return x, y


def random_spins(n, R, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(n, R)).astype(np.int8)
