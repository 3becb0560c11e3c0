"""QUBO <-> Ising conversion and energies (oracle side). Test infrastructure only.

Eq. 13 gives the QUBO objective O(a, b, T) = sum_i a_i T_i + sum_i sum_{j<i} b_ij T_i T_j.
The paper reports "Ising energies" (section "Results") without printing the
map; it is the substitution T = (1 + s)/2, s in {-1, +1}:

  O(T) = offset + sum_i ht_i s_i + sum_{i<j} (b_ij / 4) s_i s_j,
  ht_i   = a_i / 2 + (1/4) sum_{j != i} b_ij,
  offset = (1/2) sum_i a_i + (1/4) sum_{i<j} b_ij.

SB (Eq. 4) lowers -(c0/2) sum_ij J_ij x_i x_j, i.e. it maximises
(1/2) x^T J x + h^T x, so the Ising problem handed to SB is
  J_ij = -b_ij / 4 (both triangles),  h_i = -ht_i,
  E_ising(s) = -(1/2) s^T J s - h^T s,   O(T) = offset + E_ising(s).
"""
import math

import numpy as np
import scipy.sparse as sp


def qubo_energy(q, T):
    """Eq. 13 evaluated by its definition (lower-triangle double sum).

    ``T`` is a 0/1 array of shape [n] or [n, R]; returns a float or an [R] array.
    """
    T = np.asarray(T, dtype=np.float64)
    one = T.ndim == 1
    if one:
        T = T[:, None]
    E = np.zeros(T.shape[1])
    for i in range(q.n):
        E += q.lin[i] * T[i]
        for p in range(q.rowptr[i], q.rowptr[i + 1]):
            j = q.col[p]
            if j < i:
                E += q.val[p] * T[i] * T[j]
    return float(E[0]) if one else E


def to_ising(q):
    """Return (J as scipy CSR float64, h float64[n], offset float)."""
    n = q.n
    rows = np.repeat(np.arange(n), np.diff(q.rowptr))
    J = sp.csr_matrix((-q.val / 4.0, q.col, q.rowptr), shape=(n, n))
    h = np.zeros(n)
    for i in range(n):
        s = 0.0
        for p in range(q.rowptr[i], q.rowptr[i + 1]):
            s += q.val[p]
        h[i] = -(q.lin[i] / 2.0 + s / 4.0)
    lower = q.col < rows
    offset = 0.5 * float(np.sum(q.lin)) + 0.25 * float(np.sum(q.val[lower]))
    return J, h, offset


def ising_energy(J, h, s):
    """E = -(1/2) s^T J s - h^T s for s of shape [n] or [n, R]."""
    s = np.asarray(s, dtype=np.float64)
    Js = J @ s
    if s.ndim == 1:
        return float(-0.5 * s @ Js - h @ s)
    return -0.5 * np.sum(s * Js, axis=0) - h @ s


def spins_from_x(x):
    """Readout s_i = +1 if x_i > 0 else -1 (a tie at 0 leaves the triplet unselected)."""
    return np.where(np.asarray(x) > 0.0, 1.0, -1.0)


def triplets_from_spins(s):
    """T = (1 + s) / 2 as 0/1."""
    return (np.asarray(s) > 0).astype(np.int8)


def sigma_j(J, n):
    """RMS over all n(n-1) off-diagonal entries of J (zeros included)."""
    if n < 2:
        return 0.0
    return math.sqrt(float(np.sum(J.data.astype(np.float64) ** 2)) / (n * (n - 1.0)))


def c0_auto(J, n):
    """Fixed c0 = 0.5 / (sqrt(n) sigma_J) (section "Results": a fixed c0 is used)."""
    s = sigma_j(J, n)
    return 0.5 / (math.sqrt(n) * s) if s > 0 else 1.0
