"""Exhaustive enumeration for small N -- TEST INFRASTRUCTURE ONLY.

Energies of all 2^N spin states by the pairwise sum of Eq. 1, the exact ground state,
and the Boltzmann distribution exp(-beta H)/Z that a heat-bath (Glauber) sequential
update with P(s_i = +1 | rest) = (1 + tanh(beta I_i))/2 leaves invariant.
"""
from __future__ import annotations

import numpy as np


def _states(n: int) -> np.ndarray:
    """All 2^n states as rows of +-1 (bit k of the row index -> spin k)."""
    idx = np.arange(1 << n, dtype=np.int64)[:, None]
    bits = (idx >> np.arange(n, dtype=np.int64)[None, :]) & 1
    return np.where(bits == 1, 1, -1).astype(np.int8)


def all_energies(J, h) -> tuple[np.ndarray, np.ndarray]:
    """(states, energies) with H(s) = -sum_{i<j} J_ij s_i s_j - sum_i h_i s_i written as
    the explicit upper-triangle pair sum of Eq. 1 (not the quadratic form)."""
    J = np.asarray(J, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n = J.shape[0]
    S = _states(n).astype(np.float64)
    E = np.zeros(S.shape[0])
    for i in range(n):
        for j in range(i + 1, n):
            if J[i, j] != 0.0:
                E -= J[i, j] * S[:, i] * S[:, j]
        if h[i] != 0.0:
            E -= h[i] * S[:, i]
    return S.astype(np.int8), E


def ground_state(J, h) -> tuple[float, np.ndarray]:
    S, E = all_energies(J, h)
    k = int(np.argmin(E))
    return float(E[k]), S[k]


def boltzmann(J, h, beta: float) -> tuple[np.ndarray, np.ndarray]:
    """(states, p) with p proportional to exp(-beta H(s))."""
    S, E = all_energies(J, h)
    w = np.exp(-beta * (E - E.min()))
    return S, w / w.sum()
