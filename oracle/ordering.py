"""Fiedler ordering of the orbitals (TEST INFRASTRUCTURE ONLY).

Sec. 3.2 sorts the molecular orbitals of the MPS calculations along a
Fiedler vector, which narrows the band of the Hamiltonian matrix (spectral
ordering).  The orbitals are vertices of a graph with weights
W_ij = |h_ij| + |(ij|ji)| (i != j, symmetrised); the eigenvector of the
Laplacian D - W with the second smallest eigenvalue orders them.  Sign of
that eigenvector: its correlation with the input order is made >= 0; ties
keep the input order.

Pins (tests/test_ordering.py): the path-graph Laplacian's closed-form second
eigenvalue and Fiedler vector; chains hidden by a permutation, in the hopping
or only in the exchange integrals, are recovered; a chain in input order comes
back unreversed.
"""
from __future__ import annotations

import numpy as np


def weights(h: np.ndarray, eri: np.ndarray) -> np.ndarray:
    L = h.shape[0]
    K = np.array([[eri[i, j, j, i] for j in range(L)] for i in range(L)])
    W = np.abs(h) + np.abs(K)
    W = 0.5 * (W + W.T)
    np.fill_diagonal(W, 0.0)
    return W


def laplacian(W: np.ndarray) -> np.ndarray:
    return np.diag(W.sum(axis=1)) - W


def fiedler_order(h: np.ndarray, eri: np.ndarray) -> np.ndarray:
    """perm[k] = input orbital placed at position k."""
    L = h.shape[0]
    if L < 3:
        return np.arange(L)
    lam, V = np.linalg.eigh(laplacian(weights(h, eri)))
    f = V[:, np.argsort(lam, kind="stable")[1]]
    if np.dot(np.arange(L) - 0.5 * (L - 1), f) < 0:
        f = -f
    return np.argsort(f, kind="stable")
