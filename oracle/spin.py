"""Spin-parity projection for the oracle (Ms = 0).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.A.1 lets the CI expansion be projected on states of well-defined total
spin.  For n_alpha = n_beta the determinant space is mapped onto itself by
exchanging the alpha and beta strings, T: C[I_a, I_b] -> C[I_b, I_a], which
commutes with the spin-free Hamiltonian.  With the determinant convention of
this package (alpha creators first) an eigenvector of total spin S obeys
    C[I_b, I_a] = (-1)^S C[I_a, I_b],
so the two eigenspaces of T hold the even-S (singlet, quintet, ...) and the
odd-S (triplet, ...) states.  The oracle restricts H to one of them by dense
diagonalisation in the orthonormal basis
    (e_IJ + p e_JI) / sqrt(2)  (I < J),   e_II  (only for p = +1).
"""
from __future__ import annotations

import numpy as np

from .driver import _fix_sign, hmat_dense, strings


def sector_basis(N, parity, keep=None):
    """Orthonormal basis [dim][N*N] of {C : C^T = parity C} (optionally only
    over the determinants where the boolean [N][N] ``keep`` is true; keep must
    be symmetric)."""
    if parity not in (1, -1):
        raise ValueError("parity must be +1 or -1")
    cols = []
    for i in range(N):
        for j in range(i, N):
            if keep is not None and not keep[i, j]:
                continue
            v = np.zeros(N * N)
            if i == j:
                if parity < 0:
                    continue
                v[i * N + i] = 1.0
            else:
                v[i * N + j] = 1.0 / np.sqrt(2.0)
                v[j * N + i] = parity / np.sqrt(2.0)
            cols.append(v)
    return np.array(cols).reshape(len(cols), N * N)


def solve_dense_spin(norb, nel, h, eri, parity, nroots=1, keep=None):
    """Lowest eigenpairs of H in the sector C^T = parity C of the (nel, nel)
    determinant space; vectors over the full [N*N] index."""
    N = len(strings(norb, nel))
    Q = sector_basis(N, parity, keep)
    H = hmat_dense(norb, nel, nel, h, eri)
    w, U = np.linalg.eigh(Q @ H @ Q.T)
    vecs = np.array([_fix_sign(U[:, k] @ Q) for k in range(nroots)])
    return w[:nroots], vecs
