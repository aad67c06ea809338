"""Occupation-restricted CI (GAS / RAS) for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.A.1 (occupation-restricted CI): the active orbitals are split into
disjoint spaces A_1 .. A_G and the model space is cut down to the determinants
whose occupations obey per-space limits.  Reading used here: the spaces are
consecutive orbital ranges of the given sizes, and a determinant
|I_alpha> x |I_beta> is kept when, for every space g,
    gmin[g] <= (alpha electrons in A_g) + (beta electrons in A_g) <= gmax[g].
RAS is the case of three spaces with a minimum on RAS1 (at most k holes) and a
maximum on RAS3 (at most k particles).

The restricted Hamiltonian is the full one projected onto the kept
determinants, P H P; its eigenpairs are taken by dense diagonalisation of the
kept block, and its sigma as P H (P C).
"""
from __future__ import annotations

import numpy as np

from .driver import _fix_sign, hmat_dense, sigma, strings


def _space_counts(masks, spaces):
    """[N][G] electron counts of each string in each space, bit by bit."""
    out = np.zeros((len(masks), len(spaces)), dtype=np.int64)
    for i, m in enumerate(masks):
        m = int(m)
        orb = 0
        for g, size in enumerate(spaces):
            c = 0
            for _ in range(size):
                c += (m >> orb) & 1
                orb += 1
            out[i, g] = c
    return out


def gas_allowed(norb, nalpha, nbeta, spaces, gmin, gmax):
    """Boolean [N_alpha][N_beta]: which determinants the restriction keeps."""
    if sum(spaces) != norb:
        raise ValueError("space sizes must add up to norb")
    ca = _space_counts(strings(norb, nalpha), spaces)
    cb = _space_counts(strings(norb, nbeta), spaces)
    keep = np.ones((len(ca), len(cb)), dtype=bool)
    for g in range(len(spaces)):
        tot = ca[:, g][:, None] + cb[:, g][None, :]
        keep &= (tot >= gmin[g]) & (tot <= gmax[g])
    return keep


def sigma_gas(norb, nalpha, nbeta, h, eri, C, spaces, gmin, gmax):
    """P H P C for C of shape [nvec, N_alpha, N_beta] (or [nvec, Ndet])."""
    keep = gas_allowed(norb, nalpha, nbeta, spaces, gmin, gmax).reshape(-1)
    Cf = np.asarray(C, dtype=np.float64).reshape(C.shape[0], -1) * keep
    return (sigma(norb, nalpha, nbeta, h, eri, Cf) * keep).reshape(C.shape)


def solve_dense_gas(norb, nalpha, nbeta, h, eri, spaces, gmin, gmax, nroots=1):
    """Lowest eigenpairs of P H P on the kept determinants; vectors over the
    full [N_alpha * N_beta] index, zero outside the restricted space."""
    keep = gas_allowed(norb, nalpha, nbeta, spaces, gmin, gmax).reshape(-1)
    idx = np.flatnonzero(keep)
    H = hmat_dense(norb, nalpha, nbeta, h, eri)[np.ix_(idx, idx)]
    w, V = np.linalg.eigh(H)
    vecs = np.zeros((nroots, keep.size))
    for k in range(nroots):
        vecs[k, idx] = V[:, k]
        vecs[k] = _fix_sign(vecs[k])
    return w[:nroots], vecs
