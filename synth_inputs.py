"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only draws numbers: it holds none of the sigma / Davidson / RDM
arithmetic.  It is the one module both sides may import.

Integral recipe (an active-space Hamiltonian of the size class the paper lists
for FCI/CASCI, 14-16 active orbitals, Sec. II.A.1 and Table I):

* h_pq: diagonal exactly -1.0 + 0.25 p (0-based p); off-diagonal upper triangle
  drawn row-major (p < q) from N(0, 0.05^2) and mirrored.
* (pq|rs) = sum_L B^L_pq B^L_rs, a factored (density-fitting-like, Sec. III
  "Integral classes") positive semidefinite, 8-fold symmetric tensor.  For
  L = 0..n_L-1 the upper triangle of B^L including the diagonal is drawn
  row-major from N(0, 0.15^2) and mirrored.
* The draws use numpy.random.default_rng(seed) (PCG64): first the h
  off-diagonal, then B^0, B^1, ...

Hubbard ring: h_pq = -t between ring neighbours (periodic), (pp|pp) = U, every
other integral zero.  For n = 2 the ring is the dimer with a single bond.
"""
from __future__ import annotations

import math

import numpy as np

# Shapes of the CASCI workloads used throughout (orbitals, alpha, beta electrons,
# number of density-fitting factors, seed, roots).
CAS88 = dict(norb=8, nalpha=4, nbeta=4, n_l=16, seed=0, nroots=1)
CAS1212 = dict(norb=12, nalpha=6, nbeta=6, n_l=24, seed=1, nroots=4)
CAS1414 = dict(norb=14, nalpha=7, nbeta=7, n_l=28, seed=2, nroots=1)
CAS1212_SA = dict(norb=12, nalpha=6, nbeta=6, n_l=24, seed=3, nroots=3)


def integrals(norb: int, n_l: int, seed: int):
    """Return (h [n,n], eri [n,n,n,n]) as float64 C-contiguous arrays."""
    rng = np.random.default_rng(seed)
    n = norb
    h = np.zeros((n, n))
    iu = np.triu_indices(n, k=1)
    h[iu] = rng.normal(0.0, 0.05, size=len(iu[0]))
    h = h + h.T
    h[np.arange(n), np.arange(n)] = -1.0 + 0.25 * np.arange(n)
    B = np.zeros((n_l, n, n))
    iu0 = np.triu_indices(n, k=0)
    for L in range(n_l):
        b = np.zeros((n, n))
        b[iu0] = rng.normal(0.0, 0.15, size=len(iu0[0]))
        B[L] = b + np.triu(b, 1).T
    eri = np.einsum("lpq,lrs->pqrs", B, B)
    return np.ascontiguousarray(h), np.ascontiguousarray(eri)


def hubbard_ring(nsites: int, t: float, U: float):
    """Periodic 1D Hubbard ring as (h, eri)."""
    n = nsites
    h = np.zeros((n, n))
    for i in range(n):
        j = (i + 1) % n
        if i != j:
            h[i, j] = -t
            h[j, i] = -t
    eri = np.zeros((n, n, n, n))
    for p in range(n):
        eri[p, p, p, p] = U
    return h, eri


def n_strings(norb: int, nel: int) -> int:
    return math.comb(norb, nel)


def random_vectors(nvec: int, n_alpha_str: int, n_beta_str: int, seed: int = 7):
    """nvec N(0,1) vectors of shape [N_alpha][N_beta], each normalised to 1."""
    rng = np.random.default_rng(seed)
    C = rng.normal(0.0, 1.0, size=(nvec, n_alpha_str, n_beta_str))
    C /= np.sqrt((C * C).sum(axis=(1, 2), keepdims=True))
    return np.ascontiguousarray(C)


def random_rotation(n: int, seed: int):
    """A random orthogonal n x n matrix (QR of a Gaussian matrix)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(n, n)))
    return q * np.sign(np.diag(r))


def batch_instances(count: int = 512, seed: int = 4242):
    """Independent half-filled active spaces for the batched solve.

    Orbital counts uniform over {6, 8, 10, 12}, 1-3 roots each; instance i
    takes its integrals from ``integrals(n_i, 2 n_i, 1000 + i)``.  The counts
    are drawn first (all of them), then the root numbers.
    """
    rng = np.random.default_rng(seed)
    norbs = rng.choice(np.array([6, 8, 10, 12]), size=count)
    nroots = rng.integers(1, 4, size=count)
    return [dict(norb=int(n), nalpha=int(n) // 2, nbeta=int(n) // 2, n_l=2 * int(n),
                 seed=1000 + i, nroots=int(k)) for i, (n, k) in enumerate(zip(norbs, nroots))]


def _replace(mask: int, holes, particles) -> int:
    for p in holes:
        mask &= ~(1 << p)
    for p in particles:
        mask |= 1 << p
    return mask


def excitation_list(norb: int, nalpha: int, nbeta: int, max_rank: int = 2):
    """Determinant words (alpha orbital p at bit p, beta orbital p at bit norb + p)
    of the aufbau determinant (lowest orbitals occupied in both spins) and of every
    determinant within max_rank (<= 2) orbital replacements of it, sorted: the shape
    of a selected-CI space grown from one reference."""
    import itertools
    a0 = (1 << nalpha) - 1
    b0 = (1 << nbeta) - 1

    def moves(mask, nel, rank):
        occ = [p for p in range(norb) if (mask >> p) & 1]
        vir = [p for p in range(norb) if not (mask >> p) & 1]
        return [_replace(mask, h, q) for h in itertools.combinations(occ, rank)
                for q in itertools.combinations(vir, rank)]

    words = set()
    alpha = {0: [a0]}
    beta = {0: [b0]}
    for r in range(1, max_rank + 1):
        alpha[r] = moves(a0, nalpha, r)
        beta[r] = moves(b0, nbeta, r)
    for ra in range(max_rank + 1):
        for rb in range(max_rank + 1 - ra):
            for a in alpha[ra]:
                for b in beta[rb]:
                    words.add(a | (b << norb))
    return np.array(sorted(words), dtype=np.uint64)


def random_determinants(norb: int, nalpha: int, nbeta: int, count: int, seed: int):
    """count distinct determinant words with nalpha / nbeta electrons, uniformly
    drawn (same bit layout as excitation_list), in drawing order."""
    rng = np.random.default_rng(seed)
    out, seen = [], set()
    while len(out) < count:
        a = rng.choice(norb, size=nalpha, replace=False)
        b = rng.choice(norb, size=nbeta, replace=False)
        w = int(np.sum(1 << a.astype(np.uint64))) | (int(np.sum(1 << b.astype(np.uint64))) << norb)
        if w not in seen:
            seen.add(w)
            out.append(w)
    return np.array(out, dtype=np.uint64)
