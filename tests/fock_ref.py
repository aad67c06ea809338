"""Independent Fock-space construction used to pin the oracle.

The Hamiltonian here is never built from Slater-Condon rules: it is the
operator sum  H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - d_qr E_ps)
(the spin-free form of Eq. 1 with V = 0), with E_pq = sum_s a+_ps a_qs formed as
products of sparse creation/annihilation matrices on the full 2^(2n)-dimensional
Fock space.  Basis state m is the bit mask with alpha orbital p at bit p and
beta orbital p at bit n+p; a_P carries (-1)^(occupied bits below P), i.e. the
state is the ordered product of creators with all alpha ones first.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp


def annihilators(n: int):
    """List of 2n sparse matrices a_P on the 2^(2n) Fock space."""
    dim = 1 << (2 * n)
    out = []
    m = np.arange(dim, dtype=np.int64)
    for P in range(2 * n):
        occ = (m >> P) & 1
        rows = (m ^ (1 << P))[occ == 1]
        cols = m[occ == 1]
        below = np.array([bin(int(x) & ((1 << P) - 1)).count("1") for x in cols])
        vals = np.where(below % 2 == 0, 1.0, -1.0)
        out.append(sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim)))
    return out


def excitation_ops(n: int):
    """E[p][q] = sum over spin of a+_ps a_qs (sparse)."""
    a = annihilators(n)
    E = [[None] * n for _ in range(n)]
    for p in range(n):
        for q in range(n):
            E[p][q] = (a[p].T @ a[q] + a[n + p].T @ a[n + q]).tocsr()
    return E, a


def sector_states(n: int, na: int, nb: int):
    """Fock indices of the (na, nb) sector in oracle order I_alpha*N_beta + I_beta."""
    sa = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), na))
    sb = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), nb))
    return np.array([x | (y << n) for x in sa for y in sb], dtype=np.int64)


def hamiltonian(n: int, h, eri, E=None):
    """Sparse Fock-space H from E_pq products."""
    if E is None:
        E, _ = excitation_ops(n)
    dim = 1 << (2 * n)
    H = sp.csr_matrix((dim, dim))
    for p in range(n):
        for q in range(n):
            if h[p, q] != 0.0:
                H = H + h[p, q] * E[p][q]
    for p, q, r, s in itertools.product(range(n), repeat=4):
        g = eri[p, q, r, s]
        if g == 0.0:
            continue
        term = E[p][q] @ E[r][s]
        if q == r:
            term = term - E[p][s]
        H = H + 0.5 * g * term
    return H.tocsr()


def sector_matrix(n, na, nb, h, eri):
    idx = sector_states(n, na, nb)
    H = hamiltonian(n, h, eri)
    return H[idx][:, idx].toarray()


def embed(n, na, nb, vec):
    """Sector vector (oracle order) -> full Fock-space vector."""
    idx = sector_states(n, na, nb)
    out = np.zeros(1 << (2 * n))
    out[idx] = np.asarray(vec).reshape(-1)
    return out


def rdms(n, na, nb, vec, E=None):
    """Spin-free gamma_pq = <E_pq>, Gamma_pqrs = <E_pq E_rs> - d_qr <E_ps>."""
    if E is None:
        E, _ = excitation_ops(n)
    v = embed(n, na, nb, vec)
    Ev = [[E[p][q] @ v for q in range(n)] for p in range(n)]
    g1 = np.array([[v @ Ev[p][q] for q in range(n)] for p in range(n)])
    g2 = np.zeros((n,) * 4)
    for p, q, r, s in itertools.product(range(n), repeat=4):
        val = v @ (E[p][q] @ Ev[r][s])
        if q == r:
            val -= g1[p, s]
        g2[p, q, r, s] = val
    return g1, g2


def rdm3(n, na, nb, vec, E=None):
    """Spin-free Gamma3_pqrstu (pairs (p,q), (r,s), (t,u) share a spin) from
    expectation values of E-operator products and the normal-ordering identity
    E_pq E_rs E_tu = g_pqrstu + d_qt e_purs + d_st e_pqru + d_qr E_ps E_tu,
    with e the two-body operator of Gamma2 (e_pqrs = E_pq E_rs - d_qr E_ps):
      Gamma3 = <E_pq E_rs E_tu> - d_qt G2_purs - d_st G2_pqru - d_qr (G2_pstu + d_st g1_pu)."""
    if E is None:
        E, _ = excitation_ops(n)
    g1, g2 = rdms(n, na, nb, vec, E)
    v = embed(n, na, nb, vec)
    Ev = {(t, u): E[t][u] @ v for t in range(n) for u in range(n)}
    left = {(p, q): E[p][q].T @ v for p in range(n) for q in range(n)}  # (E_pq)^T v: <v|E_pq = (E_pq^T v)^T
    g3 = np.zeros((n,) * 6)
    for r, s_, t, u in itertools.product(range(n), repeat=4):
        w = E[r][s_] @ Ev[(t, u)]
        for p, q in itertools.product(range(n), repeat=2):
            val = left[(p, q)] @ w
            if q == t:
                val -= g2[p, u, r, s_]
            if s_ == t:
                val -= g2[p, q, r, u]
            if q == r:
                val -= g2[p, s_, t, u]
                if s_ == t:
                    val -= g1[p, u]
            g3[p, q, r, s_, t, u] = val
    return g3


def s2_expectation(n, na, nb, vec):
    """<S^2> from spin operators S+ = sum_p a+_pa a_pb, Sz = (Na - Nb)/2."""
    a = annihilators(n)
    splus = sum(a[p].T @ a[n + p] for p in range(n))
    v = embed(n, na, nb, vec)
    sz = 0.5 * (na - nb)
    # S^2 = S- S+ + Sz (Sz + 1)
    w = splus @ v
    return float(w @ w + sz * (sz + 1.0))


def comb(n, k):
    return math.comb(n, k)
