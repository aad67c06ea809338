"""Adaptive configuration interaction (ACI) on determinant lists, for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.A.2 (selected CI): the same selection as the grid version in aci.py -- the
2 x 2 energy estimate eps_mu of every determinant mu of the first-order interacting
space of the reference space P, exclusion of the smallest |eps| up to a total of
sigma, the model space M = P + the rest, exact diagonalisation in M, the next P
by weight 1 - gamma sigma -- but on explicit lists of determinants, so that the
space is not bounded by a CAS grid (up to 32 orbitals).  Determinants are 64-bit
words: alpha orbital p at bit p, beta orbital p at bit norb + p.

Readings (beyond those listed in aci.py, which apply unchanged):
* the first-order interacting space F(P) = every determinant reached from a
  determinant of P by one or two replacements (alpha, beta, or one of each) that is
  not in P -- the paper's definition; a determinant outside F(P) has V = 0;
* the start P is given by the caller (a list of words); for n_alpha = n_beta the
  mirror (alpha and beta strings exchanged) of every start determinant joins it, and
  |eps| and c^2 are taken as the larger of a determinant's and its mirror's value
  (both are always in the same space: F and M are closed under the exchange);
* on a CAS grid this is the grid version whenever E_P lies at or below every
  diagonal element H_mumu of the determinants outside F(P) (their eps is then 0 and
  the grid version excludes them); the tests compare the two there;
* optional exchange-parity sector (n_alpha = n_beta; +1: even S, -1: odd S): the P
  and M solves take the lowest state with c(mirror(D)) = parity c(D), in the basis
  (|D> + parity |mirror(D)>)/sqrt(2) of mirror pairs and |D> for a determinant that is
  its own mirror (even sector only); the start determinants must be able to carry
  weight there (for -1, alpha string != beta string).
"""
from __future__ import annotations

import numpy as np

from .aci import aci_epsilon, aci_excluded, aci_reference
from .driver import _fix_sign, hij, sci_sigma


def _bits(x, norb):
    return [p for p in range(norb) if (x >> p) & 1]


def _replacements(s, norb):
    """Strings reached from the occupation bit string s by one and by two replacements."""
    occ = _bits(s, norb)
    vir = [q for q in range(norb) if not (s >> q) & 1]
    one, two = [], []
    for p in occ:
        for q in vir:
            one.append(s ^ (1 << p) ^ (1 << q))
    for i, p in enumerate(occ):
        for p2 in occ[i + 1:]:
            for j, q in enumerate(vir):
                for q2 in vir[j + 1:]:
                    two.append(s ^ (1 << p) ^ (1 << p2) ^ (1 << q) ^ (1 << q2))
    return one, two


def connected(norb, det):
    """Every determinant differing from `det` by one or two replacements (same alpha and
    beta electron counts), as a set of words."""
    mask = (1 << norb) - 1
    a, b = det & mask, det >> norb
    a1, a2 = _replacements(a, norb)
    b1, b2 = _replacements(b, norb)
    out = set()
    for x in a1 + a2:
        out.add(x | (b << norb))
    for y in b1 + b2:
        out.add(a | (y << norb))
    for x in a1:
        for y in b1:
            out.add(x | (y << norb))
    return out


def mirror(norb, det):
    """The determinant with the alpha and beta strings exchanged."""
    mask = (1 << norb) - 1
    return (det >> norb) | ((det & mask) << norb)


def hmat_list(norb, dets, h, eri):
    """Dense <D_i|H|D_j> over a list (the list sigma applied to the unit vectors)."""
    m = len(dets)
    return sci_sigma(norb, np.asarray(dets, dtype=np.uint64), h, eri, np.eye(m))


def _lowest(norb, dets, h, eri, parity):
    """Lowest eigenpair of H over the list (in the exchange-parity sector when parity != 0);
    the vector over the list."""
    H = hmat_list(norb, dets, h, eri)
    if parity == 0:
        w, U = np.linalg.eigh(H)
        return w[0], U[:, 0]
    pos = {d: i for i, d in enumerate(dets)}
    rows = []
    for i, d in enumerate(dets):
        j = pos[mirror(norb, d)]
        if j < i:
            continue
        v = np.zeros(len(dets))
        if j == i:
            if parity < 0:
                continue
            v[i] = 1.0
        else:
            v[i] = 1.0 / np.sqrt(2.0)
            v[j] = parity / np.sqrt(2.0)
        rows.append(v)
    Q = np.array(rows)
    w, U = np.linalg.eigh(Q @ H @ Q.T)
    return w[0], U[:, 0] @ Q


def _mirror_max(vals, dets, norb, pair):
    if not pair:
        return vals
    pos = {d: i for i, d in enumerate(dets)}
    out = vals.copy()
    for i, d in enumerate(dets):
        j = pos.get(mirror(norb, d))
        if j is not None:
            out[i] = max(vals[i], vals[j])
    return out


def aci_list(norb, nalpha, nbeta, h, eri, start, sigma, gamma=1.0, max_iter=50, parity=0):
    """ACI from the start determinants `start` (words).  Returns dict(E=E_M,
    E_corrected=E_M + sum of the excluded eps, M=sorted words of the model space,
    P=sorted words of the last reference space, C=Psi_M over M, cycles)."""
    if not 1 <= norb <= 32:
        raise ValueError("determinant words hold at most 32 orbitals")
    if parity and nalpha != nbeta:
        raise ValueError("an exchange-parity sector needs n_alpha == n_beta")
    pair = nalpha == nbeta
    P = sorted(set(int(d) for d in start) | ({mirror(norb, int(d)) for d in start} if pair else set()))
    for d in P:
        if bin(d & ((1 << norb) - 1)).count("1") != nalpha or bin(d >> norb).count("1") != nbeta:
            raise ValueError("a start determinant is outside the (n_alpha, n_beta) sector")
    seen = []
    for cycle in range(1, max_iter + 1):
        E_P, cP = _lowest(norb, P, h, eri, parity)
        Pset = set(P)
        F = sorted(set().union(*(connected(norb, d) for d in P)) - Pset)
        # V_mu = <mu|H|Psi_P>: the list sigma over F + P of the vector (0 on F, c_P on P)
        allw = F + P
        x = np.zeros(len(allw))
        x[len(F):] = cP
        V = sci_sigma(norb, np.asarray(allw, dtype=np.uint64), h, eri, x[None, :])[0][:len(F)]
        Hmm = np.array([hij(norb, h, eri, d, d) for d in F])
        eps = aci_epsilon(E_P, Hmm, V)
        excl = aci_excluded(_mirror_max(np.abs(eps), F, norb, pair), sigma)
        M = sorted(Pset | {d for d, e in zip(F, excl) if not e})
        E_M, C = _lowest(norb, M, h, eri, parity)
        C = _fix_sign(C)
        keep = aci_reference(_mirror_max(C * C, M, norb, pair), gamma * sigma)
        newP = [d for d, k in zip(M, keep) if k]
        key = tuple(newP)
        if key in seen or cycle == max_iter:
            return dict(E=E_M, E_corrected=E_M + float(eps[excl].sum()), M=M, P=newP, C=C, cycles=cycle)
        seen.append(key)
        P = newP
