"""Adaptive configuration interaction (ACI) on the determinant grid of a CAS,
for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.A.2 (determinantal and selected CI): ACI looks for a model space M
whose variational energy E_M lies within about sigma of the CASCI energy.  It
grows a reference space P and screens the determinants mu of P's first-order
interacting space with the energy estimate of a 2 x 2 Hamiltonian built from
the current state Psi_P and Phi_mu:
    [[E_P, V_mu], [V_mu, H_mumu]],  V_mu = <Phi_mu|H|Psi_P>,
    eps_mu = lowest eigenvalue - E_P = D/2 - sqrt((D/2)^2 + V_mu^2),  D = H_mumu - E_P,
and excludes the determinants with the smallest |eps| as long as the sum of
the excluded |eps| stays at most sigma; the energy can be corrected by the
sum of the excluded eps.

Readings used here (the paper gives the criterion, not every step):
* determinants are the CAS grid I_alpha x I_beta (index I_alpha * N_beta + I_beta);
* start: P = the determinant of lowest H_II (lowest index among equals);
* F = every determinant outside P; those not connected to P have V = 0 and
  eps = 0, so the criterion always excludes them;
* excluded = {mu : S(|eps_mu|) <= sigma} with S(x) = sum of |eps_nu| over
  |eps_nu| <= x: determinants with equal |eps| leave together or not at all;
* M = P + (F - excluded), diagonalised exactly;
* next P = the determinants of M with the largest c^2 whose weights reach
  1 - gamma * sigma: {mu : T(c_mu^2) >= 1 - gamma sigma} for the largest such
  threshold, T(y) = sum of c_nu^2 over c_nu^2 >= y (ties kept together);
* stop when P repeats (or after max_iter cycles);
* for n_alpha = n_beta the exchange of alpha and beta strings commutes with H,
  so mirror determinants (I_a, I_b) and (I_b, I_a) have equal |eps| and c^2 in
  exact arithmetic; both are set to the larger of the two computed values (so
  that rounding cannot split a mirror pair at a threshold), and the start P
  holds the lowest determinant together with its mirror;
* optional exchange-parity sector (n_alpha = n_beta, parity +1: even S, -1:
  odd S): the P and M solves take the lowest state with C^T = parity C, and the
  start P is the lowest determinant that can carry weight there (for parity -1
  one with I_a != I_b) with its mirror.
"""
from __future__ import annotations

import numpy as np

from .driver import _fix_sign, hmat_dense
from .spin import sector_basis


def aci_epsilon(E, Hmm, V):
    """Energy estimate of the 2 x 2 problem [[E, V], [V, Hmm]] (lowest root - E)."""
    D = 0.5 * (np.asarray(Hmm, dtype=np.float64) - E)
    return D - np.sqrt(D * D + np.asarray(V, dtype=np.float64) ** 2)


def aci_excluded(abs_eps, sigma):
    """Boolean mask of the excluded entries: |eps| <= x* for the largest value x*
    of abs_eps whose cumulative sum S(x*) stays at most sigma."""
    a = np.asarray(abs_eps, dtype=np.float64)
    vals = np.unique(a)                       # ascending distinct values
    sums = np.array([a[a <= v].sum() for v in vals])
    ok = vals[sums <= sigma]
    if ok.size == 0:
        return np.zeros(a.shape, dtype=bool)
    return a <= ok.max()


def aci_reference(c2, gamma_sigma):
    """Boolean mask of the next reference space: c^2 >= y* for the largest value
    y* of c2 whose weight T(y*) = sum(c2[c2 >= y*]) reaches 1 - gamma_sigma."""
    c2 = np.asarray(c2, dtype=np.float64)
    vals = np.unique(c2)[::-1]                # descending distinct values
    target = 1.0 - gamma_sigma
    for v in vals:
        if c2[c2 >= v].sum() >= target:
            return c2 >= v
    return c2 >= vals[-1]


def _mirror_max(x, nalpha, nbeta):
    """max(x[Ia, Ib], x[Ib, Ia]) for n_alpha = n_beta (x over the grid); x itself otherwise."""
    if nalpha != nbeta:
        return x
    N = int(round(np.sqrt(x.size)))
    X = x.reshape(N, N)
    return np.maximum(X, X.T).reshape(-1)


def _lowest(H, idx):
    w, U = np.linalg.eigh(H[np.ix_(idx, idx)])
    return w[0], U[:, 0]


def _lowest_grid(H, mask, parity):
    """Lowest eigenpair of H restricted to the determinants in `mask` (and to the
    exchange-parity sector when parity != 0); the vector over the whole grid."""
    Nd = H.shape[0]
    if parity == 0:
        idx = np.flatnonzero(mask)
        E, c = _lowest(H, idx)
        v = np.zeros(Nd)
        v[idx] = c
        return E, v
    N = int(round(np.sqrt(Nd)))
    Q = sector_basis(N, parity, mask.reshape(N, N))
    w, U = np.linalg.eigh(Q @ H @ Q.T)
    return w[0], U[:, 0] @ Q


def aci(norb, nalpha, nbeta, h, eri, sigma, gamma=1.0, max_iter=50, parity=0):
    """ACI on the CAS grid.  Returns dict(E=E_M, E_corrected=E_M + sum of the
    excluded eps, M=bool mask, P=bool mask, C=Psi_M over the grid, cycles)."""
    if parity and nalpha != nbeta:
        raise ValueError("an exchange-parity sector needs n_alpha == n_beta")
    H = hmat_dense(norb, nalpha, nbeta, h, eri)
    Nd = H.shape[0]
    d = np.diag(H)
    P = np.zeros(Nd, dtype=bool)
    start = d.copy()
    if parity < 0:  # determinants |I>|I> carry no weight in the odd sector
        N = int(round(np.sqrt(Nd)))
        start[np.arange(N) * (N + 1)] = np.inf
    P[int(np.argmin(start))] = True
    P = _mirror_max(P.astype(np.float64), nalpha, nbeta) > 0
    seen = []
    for cycle in range(1, max_iter + 1):
        E_P, psi = _lowest_grid(H, P, parity)
        V = H @ psi                              # <Phi_mu|H|Psi_P> for every mu
        eps = aci_epsilon(E_P, d, V)
        eps[P] = 0.0
        excl = aci_excluded(_mirror_max(np.where(P, np.inf, np.abs(eps)), nalpha, nbeta), sigma) & ~P
        M = ~excl
        E_M, C = _lowest_grid(H, M, parity)
        C = _fix_sign(C)
        newP = aci_reference(_mirror_max(np.where(M, C * C, 0.0), nalpha, nbeta), gamma * sigma) & M
        key = newP.tobytes()
        if key in seen or cycle == max_iter:
            return dict(E=E_M, E_corrected=E_M + eps[excl].sum(), M=M, P=newP, C=C, cycles=cycle)
        seen.append(key)
        P = newP
