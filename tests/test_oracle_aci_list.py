"""Pins of the oracle's ACI on determinant lists (oracle/aci_list.py, Sec. II.A.2):
the replacement generator against brute force over the whole sector, the list ACI
against the grid ACI on CAS problems (same selection readings, other data path),
sigma = 0 reaching the exact sector energy, and the variational bound beyond a CAS
grid size the dense check can still hold."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth_inputs as si
from oracle import aci_list as al


def _sector(norb, na, nb):
    A = oracle.strings(norb, na)
    B = oracle.strings(norb, nb)
    return [int(a) | (int(b) << norb) for a in A for b in B]


@pytest.mark.parametrize("norb,na,nb", [(5, 2, 2), (6, 3, 1), (6, 0, 2), (7, 2, 3)])
def test_connected_determinants_are_the_sector_at_one_or_two_replacements(norb, na, nb):
    sector = _sector(norb, na, nb)
    rng = np.random.default_rng(3)
    for det in rng.choice(sector, size=min(6, len(sector)), replace=False):
        det = int(det)
        brute = {d for d in sector if bin(d ^ det).count("1") in (2, 4)}
        assert al.connected(norb, det) == brute


def test_mirror_exchanges_the_strings():
    norb = 6
    d = 0b000111 | (0b110000 << norb)
    assert al.mirror(norb, d) == 0b110000 | (0b000111 << norb)
    assert al.mirror(norb, al.mirror(norb, d)) == d


def _grid_start_word(norb, na, nb, h, eri):
    d = oracle.hdiag(norb, na, nb, h, eri)
    i = int(np.argmin(d))
    A, B = oracle.strings(norb, na), oracle.strings(norb, nb)
    Nb = len(B)
    return int(A[i // Nb]) | (int(B[i % Nb]) << norb)


def _grid_words(norb, na, nb, mask):
    A, B = oracle.strings(norb, na), oracle.strings(norb, nb)
    Nb = len(B)
    return sorted(int(A[i // Nb]) | (int(B[i % Nb]) << norb) for i in np.flatnonzero(mask))


@pytest.mark.parametrize("norb,na,nb,seed,sigma", [(6, 3, 3, 1, 1e-3), (6, 3, 3, 1, 1e-2), (6, 2, 3, 4, 1e-3),
                                                  (7, 3, 3, 2, 3e-3)])
def test_list_aci_is_the_grid_aci_on_a_cas(norb, na, nb, seed, sigma):
    h, eri = si.integrals(norb, 2 * norb, seed=seed)
    g = oracle.aci(norb, na, nb, h, eri, sigma)
    r = al.aci_list(norb, na, nb, h, eri, [_grid_start_word(norb, na, nb, h, eri)], sigma)
    assert r["cycles"] == g["cycles"]
    assert r["M"] == _grid_words(norb, na, nb, g["M"])
    assert r["P"] == _grid_words(norb, na, nb, g["P"])
    assert abs(r["E"] - g["E"]) < 1e-11
    assert abs(r["E_corrected"] - g["E_corrected"]) < 1e-11


def test_zero_threshold_reaches_the_sector_ground_state():
    # two electrons in 9 orbitals: every determinant of the sector is within two
    # replacements, so sigma = 0 ends on the sector's lowest root, leaving out only
    # determinants with no weight in it (eps = 0 exactly: here the lowest root has odd
    # S, which gives the nine determinants with both electrons in one orbital none)
    norb, na, nb = 9, 1, 1
    h, eri = si.integrals(norb, 18, seed=6)
    w, vecs = oracle.solve_dense(norb, na, nb, h, eri, nroots=1)
    r = al.aci_list(norb, na, nb, h, eri, [1 | (1 << norb)], 0.0)
    assert abs(r["E"] - w[0]) < 1e-11
    words = _grid_words(norb, na, nb, np.ones(norb * norb, dtype=bool))
    inM = set(r["M"])
    A, B = oracle.strings(norb, na), oracle.strings(norb, nb)
    for i in range(norb * norb):
        wd = int(A[i // norb]) | (int(B[i % norb]) << norb)
        if wd not in inM:
            assert abs(vecs[0][i]) < 1e-10
    assert len(inM) >= norb * (norb - 1) and set(words) >= inM


def test_beyond_a_small_grid_the_model_energy_is_variational_and_tracks_sigma():
    # 2 + 2 electrons in 9 orbitals (1296 determinants): E_M is an upper bound of the
    # sector's lowest root and approaches it as sigma falls
    norb, na, nb = 9, 2, 2
    h, eri = si.integrals(norb, 18, seed=8)
    w, _ = oracle.solve_dense(norb, na, nb, h, eri, nroots=1)
    start = [0b11 | (0b11 << norb)]
    errs = []
    for sigma in (1e-2, 1e-3):
        r = al.aci_list(norb, na, nb, h, eri, start, sigma)
        assert r["E"] >= w[0] - 1e-11
        assert len(r["M"]) < math.comb(norb, na) * math.comb(norb, nb)
        errs.append(r["E"] - w[0])
    assert errs[1] < errs[0]


def _grid_start_word_sector(norb, na, h, eri, parity):
    # the grid version's start: lowest H_II, for the odd sector among alpha != beta
    d = oracle.hdiag(norb, na, na, h, eri)
    A = oracle.strings(norb, na)
    N = len(A)
    if parity < 0:
        d = d.copy()
        d[np.arange(N) * (N + 1)] = np.inf
    i = int(np.argmin(d))
    return int(A[i // N]) | (int(A[i % N]) << norb)


@pytest.mark.parametrize("parity,sigma", [(1, 1e-3), (-1, 1e-3), (1, 0.0)])
def test_list_aci_in_a_parity_sector_is_the_grid_aci(parity, sigma):
    norb, na = 6, 3
    h, eri = si.integrals(norb, 2 * norb, seed=1)
    g = oracle.aci(norb, na, na, h, eri, sigma, parity=parity)
    r = al.aci_list(norb, na, na, h, eri, [_grid_start_word_sector(norb, na, h, eri, parity)], sigma,
                    parity=parity)
    assert r["cycles"] == g["cycles"]
    assert r["M"] == _grid_words(norb, na, na, g["M"])
    assert abs(r["E"] - g["E"]) < 1e-11
    if sigma == 0.0:
        w = np.linalg.eigvalsh(oracle.hmat_dense(norb, na, na, h, eri))
        Q = oracle.sector_basis(len(oracle.strings(norb, na)), parity)
        ws = np.linalg.eigvalsh(Q @ oracle.hmat_dense(norb, na, na, h, eri) @ Q.T)
        assert abs(r["E"] - ws[0]) < 1e-10 and r["E"] >= w[0] - 1e-12
