"""Pins of the CPU oracle against facts it does not compute itself.

Each test names the passage or mathematical fact it rests on.  None of them
retypes the oracle's own formulas: the Hamiltonian is rebuilt from sparse
Fock-space operator products (tests/fock_ref.py), the string tables are checked
through the gl(n) commutation relations, and the solvers against closed forms.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth_inputs as si
import fock_ref


# ---------------------------------------------------------------- strings
@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (4, 2), (6, 3), (8, 4), (10, 3), (14, 7)])
def test_strings_are_all_combinations_in_ascending_order(n, k):
    # Sec. II.A.1: every string gets a gap-free index; our ordering is ascending mask value.
    want = sorted(sum(1 << i for i in c) for c in itertools.combinations(range(n), k))
    got = oracle.strings(n, k)
    assert len(got) == math.comb(n, k)
    assert list(map(int, got)) == want


def _table_matrices(n, k):
    J, s = oracle.single_table(n, k)
    N = J.shape[0]
    E = np.zeros((n, n, N, N))
    for I in range(N):
        for p in range(n):
            for q in range(n):
                if J[I, p, q] >= 0:
                    E[p, q, J[I, p, q], I] = s[I, p, q]
    return E


@pytest.mark.parametrize("n,k", [(4, 2), (5, 2), (6, 3), (5, 4)])
def test_single_table_obeys_gl_n_commutators(n, k):
    # a+_p a_q of one spin satisfy [E_pq, E_rs] = d_qr E_ps - d_ps E_rq,
    # E_pq^T = E_qp and E_pp = occupation.  A wrong phase or index breaks these.
    E = _table_matrices(n, k)
    for p, q, r, s in itertools.product(range(n), repeat=4):
        lhs = E[p, q] @ E[r, s] - E[r, s] @ E[p, q]
        rhs = (q == r) * E[p, s] - (p == s) * E[r, q]
        assert np.array_equal(lhs, rhs), (p, q, r, s)
    for p, q in itertools.product(range(n), repeat=2):
        assert np.array_equal(E[p, q].T, E[q, p])
    strs = oracle.strings(n, k)
    for p in range(n):
        assert np.array_equal(np.diag(E[p, p]), (strs >> p) & 1)


def test_single_table_matches_fock_space_operators():
    n, k = 5, 2
    _, a = fock_ref.excitation_ops(n)
    idx = fock_ref.sector_states(n, k, 0)  # alpha strings only (beta empty)
    E = _table_matrices(n, k)
    for p, q in itertools.product(range(n), repeat=2):
        M = (a[p].T @ a[q])[idx][:, idx].toarray()
        assert np.array_equal(M, E[p, q])


# ---------------------------------------------------------------- Hamiltonian
CASES = [(2, 1, 1), (3, 1, 1), (3, 2, 1), (4, 2, 2), (4, 3, 1), (4, 1, 0), (5, 2, 3)]


@pytest.mark.parametrize("n,na,nb", CASES)
def test_hamiltonian_equals_operator_form(n, na, nb):
    # Eq. 1 (V = 0) written with spin-free generators: the oracle's Slater-Condon
    # matrix must equal the operator-product matrix element by element.
    h, eri = si.integrals(n, 2 * n, seed=11 + n + 7 * na + 3 * nb)
    H_sc = oracle.hmat_dense(n, na, nb, h, eri)
    H_op = fock_ref.sector_matrix(n, na, nb, h, eri)
    assert np.abs(H_sc - H_op).max() < 1e-13


def test_hamiltonian_is_symmetric():
    h, eri = si.integrals(6, 12, seed=5)
    H = oracle.hmat_dense(6, 3, 3, h, eri)
    assert np.abs(H - H.T).max() < 1e-14


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.5, 1.0), (1.0, 0.0), (0.3, 8.0)])
def test_hubbard_dimer_closed_form(t, U):
    # Two-site Hubbard model at half filling: E0 = (U - sqrt(U^2 + 16 t^2)) / 2.
    h, eri = si.hubbard_ring(2, t, U)
    w, _ = oracle.solve_dense(2, 1, 1, h, eri, nroots=1)
    assert abs(w[0] - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-14


@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (6, 2, 3), (7, 3, 2)])
def test_noninteracting_limit(n, na, nb):
    # g = 0: ground energy = sum of the lowest na + lowest nb eigenvalues of h.
    h, _ = si.integrals(n, 2, seed=3)
    eri = np.zeros((n,) * 4)
    eps = np.linalg.eigvalsh(h)
    w, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=1)
    assert abs(w[0] - (eps[:na].sum() + eps[:nb].sum())) < 1e-12


@pytest.mark.parametrize("nsites", [4, 6])
def test_hubbard_ring_matches_fock_space_diagonalisation(nsites):
    h, eri = si.hubbard_ring(nsites, 1.0, 4.0)
    k = nsites // 2
    w_or, _ = oracle.solve_dense(nsites, k, k, h, eri, nroots=6)
    H_op = fock_ref.sector_matrix(nsites, k, k, h, eri)
    w_op = np.linalg.eigvalsh(H_op)[:6]
    assert np.abs(w_or - w_op).max() < 1e-12


def test_energy_invariant_under_orbital_rotation():
    # Full CI in the active space is invariant under orthogonal orbital rotations.
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 12, seed=21)
    Q = si.random_rotation(n, seed=4)
    h2 = Q.T @ h @ Q
    eri2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", eri, Q, Q, Q, Q)
    w1, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=3)
    w2, _ = oracle.solve_dense(n, na, nb, h2, eri2, nroots=3)
    assert np.abs(w1 - w2).max() < 1e-12


# ---------------------------------------------------------------- sigma
@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (5, 2, 3), (6, 1, 4)])
def test_direct_sigma_equals_dense_product(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=8)
    H = oracle.hmat_dense(n, na, nb, h, eri)
    Na, Nb = math.comb(n, na), math.comb(n, nb)
    C = si.random_vectors(3, Na, Nb, seed=2).reshape(3, -1)
    S = oracle.sigma(n, na, nb, h, eri, C)
    assert np.abs(S - C @ H.T).max() < 1e-13
    rows = np.array([0, Na * Nb - 1, 7 % (Na * Nb), (Na * Nb) // 2])
    Sr = oracle.sigma(n, na, nb, h, eri, C, rows=rows)
    assert np.abs(Sr - S[:, rows]).max() < 1e-14


# ---------------------------------------------------------------- Davidson
def test_davidson_matches_dense_cas88():
    cfg = si.CAS88
    h, eri = si.integrals(cfg["norb"], cfg["n_l"], cfg["seed"])
    w_d, V_d = oracle.solve_dense(8, 4, 4, h, eri, nroots=3)
    w, V, rn, it = oracle.davidson(8, 4, 4, h, eri, nroots=3, tol=1e-10)
    assert np.all(rn < 1e-10)
    assert np.abs(w - w_d).max() < 1e-11
    for k in range(3):
        assert abs(abs(V[k] @ V_d[k]) - 1.0) < 1e-10


# ---------------------------------------------------------------- RDMs
def _ground(n, na, nb, seed, nroots=1):
    h, eri = si.integrals(n, 2 * n, seed=seed)
    w, V = oracle.solve_dense(n, na, nb, h, eri, nroots=nroots)
    return h, eri, w, V


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (4, 2, 1), (5, 3, 2)])
def test_rdms_match_fock_space_expectations(n, na, nb):
    h, eri, w, V = _ground(n, na, nb, seed=31)
    g1, g2 = oracle.rdm12(n, na, nb, V[0])
    f1, f2 = fock_ref.rdms(n, na, nb, V[0])
    assert np.abs(g1 - f1).max() < 1e-13
    assert np.abs(g2 - f2).max() < 1e-13


@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (6, 2, 3)])
def test_rdm_invariants(n, na, nb):
    h, eri, w, V = _ground(n, na, nb, seed=41)
    N = na + nb
    g1, g2 = oracle.rdm12(n, na, nb, V[0])
    assert abs(np.trace(g1) - N) < 1e-12
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-11
    assert np.abs(np.einsum("pqrr->pq", g2) - (N - 1) * g1).max() < 1e-12
    # Energy from the RDMs (the Lagrangian's CI part in Sec. II.B)
    E = np.einsum("pq,pq->", h, g1) + 0.5 * np.einsum("pqrs,pqrs->", eri, g2)
    assert abs(E - w[0]) < 1e-12
    # Hermiticity / particle exchange
    assert np.abs(g1 - g1.T).max() < 1e-13
    assert np.abs(g2 - g2.transpose(2, 3, 0, 1)).max() < 1e-13
    assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-13


@pytest.mark.parametrize("n,na,nb", [(3, 2, 1), (4, 2, 2), (4, 1, 2)])
def test_rdm3_matches_fock_space_identity(n, na, nb):
    """The oracle's 3-RDM (operator strings on determinants) against expectation
    values of E-operator products on the Fock space, reduced by the normal-ordering
    identity (fock_ref.rdm3)."""
    h, eri, w, V = _ground(n, na, nb, seed=61)
    g3 = oracle.rdm3(n, na, nb, V[0])
    f3 = fock_ref.rdm3(n, na, nb, V[0])
    assert np.abs(g3 - f3).max() < 1e-13


@pytest.mark.parametrize("n,na,nb", [(5, 3, 2), (6, 3, 3)])
def test_rdm3_invariants(n, na, nb):
    h, eri, w, V = _ground(n, na, nb, seed=71)
    N = na + nb
    g1, g2 = oracle.rdm12(n, na, nb, V[0])
    g3 = oracle.rdm3(n, na, nb, V[0])
    assert abs(np.einsum("pprrtt->", g3) - N * (N - 1) * (N - 2)) < 1e-10
    assert np.abs(np.einsum("pqrstt->pqrs", g3) - (N - 2) * g2).max() < 1e-12
    # the three (creator, annihilator) pairs commute as units
    assert np.abs(g3 - g3.transpose(2, 3, 0, 1, 4, 5)).max() < 1e-13
    assert np.abs(g3 - g3.transpose(4, 5, 2, 3, 0, 1)).max() < 1e-13
    # Hermiticity for a real vector
    assert np.abs(g3 - g3.transpose(1, 0, 3, 2, 5, 4)).max() < 1e-13


def test_rdm3_of_a_single_determinant():
    """For one determinant Gamma3 is the antisymmetrised product of occupations:
    sum over spin assignments of det[[d_pq, d_ps, d_pu], [d_rq, d_rs, d_ru], [d_tq, d_ts, d_tu]]
    restricted to occupied spin orbitals; checked on its diagonal and exchange elements."""
    n, na, nb = 4, 2, 1  # |alpha 0,1 ; beta 0>
    v = np.zeros(6 * 4)
    v[0] = 1.0  # alpha string {0,1} (index 0) x beta string {0} (index 0)
    g3 = oracle.rdm3(n, na, nb, v)
    occ = {(0, 0), (1, 0), (0, 1)}  # (orbital, spin)
    so = sorted(occ)
    ref = np.zeros((n,) * 6)
    import itertools as it
    for (p, sp_), (r, sr), (t, st) in it.product(so, repeat=3):
        for perm, sign in (((0, 1, 2), 1), ((1, 0, 2), -1), ((0, 2, 1), -1), ((2, 1, 0), -1), ((1, 2, 0), 1), ((2, 0, 1), 1)):
            ann = [(p, sp_), (r, sr), (t, st)]
            a_q, a_s, a_u = ann[perm[0]], ann[perm[1]], ann[perm[2]]
            # pair spins must match: (p,q), (r,s), (t,u)
            if a_q[1] != sp_ or a_s[1] != sr or a_u[1] != st:
                continue
            if len({(p, sp_), (r, sr), (t, st)}) < 3:
                continue
            ref[p, a_q[0], r, a_s[0], t, a_u[0]] += sign
    assert np.abs(g3 - ref).max() < 1e-14


def _s2_from_rdms(g1, g2, N):
    # <S^2> = -1/2 sum_pq Gamma_pqqp + N (4 - N) / 4 for spin-free RDMs.
    return -0.5 * np.einsum("pqqp->", g2) + N * (4 - N) / 4.0


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (5, 3, 2)])
def test_s2_from_rdms_matches_spin_operators(n, na, nb):
    h, eri, w, V = _ground(n, na, nb, seed=51, nroots=3)
    for k in range(3):
        g1, g2 = oracle.rdm12(n, na, nb, V[k])
        assert abs(_s2_from_rdms(g1, g2, na + nb) - fock_ref.s2_expectation(n, na, nb, V[k])) < 1e-12


def test_dimer_ground_state_is_singlet():
    h, eri = si.hubbard_ring(2, 1.0, 4.0)
    w, V = oracle.solve_dense(2, 1, 1, h, eri, nroots=1)
    g1, g2 = oracle.rdm12(2, 1, 1, V[0])
    assert abs(_s2_from_rdms(g1, g2, 2)) < 1e-13


def test_rdm2_elements_agree_with_full_rdm():
    n, na, nb = 6, 3, 3
    h, eri, w, V = _ground(n, na, nb, seed=61)
    _, g2 = oracle.rdm12(n, na, nb, V[0], one=False)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, size=(40, 4))
    got = oracle.rdm2_elements(n, na, nb, V[0], idx)
    assert np.abs(got - g2[tuple(idx.T)]).max() < 1e-14


def test_transition_rdm_matches_fock_space():
    # One-body transition density matrix <Psi_a| a+_x a_u |Psi_b> (Sec. II.A.1).
    n, na, nb = 4, 2, 2
    h, eri, w, V = _ground(n, na, nb, seed=71, nroots=2)
    t1, _ = oracle.rdm12(n, na, nb, V[0], V[1], two=False)
    E, _ = fock_ref.excitation_ops(n)
    bra, ket = fock_ref.embed(n, na, nb, V[0]), fock_ref.embed(n, na, nb, V[1])
    want = np.array([[bra @ (E[p][q] @ ket) for q in range(n)] for p in range(n)])
    assert np.abs(t1 - want).max() < 1e-13


def test_splitmix64_published_value():
    # splitmix64 seeded with 0 gives 0xE220A8397B1DCDAF as its first output
    # (the reference generator of Steele, Lea & Flood 2014).
    from oracle.driver import _splitmix64
    assert int(_splitmix64(np.array([0], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("n,na,nb,seed,nroots", [(6, 3, 3, 0, 2), (4, 2, 2, 5, 1), (4, 2, 2, 12, 3)])
def test_davidson_finds_roots_of_both_spin_flip_sectors(n, na, nb, seed, nroots):
    # With closed-shell guesses the subspace would stay in one spin-flip sector;
    # the lowest roots of the determinant space (any S) must all be found.
    h, eri = si.integrals(n, 2 * n, seed=seed)
    w_d, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=nroots)
    w, V, rn, it = oracle.davidson(n, na, nb, h, eri, nroots=nroots, tol=1e-10)
    assert np.abs(w - w_d).max() < 1e-10


# ---------------------------------------------------------------- occupation-restricted CI
# (Sec. II.A.1: GAS / RAS restrictions on the per-space occupations)
GAS_SETS = [
    # n, na, nb, spaces, gmin, gmax
    (6, 3, 3, (2, 2, 2), (2, 0, 0), (4, 4, 2)),       # RAS: <= 2 holes in RAS1, <= 2 particles in RAS3
    (6, 3, 2, (1, 3, 2), (1, 1, 0), (2, 5, 1)),
    (6, 3, 3, (3, 3), (4, 0), (6, 2)),
    (6, 2, 3, (2, 2, 2), (0, 1, 0), (3, 3, 3)),
]


@pytest.mark.parametrize("n,na,nb,spaces,gmin,gmax", GAS_SETS)
def test_gas_size_matches_occupation_counting(n, na, nb, spaces, gmin, gmax):
    # Number of kept determinants = sum over per-space occupations (a_g, b_g)
    # obeying the limits of prod_g C(size_g, a_g) C(size_g, b_g).
    count = 0
    for a in itertools.product(*[range(s + 1) for s in spaces]):
        if sum(a) != na:
            continue
        for b in itertools.product(*[range(s + 1) for s in spaces]):
            if sum(b) != nb:
                continue
            if all(gmin[g] <= a[g] + b[g] <= gmax[g] for g in range(len(spaces))):
                count += math.prod(math.comb(s, x) * math.comb(s, y) for s, x, y in zip(spaces, a, b))
    keep = oracle.gas_allowed(n, na, nb, spaces, gmin, gmax)
    assert int(keep.sum()) == count


@pytest.mark.parametrize("n,na,nb,spaces,gmin,gmax", GAS_SETS)
def test_gas_eigenvalues_match_fock_space_projection(n, na, nb, spaces, gmin, gmax):
    # Independent route: the operator-product Hamiltonian on the (na, nb) sector,
    # restricted to the Fock states whose per-space occupation (counted from the
    # Fock bit masks) obeys the limits.
    idx = fock_ref.sector_states(n, na, nb)
    H = fock_ref.sector_matrix(n, na, nb, *si.integrals(n, 2 * n, seed=n + na))
    ok = []
    for m in idx:
        m = int(m)
        occ, start = [], 0
        for s in spaces:
            block = ((1 << s) - 1) << start
            occ.append(bin(m & block).count("1") + bin((m >> n) & block).count("1"))
            start += s
        ok.append(all(gmin[g] <= occ[g] <= gmax[g] for g in range(len(spaces))))
    ok = np.array(ok)
    w_op = np.linalg.eigvalsh(H[np.ix_(ok, ok)])[:4]
    h, eri = si.integrals(n, 2 * n, seed=n + na)
    w, V = oracle.solve_dense_gas(n, na, nb, h, eri, spaces, gmin, gmax, nroots=4)
    assert np.abs(w - w_op).max() < 1e-11
    # eigenvectors vanish outside the restricted space and satisfy P H P v = w v
    keep = oracle.gas_allowed(n, na, nb, spaces, gmin, gmax).reshape(-1)
    assert np.all(V[:, ~keep] == 0.0)
    S = oracle.sigma_gas(n, na, nb, h, eri, V, spaces, gmin, gmax)
    assert np.abs(S - w[:, None] * V).max() < 1e-11
    # the same kept set from both routes; P H P C for a vector with weight everywhere
    assert np.array_equal(ok, keep)
    C = np.random.default_rng(5).normal(size=(1, keep.size))
    S = oracle.sigma_gas(n, na, nb, h, eri, C, spaces, gmin, gmax)[0]
    assert np.all(S[~keep] == 0.0)
    assert np.abs(S[keep] - H[np.ix_(ok, ok)] @ C[0, ok]).max() < 1e-11


def test_gas_without_restriction_is_cas():
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 12, seed=8)
    keep = oracle.gas_allowed(n, na, nb, (2, 4), (0, 0), (4, 8))
    assert keep.all()
    w, _ = oracle.solve_dense_gas(n, na, nb, h, eri, (2, 4), (0, 0), (4, 8), nroots=3)
    w0, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=3)
    assert np.abs(w - w0).max() < 1e-12


def test_gas_frozen_doubly_occupied_space_closed_form():
    # A space held at full occupation is a frozen core: E = E_core + CAS on the
    # other orbitals with h'_pq = h_pq + sum_c [2 (pq|cc) - (pc|cq)] and
    # E_core = sum_c 2 h_cc + sum_cd [2 (cc|dd) - (cd|dc)]  (textbook closed-shell energy).
    n, na, nb, nc = 7, 4, 3, 2
    h, eri = si.integrals(n, 14, seed=17)
    w, _ = oracle.solve_dense_gas(n, na, nb, h, eri, (nc, n - nc), (2 * nc, 0), (2 * nc, 2 * (n - nc)), nroots=3)
    c, a = slice(0, nc), slice(nc, n)
    e_core = 2 * np.trace(h[c, c]) + 2 * np.einsum("ccdd->", eri[c, c, c, c]) - np.einsum("cddc->", eri[c, c, c, c])
    h_eff = h[a, a] + 2 * np.einsum("pqcc->pq", eri[a, a, c, c]) - np.einsum("pccq->pq", eri[a, c, c, a])
    w_act, _ = oracle.solve_dense(n - nc, na - nc, nb - nc, h_eff, eri[a, a, a, a].copy(), nroots=3)
    assert np.abs(w - (e_core + w_act)).max() < 1e-11


def test_gas_empty_space_deletes_orbitals():
    # A space held empty removes its orbitals: CAS on the others with h, eri restricted.
    n, na, nb = 7, 3, 3
    h, eri = si.integrals(n, 14, seed=19)
    w, _ = oracle.solve_dense_gas(n, na, nb, h, eri, (5, 2), (0, 0), (10, 0), nroots=3)
    k = slice(0, 5)
    w_sub, _ = oracle.solve_dense(5, na, nb, h[k, k].copy(), eri[k, k, k, k].copy(), nroots=3)
    assert np.abs(w - w_sub).max() < 1e-12


# ---------------------------------------------------------------- spin parity (Ms = 0)
# (Sec. II.A.1: projection on states of well-defined total spin)
@pytest.mark.parametrize("n,m", [(4, 2), (5, 2), (4, 1), (5, 3)])
def test_spin_sectors_partition_the_spectrum_by_parity_of_s(n, m):
    # Exchange of alpha and beta strings commutes with H: the two sectors together
    # hold every eigenvalue once, and every state of the even (odd) sector has even
    # (odd) total spin by the spin operators of the Fock-space route.
    h, eri = si.integrals(n, 2 * n, seed=n + 7 * m)
    N = math.comb(n, m)
    w_all = np.linalg.eigvalsh(fock_ref.sector_matrix(n, m, m, h, eri))
    both = []
    for p in (1, -1):
        dim = N * (N + p) // 2
        assert oracle.sector_basis(N, p).shape == (dim, N * N)
        w, V = oracle.solve_dense_spin(n, m, h, eri, p, nroots=dim)
        both.append(w)
        for k in range(min(dim, 6)):
            s2 = fock_ref.s2_expectation(n, m, m, V[k])
            S = (math.sqrt(1.0 + 4.0 * s2) - 1.0) / 2.0
            assert abs(S - round(S)) < 1e-9 and (-1) ** round(S) == p
    assert np.abs(np.sort(np.concatenate(both)) - w_all).max() < 1e-11


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.5, 1.0)])
def test_spin_sectors_of_the_hubbard_dimer(t, U):
    # Two sites, one electron of each spin: the even sector holds the singlets
    # (lowest (U - sqrt(U^2 + 16 t^2)) / 2, then U, then (U + sqrt(...)) / 2), the odd
    # sector the Ms = 0 triplet at energy 0.
    h, eri = si.hubbard_ring(2, t, U)
    r = math.sqrt(U * U + 16 * t * t)
    w, _ = oracle.solve_dense_spin(2, 1, h, eri, 1, nroots=3)
    assert np.abs(w - np.array([(U - r) / 2, U, (U + r) / 2])).max() < 1e-14
    w, _ = oracle.solve_dense_spin(2, 1, h, eri, -1, nroots=1)
    assert abs(w[0]) < 1e-14


# ---------------------------------------------------------------- adaptive CI
# (Sec. II.A.2: 2 x 2 energy estimates, exclusion of determinants whose summed
# estimates stay below sigma, |E_M - E_CASCI| ~ sigma)
def test_aci_epsilon_is_the_lowest_root_of_the_2x2_problem():
    rng = np.random.default_rng(3)
    E = -5.0
    Hmm = E + rng.uniform(-1.0, 4.0, size=200)
    V = rng.normal(0.0, 0.3, size=200)
    V[:10] = 0.0
    eps = oracle.aci_epsilon(E, Hmm, V)
    ref = [np.linalg.eigvalsh(np.array([[E, v], [v, hm]]))[0] - E for hm, v in zip(Hmm, V)]
    assert np.abs(eps - np.array(ref)).max() < 1e-13


def test_aci_selection_rules_match_sorted_prefixes():
    rng = np.random.default_rng(9)
    a = rng.exponential(1e-4, size=500)
    for sigma in (0.0, 1e-4, 3e-3, 1.0):
        excl = oracle.aci_excluded(a, sigma)
        order = np.argsort(a)
        k = int(np.sum(np.cumsum(a[order]) <= sigma))
        assert set(np.flatnonzero(excl)) == set(order[:k].tolist())
    # equal values leave together or not at all
    b = np.array([1.0, 1.0, 1.0, 5.0])
    assert oracle.aci_excluded(b, 2.5).sum() == 0 and oracle.aci_excluded(b, 3.0).sum() == 3
    c2 = rng.dirichlet(np.ones(300))
    for gs in (0.5, 1e-2, 1e-4):
        keep = oracle.aci_reference(c2, gs)
        order = np.argsort(-c2)
        k = int(np.searchsorted(np.cumsum(c2[order]), 1.0 - gs) + 1)
        assert set(np.flatnonzero(keep)) == set(order[:k].tolist())


@pytest.mark.parametrize("n,na,nb,seed", [(6, 3, 3, 1), (7, 3, 2, 5)])
def test_aci_zero_threshold_reaches_casci(n, na, nb, seed):
    h, eri = si.integrals(n, 2 * n, seed=seed)
    w, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=1)
    r = oracle.aci(n, na, nb, h, eri, 0.0)
    assert abs(r["E"] - w[0]) < 1e-10


@pytest.mark.parametrize("sigma", [1e-2, 1e-3, 1e-4])
def test_aci_energy_error_tracks_sigma(sigma):
    # Variational in M and within a few sigma of CASCI; E_M is the lowest root of
    # the operator-product Hamiltonian restricted to M (independent route).
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 12, seed=1)
    w, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=1)
    r = oracle.aci(n, na, nb, h, eri, sigma)
    assert 0.0 <= r["E"] - w[0] <= 3.0 * sigma
    assert abs(r["E_corrected"] - w[0]) < abs(r["E"] - w[0])
    H = fock_ref.sector_matrix(n, na, nb, h, eri)
    M = r["M"]
    assert abs(np.linalg.eigvalsh(H[np.ix_(M, M)])[0] - r["E"]) < 1e-11
    assert np.all(r["C"][~M] == 0.0) and np.all(r["P"] <= M)


def test_aci_spaces_are_mirror_symmetric_for_equal_spin_counts():
    # n_alpha = n_beta: H commutes with the alpha <-> beta exchange, so the model and
    # reference spaces are closed under it (mirror determinants share estimates).
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 12, seed=1)
    N = math.comb(n, na)
    for sigma in (1e-2, 1e-3):
        r = oracle.aci(n, na, nb, h, eri, sigma)
        for key in ("M", "P"):
            X = r[key].reshape(N, N)
            assert np.array_equal(X, X.T)


@pytest.mark.parametrize("parity", [1, -1])
def test_aci_in_a_parity_sector_reaches_the_sector_casci(parity):
    # sigma = 0 in the even (odd) sector ends at the lowest even-S (odd-S) root, and the
    # vector has the sector's exchange symmetry.
    n, m = 6, 3
    h, eri = si.integrals(n, 12, seed=1)
    w, _ = oracle.solve_dense_spin(n, m, h, eri, parity, nroots=1)
    r = oracle.aci(n, m, m, h, eri, 0.0, parity=parity)
    assert abs(r["E"] - w[0]) < 1e-10
    N = math.comb(n, m)
    C = r["C"].reshape(N, N)
    assert np.abs(C - parity * C.T).max() < 1e-12
    r = oracle.aci(n, m, m, h, eri, 1e-3, parity=parity)
    assert 0.0 <= r["E"] - w[0] <= 3e-3


def test_spin_sectors_partition_an_occupation_restricted_spectrum():
    # The restriction acts on alpha + beta counts, so the kept set is closed under the
    # exchange; the two sectors over it hold the restricted spectrum exactly once.
    n, m = 6, 3
    spaces, gmin, gmax = (2, 2, 2), (2, 0, 0), (4, 4, 2)
    h, eri = si.integrals(n, 12, seed=6)
    keep = oracle.gas_allowed(n, m, m, spaces, gmin, gmax)
    assert np.array_equal(keep, keep.T)
    nd = int(keep.sum())
    w_all, _ = oracle.solve_dense_gas(n, m, m, h, eri, spaces, gmin, gmax, nroots=nd)
    both = []
    for p in (1, -1):
        dim = oracle.sector_basis(keep.shape[0], p, keep).shape[0]
        w, _ = oracle.solve_dense_spin(n, m, h, eri, p, nroots=dim, keep=keep)
        both.append(w)
    assert np.abs(np.sort(np.concatenate(both)) - w_all).max() < 1e-11


# ---------------------------------------------------------------- determinant-list sigma
# (Sec. II.A.2: selected CI works on an arbitrary list of determinants)
def test_sci_sigma_matches_fock_space_on_a_mixed_determinant_list():
    # Random determinants from several (n_alpha, n_beta) sectors, in random order:
    # sigma equals the operator-product Hamiltonian restricted to the list.
    n = 5
    h, eri = si.integrals(n, 10, seed=12)
    rng = np.random.default_rng(4)
    words = []
    # sectors (3, 3), (4, 2) and (1, 1) differ from (2, 2) by two electrons, so their
    # XOR with it can have 2 or 4 bits set while H must still give zero between them
    for na, nb in [(2, 2), (2, 3), (3, 2), (3, 3), (4, 2), (1, 1)]:
        sa, sb = oracle.strings(n, na), oracle.strings(n, nb)
        words += list(oracle.det_words(n, rng.choice(sa, 30), rng.choice(sb, 30)))
    dets = np.unique(np.array(words, dtype=np.uint64))
    rng.shuffle(dets)
    C = rng.normal(size=(2, dets.size))
    H = fock_ref.hamiltonian(n, h, eri)
    idx = dets.astype(np.int64)
    ref = (H[idx][:, idx] @ C.T).T
    assert np.abs(oracle.sci_sigma(n, dets, h, eri, C) - ref).max() < 1e-12


def _det_energy(h, eri, A, B):
    """<D|H|D> from the closed-shell-style sums over occupied alpha (A) and beta (B) orbitals."""
    e = sum(h[a, a] for a in A) + sum(h[b, b] for b in B)
    for S in (A, B):
        e += 0.5 * sum(eri[p, p, q, q] - eri[p, q, q, p] for p in S for q in S)
    e += sum(eri[a, a, b, b] for a in A for b in B)
    return e


def _masks(n, k):
    """All k-of-n occupation masks in ascending order (string addresses, Sec. II.A.1)."""
    return sorted(sum(1 << p for p in c) for c in itertools.combinations(range(n), k))


@pytest.mark.parametrize("n,na,nb", [(5, 3, 1), (6, 2, 4), (6, 3, 3), (7, 4, 2), (4, 0, 2)])
def test_hdiag_matches_closed_form_and_dense_diagonal(n, na, nb):
    # The determinant diagonal (the Davidson preconditioner) at index
    # I_alpha * N_beta + I_beta: the Slater-Condon diagonal written as sums over the
    # occupied orbitals, and the diagonal of the Fock-space-pinned dense H.  Unequal
    # alpha and beta counts make a transposed index visible.
    h, eri = si.integrals(n, 2 * n, seed=40 + n + na)
    d = oracle.hdiag(n, na, nb, h, eri)
    sa, sb = _masks(n, na), _masks(n, nb)
    assert d.shape == (len(sa) * len(sb),)
    ref = np.array([_det_energy(h, eri, [p for p in range(n) if (a >> p) & 1],
                                [p for p in range(n) if (b >> p) & 1]) for a in sa for b in sb])
    assert np.abs(d - ref).max() < 1e-12
    assert np.abs(d - np.diag(oracle.hmat_dense(n, na, nb, h, eri))).max() < 1e-13


def test_sci_sigma_beyond_sixteen_orbitals():
    # 20 orbitals (beta spin orbitals in bits 20..39): Hermiticity, the determinant
    # energy and the single-replacement element in closed form.
    n = 20
    h, eri = si.integrals(n, 40, seed=3)
    rng = np.random.default_rng(6)
    A0, B0 = [0, 1, 2], [0, 1, 3]
    base = sum(1 << a for a in A0) | (sum(1 << b for b in B0) << n)
    singles = []
    for s_ in A0:
        for r in range(n):
            if r not in A0:
                singles.append((r, s_, base ^ (1 << s_) ^ (1 << r)))
    others = [sum(1 << int(x) for x in rng.choice(n, 3, replace=False))
              | (sum(1 << int(x) for x in rng.choice(n, 3, replace=False)) << n) for _ in range(40)]
    dets = np.unique(np.array([base] + [d for _, _, d in singles] + others, dtype=np.uint64))
    H = oracle.sci_sigma(n, dets, h, eri, np.eye(dets.size))
    assert np.abs(H - H.T).max() < 1e-12
    for k, d in enumerate(dets):
        d = int(d)
        A = [p for p in range(n) if (d >> p) & 1]
        B = [p for p in range(n) if (d >> (n + p)) & 1]
        assert abs(H[k, k] - _det_energy(h, eri, A, B)) < 1e-11
    i0 = int(np.flatnonzero(dets == np.uint64(base))[0])
    for r, s_, d in singles:
        j = int(np.flatnonzero(dets == np.uint64(d))[0])
        lo, hi = min(r, s_), max(r, s_)
        sign = (-1) ** sum(1 for a in A0 if lo < a < hi)
        v = h[r, s_] + sum(eri[r, s_, k, k] - eri[r, k, k, s_] for k in A0) + sum(eri[r, s_, k, k] for k in B0)
        assert abs(H[j, i0] - sign * v) < 1e-12
