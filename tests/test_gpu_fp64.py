"""GPU parity of the FP64 path against the CPU oracle (element by element on
small spaces, sampled rows at the CAS(12,12) and CAS(14,14) sizes).

Tolerances: string tables bit-exact; sigma max|S - S_ref| / max|S_ref| <= 1e-12;
energies 1e-10 Eh; RDMs 1e-9 max-abs."""
import math

import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

SMALL = [(2, 1, 1), (3, 3, 3), (4, 0, 2), (4, 2, 0), (4, 1, 3), (5, 2, 3), (6, 3, 3), (6, 1, 4),
         (7, 3, 2), (7, 4, 4), (8, 4, 4), (9, 2, 5)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n,na,nb", SMALL)
def test_string_tables_bit_exact(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=1)
    prob = fg.CASProblem(n, na, nb, h, eri)
    for spin, ne in ((0, na), (1, nb)):
        s, J, g = prob.string_tables(spin)
        assert np.array_equal(s, oracle.strings(n, ne))
        Jr, gr = oracle.single_table(n, ne)
        assert np.array_equal(J, Jr)
        assert np.array_equal(g, gr)
    prob.close()


@pytest.mark.parametrize("n,na,nb", SMALL)
def test_sigma_fp64_matches_oracle(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=n + 10 * na + 100 * nb)
    prob = fg.CASProblem(n, na, nb, h, eri)
    C = si.random_vectors(3, prob.na, prob.nb, seed=5)
    S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
    S_ref = oracle.sigma(n, na, nb, h, eri, C)
    for v in range(3):
        assert _rel(S[v], S_ref[v]) <= 1e-12
    hd = prob.hdiag().cpu().numpy().reshape(-1)
    assert np.abs(hd - oracle.hdiag(n, na, nb, h, eri)).max() <= 1e-12 * max(1, np.abs(hd).max())
    prob.close()


def _sampled_sigma_check(cfg, nvec, nrows, seed):
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(n, na, nb, h, eri)
    C = si.random_vectors(nvec, prob.na, prob.nb, seed=seed)
    Cd = torch.tensor(C, device="cuda")
    S = prob.sigma(Cd).cpu().numpy().reshape(nvec, -1)
    rng = np.random.default_rng(seed)
    nd = prob.ndet
    rows = np.unique(np.concatenate([[0, nd - 1, prob.nb - 1, nd - prob.nb],
                                     rng.integers(0, nd, size=nrows)]))
    S_ref = oracle.sigma(n, na, nb, h, eri, C.reshape(nvec, -1), rows=rows)
    scale = np.abs(S).max(axis=1)
    for v in range(nvec):
        err = np.abs(S[v, rows] - S_ref[v]).max() / scale[v]
        assert err <= 1e-12, err
    prob.close()


def test_sigma_cas1212_sampled_rows():
    _sampled_sigma_check(si.CAS1212, nvec=4, nrows=400, seed=11)


def test_sigma_cas1414_sampled_rows():
    _sampled_sigma_check(si.CAS1414, nvec=1, nrows=60, seed=12)


def test_sigma_nvec_zero_and_overlap_errors():
    h, eri = si.integrals(4, 8, seed=0)
    prob = fg.CASProblem(4, 2, 2, h, eri)
    C = torch.zeros(2, prob.na, prob.nb, dtype=torch.float64, device="cuda")
    fg.forte_sigma(prob.ctx, C, C, 0)
    with pytest.raises(fg.ForteError):
        fg.forte_sigma(prob.ctx, C, C, 1)
    prob.close()


def test_sigma_is_symmetric_operator_on_random_vectors():
    # x^T H y = y^T H x holds for any size (H symmetric)
    cfg = si.CAS1212
    h, eri = si.integrals(cfg["norb"], cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    C = torch.tensor(si.random_vectors(2, prob.na, prob.nb, seed=3), device="cuda")
    S = prob.sigma(C)
    a = float((C[0] * S[1]).sum())
    b = float((C[1] * S[0]).sum())
    assert abs(a - b) < 1e-12 * max(1.0, abs(a))
    prob.close()


def test_davidson_cas88_matches_dense():
    cfg = si.CAS88
    h, eri = si.integrals(8, cfg["n_l"], cfg["seed"])
    w, V = oracle.solve_dense(8, 4, 4, h, eri, nroots=4)
    prob = fg.CASProblem(8, 4, 4, h, eri)
    E, C, rn, it = prob.davidson(nroots=4, tol=1e-10)
    assert np.all(rn < 1e-10)
    assert np.abs(E - w).max() < 1e-10
    Cn = C.cpu().numpy().reshape(4, -1)
    for k in range(4):
        if min(abs(w[k] - w[j]) for j in range(4) if j != k) > 1e-6:
            assert abs(abs(Cn[k] @ V[k]) - 1) < 1e-9
    prob.close()


@pytest.mark.parametrize("nsites", [4, 6, 8])
def test_davidson_hubbard_ring_ground_state_is_singlet(nsites):
    h, eri = si.hubbard_ring(nsites, 1.0, 4.0)
    k = nsites // 2
    w, _ = oracle.solve_dense(nsites, k, k, h, eri, nroots=1)
    prob = fg.CASProblem(nsites, k, k, h, eri)
    E, C, rn, it = prob.davidson(nroots=1, tol=1e-10)
    assert abs(E[0] - w[0]) < 1e-10
    g1, g2 = prob.rdms(C[0])
    g2 = g2.cpu().numpy()
    N = 2 * k
    s2 = -0.5 * np.einsum("pqqp->", g2) + N * (4 - N) / 4.0
    assert abs(s2) < 1e-8
    prob.close()


def test_davidson_dimer_closed_form():
    t, U = 1.0, 4.0
    h, eri = si.hubbard_ring(2, t, U)
    prob = fg.CASProblem(2, 1, 1, h, eri)
    E, C, rn, it = prob.davidson(nroots=1, tol=1e-12)
    assert abs(E[0] - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12
    prob.close()


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (5, 2, 3), (6, 3, 3), (7, 3, 2), (8, 4, 4)])
def test_rdms_match_oracle(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=40 + n)
    w, V = oracle.solve_dense(n, na, nb, h, eri, nroots=2)
    prob = fg.CASProblem(n, na, nb, h, eri)
    Vd = torch.tensor(V.reshape(2, prob.na, prob.nb), device="cuda")
    g1, g2 = prob.rdms(Vd[0])
    r1, r2 = oracle.rdm12(n, na, nb, V[0])
    assert np.abs(g1.cpu().numpy() - r1).max() < 1e-9
    assert np.abs(g2.cpu().numpy() - r2).max() < 1e-9
    t1 = prob.tdm1(Vd[0], Vd[1]).cpu().numpy()
    q1, _ = oracle.rdm12(n, na, nb, V[0], V[1], two=False)
    assert np.abs(t1 - q1).max() < 1e-9
    prob.close()


def test_rdms_cas1212_sampled_elements_and_invariants():
    cfg = si.CAS1212
    n = 12
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(n, 6, 6, h, eri)
    Ch = si.random_vectors(1, prob.na, prob.nb, seed=9)[0]
    C = torch.tensor(Ch, device="cuda")
    g1, g2 = prob.rdms(C)
    g1, g2 = g1.cpu().numpy(), g2.cpu().numpy()
    N = 12
    assert abs(np.trace(g1) - N) < 1e-9
    assert abs(np.einsum("pprr->", g2) - N * (N - 1)) < 1e-8
    assert np.abs(np.einsum("pqrr->pq", g2) - (N - 1) * g1).max() < 1e-9
    rng = np.random.default_rng(1)
    idx = rng.integers(0, n, size=(24, 4))
    ref = oracle.rdm2_elements(n, 6, 6, Ch, idx)
    assert np.abs(g2[tuple(idx.T)] - ref).max() < 1e-9
    # energy expectation from RDMs equals <C|H|C> from sigma
    S = prob.sigma(C.reshape(1, prob.na, prob.nb))
    e_sig = float((C.reshape(-1) * S.reshape(-1)).sum())
    e_rdm = np.einsum("pq,pq->", h, g1) + 0.5 * np.einsum("pqrs,pqrs->", eri, g2)
    assert abs(e_sig - e_rdm) < 1e-9
    prob.close()


def test_guess_restart_converges_immediately():
    h, eri = si.integrals(8, 16, seed=0)
    prob = fg.CASProblem(8, 4, 4, h, eri)
    E, C, rn, it = prob.davidson(nroots=2, tol=1e-10)
    fg.forte_set_guess(prob.ctx, C, 2)
    E2, C2, rn2, it2 = prob.davidson(nroots=2, tol=1e-10)
    assert np.abs(E2 - E).max() < 1e-10
    assert it2 <= 2
    prob.close()


def test_not_converged_status():
    h, eri = si.integrals(8, 16, seed=0)
    prob = fg.CASProblem(8, 4, 4, h, eri)
    fg.forte_set_davidson_params(prob.ctx, 12, 2, 1, 1e-8)
    with pytest.raises(fg.ForteError) as ei:
        fg.forte_davidson(prob.ctx, 1, 1e-12)
    assert ei.value.code == fg.FORTE_ERR_NOT_CONVERGED
    E, rn, it = fg.forte_get_roots(prob.ctx, 1)
    assert it == 1 and np.isfinite(E[0])
    prob.close()


@pytest.mark.parametrize("n,na,nb,seed,nroots", [(6, 3, 3, 0, 2), (4, 2, 2, 5, 1), (4, 2, 2, 12, 3),
                                                 (6, 2, 4, 3, 3)])
def test_davidson_finds_roots_of_both_spin_flip_sectors(n, na, nb, seed, nroots):
    h, eri = si.integrals(n, 2 * n, seed=seed)
    w, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=nroots)
    prob = fg.CASProblem(n, na, nb, h, eri)
    E, C, rn, it = prob.davidson(nroots=nroots, tol=1e-10)
    assert np.abs(E - w).max() < 1e-10
    prob.close()


@pytest.mark.parametrize("n,na,nb,nroots", [(5, 1, 0, 3), (3, 1, 1, 4), (4, 2, 1, 3), (2, 1, 1, 4)])
def test_davidson_tiny_spaces_with_many_roots(n, na, nb, nroots):
    # subspace limit capped by the dimension: the collapse must never shrink below
    # what the space already holds
    h, eri = si.integrals(n, 2 * n, seed=31 + n)
    w, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=nroots)
    prob = fg.CASProblem(n, na, nb, h, eri)
    E, C, rn, it = prob.davidson(nroots=nroots, tol=1e-10)
    assert np.abs(E - w).max() < 1e-10
    prob.close()


def test_profile_counts_launches():
    h, eri = si.integrals(6, 12, seed=0)
    prob = fg.CASProblem(6, 3, 3, h, eri)
    C = torch.tensor(si.random_vectors(1, prob.na, prob.nb), device="cuda")
    fg.forte_profile_enable(prob.ctx, 1)
    prob.sigma(C)
    fg.forte_profile_enable(prob.ctx, 0)
    table = fg.profile_table(prob.ctx)
    assert table["ab_fp64"][0] == 1 and table["ss_spmm"][0] == 2
    assert fg.forte_get_counters(prob.ctx)[0] == 1
    prob.close()
