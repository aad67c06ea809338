"""Determinant-list sigma (forte_sci_sigma, the selected-CI data path of
Sec. II.A.2) against the oracle's Slater-Condon sigma over the same list
(oracle.sci_sigma, oracle.hij), and against the grid sigma on a complete list."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402


def _dev_words(words):
    return torch.tensor(np.asarray(words, dtype=np.uint64).view(np.int64), device="cuda")


def _sci_sigma(n, h, eri, words, C):
    sci = fg.forte_sci_create(n, h, eri)
    try:
        Ct = torch.tensor(np.ascontiguousarray(C), device="cuda")
        S = torch.full_like(Ct, np.nan)
        fg.forte_sci_sigma(sci, _dev_words(words), Ct, S, C.shape[0])
        torch.cuda.synchronize()
        return S.cpu().numpy()
    finally:
        fg.forte_sci_destroy(sci)


def _mixed_list(n, na, nb, count, seed):
    # a subset of the reference's singles and doubles (many connected pairs), random
    # determinants of the same sector, and a second sector (na + 1, nb - 1)
    rng = np.random.default_rng(seed)
    exc = si.excitation_list(n, na, nb)
    pick = exc[rng.choice(len(exc), size=min(len(exc), count // 2), replace=False)]
    rand = si.random_determinants(n, na, nb, count // 4, seed + 1)
    other = si.random_determinants(n, na + 1, nb - 1, count // 4, seed + 2)
    words = np.unique(np.concatenate([pick, rand, other]))
    return words[rng.permutation(len(words))]


@pytest.mark.parametrize("n,na,nb,count", [(6, 3, 3, 300), (8, 4, 3, 600), (16, 5, 5, 1200), (24, 6, 6, 1600),
                                           (30, 8, 8, 1600), (32, 7, 6, 1200)])
def test_sci_sigma_matches_oracle(n, na, nb, count):
    h, eri = si.integrals(n, 2 * n, seed=40 + n)
    words = _mixed_list(n, na, nb, count, seed=n)
    rng = np.random.default_rng(n)
    C = rng.normal(size=(2, len(words)))
    S = _sci_sigma(n, h, eri, words, C)
    S_ref = oracle.sci_sigma(n, words, h, eri, C)
    assert np.abs(S - S_ref).max() <= 1e-12 * np.abs(S_ref).max()


def test_sci_sigma_complete_list_equals_grid_sigma():
    # every determinant of CAS(6,6) in grid order: the list sigma is the grid sigma
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 2 * n, seed=3)
    A, B = oracle.strings(n, na), oracle.strings(n, nb)
    words = oracle.det_words(n, np.repeat(A, len(B)), np.tile(B, len(A)))
    C = si.random_vectors(3, len(A), len(B), seed=5).reshape(3, -1)
    S = _sci_sigma(n, h, eri, words, C)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        Sg = prob.sigma(torch.tensor(C.reshape(3, len(A), len(B)), device="cuda")).cpu().numpy().reshape(3, -1)
    finally:
        prob.close()
    assert np.abs(S - Sg).max() <= 1e-12 * np.abs(Sg).max()
    assert np.abs(S - oracle.sigma(n, na, nb, h, eri, C)).max() <= 1e-12 * np.abs(Sg).max()


def test_sci_sigma_large_list_sampled_rows():
    # the singles and doubles of the aufbau determinant of 30 orbitals, 10 + 10
    # electrons (57,501 determinants), 5 vectors (two launches of the kernel):
    # sampled rows against the oracle's matrix elements, summed row by row
    n, na, nb = 30, 10, 10
    h, eri = si.integrals(n, 2 * n, seed=77)
    words = si.excitation_list(n, na, nb)
    rng = np.random.default_rng(1)
    C = rng.normal(size=(5, len(words)))
    S = _sci_sigma(n, h, eri, words, C)
    assert np.all(np.isfinite(S))
    pc = np.vectorize(lambda x: bin(int(x)).count("1"))
    for i in list(rng.choice(len(words), size=6, replace=False)) + [0, len(words) - 1]:
        x = words ^ words[i]
        near = np.nonzero(pc(x) <= 4)[0]
        hrow = np.array([oracle.hij(n, h, eri, int(words[i]), int(words[j])) for j in near])
        ref = C[:, near] @ hrow
        assert np.abs(S[:, i] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), i


def test_sci_sigma_empty_and_errors():
    n = 4
    h, eri = si.integrals(n, 8, seed=0)
    sci = fg.forte_sci_create(n, h, eri)
    try:
        d = _dev_words(np.zeros(0, dtype=np.uint64))
        C = torch.zeros(0, dtype=torch.float64, device="cuda")
        assert fg.forte_sci_sigma(sci, d, C, C, 1) == fg.FORTE_OK
        assert fg.library().forte_sci_sigma(sci, -1, None, None, None, 1) == fg.FORTE_ERR_ARG
        assert fg.library().forte_sci_sigma(sci, 8, None, None, None, 1) == fg.FORTE_ERR_ARG
    finally:
        fg.forte_sci_destroy(sci)
    with pytest.raises(fg.ForteError):
        fg.forte_sci_create(33, np.zeros((33, 33)), np.zeros((33,) * 4))
