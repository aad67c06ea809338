"""GPU parity of the FP64-class sigma whose alpha-beta term is formed from exact
digit products on the tensor cores (FORTE_OZ64) against the CPU oracle and the
FP64 path, and of Davidson solves that use it.

Error bound: each integral row and each 64-string tile of C is held in 45-bit
fixed point relative to its own maximum (2^-46 relative), the digit products are exact
up to the dropped levels (~2^-50 of K times the product of the two scales) and every
contribution is rounded once onto a 64-bit grid 2^-62 below the bound
n_kl(alpha) n_kl(beta) max|g| max|C|.  Per term that is ~2^-45 of |g| |C| at the
row / column maxima; with a few thousand terms per element the error stays below
1e-12 of max |sigma| for normalised vectors, the tolerance of the double-FP32
same-spin part as well.  The tests use 1e-12 (relative to max |S|)."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

TOL = 1e-12
# several 64-string tiles with ragged tails, unequal alpha / beta strings, one
# empty spin, n_kl from 1 to 56
CASES = [(2, 1, 1), (4, 2, 2), (5, 2, 3), (6, 3, 3), (7, 3, 2), (8, 4, 4), (9, 2, 5), (10, 5, 5), (11, 5, 4),
         (6, 3, 0), (5, 0, 2)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n,na,nb", CASES)
def test_oz64_sigma_matches_oracle(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=7 * n + na + 5 * nb)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=fg.FORTE_OZ64)
    try:
        C = si.random_vectors(2, prob.na, prob.nb, seed=3)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
        S_ref = oracle.sigma(n, na, nb, h, eri, C)
        for v in range(2):
            assert _rel(S[v], S_ref[v]) < TOL
    finally:
        prob.close()


def test_oz64_sigma_agrees_with_fp64_path_cas1212():
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    try:
        C = torch.tensor(si.random_vectors(3, prob.na, prob.nb, seed=6), device="cuda")
        S64 = prob.sigma(C)
        prob.set_precision(fg.FORTE_OZ64)
        So = prob.sigma(C)
        assert float((So - S64).abs().max() / S64.abs().max()) < TOL
        # integer sums: a second call is bit-identical
        So2 = prob.sigma(C)
        assert torch.equal(So, So2)
    finally:
        prob.close()


def test_oz64_sigma_cas1414_sampled_rows():
    """The CAS(14,14) workload (11.8 M determinants, 54 tiles per alpha string)."""
    cfg = si.CAS1414
    h, eri = si.integrals(14, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(14, 7, 7, h, eri, precision=fg.FORTE_OZ64)
    try:
        C = si.random_vectors(1, prob.na, prob.nb, seed=13)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy().reshape(-1)
        rng = np.random.default_rng(8)
        rows = np.unique(np.concatenate([[0, prob.ndet - 1], rng.integers(0, prob.ndet, size=32)]))
        S_ref = oracle.sigma(14, 7, 7, h, eri, C.reshape(1, -1), rows=rows)[0]
        assert np.abs(S[rows] - S_ref).max() / np.abs(S).max() < TOL
    finally:
        prob.close()


def test_oz64_wide_dynamic_range_and_scaling():
    """Entries from 1e-14 to 1 (per-column fixed point keeps the small columns), a
    vector scaled by 1e-7 (the scales follow max |C|) and the zero vector."""
    n, na, nb = 8, 4, 4
    h, eri = si.integrals(n, 16, seed=21)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        rng = np.random.default_rng(4)
        x = np.exp(rng.uniform(np.log(1e-14), 0.0, size=prob.ndet)) * rng.choice([-1.0, 1.0], size=prob.ndet)
        x /= np.linalg.norm(x)
        C = torch.tensor(x.reshape(1, prob.na, prob.nb), device="cuda")
        S64 = prob.sigma(C).cpu().numpy()
        prob.set_precision(fg.FORTE_OZ64)
        So = prob.sigma(C).cpu().numpy()
        assert _rel(So, S64) < TOL
        Ss = prob.sigma(C * 1e-7).cpu().numpy()
        assert _rel(Ss * 1e7, S64) < TOL
        Z = prob.sigma(torch.zeros_like(C))
        assert float(Z.abs().max()) == 0.0
    finally:
        prob.close()


@pytest.mark.parametrize("n,na,nb", [(15, 1, 2), (16, 1, 1)])
def test_oz64_largest_orbital_counts(n, na, nb):
    """n = 15 (120 symmetric pairs) is the largest on the tensor-core path; n = 16
    (136 pairs) uses the double-FP32 alpha-beta term."""
    h, eri = si.integrals(n, 2 * n, seed=2)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=fg.FORTE_OZ64)
    try:
        C = si.random_vectors(1, prob.na, prob.nb, seed=1)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
        assert _rel(S[0], oracle.sigma(n, na, nb, h, eri, C)[0]) < TOL
    finally:
        prob.close()


def test_oz64_davidson_matches_dense():
    cfg = si.CAS88
    h, eri = si.integrals(8, cfg["n_l"], cfg["seed"])
    w, _ = oracle.solve_dense(8, 4, 4, h, eri, nroots=3)
    prob = fg.CASProblem(8, 4, 4, h, eri, precision=fg.FORTE_OZ64)
    try:
        E, C, rn, it = prob.davidson(nroots=3, tol=1e-10)
        assert np.all(rn < 1e-10)
        assert np.abs(E - w).max() < 1e-10
        n64, nmix = fg.forte_get_counters(prob.ctx)
        assert n64 > 0 and nmix == 0
    finally:
        prob.close()


def test_mixed_refinement_reaches_tight_tolerance_cas1212():
    """BF16X2 Davidson refined with the FORTE_OZ64 sigma to 1e-9 against the FP64 solve."""
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    try:
        E64, _, _, _ = prob.davidson(nroots=2, tol=1e-9)
        prob.set_precision(fg.FORTE_BF16X2)
        E, C, rn, it = prob.davidson(nroots=2, tol=1e-9)
        assert np.all(np.asarray(rn) < 1e-9)
        assert np.abs(np.asarray(E) - np.asarray(E64)).max() < 1e-11
    finally:
        prob.close()
