"""GPU parity of the FP64-class double-FP32 sigma (FORTE_DF32) against the CPU
oracle and the FP64 path, and of a Davidson solve run entirely on it.

Error bound: each operand is held to 2^-48 relative as hi + lo FP32 values,
each product drops only lo*lo (2^-48) and the hi*hi rounding is recovered by the
FMA, the sums are compensated; per term the relative error is about 2^-46, and
the sums of a few thousand terms per sigma element stay below 1e-12 of
max |sigma| for normalised vectors.  Tests use 1e-12 (relative to max |S|)."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

CASES = [(2, 1, 1), (4, 2, 2), (5, 2, 3), (6, 3, 3), (7, 3, 2), (8, 4, 4), (9, 2, 5), (10, 5, 5), (6, 3, 0),
         (5, 0, 2)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n,na,nb", CASES)
def test_df_sigma_matches_oracle(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=5 * n + na + 3 * nb)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=fg.FORTE_DF32)
    try:
        C = si.random_vectors(2, prob.na, prob.nb, seed=8)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
        S_ref = oracle.sigma(n, na, nb, h, eri, C)
        for v in range(2):
            assert _rel(S[v], S_ref[v]) < 1e-12
    finally:
        prob.close()


def test_df_sigma_agrees_with_fp64_path_cas1212():
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    try:
        C = torch.tensor(si.random_vectors(3, prob.na, prob.nb, seed=6), device="cuda")
        S64 = prob.sigma(C)
        prob.set_precision(fg.FORTE_DF32)
        Sd = prob.sigma(C)
        assert float((Sd - S64).abs().max() / S64.abs().max()) < 1e-12
    finally:
        prob.close()


def test_df_sigma_cas1414_sampled_rows():
    cfg = si.CAS1414
    h, eri = si.integrals(14, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(14, 7, 7, h, eri, precision=fg.FORTE_DF32)
    try:
        C = si.random_vectors(1, prob.na, prob.nb, seed=12)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy().reshape(-1)
        rng = np.random.default_rng(5)
        rows = np.unique(np.concatenate([[0, prob.ndet - 1], rng.integers(0, prob.ndet, size=32)]))
        S_ref = oracle.sigma(14, 7, 7, h, eri, C.reshape(1, -1), rows=rows)[0]
        assert np.abs(S[rows] - S_ref).max() / np.abs(S).max() < 1e-12
    finally:
        prob.close()


def test_df_davidson_matches_dense():
    cfg = si.CAS88
    h, eri = si.integrals(8, cfg["n_l"], cfg["seed"])
    w, _ = oracle.solve_dense(8, 4, 4, h, eri, nroots=3)
    prob = fg.CASProblem(8, 4, 4, h, eri, precision=fg.FORTE_DF32)
    try:
        E, C, rn, it = prob.davidson(nroots=3, tol=1e-10)
        assert np.all(rn < 1e-10)
        assert np.abs(E - w).max() < 1e-10
        n64, nmix = fg.forte_get_counters(prob.ctx)
        assert n64 > 0 and nmix == 0
    finally:
        prob.close()


def test_df_mode_is_accepted_by_the_batch_solver():
    probs = []
    for i in range(4):
        h, eri = si.integrals(6, 12, seed=900 + i)
        probs.append(dict(norb=6, nalpha=3, nbeta=3, nroots=2, h=h, eri=eri))
    E, st = fg.forte_batch_solve(probs, precision=fg.FORTE_DF32, tol=1e-10)
    assert np.all(st == 0)
    for p, e in zip(probs, E):
        w, _ = oracle.solve_dense(6, 3, 3, p["h"], p["eri"], nroots=2)
        assert np.abs(e - w).max() < 1e-10
