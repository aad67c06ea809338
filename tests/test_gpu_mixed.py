"""GPU parity of the reduced-precision sigma (tcgen05 alpha-beta GEMM and dense
tcgen05 same-spin GEMM, in TF32 or split BF16) and of the mixed-precision Davidson with FP64
refinement, against the CPU oracle.

Tolerances (max|S - S_ref| / max|S_ref|), from the arithmetic:
  BF16X2: operands carry 16-17 significant bits (|x - hi - lo| <= 2^-17 |x|), the
          dropped lo*lo term is <= 2^-16 |ab|, FP32 accumulation adds ~2^-24 per term;
          the same-spin FP32 path rounds C to 2^-24.  Bound used: 5e-5.
  TF32:   operands rounded to 11 significant bits (2^-11 relative each, ~2^-10 per
          product); bound used: 5e-3.
Energies after the FP64 refinement meet the FP64 tolerance (1e-10 Eh)."""
import os

import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

TOL = {fg.FORTE_BF16X2: 5e-5, fg.FORTE_TF32: 5e-3}
MODES = [fg.FORTE_BF16X2, fg.FORTE_TF32]
CASES = [(2, 1, 1), (4, 2, 2), (5, 2, 3), (6, 3, 3), (7, 3, 2), (8, 4, 4), (9, 2, 5), (10, 5, 5), (6, 3, 0),
         (5, 0, 2), (11, 5, 4)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,na,nb", CASES)
def test_mixed_sigma_matches_oracle(mode, n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=3 * n + na + 7 * nb)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=mode)
    C = si.random_vectors(2, prob.na, prob.nb, seed=4)
    S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    S_ref = oracle.sigma(n, na, nb, h, eri, C)
    for v in range(2):
        err = _rel(S[v], S_ref[v])
        assert err <= TOL[mode], (mode, err)
    prob.close()


@pytest.mark.parametrize("mode", MODES)
def test_mixed_sigma_cas1414_sampled_rows(mode):
    cfg = si.CAS1414
    h, eri = si.integrals(14, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(14, 7, 7, h, eri, precision=mode)
    C = si.random_vectors(1, prob.na, prob.nb, seed=12)
    S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy().reshape(-1)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[0, prob.ndet - 1], rng.integers(0, prob.ndet, size=40)]))
    S_ref = oracle.sigma(14, 7, 7, h, eri, C.reshape(1, -1), rows=rows)[0]
    err = np.abs(S[rows] - S_ref).max() / np.abs(S).max()
    assert err <= TOL[mode], err
    prob.close()


@pytest.mark.parametrize("mode", MODES)
def test_mixed_sigma_agrees_with_fp64_path_cas1212(mode):
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    C = torch.tensor(si.random_vectors(4, prob.na, prob.nb, seed=2), device="cuda")
    S64 = prob.sigma(C)
    prob.set_precision(mode)
    Sm = prob.sigma(C)
    err = float((Sm - S64).abs().max() / S64.abs().max())
    assert err <= TOL[mode], err
    prob.close()


def test_split_operands_round_to_nearest_even():
    # The BF16 hi/lo split reproduces x to ~2^-17 and TF32 to 2^-11 relative; an
    # all-ones vector sigma equals the FP64 one within the TF32 bound.
    h, eri = si.integrals(6, 12, seed=1)
    prob = fg.CASProblem(6, 3, 3, h, eri, precision=fg.FORTE_BF16X2)
    C = torch.ones(1, prob.na, prob.nb, dtype=torch.float64, device="cuda")
    Sm = prob.sigma(C)
    prob.set_precision(fg.FORTE_FP64)
    S64 = prob.sigma(C)
    assert float((Sm - S64).abs().max() / S64.abs().max()) < 5e-5
    prob.close()


@pytest.mark.parametrize("mode", MODES)
def test_mixed_davidson_refines_to_fp64_accuracy(mode):
    cfg = si.CAS88
    h, eri = si.integrals(8, cfg["n_l"], cfg["seed"])
    w, _ = oracle.solve_dense(8, 4, 4, h, eri, nroots=3)
    prob = fg.CASProblem(8, 4, 4, h, eri, precision=mode)
    E, C, rn, it = prob.davidson(nroots=3, tol=1e-10)
    assert np.all(rn < 1e-10)
    assert np.abs(E - w).max() < 1e-10
    n64, nmix = fg.forte_get_counters(prob.ctx)
    assert nmix > 0 and n64 > 0
    prob.close()


def test_mixed_davidson_cas1212_hubbard():
    h, eri = si.hubbard_ring(12, 1.0, 4.0)
    prob64 = fg.CASProblem(12, 6, 6, h, eri)
    E64, _, _, _ = prob64.davidson(nroots=1, tol=1e-8)
    prob64.close()
    prob = fg.CASProblem(12, 6, 6, h, eri, precision=fg.FORTE_BF16X2)
    E, C, rn, it = prob.davidson(nroots=1, tol=1e-8)
    assert abs(E[0] - E64[0]) < 1e-10
    prob.close()
