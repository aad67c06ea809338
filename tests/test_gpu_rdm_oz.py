"""GPU parity of the tensor-core 2-RDM (reduced-precision modes) against the CPU
oracle and against the FP64 Gram path.

In FORTE_BF16X2 / FORTE_TF32 mode forte_rdms forms the 2-RDM from the Gram
matrices of the symmetric and antisymmetric one-body images, computed with exact
integer products of 8-bit digit slices on the BF16 tensor cores; the cross block
comes from the 1-RDM.  Error bound: every element of a Gram row is held to
2^-46 of the row maximum and digit products below 2^-50 of the product of the two
row maxima are dropped, so for normalised vectors an absolute error of 1e-11 on
every RDM element is a wide margin; the tests use that bound."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

TOL = 1e-11
# (n, na, nb): every padded row count of the kernel (16..112 for the symmetric rows,
# 16..96 for the antisymmetric ones), unequal alpha / beta strings, ragged chunks
CASES = [(2, 1, 1), (3, 1, 2), (4, 2, 2), (5, 2, 3), (6, 3, 3), (7, 3, 2), (8, 4, 4), (9, 2, 5), (10, 5, 5),
         (11, 3, 3), (12, 2, 3), (13, 2, 2), (14, 2, 3)]


def _rdms(prob, C, mode):
    prob.set_precision(mode)
    g1, g2 = prob.rdms(C)
    return g1.cpu().numpy(), g2.cpu().numpy()


def _wide_range_vector(na, nb, seed):
    """Normalised vector whose magnitudes span 1e-14 .. 1 (log-uniform), random signs."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(1e-14), 0.0, size=na * nb)) * rng.choice([-1.0, 1.0], size=na * nb)
    return x / np.linalg.norm(x)


@pytest.mark.parametrize("mode", [fg.FORTE_BF16X2, fg.FORTE_TF32])
@pytest.mark.parametrize("n,na,nb", CASES)
def test_oz_rdms_match_oracle(mode, n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=60 + n)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        if prob.ndet <= 4000:
            _, V = oracle.solve_dense(n, na, nb, h, eri, nroots=1)
            c = V[0]
        else:
            c = si.random_vectors(1, prob.na, prob.nb, seed=n)[0].reshape(-1)
        C = torch.tensor(c.reshape(prob.na, prob.nb), device="cuda")
        g1, g2 = _rdms(prob, C, mode)
        r1, r2 = oracle.rdm12(n, na, nb, c)
        assert np.abs(g1 - r1).max() < 1e-12
        assert np.abs(g2 - r2).max() < TOL
    finally:
        prob.close()


@pytest.mark.parametrize("n,na,nb", [(6, 3, 3), (8, 3, 4), (10, 5, 5)])
def test_oz_rdms_wide_dynamic_range(n, na, nb):
    """Entries from 1e-14 to 1: per-row fixed point must keep the small ones."""
    h, eri = si.integrals(n, 2 * n, seed=7)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        c = _wide_range_vector(prob.na, prob.nb, seed=n)
        C = torch.tensor(c.reshape(prob.na, prob.nb), device="cuda")
        _, g2o = _rdms(prob, C, fg.FORTE_BF16X2)
        _, g2d = _rdms(prob, C, fg.FORTE_FP64)
        _, r2 = oracle.rdm12(n, na, nb, c)
        assert np.abs(g2d - r2).max() < 1e-12
        assert np.abs(g2o - r2).max() < TOL
    finally:
        prob.close()


def test_oz_rdms_scaled_vector_is_homogeneous():
    """Gamma(c C) = c^2 Gamma(C): the fixed-point scale follows max |C|."""
    n, na, nb = 8, 4, 4
    h, eri = si.integrals(n, 16, seed=3)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=fg.FORTE_BF16X2)
    try:
        c = si.random_vectors(1, prob.na, prob.nb, seed=5)[0]
        C = torch.tensor(c, device="cuda")
        _, g2 = prob.rdms(C)
        _, g2s = prob.rdms(C * 1e-7)
        g2, g2s = g2.cpu().numpy(), g2s.cpu().numpy()
        assert np.abs(g2s * 1e14 - g2).max() < TOL
        Z = torch.zeros_like(C)
        g1z, g2z = prob.rdms(Z)
        assert float(g1z.abs().max()) == 0.0 and float(g2z.abs().max()) == 0.0
    finally:
        prob.close()


def test_oz_rdms_cas1212_match_fp64_path_and_invariants():
    cfg = si.CAS1212
    n = 12
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(n, 6, 6, h, eri)
    try:
        Ch = si.random_vectors(1, prob.na, prob.nb, seed=9)[0]
        C = torch.tensor(Ch, device="cuda")
        g1d, g2d = _rdms(prob, C, fg.FORTE_FP64)
        g1o, g2o = _rdms(prob, C, fg.FORTE_BF16X2)
        assert np.abs(g1o - g1d).max() == 0.0  # the 1-RDM is the FP64 one in every mode
        assert np.abs(g2o - g2d).max() < TOL
        N = 12
        assert abs(np.einsum("pprr->", g2o) - N * (N - 1)) < 1e-9
        assert np.abs(np.einsum("pqrr->pq", g2o) - (N - 1) * g1o).max() < 1e-10
        assert np.abs(g2o - g2o.transpose(2, 3, 0, 1)).max() < TOL
        rng = np.random.default_rng(2)
        idx = rng.integers(0, n, size=(16, 4))
        ref = oracle.rdm2_elements(n, 6, 6, Ch, idx)
        assert np.abs(g2o[tuple(idx.T)] - ref).max() < TOL
    finally:
        prob.close()


def test_oz_rdms_cas1414_match_fp64_path_and_oracle_elements():
    """The CAS(14,14) workload: 11.8 M determinants, 105 + 91 Gram rows.  The
    tensor-core 2-RDM equals the FP64 path everywhere and the oracle's operator
    application on sampled elements (random ones, and the diagonal-type
    Gamma_ppqq / Gamma_pqqp that carry the largest values)."""
    cfg = si.CAS1414
    n = 14
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(n, 7, 7, h, eri)
    try:
        Ch = si.random_vectors(1, prob.na, prob.nb, seed=11)[0]
        C = torch.tensor(Ch, device="cuda")
        _, g2d = _rdms(prob, C, fg.FORTE_FP64)
        _, g2o = _rdms(prob, C, fg.FORTE_BF16X2)
        assert np.abs(g2o - g2d).max() < TOL
        rng = np.random.default_rng(14)
        idx = np.vstack([rng.integers(0, n, size=(12, 4)),
                         [[0, 0, 13, 13], [5, 5, 5, 5], [2, 9, 9, 2], [13, 6, 6, 13]]])
        ref = oracle.rdm2_elements(n, 7, 7, Ch, idx)
        assert np.abs(g2o[tuple(idx.T)] - ref).max() < TOL
    finally:
        prob.close()


def test_oz_state_averaged_gradient_uses_tensor_core_rdms():
    """forte_sa_gradient in BF16X2 mode equals the FP64-mode gradient to the RDM bound."""
    n, na, nb = 8, 4, 4
    h, eri = si.integrals(n, 16, seed=12)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        _, V = oracle.solve_dense(n, na, nb, h, eri, nroots=2)
        C = torch.tensor(V.reshape(2, prob.na, prob.nb), device="cuda")
        w = np.array([0.5, 0.5])
        out = []
        for mode in (fg.FORTE_FP64, fg.FORTE_BF16X2):
            prob.set_precision(mode)
            dh = torch.zeros(n, n, dtype=torch.float64, device="cuda")
            de = torch.zeros((n,) * 4, dtype=torch.float64, device="cuda")
            fg.forte_sa_gradient(prob.ctx, 2, w, C, 1.0, dh, de, n)
            out.append((dh.cpu().numpy(), de.cpu().numpy()))
        assert np.abs(out[0][0] - out[1][0]).max() < 1e-12
        assert np.abs(out[0][1] - out[1][1]).max() < TOL
    finally:
        prob.close()
