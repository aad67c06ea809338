"""GPU parity of the spin-free 3-RDM (Sec. II.A.1, gamma_3 summed over spin)
against the CPU oracle, element by element, and its invariants at a size the
oracle is not run on.  FP64 on both sides: the GPU sums the same products in
another order, so the tolerance is 1e-12 of max |Gamma3|."""
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
# one or several Gram tiles (n^2 = 9 .. 49), one empty spin, a single electron
CASES = [(3, 1, 1), (4, 2, 2), (5, 2, 3), (6, 3, 3), (6, 3, 0), (7, 3, 2), (5, 1, 0)]


def _unit(C):
    return C / np.linalg.norm(C)


@pytest.mark.parametrize("n,na,nb", CASES)
def test_rdm3_matches_oracle(n, na, nb):
    h, eri = si.integrals(n, 2 * n, seed=5 * n + na)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        C = _unit(si.random_vectors(1, prob.na, prob.nb, seed=n + nb)[0])
        g3 = prob.rdm3(torch.tensor(C, device="cuda")).cpu().numpy()
        ref = oracle.rdm3(n, na, nb, C)
        scale = max(np.abs(ref).max(), 1.0)
        assert np.abs(g3 - ref).max() < TOL * scale
    finally:
        prob.close()


def test_rdm3_ground_state_invariants_cas88():
    """CAS(8,8) ground state (4900 determinants): partial traces give the 2-RDM,
    the full trace N(N-1)(N-2), and the 3-RDM is symmetric under exchange of the
    pairs and under bra-ket transposition."""
    cfg = si.CAS88
    n, N = 8, 8
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(n, 4, 4, h, eri)
    try:
        E, C, rn, it = prob.davidson(nroots=1, tol=1e-10)
        g1, g2 = (x.cpu().numpy() for x in prob.rdms(C[0]))
        g3 = prob.rdm3(C[0]).cpu().numpy()
        assert np.abs(np.einsum("pqrstt->pqrs", g3) - (N - 2) * g2).max() < 1e-11
        assert abs(np.einsum("ppqqrr->", g3) - N * (N - 1) * (N - 2)) < 1e-9
        assert np.abs(g3 - g3.transpose(2, 3, 0, 1, 4, 5)).max() < 1e-12
        assert np.abs(g3 - g3.transpose(0, 1, 4, 5, 2, 3)).max() < 1e-12
        assert np.abs(g3 - g3.transpose(1, 0, 3, 2, 5, 4)).max() < 1e-12
    finally:
        prob.close()


def test_rdm3_is_fp64_in_reduced_precision_mode():
    """The 3-RDM takes the FP64 1-/2-RDMs whatever the sigma precision."""
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 12, seed=3)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=fg.FORTE_BF16X2)
    try:
        C = _unit(si.random_vectors(1, prob.na, prob.nb, seed=9)[0])
        g3 = prob.rdm3(torch.tensor(C, device="cuda")).cpu().numpy()
        ref = oracle.rdm3(n, na, nb, C)
        assert np.abs(g3 - ref).max() < TOL * max(np.abs(ref).max(), 1.0)
    finally:
        prob.close()
