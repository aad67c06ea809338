"""GPU parity of adaptive CI (Sec. II.A.2) on the CAS determinant grid against
the CPU oracle, cycle by cycle the same spaces: E_M, the corrected energy, the
sizes of M and of the final reference space, the number of cycles and Psi_M."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402


@pytest.mark.parametrize("sigma", [0.0, 1e-2, 1e-3, 1e-4])
@pytest.mark.parametrize("n,na,nb,seed", [(6, 3, 3, 1), (7, 3, 2, 5), (7, 3, 3, 8)])
def test_aci_matches_oracle(n, na, nb, seed, sigma):
    h, eri = si.integrals(n, 2 * n, seed=seed)
    ref = oracle.aci(n, na, nb, h, eri, sigma)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        E, Ec, C, nM, nP, cyc = prob.aci(sigma, tol=1e-11)
        assert abs(E - ref["E"]) < 1e-9
        assert abs(Ec - ref["E_corrected"]) < 1e-9
        if sigma == 0.0:
            # every |eps| > 0 is kept, also the rounding noise (~1e-30) of determinants
            # whose exact V is zero: the sets depend on rounding, the energy does not
            return
        assert nM == int(ref["M"].sum()) and nP == int(ref["P"].sum()) and cyc == ref["cycles"]
        Cn = C.cpu().numpy().reshape(-1)
        assert np.all(Cn[~ref["M"]] == 0.0)
        assert abs(abs(Cn @ ref["C"]) - 1.0) < 1e-9
    finally:
        prob.close()


@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("n,m,seed,sigma", [(6, 3, 1, 1e-2), (6, 3, 1, 1e-3), (7, 3, 8, 1e-3)])
def test_aci_parity_sector_matches_oracle(n, m, seed, sigma, parity):
    h, eri = si.integrals(n, 2 * n, seed=seed)
    ref = oracle.aci(n, m, m, h, eri, sigma, parity=parity)
    prob = fg.CASProblem(n, m, m, h, eri)
    try:
        E, Ec, C, nM, nP, cyc = prob.aci(sigma, tol=1e-11, parity=parity)
        assert abs(E - ref["E"]) < 1e-9 and abs(Ec - ref["E_corrected"]) < 1e-9
        assert nM == int(ref["M"].sum()) and nP == int(ref["P"].sum()) and cyc == ref["cycles"]
        Cn = C.cpu().numpy()
        assert np.abs(Cn - parity * Cn.T).max() <= 1e-15
        # the sector is left again afterwards
        E0, _, _, _ = prob.davidson(nroots=1, tol=1e-10)
        assert E0[0] <= E + 1e-10
    finally:
        prob.close()


def test_aci_tensor_core_precision_mode():
    n, na, nb = 7, 3, 3
    h, eri = si.integrals(n, 14, seed=8)
    ref = oracle.aci(n, na, nb, h, eri, 1e-3)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=fg.FORTE_OZ64)
    try:
        E, Ec, C, nM, nP, cyc = prob.aci(1e-3, tol=1e-11)
        assert nM == int(ref["M"].sum()) and abs(E - ref["E"]) < 1e-9
    finally:
        prob.close()


def test_aci_arguments():
    n = 6
    h, eri = si.integrals(n, 12, seed=2)
    prob = fg.CASProblem(n, 3, 3, h, eri)
    try:
        with pytest.raises(fg.ForteError):
            prob.aci(-1.0)
        with pytest.raises(fg.ForteError):
            prob.aci(1e-3, parity=2)
        prob.set_gas((2, 4), (2, 0), (4, 8))
        with pytest.raises(fg.ForteError):
            prob.aci(1e-3)
    finally:
        prob.close()
