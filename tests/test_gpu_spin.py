"""GPU parity of the Ms = 0 spin-parity sectors (Sec. II.A.1, projection on
states of well-defined total spin) against the CPU oracle: Davidson roots in
the even-S and odd-S sectors, alone and combined with an occupation
restriction, in the FP64, FORTE_OZ64 and BF16x2 modes; the exact exchange
symmetry of the returned vectors; and at CAS(12,12) the sector roots against
the unrestricted solve."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

MODES = [fg.FORTE_FP64, fg.FORTE_OZ64, fg.FORTE_BF16X2]


def _exchange_error(C, parity):
    C = C.cpu().numpy()
    return float(np.abs(C - parity * np.swapaxes(C, -1, -2)).max())


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (8, 4), (7, 2)])
def test_spin_sector_roots_match_oracle(n, m, parity, mode):
    h, eri = si.integrals(n, 2 * n, seed=3 * n + m)
    w, V = oracle.solve_dense_spin(n, m, h, eri, parity, nroots=3)
    prob = fg.CASProblem(n, m, m, h, eri, precision=mode)
    try:
        prob.set_spin_parity(parity)
        E, C, rn, it = prob.davidson(nroots=3, tol=1e-9)
        assert np.all(np.asarray(rn) < 1e-9)
        assert np.abs(np.asarray(E) - w).max() < 1e-10
        assert _exchange_error(C, parity) == 0.0
        assert abs(abs(C[0].cpu().numpy().reshape(-1) @ V[0]) - 1.0) < 1e-9
    finally:
        prob.close()


@pytest.mark.parametrize("parity", [1, -1])
def test_spin_sector_with_occupation_restriction(parity):
    n, m = 8, 4
    spaces, gmin, gmax = (2, 4, 2), (2, 0, 0), (4, 8, 2)
    h, eri = si.integrals(n, 16, seed=41)
    keep = oracle.gas_allowed(n, m, m, spaces, gmin, gmax)
    w, _ = oracle.solve_dense_spin(n, m, h, eri, parity, nroots=3, keep=keep)
    prob = fg.CASProblem(n, m, m, h, eri)
    try:
        prob.set_gas(spaces, gmin, gmax)
        prob.set_spin_parity(parity)
        E, C, rn, it = prob.davidson(nroots=3, tol=1e-9)
        assert np.abs(np.asarray(E) - w).max() < 1e-10
        Cn = C.cpu().numpy()
        assert np.all(Cn[:, ~keep] == 0.0)
        assert _exchange_error(C, parity) == 0.0
    finally:
        prob.close()


def test_spin_sectors_against_unrestricted_solve_cas1212():
    """The lowest even-S and odd-S roots equal the lowest unrestricted roots of
    that exchange parity (853776 determinants)."""
    cfg = si.CAS1212
    h, eri = si.integrals(12, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(12, 6, 6, h, eri)
    try:
        E, C, rn, it = prob.davidson(nroots=6, tol=1e-9)
        par = [float((c * c.T).sum()) for c in C]
        assert all(abs(abs(p) - 1.0) < 1e-8 for p in par)
        for parity in (1, -1):
            mine = [e for e, p in zip(E, par) if np.sign(p) == parity]
            if not mine:
                continue
            prob.set_spin_parity(parity)
            Es, Cs, rns, _ = prob.davidson(nroots=1, tol=1e-9)
            assert abs(Es[0] - mine[0]) < 1e-9
            assert _exchange_error(Cs, parity) == 0.0
        prob.set_spin_parity(0)
    finally:
        prob.close()


def test_spin_parity_arguments():
    n = 6
    h, eri = si.integrals(n, 12, seed=2)
    prob = fg.CASProblem(n, 3, 2, h, eri)
    try:
        with pytest.raises(fg.ForteError):
            prob.set_spin_parity(1)   # n_alpha != n_beta
        prob.set_spin_parity(0)
    finally:
        prob.close()
    prob = fg.CASProblem(n, 3, 3, h, eri)
    try:
        with pytest.raises(fg.ForteError):
            prob.set_spin_parity(2)
        # the odd sector of CAS(2,2) with one electron per spin has dimension 1
        sub = fg.CASProblem(2, 1, 1, *si.hubbard_ring(2, 1.0, 4.0))
        try:
            sub.set_spin_parity(-1)
            E, C, rn, it = sub.davidson(nroots=1, tol=1e-12)
            assert abs(E[0]) < 1e-13
            with pytest.raises(fg.ForteError):
                sub.davidson(nroots=2, tol=1e-12)
        finally:
            sub.close()
    finally:
        prob.close()
