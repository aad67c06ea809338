"""GPU parity of occupation-restricted CI (GAS / RAS, Sec. II.A.1) against the
CPU oracle: the kept-determinant count, P H P C element by element in the
FP64-class precision modes, Davidson roots of P H P, and at CAS(12,12) the
frozen-core closed form (a space held doubly occupied equals a smaller CAS with
the core's mean field folded into h)."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

# n, na, nb, spaces, gmin, gmax: RAS with 1 and 2 holes / particles, four
# spaces, unequal alpha / beta counts, several 64-string tiles
GAS_SETS = [
    (6, 3, 3, (2, 2, 2), (2, 0, 0), (4, 4, 2)),
    (6, 3, 2, (1, 3, 2), (1, 1, 0), (2, 5, 1)),
    (8, 4, 4, (3, 2, 3), (5, 0, 0), (6, 4, 1)),
    (9, 4, 3, (2, 2, 2, 3), (2, 1, 0, 0), (4, 4, 3, 2)),
    (10, 5, 5, (3, 4, 3), (4, 0, 0), (6, 8, 2)),
]
MODES = [fg.FORTE_FP64, fg.FORTE_DF32, fg.FORTE_OZ64]


def _problem(n, na, nb, spaces, gmin, gmax, precision=fg.FORTE_FP64, seed=None):
    h, eri = si.integrals(n, 2 * n, seed=n + na if seed is None else seed)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=precision)
    nd = prob.set_gas(spaces, gmin, gmax)
    return prob, h, eri, nd


@pytest.mark.parametrize("route", [-1, 0, 1])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,na,nb,spaces,gmin,gmax", GAS_SETS)
def test_gas_sigma_matches_oracle(n, na, nb, spaces, gmin, gmax, mode, route):
    # route -1: timed choice, 0: full grid + projection, 1: kept-determinant kernel
    prob, h, eri, nd = _problem(n, na, nb, spaces, gmin, gmax, mode)
    fg.forte_set_gas_route(prob.ctx, route)
    try:
        keep = oracle.gas_allowed(n, na, nb, spaces, gmin, gmax)
        assert nd == int(keep.sum())
        # weight on every determinant, also the excluded ones: they must count as zero
        C = si.random_vectors(2, prob.na, prob.nb, seed=n)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
        S_ref = oracle.sigma_gas(n, na, nb, h, eri, C, spaces, gmin, gmax)
        assert np.all(S[:, ~keep] == 0.0)
        assert np.abs(S - S_ref).max() < 1e-12 * np.abs(S_ref).max()
        hd = prob.hdiag().cpu().numpy()
        assert np.all(np.isinf(hd[~keep])) and np.all(np.isfinite(hd[keep]))
        assert np.abs(hd[keep] - oracle.hdiag(n, na, nb, h, eri).reshape(keep.shape)[keep]).max() < 1e-11
    finally:
        prob.close()


@pytest.mark.parametrize("route", [0, 1])
@pytest.mark.parametrize("mode", [fg.FORTE_FP64, fg.FORTE_OZ64, fg.FORTE_BF16X2])
@pytest.mark.parametrize("n,na,nb,spaces,gmin,gmax", GAS_SETS[:3])
def test_gas_davidson_matches_dense(n, na, nb, spaces, gmin, gmax, mode, route):
    # route 1 in the BF16x2 mode runs the FP32 kept-determinant kernel in the
    # reduced-precision phase and the FP64 one in the refinement
    prob, h, eri, nd = _problem(n, na, nb, spaces, gmin, gmax, mode)
    fg.forte_set_gas_route(prob.ctx, route)
    try:
        w, V = oracle.solve_dense_gas(n, na, nb, h, eri, spaces, gmin, gmax, nroots=3)
        E, C, rn, it = prob.davidson(nroots=3, tol=1e-9)
        assert np.all(np.asarray(rn) < 1e-9)
        assert np.abs(np.asarray(E) - w).max() < 1e-10
        Cn = C.cpu().numpy().reshape(3, -1)
        keep = oracle.gas_allowed(n, na, nb, spaces, gmin, gmax).reshape(-1)
        assert np.all(Cn[:, ~keep] == 0.0)
        # the ground state is non-degenerate: same vector up to the sign convention
        assert abs(abs(Cn[0] @ V[0]) - 1.0) < 1e-9
    finally:
        prob.close()


def test_gas_frozen_core_closed_form_cas1212():
    """CAS(12,12), 853776 determinants; two orbitals held doubly occupied keep
    the 44100 determinants of CAS(10,8): E = E_core + E_CAS(10,8)(h_eff)."""
    n, na, nb, nc = 12, 6, 6, 2
    cfg = si.CAS1212
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    prob = fg.CASProblem(n, na, nb, h, eri)
    sub = None
    try:
        nd = prob.set_gas((nc, n - nc), (2 * nc, 0), (2 * nc, 2 * (n - nc)))
        assert nd == 210 * 210
        E, C, rn, it = prob.davidson(nroots=2, tol=1e-9)
        c, a = slice(0, nc), slice(nc, n)
        e_core = (2 * np.trace(h[c, c]) + 2 * np.einsum("ccdd->", eri[c, c, c, c])
                  - np.einsum("cddc->", eri[c, c, c, c]))
        h_eff = h[a, a] + 2 * np.einsum("pqcc->pq", eri[a, a, c, c]) - np.einsum("pccq->pq", eri[a, c, c, a])
        sub = fg.CASProblem(n - nc, na - nc, nb - nc, np.ascontiguousarray(h_eff),
                            np.ascontiguousarray(eri[a, a, a, a]))
        E2, _, rn2, _ = sub.davidson(nroots=2, tol=1e-9)
        assert np.abs(np.asarray(E) - (e_core + np.asarray(E2))).max() < 1e-9
    finally:
        prob.close()
        if sub is not None:
            sub.close()


def test_gas_reset_and_errors():
    n, na, nb = 6, 3, 3
    h, eri = si.integrals(n, 12, seed=4)
    prob = fg.CASProblem(n, na, nb, h, eri)
    try:
        C = torch.tensor(si.random_vectors(1, prob.na, prob.nb, seed=2), device="cuda")
        S_full = prob.sigma(C)
        nd = prob.set_gas((2, 4), (2, 0), (4, 4))
        assert 0 < nd < prob.ndet
        for bad in [((2, 3), (0, 0), (4, 6)),        # sizes do not add up to n
                    ((2, 4), (3, 0), (2, 8)),        # gmin > gmax
                    ((0, 6), (0, 0), (0, 12)),       # empty space
                    ((3, 3), (6, 6), (6, 6))]:       # keeps no determinant
            with pytest.raises(fg.ForteError):
                prob.set_gas(*bad)
        # a rejected call leaves the previous restriction in force
        S = prob.sigma(C)
        keep = oracle.gas_allowed(n, na, nb, (2, 4), (2, 0), (4, 4))
        assert np.all(S.cpu().numpy()[:, ~keep] == 0.0)
        assert prob.set_gas((), (), ()) == prob.ndet
        assert float((prob.sigma(C) - S_full).abs().max()) <= 1e-13 * float(S_full.abs().max())
        assert bool(torch.isfinite(prob.hdiag()).all())
    finally:
        prob.close()


def test_gas_timed_route_records_both_timings():
    # CAS(10,10) under RAS(2h, 2p) keeps well below a quarter of the determinants:
    # the first sigma times both routes and keeps the faster
    n, na, nb, spaces, gmin, gmax = 10, 5, 5, (3, 4, 3), (4, 0, 0), (6, 10, 2)
    prob, h, eri, nd = _problem(n, na, nb, spaces, gmin, gmax, fg.FORTE_FP64)
    try:
        assert 4 * nd <= prob.ndet
        assert fg.forte_get_gas_route(prob.ctx)[0] == -1
        C = si.random_vectors(1, prob.na, prob.nb, seed=4)
        S = prob.sigma(torch.tensor(C, device="cuda")).cpu().numpy()
        r64, r32, ms = fg.forte_get_gas_route(prob.ctx)
        assert r64 in (0, 1) and ms[0] > 0 and ms[1] > 0
        assert r64 == (1 if ms[1] <= ms[0] else 0)
        S_ref = oracle.sigma_gas(n, na, nb, h, eri, C, spaces, gmin, gmax)
        assert np.abs(S - S_ref).max() < 1e-12 * np.abs(S_ref).max()
        with pytest.raises(fg.ForteError):
            fg.forte_set_gas_route(prob.ctx, 2)
    finally:
        prob.close()
