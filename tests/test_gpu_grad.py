"""Differentiation of the state-averaged energy E_SA = sum_k w_k E_k (Sec. II.B
Lagrangian, CI part): the backward of `sa_energy` is the library's adjoint
kernel (forte_sa_gradient), dE/dh = sum w gamma and dE/d(pq|rs) = 1/2 sum w Gamma.

Checked against (i) the oracle's RDMs of its own dense eigenvectors and (ii)
central finite differences (step 1e-5) along symmetry orbits of the integrals
(h_pq with h_qp; the 8 equivalents of (pq|rs)), so that the convention for the
split of the derivative among equivalent entries cancels.  Tolerance 1e-6
absolute for the finite differences (energy noise ~1e-12 / step + O(step^2))."""
import itertools
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


def _orbit_h(n, p, q):
    m = np.zeros((n, n))
    m[p, q] = m[q, p] = 1.0
    return m


def _orbit_eri(n, p, q, r, s):
    m = np.zeros((n,) * 4)
    for a, b, c, d in {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                       (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}:
        m[a, b, c, d] = 1.0
    return m


def _energy(h, eri, n, na, nb, w, precision=fg.FORTE_FP64):
    with torch.no_grad():
        e = fg.sa_energy(torch.tensor(h), torch.tensor(eri), n, na, nb, w, precision=precision, tol=1e-10)
    return float(e)


@pytest.mark.parametrize("n,na,nb,seed", [(6, 3, 3, 3), (6, 2, 3, 4)])
def test_sa_gradient_equals_weighted_oracle_rdms(n, na, nb, seed):
    h, eri = si.integrals(n, 2 * n, seed=seed)
    w = [1 / 3, 1 / 3, 1 / 3]
    ev, V = oracle.solve_dense(n, na, nb, h, eri, nroots=4)
    assert ev[3] - ev[2] > 1e-4 and min(np.diff(ev[:3])) > 1e-6
    ht = torch.tensor(h, requires_grad=True)
    et = torch.tensor(eri, requires_grad=True)
    E = fg.sa_energy(ht, et, n, na, nb, w)
    E.backward()
    assert abs(float(E.detach()) - sum(wi * e for wi, e in zip(w, ev[:3]))) < 1e-10
    g1 = sum(wi * oracle.rdm12(n, na, nb, V[k], two=False)[0] for k, wi in enumerate(w))
    g2 = sum(wi * oracle.rdm12(n, na, nb, V[k], one=False)[1] for k, wi in enumerate(w))
    assert np.abs(ht.grad.numpy() - g1).max() < 1e-9
    assert np.abs(et.grad.numpy() - 0.5 * g2).max() < 1e-9


def test_sa_gradient_central_differences_small():
    n, na, nb, seed = 6, 3, 3, 3
    h, eri = si.integrals(n, 2 * n, seed=seed)
    w = [1 / 3, 1 / 3, 1 / 3]
    ht = torch.tensor(h, requires_grad=True)
    et = torch.tensor(eri, requires_grad=True)
    fg.sa_energy(ht, et, n, na, nb, w).backward()
    gh, ge = ht.grad.numpy(), et.grad.numpy()
    rng = np.random.default_rng(17)
    step = 1e-5
    for _ in range(8):
        p, q = rng.integers(0, n, size=2)
        d = _orbit_h(n, p, q)
        fd = (_energy(h + step * d, eri, n, na, nb, w) - _energy(h - step * d, eri, n, na, nb, w)) / (2 * step)
        assert abs(fd - (gh * d).sum()) < 1e-6, ("h", p, q)
    for _ in range(8):
        p, q, r, s = rng.integers(0, n, size=4)
        d = _orbit_eri(n, p, q, r, s)
        fd = (_energy(h, eri + step * d, n, na, nb, w) - _energy(h, eri - step * d, n, na, nb, w)) / (2 * step)
        assert abs(fd - (ge * d).sum()) < 1e-6, ("eri", p, q, r, s)


GOLDEN_SA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cas1212_seed3_3roots.json")


def _orbits64(n, seed=3):
    """32 symmetry orbits of h (p <= q) and 32 of (pq|rs), drawn from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < 32:
        p, q = sorted(int(x) for x in rng.integers(0, n, size=2))
        if ("h", p, q) not in out:
            out.append(("h", p, q))
    while len(out) < 64:
        p, q, r, s_ = (int(x) for x in rng.integers(0, n, size=4))
        out.append(("eri", p, q, r, s_))
    return out


def _sa_energy_warm(n, na, nb, h, eri, w, guess, precision, tol):
    """E_SA of the perturbed problem, Davidson started from the unperturbed roots."""
    ctx = fg.forte_cas_create(n, na, nb, h, eri)
    try:
        fg.forte_set_precision(ctx, precision)
        fg.forte_set_guess(ctx, guess, len(w))
        fg.forte_davidson(ctx, len(w), tol)
        return fg.forte_sa_energy(ctx, w)
    finally:
        fg.forte_destroy(ctx)


@pytest.mark.parametrize("precision", [fg.FORTE_FP64, fg.FORTE_BF16X2])
def test_sa_gradient_cas1212_three_roots_64_orbits(precision):
    """The differentiation workload at its stated size: CAS(12,12), seed 3, equal
    weights over 3 roots.  (i) The averaged 1-RDM and sampled 2-RDM elements of the
    backward equal the oracle's (its own eigenvectors, residual 1e-10; stored by
    tests/golden/make_golden.py) to 1e-9.  (ii) Central differences (step 1e-5) on
    64 symmetry orbits -- 32 of h, 32 of (pq|rs) -- match the analytic gradient to
    1e-6.  The perturbed solves start from the unperturbed roots and stop at a
    residual of 1e-8: the energy error r^2 / gap (< 1e-14 Eh for the gaps here)
    contributes < 1e-9 to each difference quotient."""
    import json
    g = json.load(open(GOLDEN_SA))
    cfg = si.CAS1212_SA
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    w = np.array(g["sa_weights"])
    prob = fg.CASProblem(n, na, nb, h, eri, precision=precision)
    try:
        E, C, rn, it = prob.davidson(nroots=3, tol=1e-10)
        assert np.all(np.asarray(rn) < 1e-10)
        np.testing.assert_allclose(np.asarray(E), np.array(g["energies"]), rtol=0, atol=1e-10)
        assert abs(fg.forte_sa_energy(prob.ctx, w) - float(w @ np.array(g["energies"]))) < 1e-10
        dh = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        de = torch.zeros((n,) * 4, dtype=torch.float64, device="cuda")
        fg.forte_sa_gradient(prob.ctx, 3, w, C, 1.0, dh, de, n)
        gh, ge = dh.cpu().numpy(), de.cpu().numpy()
        # (i) against the oracle's state-averaged RDMs: gamma = dE/dh, Gamma = 2 dE/d(pq|rs)
        assert np.abs(gh - np.array(g["sa_gamma1"])).max() < 1e-9
        idx = np.array(g["sa_gamma2_index"])
        assert np.abs(2 * ge[tuple(idx.T)] - np.array(g["sa_gamma2"])).max() < 1e-9
        # (ii) central differences on 64 orbits
        step = 1e-5
        worst = 0.0
        for orb in _orbits64(n):
            if orb[0] == "h":
                d = _orbit_h(n, *orb[1:])
                args_p, args_m, an = (h + step * d, eri), (h - step * d, eri), (gh * d).sum()
            else:
                d = _orbit_eri(n, *orb[1:])
                args_p, args_m, an = (h, eri + step * d), (h, eri - step * d), (ge * d).sum()
            ep = _sa_energy_warm(n, na, nb, *args_p, w, C, precision, 1e-8)
            em = _sa_energy_warm(n, na, nb, *args_m, w, C, precision, 1e-8)
            dev = abs((ep - em) / (2 * step) - an)
            worst = max(worst, dev)
            assert dev < 1e-6, (orb, dev)
    finally:
        prob.close()


def test_sa_gradient_oz64_mode_matches_fp64_mode():
    """forte_sa_gradient after FORTE_OZ64 solves equals the FP64-mode gradient.  Both
    solves stop at residual 1e-9, so the gradients agree to ~residual / gap (gaps
    0.13 and 0.15 here); the energies differ by the sigma error of the mode (1e-12 of
    max |sigma|, ~1e-11 Eh here)."""
    n, na, nb = 8, 4, 4
    h, eri = si.integrals(n, 16, seed=3)
    w = [0.5, 0.5]
    out = []
    for mode in (fg.FORTE_FP64, fg.FORTE_OZ64):
        ht = torch.tensor(h, requires_grad=True)
        et = torch.tensor(eri, requires_grad=True)
        E = fg.sa_energy(ht, et, n, na, nb, w, precision=mode, tol=1e-9)
        E.backward()
        out.append((float(E.detach()), ht.grad.numpy().copy(), et.grad.numpy().copy()))
    de = abs(out[0][0] - out[1][0])
    dh = np.abs(out[0][1] - out[1][1]).max()
    dg = np.abs(out[0][2] - out[1][2]).max()
    assert de < 1e-10 and dh < 1e-7 and dg < 1e-7, (de, dh, dg)
