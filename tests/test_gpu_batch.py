"""Batched solve (forte_batch_solve) of independent active-space problems of
uneven size and root count, against the oracle (dense diagonalisation) and,
for the batch workload's larger instances, across precisions."""
import math

import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402


def _small_batch(count, seed):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        n = int(rng.choice([2, 3, 4, 5, 6]))
        na = int(rng.integers(0, n + 1))
        nb = int(rng.integers(0, n + 1))
        ndet = math.comb(n, na) * math.comb(n, nb)
        nr = int(min(ndet, rng.integers(1, 4)))
        h, eri = si.integrals(n, 2 * n, seed=500 + i)
        probs.append(dict(norb=n, nalpha=na, nbeta=nb, nroots=nr, h=h, eri=eri))
    return probs


@pytest.mark.parametrize("precision", [fg.FORTE_FP64, fg.FORTE_BF16X2, fg.FORTE_OZ64])
def test_batch_matches_oracle_dense(precision):
    probs = _small_batch(40, seed=3)
    E, st = fg.forte_batch_solve(probs, precision=precision, tol=1e-10, nworkers=6)
    assert np.all(st == 0)
    for p, e in zip(probs, E):
        w, _ = oracle.solve_dense(p["norb"], p["nalpha"], p["nbeta"], p["h"], p["eri"], nroots=p["nroots"])
        assert np.abs(e - w).max() < 1e-9, p


def test_batch_workload_head_fp64_vs_mixed():
    # first instances of the batched workload (orbital counts {6,8,10,12}, 1-3 roots)
    inst = si.batch_instances()[:16]
    probs = []
    for q in inst:
        h, eri = si.integrals(q["norb"], q["n_l"], q["seed"])
        probs.append(dict(norb=q["norb"], nalpha=q["nalpha"], nbeta=q["nbeta"], nroots=q["nroots"], h=h, eri=eri))
    E64, st64 = fg.forte_batch_solve(probs, precision=fg.FORTE_FP64, tol=1e-6)
    Em, stm = fg.forte_batch_solve(probs, precision=fg.FORTE_BF16X2, tol=1e-6)
    assert np.all(st64 == 0) and np.all(stm == 0)
    for a, b in zip(E64, Em):
        assert np.abs(a - b).max() < 1e-8
    # the n = 6 instances also against the oracle
    for p, e in zip(probs, E64):
        if p["norb"] == 6:
            w, _ = oracle.solve_dense(6, 3, 3, p["h"], p["eri"], nroots=p["nroots"])
            assert np.abs(e - w).max() < 1e-9


def test_batch_reports_bad_input():
    h, eri = si.integrals(4, 8, seed=0)
    bad = h.copy()
    bad[0, 1] = np.nan
    probs = [dict(norb=4, nalpha=2, nbeta=2, nroots=1, h=h, eri=eri),
             dict(norb=4, nalpha=2, nbeta=2, nroots=1, h=bad, eri=eri)]
    with pytest.raises(fg.ForteError):
        fg.forte_batch_solve(probs)
