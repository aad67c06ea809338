"""Batched solve (forte_batch_solve): one launch per size class, one CTA per
problem running the whole Davidson solve, against the oracle (dense
diagonalisation, stored oracle energies) and across precisions."""
import glob
import json
import math
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

HERE = os.path.dirname(os.path.abspath(__file__))


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
    # mixed classes, empty spins (n_alpha or n_beta = 0), spaces smaller than the subspace
    probs = _small_batch(40, seed=3)
    E, st = fg.forte_batch_solve(probs, precision=precision, tol=1e-10)
    assert np.all(st == 0)
    for p, e in zip(probs, E):
        w, _ = oracle.solve_dense(p["norb"], p["nalpha"], p["nbeta"], p["h"], p["eri"], nroots=p["nroots"])
        assert np.abs(e - w).max() < 1e-10, p


def _workload(count, max_norb=12):
    probs = []
    for q in si.batch_instances():
        if len(probs) == count:
            break
        if q["norb"] > max_norb:
            continue
        h, eri = si.integrals(q["norb"], q["n_l"], q["seed"])
        probs.append(dict(norb=q["norb"], nalpha=q["nalpha"], nbeta=q["nbeta"], nroots=q["nroots"], h=h, eri=eri))
    return probs


def test_batch_workload_head_fp64_vs_mixed_and_oracle():
    # the first instances of the batched workload with up to 10 orbitals (1-3 roots):
    # FP64 and mixed agree; the n = 6 and n = 8 instances match the oracle's dense
    # diagonalisation to 1e-9 Eh
    probs = _workload(16, max_norb=10)
    E64, st64 = fg.forte_batch_solve(probs, precision=fg.FORTE_FP64, tol=1e-7)
    Em, stm = fg.forte_batch_solve(probs, precision=fg.FORTE_BF16X2, tol=1e-7)
    assert np.all(st64 == 0) and np.all(stm == 0)
    for a, b in zip(E64, Em):
        assert np.abs(a - b).max() < 1e-9
    checked = 0
    for p, e in zip(probs, E64):
        if p["norb"] <= 8:
            w, _ = oracle.solve_dense(p["norb"], p["nalpha"], p["nbeta"], p["h"], p["eri"], nroots=p["nroots"])
            assert np.abs(e - w).max() < 1e-9
            checked += 1
    assert checked >= 4


def test_batch_autotuner_reports_every_class():
    probs = _workload(12, max_norb=10)
    fg.forte_batch_solve(probs, precision=fg.FORTE_BF16X2, tol=1e-6)
    tun = fg.forte_batch_tuning()
    classes = {(p["norb"], p["nalpha"], p["nbeta"]) for p in probs}
    assert {(t["norb"], t["nalpha"], t["nbeta"]) for t in tun} == classes
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for t in tun:
        assert t["threads"] in (128, 256, 512) and t["tile"] in (16, 32, 64) and t["sigma_ms"] > 0
        assert t["single_iter_ms"] > 0 and t["ctas_per_sm"] >= 1
        assert t["problems"] == sum(1 for p in probs if (p["norb"], p["nalpha"], p["nbeta"]) ==
                                    (t["norb"], t["nalpha"], t["nbeta"]))
        # the documented rule: class launch when one sigma round of the class costs
        # no more than one single-path iteration of each of its problems
        waves = math.ceil(t["problems"] / (t["ctas_per_sm"] * nsm))
        cta = t["sigma_ms"] * waves <= t["problems"] * t["single_iter_ms"]
        assert t["path"] == ("class launch" if cta else "single-problem path")


@pytest.mark.parametrize("precision", [fg.FORTE_FP64, fg.FORTE_BF16X2])
@pytest.mark.parametrize("name", ["cas1010_seed5_3roots", "cas1212_seed1_4roots", "batch1058_cas1010"])
def test_batch_matches_stored_oracle_energies(name, precision):
    # the stored oracle energies (residual bound below 5e-12 Eh) of CAS(10,10) and
    # CAS(12,12), solved as members of a batch (up to three roots each); batch1058 is
    # the batched workload's instance whose FP64 in-CTA Davidson-Liu stalls: it is
    # solved again on the single-problem path (Jacobi-Davidson after the stall)
    g = json.load(open(os.path.join(HERE, "golden", name + ".json")))
    h, eri = si.integrals(g["norb"], g["n_l"], g["seed"])
    nr = min(3, g["nroots"])
    small = _workload(6, max_norb=8)
    probs = small + [dict(norb=g["norb"], nalpha=g["nalpha"], nbeta=g["nbeta"], nroots=nr, h=h, eri=eri)]
    E, st = fg.forte_batch_solve(probs, precision=precision, tol=1e-8)
    assert np.all(st == 0)
    np.testing.assert_allclose(E[-1], np.array(g["energies"][:nr]), rtol=0, atol=1e-10)
    stats = fg.forte_batch_stats()
    assert stats["class_launch"] + stats["single_path"] == len(probs)


def test_batch_reports_bad_input():
    h, eri = si.integrals(4, 8, seed=0)
    bad = h.copy()
    bad[0, 1] = np.nan
    probs = [dict(norb=4, nalpha=2, nbeta=2, nroots=1, h=h, eri=eri),
             dict(norb=4, nalpha=2, nbeta=2, nroots=1, h=bad, eri=eri)]
    with pytest.raises(fg.ForteError):
        fg.forte_batch_solve(probs)


def test_batch_head_128_mixed_instance_1058_matches_oracle():
    # The first 128 instances of the batched workload in the mixed mode: three size
    # classes in one graph next to the single-problem path.  Instance 58 (seed 1058)
    # is the one whose in-CTA Davidson-Liu does not converge within the iteration cap;
    # its status must reach the host at its own batch index, so that it is solved
    # again on the single-problem path (a status written at the CTA's index within
    # its class was read as converged, 8.5e-4 Eh above the ground state).
    g = json.load(open(os.path.join(HERE, "golden", "batch1058_cas1010.json")))
    probs = _workload(128)
    k = [i for i, q in enumerate(si.batch_instances()[:128]) if q["seed"] == 1058][0]
    E, st = fg.forte_batch_solve(probs, precision=fg.FORTE_BF16X2, tol=1e-7)
    assert np.all(st == 0)
    assert abs(E[k][0] - g["energies"][0]) < 1e-9
