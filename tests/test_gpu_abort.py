"""Failure path of the bounded device waits (no counterpart in the paper; the
library's promise that errors never trap the GPU).

With a wait budget of a few clock cycles (forte_set_wait_budget) every pipeline
wait of the tensor-core kernels expires: the CTA raises the context's status
flag, stops its other roles, waits for its own MMAs and copies in flight, frees
its tensor memory and exits.  The test checks that each kernel -- alpha-beta MMA,
same-spin MMA, digit-slice alpha-beta, digit-slice 2-RDM Gram -- reports the
expiry (FORTE_ERR_TIMEOUT naming it), that the same context then computes the
right result with the default budget, and that a fresh context solves
correctly.  Nothing here makes the GPU fault or hang: every wait is bounded."""
import numpy as np
import pytest

import oracle
import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2405_10197_gb300 as fg  # noqa: E402

CASES = [
    # (precision, call, n, na, nb, kernel named in the error)
    (fg.FORTE_BF16X2, "sigma", 8, 4, 4, "alpha-beta MMA"),
    (fg.FORTE_BF16X2, "sigma", 8, 0, 4, "same-spin MMA"),   # no alpha replacements: same-spin GEMM only
    (fg.FORTE_OZ64, "sigma", 8, 4, 4, "digit-slice alpha-beta"),
    (fg.FORTE_BF16X2, "rdms", 8, 4, 4, "digit-slice 2-RDM Gram"),
]


def _run(prob, call, C):
    if call == "sigma":
        S = torch.empty_like(C)
        fg.forte_sigma(prob.ctx, C, S, 1)
        return S
    n = prob.norb
    g1 = torch.empty(n, n, dtype=torch.float64, device="cuda")
    g2 = torch.empty((n,) * 4, dtype=torch.float64, device="cuda")
    fg.forte_rdms(prob.ctx, C[0], g1, g2, n)
    return g2


@pytest.mark.parametrize("mode,call,n,na,nb,name", CASES, ids=[c[5] for c in CASES])
def test_expired_waits_report_timeout_and_the_context_stays_usable(mode, call, n, na, nb, name):
    h, eri = si.integrals(n, 2 * n, seed=31)
    prob = fg.CASProblem(n, na, nb, h, eri, precision=mode)
    try:
        C = torch.tensor(si.random_vectors(1, prob.na, prob.nb, seed=8), device="cuda")
        C /= C.norm()
        fg.forte_set_wait_budget(prob.ctx, 4)
        if call == "sigma":
            _run(prob, call, C)
            assert fg.forte_get_status(prob.ctx, allow=(fg.FORTE_ERR_TIMEOUT,)) == fg.FORTE_ERR_TIMEOUT
        else:
            with pytest.raises(fg.ForteError) as ex:
                _run(prob, call, C)
            assert ex.value.code == fg.FORTE_ERR_TIMEOUT
        assert name in fg.forte_last_error()
        # default budget: the same context gives the right answer again
        fg.forte_set_wait_budget(prob.ctx, 0)
        out = _run(prob, call, C)
        assert fg.forte_get_status(prob.ctx) == fg.FORTE_OK
        prob.set_precision(fg.FORTE_FP64)
        ref = _run(prob, call, C)
        tol = 5e-5 if (mode == fg.FORTE_BF16X2 and call == "sigma") else 1e-11
        assert float((out - ref).abs().max() / ref.abs().max()) < tol
    finally:
        prob.close()
    # a fresh context on the same device solves correctly
    p2 = fg.CASProblem(n, na, nb, h, eri, precision=mode)
    try:
        E, _, rn, _ = p2.davidson(nroots=1, tol=1e-9)
        w, _ = oracle.solve_dense(n, na, nb, h, eri, nroots=1)
        assert abs(E[0] - w[0]) < 1e-9
    finally:
        p2.close()
