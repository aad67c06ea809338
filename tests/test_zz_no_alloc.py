"""forte_sigma_fp64_noalloc: the FP64 sigma for callers that cannot allocate
device memory during a call (their memory belongs to another allocator, or a
cudaMalloc/cudaFree synchronisation is unacceptable in their loop).

Called through the C ABI (ctypes on libforte_gpu.so) and compared, on two calls
in a row, with the regular forte_sigma and with the CPU oracle's direct
Slater-Condon sigma (every element for the small spaces, sampled rows for
CAS(12,12)), within the sigma tolerance of the other parity tests (max-abs
relative 1e-12).  Kept in its own file, named to be collected last."""
import ctypes

import numpy as np
import pytest

import synth_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_2405_10197_gb300 as fg  # noqa: E402

TOL = 1e-12


def _inputs(n, na):
    return si.integrals(n, 2 * n, seed=n + na)


def _ctx(n, na, nb):
    h, eri = _inputs(n, na)
    return fg.forte_cas_create(n, na, nb, h, eri)


@pytest.mark.parametrize("n,na,nb,nvec", [(8, 4, 4, 3), (9, 2, 5, 2), (12, 6, 6, 1)])
def test_noalloc_sigma_matches_forte_sigma_and_oracle_twice(n, na, nb, nvec):
    lib = fg.library()
    h, eri = _inputs(n, na)
    ctx = _ctx(n, na, nb)
    NA, NB = fg.forte_get_sizes(ctx)
    rows = None
    if NA * NB > 20000:  # oracle rows sampled at CAS(12,12), incl. the first and last
        rows = np.unique(np.concatenate([[0, NA * NB - 1],
                                         np.random.default_rng(5).integers(0, NA * NB, 3000)]))
    for call, seed in enumerate((21, 22)):
        Ch = si.random_vectors(nvec, NA, NB, seed=seed)
        C = torch.tensor(Ch, device="cuda")
        S_ref = torch.empty_like(C)
        S = torch.full_like(C, float("nan"))
        assert lib.forte_sigma(ctx, C.data_ptr(), S_ref.data_ptr(), nvec) == 0
        rc = lib.forte_sigma_fp64_noalloc(ctx, C.data_ptr(), S.data_ptr(), nvec)
        assert rc == 0, lib.forte_last_error().decode()
        torch.cuda.synchronize()
        err = float((S - S_ref).abs().max() / S_ref.abs().max())
        assert err <= TOL, (call, err)
        So = oracle.sigma(n, na, nb, h, eri, Ch.reshape(nvec, -1), rows=rows)
        Sg = S.reshape(nvec, -1).cpu().numpy()
        if rows is not None:
            Sg = Sg[:, rows]
        for v in range(nvec):
            err_o = float(np.abs(Sg[v] - So[v]).max() / np.abs(So[v]).max())
            assert err_o <= TOL, (call, v, err_o)
    fg.forte_destroy(ctx)


def test_noalloc_rejects_requests_beyond_its_scratch():
    lib = fg.library()
    ctx = _ctx(12, 6, 6)
    NA, NB = fg.forte_get_sizes(ctx)
    C = torch.zeros(2, NA, NB, dtype=torch.float64, device="cuda")
    S = torch.zeros_like(C)
    rc = lib.forte_sigma_fp64_noalloc(ctx, C.data_ptr(), S.data_ptr(), 2)
    assert rc == fg.FORTE_ERR_ARG
    assert "scratch limit" in lib.forte_last_error().decode()
    assert lib.forte_sigma_fp64_noalloc(ctx, ctypes.c_void_p(0), ctypes.c_void_p(0), 0) == 0
    fg.forte_destroy(ctx)
