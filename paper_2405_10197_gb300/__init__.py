"""Python binding of libforte_gpu.so, the GB300 CASCI engine.

The functions below carry the names of the C ABI in include/forte_gpu.h and
only marshal arguments (torch tensors or integer addresses to pointers, status
codes to exceptions).  Every step of the computation runs in the library's
CUDA kernels; there is no CPU fallback: if the shared library is missing this
module raises on first use.

``CASProblem`` is a small convenience wrapper that allocates the outputs with
torch (device memory only) and calls the same entry points.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libforte_gpu.so")

FORTE_OK = 0
FORTE_ERR_ARG = 1
FORTE_ERR_ALLOC = 2
FORTE_ERR_CUDA = 3
FORTE_ERR_NOT_CONVERGED = 4
FORTE_ERR_NUMERIC = 5
FORTE_ERR_TIMEOUT = 6

FORTE_FP64 = 0
FORTE_TF32 = 1
FORTE_BF16X2 = 2
FORTE_DF32 = 3
FORTE_OZ64 = 4

_ERRNAMES = {1: "FORTE_ERR_ARG", 2: "FORTE_ERR_ALLOC", 3: "FORTE_ERR_CUDA",
             4: "FORTE_ERR_NOT_CONVERGED", 5: "FORTE_ERR_NUMERIC", 6: "FORTE_ERR_TIMEOUT"}


class ForteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library():
    """Load libforte_gpu.so (built by build.py); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the CUDA library is required; there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    L.forte_cas_create.restype = vp
    L.forte_cas_create.argtypes = [i, i, i, vp, vp]
    L.forte_destroy.restype = None
    L.forte_destroy.argtypes = [vp]
    L.forte_sci_create.restype = vp
    L.forte_sci_create.argtypes = [i, vp, vp]
    L.forte_sci_destroy.restype = None
    L.forte_sci_destroy.argtypes = [vp]
    L.forte_last_error.restype = ctypes.c_char_p
    L.forte_last_error.argtypes = []
    sigs = {
        "forte_set_stream": [vp, vp],
        "forte_set_precision": [vp, i],
        "forte_get_sizes": [vp, vp, vp],
        "forte_get_string_tables": [vp, i, vp, vp, vp],
        "forte_get_hdiag": [vp, vp],
        "forte_sigma": [vp, vp, vp, i],
        "forte_davidson": [vp, i, d],
        "forte_set_davidson_params": [vp, i, i, i, d],
        "forte_get_roots": [vp, vp, vp, vp, vp],
        "forte_set_guess": [vp, vp, i],
        "forte_rdms": [vp, vp, vp, vp],
        "forte_tdm1": [vp, vp, vp, vp],
        "forte_rdm3": [vp, vp, vp],
        "forte_set_gas": [vp, i, vp, vp, vp, vp],
        "forte_set_gas_route": [vp, i],
        "forte_get_gas_route": [vp, vp, vp, vp],
        "forte_set_spin_parity": [vp, i],
        "forte_aci": [vp, d, d, i, d, i, vp, vp, vp, vp, vp],
        "forte_sigma_fp64_noalloc": [vp, vp, vp, i],
        "forte_sa_gradient": [vp, i, vp, vp, d, vp, vp],
        "forte_sa_energy": [vp, i, vp, vp],
        "forte_get_status": [vp],
        "forte_set_wait_budget": [vp, ctypes.c_ulonglong],
        "forte_batch_solve": [i, vp, vp, vp, vp, vp, vp, i, d, i, vp, vp],
        "forte_batch_tuning": [i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
        "forte_batch_stats": [vp, vp, vp],
        "forte_sci_set_stream": [vp, vp],
        "forte_sci_sigma": [vp, ll, vp, vp, vp, i],
        "forte_profile_enable": [vp, i],
        "forte_profile_query": [vp, ctypes.c_char_p, vp, vp],
        "forte_get_counters": [vp, vp, vp],
    }
    L.forte_profile_kernel_name.restype = ctypes.c_char_p
    L.forte_profile_kernel_name.argtypes = [vp, i]
    for name, args in sigs.items():
        f = getattr(L, name)
        f.restype = i
        f.argtypes = args
    _ = ll
    _lib = L
    return L


def _check(code, allow=()):
    if code != FORTE_OK and code not in allow:
        raise ForteError(code, forte_last_error())
    return code


def _ptr(x, numel=None, dtype="float64"):
    """Device pointer of a torch tensor (dtype/contiguity/size checked) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    want = {"float64": torch.float64}[dtype]
    if not isinstance(x, torch.Tensor):
        raise TypeError("expected a torch tensor or an integer device address")
    if x.dtype != want or not x.is_cuda or not x.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor, got {x.dtype} on {x.device}")
    if numel is not None and x.numel() < numel:
        raise ValueError(f"tensor has {x.numel()} elements, need {numel}")
    return x.data_ptr()


def _host_f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        a = a.reshape(shape)
    return a


# --------------------------------------------------------------- C ABI names

def forte_last_error() -> str:
    return library().forte_last_error().decode()


def forte_cas_create(norb, nalpha, nbeta, h, eri):
    """Return an opaque context handle (int).  h, eri: host arrays."""
    h = _host_f64(h, (norb, norb))
    eri = _host_f64(eri, (norb,) * 4)
    ctx = library().forte_cas_create(norb, nalpha, nbeta, h.ctypes.data, eri.ctypes.data)
    if not ctx:
        raise ForteError(FORTE_ERR_ARG, forte_last_error())
    return ctx


def forte_destroy(ctx):
    library().forte_destroy(ctx)


def forte_set_stream(ctx, stream):
    """stream: a torch.cuda.Stream, an integer cudaStream_t, or None (legacy default)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(library().forte_set_stream(ctx, s))


def forte_set_precision(ctx, mode):
    return _check(library().forte_set_precision(ctx, int(mode)))


def forte_get_sizes(ctx):
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(library().forte_get_sizes(ctx, ctypes.addressof(a), ctypes.addressof(b)))
    return a.value, b.value


def forte_get_string_tables(ctx, spin, norb):
    na, nb = forte_get_sizes(ctx)
    N = na if spin == 0 else nb
    s = np.zeros(N, dtype=np.uint32)
    J = np.zeros((N, norb, norb), dtype=np.int32)
    g = np.zeros((N, norb, norb), dtype=np.int8)
    _check(library().forte_get_string_tables(ctx, spin, s.ctypes.data, J.ctypes.data, g.ctypes.data))
    return s, J, g


def forte_get_hdiag(ctx, out):
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_get_hdiag(ctx, _ptr(out, na * nb)))


def forte_sigma(ctx, C, S, nvec):
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_sigma(ctx, _ptr(C, nvec * na * nb), _ptr(S, nvec * na * nb), int(nvec)))


def forte_sigma_fp64_noalloc(ctx, C, S, nvec):
    """FP64 sigma through the entry point that allocates no device memory
    (scratch is a fixed array inside the library; nvec * N_det <= 2^20)."""
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_sigma_fp64_noalloc(ctx, _ptr(C, nvec * na * nb), _ptr(S, nvec * na * nb),
                                                     int(nvec)))


def forte_davidson(ctx, nroots, tol, allow_not_converged=False):
    allow = (FORTE_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    return _check(library().forte_davidson(ctx, int(nroots), float(tol)), allow)


def forte_set_davidson_params(ctx, max_subspace_per_root, collapse_per_root, max_iter, denom_guard):
    return _check(library().forte_set_davidson_params(ctx, int(max_subspace_per_root),
                                                      int(collapse_per_root), int(max_iter),
                                                      float(denom_guard)))


def forte_get_roots(ctx, nroots, C=None):
    """Returns (E, rnorm, iters); copies eigenvectors into the device tensor C if given."""
    na, nb = forte_get_sizes(ctx)
    E = np.zeros(nroots)
    rn = np.zeros(nroots)
    it = ctypes.c_int()
    _check(library().forte_get_roots(ctx, E.ctypes.data, _ptr(C, nroots * na * nb), rn.ctypes.data,
                                     ctypes.addressof(it)))
    return E, rn, it.value


def forte_set_guess(ctx, C, nvec):
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_set_guess(ctx, _ptr(C, nvec * na * nb) if nvec else None, int(nvec)))


def forte_rdms(ctx, C, g1, g2, norb):
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_rdms(ctx, _ptr(C, na * nb), _ptr(g1, norb * norb),
                                       _ptr(g2, norb ** 4)))


def forte_tdm1(ctx, bra, ket, t1, norb):
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_tdm1(ctx, _ptr(bra, na * nb), _ptr(ket, na * nb),
                                       _ptr(t1, norb * norb)))


def forte_rdm3(ctx, C, g3, norb):
    na, nb = forte_get_sizes(ctx)
    return _check(library().forte_rdm3(ctx, _ptr(C, na * nb), _ptr(g3, norb ** 6)))


def forte_set_gas(ctx, spaces, gmin, gmax):
    """Occupation restriction (GAS / RAS): consecutive spaces of the given sizes,
    per-space limits on the alpha + beta electron count.  Empty ``spaces``
    removes it.  Returns the number of kept determinants."""
    G = len(spaces)
    if len(gmin) != G or len(gmax) != G:
        raise ValueError("spaces, gmin and gmax need the same length")
    arr = ctypes.c_int * max(G, 1)
    nd = ctypes.c_longlong()
    _check(library().forte_set_gas(ctx, G, arr(*spaces), arr(*gmin), arr(*gmax), ctypes.byref(nd)))
    return nd.value


def forte_set_gas_route(ctx, route):
    """Restricted sigma route: -1 timed choice (default), 0 full grid, 1 kept determinants."""
    return _check(library().forte_set_gas_route(ctx, int(route)))


def forte_get_gas_route(ctx):
    """(route for FP64 vectors, route for FP32 vectors, timings [4] in ms)."""
    r64, r32 = ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(4)
    _check(library().forte_get_gas_route(ctx, ctypes.byref(r64), ctypes.byref(r32), ms.ctypes.data))
    return r64.value, r32.value, ms


def forte_set_spin_parity(ctx, parity):
    """Davidson sector C^T = parity C for Ms = 0: +1 even S, -1 odd S, 0 off."""
    return _check(library().forte_set_spin_parity(ctx, int(parity)))


def forte_aci(ctx, sigma, gamma=1.0, max_cycles=50, tol=1e-10, C=None, parity=0):
    """Adaptive CI on the CAS grid: returns (E_M, E_corrected, nM, nP, cycles);
    Psi_M goes into the device tensor C when given.  parity: exchange-parity
    sector of the target (+1 even S, -1 odd S, 0 none)."""
    na, nb = forte_get_sizes(ctx)
    E = (ctypes.c_double * 2)()
    nM, nP, cyc = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
    _check(library().forte_aci(ctx, float(sigma), float(gamma), int(max_cycles), float(tol), int(parity), E,
                               _ptr(C, na * nb) if C is not None else None, ctypes.byref(nM), ctypes.byref(nP),
                               ctypes.byref(cyc)))
    return E[0], E[1], nM.value, nP.value, cyc.value


def forte_sa_gradient(ctx, nstates, weights, C, scale, dh, deri, norb):
    """Accumulate scale * d(sum_k w_k E_k)/d(h, eri) into the device tensors dh, deri."""
    na, nb = forte_get_sizes(ctx)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.size != nstates:
        raise ValueError("need one weight per state")
    return _check(library().forte_sa_gradient(ctx, int(nstates), w.ctypes.data, _ptr(C, nstates * na * nb),
                                              float(scale), _ptr(dh, norb * norb), _ptr(deri, norb ** 4)))


def forte_sa_energy(ctx, weights):
    """E_SA = sum_k w_k E_k over the first len(weights) roots of the last forte_davidson."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    out = ctypes.c_double()
    _check(library().forte_sa_energy(ctx, int(w.size), w.ctypes.data, ctypes.byref(out)))
    return out.value


def forte_get_status(ctx, allow=()):
    """FORTE_OK, or FORTE_ERR_TIMEOUT when a bounded device wait expired (raises unless allowed)."""
    return _check(library().forte_get_status(ctx), allow)


def forte_set_wait_budget(ctx, cycles):
    return _check(library().forte_set_wait_budget(ctx, int(cycles)))


def forte_batch_solve(problems, precision=FORTE_FP64, tol=1e-8, max_iter=400, allow_not_converged=False):
    """Solve a list of independent problems (one CTA per problem, one launch per size class).

    problems: sequence of dicts with norb, nalpha, nbeta, nroots, h, eri (host arrays).
    Returns (list of energy arrays, per-problem status array)."""
    P = len(problems)
    if P == 0:
        return [], np.zeros(0, dtype=np.int32)
    norb = np.array([p["norb"] for p in problems], dtype=np.int32)
    na = np.array([p["nalpha"] for p in problems], dtype=np.int32)
    nb = np.array([p["nbeta"] for p in problems], dtype=np.int32)
    nr = np.array([p["nroots"] for p in problems], dtype=np.int32)
    hs = [_host_f64(p["h"], (int(n), int(n))) for p, n in zip(problems, norb)]
    es = [_host_f64(p["eri"], (int(n),) * 4) for p, n in zip(problems, norb)]
    hp = (ctypes.c_void_p * P)(*[a.ctypes.data for a in hs])
    ep = (ctypes.c_void_p * P)(*[a.ctypes.data for a in es])
    E = np.zeros(int(nr.sum()))
    st = np.zeros(P, dtype=np.int32)
    code = library().forte_batch_solve(P, norb.ctypes.data, na.ctypes.data, nb.ctypes.data, nr.ctypes.data,
                                       ctypes.cast(hp, ctypes.c_void_p), ctypes.cast(ep, ctypes.c_void_p),
                                       int(precision), float(tol), int(max_iter), E.ctypes.data, st.ctypes.data)
    _check(code, (FORTE_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    out, o = [], 0
    for k in nr:
        out.append(E[o:o + k].copy())
        o += k
    return out, st


def forte_batch_tuning():
    """Autotuner choices of the last forte_batch_solve: list of dicts per size class."""
    cap = 64
    nc = ctypes.c_int()
    arrs = [np.zeros(cap, dtype=np.int32) for _ in range(5)]
    ms = np.zeros(cap)
    path = np.zeros(cap, dtype=np.int32)
    single = np.zeros(cap)
    nprob = np.zeros(cap, dtype=np.int32)
    occ = np.zeros(cap, dtype=np.int32)
    _check(library().forte_batch_tuning(cap, ctypes.byref(nc), *[a.ctypes.data for a in arrs], ms.ctypes.data,
                                        path.ctypes.data, single.ctypes.data, nprob.ctypes.data, occ.ctypes.data))
    out = []
    for k in range(min(nc.value, cap)):
        out.append(dict(norb=int(arrs[0][k]), nalpha=int(arrs[1][k]), nbeta=int(arrs[2][k]),
                        threads=int(arrs[3][k]), tile=int(arrs[4][k]), sigma_ms=float(ms[k]),
                        path="class launch" if path[k] == 0 else "single-problem path",
                        single_iter_ms=float(single[k]), problems=int(nprob[k]), ctas_per_sm=int(occ[k])))
    return out


def forte_batch_stats():
    """Problem counts of the last forte_batch_solve: class launches, single-problem path, retried."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(library().forte_batch_stats(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(class_launch=a.value, single_path=b.value, retried=c.value)


def forte_sci_create(norb, h, eri):
    """Handle for sigma over determinant lists (norb <= 32); h, eri: host arrays."""
    h = _host_f64(h, (norb, norb))
    eri = _host_f64(eri, (norb,) * 4)
    sci = library().forte_sci_create(norb, h.ctypes.data, eri.ctypes.data)
    if not sci:
        raise ForteError(FORTE_ERR_ARG, forte_last_error())
    return sci


def forte_sci_destroy(sci):
    library().forte_sci_destroy(sci)


def forte_sci_set_stream(sci, stream):
    s = getattr(stream, "cuda_stream", stream)
    return _check(library().forte_sci_set_stream(sci, s))


def forte_sci_sigma(sci, dets, C, S, nvec):
    """dets: CUDA int64/uint64 tensor [ndet] of determinant words; C, S: CUDA FP64 [nvec][ndet]."""
    import torch
    if not isinstance(dets, torch.Tensor) or not dets.is_cuda or dets.dtype not in (torch.int64, torch.uint64) \
            or not dets.is_contiguous():
        raise ValueError("dets must be a contiguous CUDA int64 tensor of determinant words")
    nd = dets.numel()
    return _check(library().forte_sci_sigma(sci, nd, dets.data_ptr(), _ptr(C, nvec * nd), _ptr(S, nvec * nd),
                                            int(nvec)))


def forte_profile_enable(ctx, on):
    return _check(library().forte_profile_enable(ctx, int(on)))


def forte_profile_query(ctx, kernel=None):
    """(launches, total_ms) of the recorded launches of `kernel` (None: all)."""
    n = ctypes.c_int()
    ms = ctypes.c_double()
    k = kernel.encode() if kernel else None
    _check(library().forte_profile_query(ctx, k, ctypes.addressof(n), ctypes.addressof(ms)))
    return n.value, ms.value


def forte_profile_kernel_name(ctx, i):
    r = library().forte_profile_kernel_name(ctx, int(i))
    return r.decode() if r else None


def forte_get_counters(ctx):
    """(sigma vectors built in FP64, sigma vectors built in a reduced-precision mode)."""
    a, b = ctypes.c_longlong(), ctypes.c_longlong()
    _check(library().forte_get_counters(ctx, ctypes.addressof(a), ctypes.addressof(b)))
    return a.value, b.value


def profile_table(ctx):
    """{kernel name: (launches, total_ms)} of the recorded launches."""
    out = {}
    i = 0
    while True:
        name = forte_profile_kernel_name(ctx, i)
        if name is None:
            return out
        out[name] = forte_profile_query(ctx, name)
        i += 1


# --------------------------------------------------------------- convenience

class CASProblem:
    """One active-space problem on the current CUDA device."""

    def __init__(self, norb, nalpha, nbeta, h, eri, precision=FORTE_FP64, stream=None):
        import torch
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta
        self.ctx = forte_cas_create(norb, nalpha, nbeta, h, eri)
        self.na, self.nb = forte_get_sizes(self.ctx)
        self.ndet = self.na * self.nb
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is not None:
            forte_set_stream(self.ctx, stream)
        forte_set_precision(self.ctx, precision)

    def close(self):
        if getattr(self, "ctx", None):
            forte_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, mode):
        forte_set_precision(self.ctx, mode)

    def sigma(self, C):
        import torch
        C = C.reshape(-1, self.na, self.nb)
        S = torch.empty_like(C)
        forte_sigma(self.ctx, C, S, C.shape[0])
        return S

    def set_gas(self, spaces, gmin, gmax):
        return forte_set_gas(self.ctx, spaces, gmin, gmax)

    def set_spin_parity(self, parity):
        forte_set_spin_parity(self.ctx, parity)

    def aci(self, sigma, gamma=1.0, max_cycles=50, tol=1e-10, parity=0):
        """(E_M, E_corrected, Psi_M [N_alpha][N_beta], nM, nP, cycles)."""
        import torch
        C = torch.empty(self.na, self.nb, dtype=torch.float64, device=self.device)
        e, ec, nm, np_, cyc = forte_aci(self.ctx, sigma, gamma, max_cycles, tol, C, parity)
        return e, ec, C, nm, np_, cyc

    def hdiag(self):
        import torch
        out = torch.empty(self.na, self.nb, dtype=torch.float64, device=self.device)
        forte_get_hdiag(self.ctx, out)
        return out

    def davidson(self, nroots=1, tol=1e-10, allow_not_converged=False):
        import torch
        forte_davidson(self.ctx, nroots, tol, allow_not_converged)
        C = torch.empty(nroots, self.na, self.nb, dtype=torch.float64, device=self.device)
        E, rn, it = forte_get_roots(self.ctx, nroots, C)
        return E, C, rn, it

    def rdms(self, C):
        import torch
        g1 = torch.empty(self.norb, self.norb, dtype=torch.float64, device=self.device)
        g2 = torch.empty((self.norb,) * 4, dtype=torch.float64, device=self.device)
        forte_rdms(self.ctx, C.contiguous(), g1, g2, self.norb)
        return g1, g2

    def rdm3(self, C):
        import torch
        g3 = torch.empty((self.norb,) * 6, dtype=torch.float64, device=self.device)
        forte_rdm3(self.ctx, C.contiguous(), g3, self.norb)
        return g3

    def tdm1(self, bra, ket):
        import torch
        t1 = torch.empty(self.norb, self.norb, dtype=torch.float64, device=self.device)
        forte_tdm1(self.ctx, bra.contiguous(), ket.contiguous(), t1, self.norb)
        return t1

    def string_tables(self, spin):
        return forte_get_string_tables(self.ctx, spin, self.norb)


# --------------------------------------------------------------- differentiable SA energy

def _make_sa_energy():
    import torch

    class SAEnergy(torch.autograd.Function):
        """E_SA(h, eri) = sum_k w_k E_k over the lowest len(weights) roots.

        forward: forte_cas_create + forte_davidson + forte_sa_energy; backward: forte_sa_gradient,
        the library's adjoint kernel (dE/dh = sum w gamma, dE/d(pq|rs) = 1/2 sum w Gamma).
        """

        @staticmethod
        def forward(fctx, h, eri, norb, nalpha, nbeta, weights, precision=FORTE_FP64, tol=1e-10):
            hn = h.detach().to("cpu", torch.float64).numpy()
            en = eri.detach().to("cpu", torch.float64).numpy()
            prob = CASProblem(norb, nalpha, nbeta, hn, en, precision=precision)
            w = np.asarray(weights, dtype=np.float64)
            E, C, rn, it = prob.davidson(len(w), tol)
            fctx.prob, fctx.C, fctx.w = prob, C, w
            fctx.meta = (h.device, h.dtype, eri.device, eri.dtype)
            fctx.energies, fctx.residuals = E, rn
            return torch.tensor(forte_sa_energy(prob.ctx, w), dtype=h.dtype, device=h.device)

        @staticmethod
        def backward(fctx, grad):
            import torch as T
            prob = fctx.prob
            n = prob.norb
            dh = T.zeros(n, n, dtype=T.float64, device=prob.device)
            deri = T.zeros((n,) * 4, dtype=T.float64, device=prob.device)
            forte_sa_gradient(prob.ctx, len(fctx.w), fctx.w, fctx.C, float(grad), dh, deri, n)
            hdev, hdt, edev, edt = fctx.meta
            return dh.to(hdev, hdt), deri.to(edev, edt), None, None, None, None, None, None

    return SAEnergy


_SAEnergy = None


def sa_energy(h, eri, norb, nalpha, nbeta, weights, precision=FORTE_FP64, tol=1e-10):
    """Differentiable state-averaged CASCI energy (torch scalar)."""
    global _SAEnergy
    if _SAEnergy is None:
        _SAEnergy = _make_sa_energy()
    return _SAEnergy.apply(h, eri, norb, nalpha, nbeta, tuple(weights), precision, tol)
