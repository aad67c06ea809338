"""Python driver of the oracle: loads ``oracle_core.c`` (compiled with gcc) and
adds the textbook solvers on top of it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sources followed:
* string-based CI, determinant = alpha string x beta string, coefficients as a
  matrix C[I_alpha, I_beta]: Sec. II.A.1 (string-based CI of Handy);
* Davidson-Liu diagonalization: Sec. II.A.1 names the method only; the steps
  below are the textbook ones (subspace Rayleigh-Ritz, residual, diagonal
  preconditioner, Gram-Schmidt, collapse);
* 1-, 2- and 3-RDM definitions: Sec. II.A.1, Eqs. for gamma_1, gamma_2 and
  gamma_3, summed over spin into the spin-free (chemist-order) quantities.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_core.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile oracle_core.c into oracle/liboracle.so (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.ora_hij.restype = ctypes.c_double
            lib.ora_hij.argtypes = [ctypes.c_int, dp, dp, ctypes.c_uint64, ctypes.c_uint64]
            lib.ora_strings.restype = ctypes.c_long
            lib.ora_strings.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            lib.ora_single_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_hmat_dense.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp]
            lib.ora_hdiag.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp]
            lib.ora_sigma.argtypes = [ctypes.c_int] * 3 + [dp, dp, ctypes.c_int, dp, dp,
                                                           ctypes.c_long, ctypes.c_void_p]
            lib.ora_rdm12.argtypes = [ctypes.c_int] * 3 + [dp, dp, ctypes.c_void_p, ctypes.c_void_p]
            lib.ora_rdm3.argtypes = [ctypes.c_int] * 3 + [dp, dp, ctypes.c_void_p]
            lib.ora_rdm2_elements.argtypes = [ctypes.c_int] * 3 + [dp, dp, ctypes.c_long,
                                                                   ctypes.c_void_p, dp]
            lib.ora_sci_sigma.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_void_p, dp, dp, ctypes.c_int,
                                          dp, dp]
            lib.ora_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    """OpenMP threads the oracle uses (1 when built without OpenMP)."""
    return int(_L().ora_num_threads())


def strings(norb: int, nel: int) -> np.ndarray:
    """All norb-bit masks with nel bits set, ascending (uint32)."""
    n = _L().ora_strings(norb, nel, None)
    out = np.zeros(n, dtype=np.uint32)
    _L().ora_strings(norb, nel, out.ctypes.data)
    return out


def single_table(norb: int, nel: int):
    """(J [N][n][n] int32, sgn [N][n][n] int8): J = address of E_pq|I>, -1 if zero."""
    N = len(strings(norb, nel))
    J = np.zeros((N, norb, norb), dtype=np.int32)
    s = np.zeros((N, norb, norb), dtype=np.int8)
    _L().ora_single_table(norb, nel, J.ctypes.data, s.ctypes.data)
    return J, s


def hij(norb, h, eri, I: int, J: int) -> float:
    h, eri = _f64(h), _f64(eri)
    return float(_L().ora_hij(norb, _dp(h), _dp(eri), I, J))


def hmat_dense(norb, nalpha, nbeta, h, eri) -> np.ndarray:
    """Full Hamiltonian in the determinant basis, index = I_alpha*N_beta + I_beta."""
    h, eri = _f64(h), _f64(eri)
    Nd = len(strings(norb, nalpha)) * len(strings(norb, nbeta))
    H = np.zeros((Nd, Nd))
    _L().ora_hmat_dense(norb, nalpha, nbeta, _dp(h), _dp(eri), _dp(H))
    return H


def hdiag(norb, nalpha, nbeta, h, eri) -> np.ndarray:
    h, eri = _f64(h), _f64(eri)
    Nd = len(strings(norb, nalpha)) * len(strings(norb, nbeta))
    d = np.zeros(Nd)
    _L().ora_hdiag(norb, nalpha, nbeta, _dp(h), _dp(eri), _dp(d))
    return d


def sigma(norb, nalpha, nbeta, h, eri, C, rows=None) -> np.ndarray:
    """Direct sigma = H C.  C has shape [nvec, Ndet] (or [nvec, Na, Nb]).

    With ``rows`` (determinant indices) only those outputs are formed and the
    result has shape [nvec, len(rows)].
    """
    h, eri = _f64(h), _f64(eri)
    C = _f64(C)
    nvec = C.shape[0] if C.ndim > 1 else 1
    Cf = C.reshape(nvec, -1)
    Cf = _f64(Cf)
    if rows is None:
        S = np.zeros_like(Cf)
        _L().ora_sigma(norb, nalpha, nbeta, _dp(h), _dp(eri), nvec, _dp(Cf), _dp(S), 0, None)
        return S.reshape(C.shape)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    S = np.zeros((nvec, len(rows)))
    _L().ora_sigma(norb, nalpha, nbeta, _dp(h), _dp(eri), nvec, _dp(Cf), _dp(S),
                   len(rows), rows.ctypes.data)
    return S


def _fix_sign(v):
    """Largest-|c| component positive (ties: lowest index)."""
    k = int(np.argmax(np.abs(v)))
    return v if v[k] >= 0 else -v


def solve_dense(norb, nalpha, nbeta, h, eri, nroots=1):
    """Lowest eigenpairs by dense diagonalisation (LAPACK syevd via numpy)."""
    H = hmat_dense(norb, nalpha, nbeta, h, eri)
    w, V = np.linalg.eigh(H)
    vecs = np.array([_fix_sign(V[:, k]) for k in range(nroots)])
    return w[:nroots], vecs


_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x):
    """splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = x + _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def guess_perturbation(nd, k, amp=0.02):
    """Deterministic symmetry-breaking perturbation of guess vector k: entries
    amp * sqrt(12/nd) * (u - 1/2), u uniform in [0, 1) from splitmix64 of
    (i + (k+1) * golden gamma).  Its norm is about amp.  Without it a
    closed-shell guess keeps the subspace inside one spin-flip symmetry sector
    and roots of the other sector are never found."""
    with np.errstate(over="ignore"):
        x = np.arange(nd, dtype=np.uint64) + np.uint64(k + 1) * _SM_GAMMA
    u = (_splitmix64(x) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return amp * np.sqrt(12.0 / nd) * (u - 0.5)


def davidson(norb, nalpha, nbeta, h, eri, nroots=1, tol=1e-10, max_iter=200,
             max_sub_per_root=12, collapse_per_root=2, guard=1e-8, verbose=False):
    """Textbook Davidson-Liu with the oracle's direct sigma (all FP64).

    Guess: unit vectors at the lowest diagonal elements (ties: lowest index)
    plus the small deterministic perturbation of ``guess_perturbation``,
    orthonormalised.
    Preconditioner: (theta - H_II)^-1, denominators below ``guard`` in size
    replaced by +-guard.  Orthogonalisation: classical Gram-Schmidt applied
    twice.  Converged when every root's residual 2-norm is below ``tol``.
    Returns (energies, vectors [nroots, Ndet], residual norms, iterations).
    """
    d = hdiag(norb, nalpha, nbeta, h, eri)
    Nd = d.size
    order = np.argsort(d, kind="stable")
    nguess = min(nroots, Nd)
    B = np.zeros((nguess, Nd))
    for k in range(nguess):
        B[k] = guess_perturbation(Nd, k)
        B[k, order[k]] += 1.0
    q, _ = np.linalg.qr(B.T)
    B = np.ascontiguousarray(q.T)
    S = sigma(norb, nalpha, nbeta, h, eri, B)
    max_sub = max(max_sub_per_root * nroots, nroots + 1)
    it = 0
    while True:
        it += 1
        G = B @ S.T
        G = 0.5 * (G + G.T)
        w, U = np.linalg.eigh(G)
        theta = w[:nroots]
        X = U[:, :nroots].T @ B
        HX = U[:, :nroots].T @ S
        R = HX - theta[:, None] * X
        rn = np.sqrt((R * R).sum(axis=1))
        if verbose:
            print(f"oracle davidson it {it} dim {B.shape[0]} E {theta} |r| {rn}")
        if np.all(rn < tol) or it >= max_iter or B.shape[0] >= Nd:
            vecs = np.array([_fix_sign(x / np.linalg.norm(x)) for x in X])
            return theta, vecs, rn, it
        new = []
        for k in range(nroots):
            if rn[k] < tol:
                continue
            den = theta[k] - d
            small = np.abs(den) < guard
            den[small] = np.where(den[small] >= 0, guard, -guard)
            new.append(R[k] / den)
        if B.shape[0] + len(new) > max_sub:
            keep = collapse_per_root * nroots
            B = U[:, :keep].T @ B
            S = U[:, :keep].T @ S
            # re-orthonormalise the collapsed basis (it is orthonormal up to rounding)
            q, r = np.linalg.qr(B.T)
            B = q.T
            S = np.linalg.solve(r.T, S)
        added = []
        for v in new:
            for _ in range(2):
                v = v - B.T @ (B @ v)
                for a in added:
                    v = v - a * (a @ v)
            nv = np.linalg.norm(v)
            if nv < 1e-12:
                continue
            added.append(v / nv)
        if not added:
            vecs = np.array([_fix_sign(x / np.linalg.norm(x)) for x in X])
            return theta, vecs, rn, it
        A = np.array(added)
        SA = sigma(norb, nalpha, nbeta, h, eri, A)
        B = np.vstack([B, A])
        S = np.vstack([S, SA])


def det_words(norb, alpha_strings, beta_strings):
    """64-bit determinant words: alpha orbital p at bit p, beta orbital p at bit norb + p
    (2 norb <= 64 spin orbitals, so norb <= 32)."""
    if not 1 <= norb <= 32:
        raise ValueError("determinant words hold at most 32 orbitals")
    a = np.asarray(alpha_strings, dtype=np.uint64)
    b = np.asarray(beta_strings, dtype=np.uint64)
    return a | (b << np.uint64(norb))


def sci_sigma(norb, dets, h, eri, C):
    """Sigma over an arbitrary list of determinants (64-bit words, norb <= 32):
    S[v][i] = sum_j <D_i|H|D_j> C[v][j].  C has shape [nvec, len(dets)].  The list
    may mix (n_alpha, n_beta) sectors; determinants of different sectors do not couple."""
    if not 1 <= norb <= 32:
        raise ValueError("determinant words hold at most 32 orbitals")
    h, eri = _f64(h), _f64(eri)
    dets = np.ascontiguousarray(dets, dtype=np.uint64)
    Cf = _f64(np.atleast_2d(C))
    S = np.zeros_like(Cf)
    _L().ora_sci_sigma(norb, len(dets), dets.ctypes.data, _dp(h), _dp(eri), Cf.shape[0], _dp(Cf), _dp(S))
    return S


def rdm12(norb, nalpha, nbeta, bra, ket=None, one=True, two=True):
    """Spin-free gamma1 [n,n] and Gamma2 [n,n,n,n] (chemist order) by operator
    application on every determinant; bra = ket when ket is None."""
    bra = _f64(bra).reshape(-1)
    ket = bra if ket is None else _f64(ket).reshape(-1)
    g1 = np.zeros((norb, norb)) if one else None
    g2 = np.zeros((norb,) * 4) if two else None
    _L().ora_rdm12(norb, nalpha, nbeta, _dp(bra), _dp(ket),
                   g1.ctypes.data if one else None, g2.ctypes.data if two else None)
    return g1, g2


def rdm3(norb, nalpha, nbeta, bra, ket=None):
    """Spin-free Gamma3 [n]*6: g3[p,q,r,s,t,u] = sum over spins of
    <bra| a+_p a+_r a+_t a_u a_s a_q |ket> (pairs (p,q), (r,s), (t,u) share a spin),
    by operator application on every determinant; bra = ket when ket is None."""
    bra = _f64(bra).reshape(-1)
    ket = bra if ket is None else _f64(ket).reshape(-1)
    g3 = np.zeros((norb,) * 6)
    _L().ora_rdm3(norb, nalpha, nbeta, _dp(bra), _dp(ket), g3.ctypes.data)
    return g3


def rdm2_elements(norb, nalpha, nbeta, vec, idx):
    """Selected Gamma2[p,q,r,s] for idx = [[p,q,r,s], ...] (one vector)."""
    v = _f64(vec).reshape(-1)
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 4)
    out = np.zeros(len(idx))
    _L().ora_rdm2_elements(norb, nalpha, nbeta, _dp(v), _dp(v), len(idx), idx.ctypes.data, _dp(out))
    return out
