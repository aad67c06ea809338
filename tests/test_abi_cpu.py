"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, exports every entry point the header declares, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "forte_gpu.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2405_10197_gb300 import build
    path = build.build()
    import paper_2405_10197_gb300 as fg
    return fg.library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(forte_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_four_core_calls():
    names = declared_functions()
    for core in ("forte_cas_create", "forte_sigma", "forte_davidson", "forte_rdms"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"


def test_library_targets_sm_103a():
    from paper_2405_10197_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def _create(lib, n, na, nb, h, eri):
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    return lib.forte_cas_create(n, na, nb, h.ctypes.data, eri.ctypes.data)


@pytest.mark.parametrize("n,na,nb", [(0, 0, 0), (17, 1, 1), (4, 5, 1), (4, 1, -1)])
def test_create_rejects_bad_sizes(lib, n, na, nb):
    m = max(n, 1)
    assert not _create(lib, n, na, nb, np.zeros((m, m)), np.zeros((m,) * 4))
    assert "invalid sizes" in lib.forte_last_error().decode()


def test_create_rejects_null_pointers(lib):
    assert not lib.forte_cas_create(4, 2, 2, None, None)
    assert "non-NULL" in lib.forte_last_error().decode()


def test_create_rejects_nan_and_asymmetry(lib):
    import synth_inputs as si
    h, eri = si.integrals(4, 8, seed=0)
    bad = h.copy()
    bad[1, 2] = np.nan
    assert not _create(lib, 4, 2, 2, bad, eri)
    assert "NaN" in lib.forte_last_error().decode()
    bad = h.copy()
    bad[0, 1] += 1e-6
    assert not _create(lib, 4, 2, 2, bad, eri)
    assert "symmetric" in lib.forte_last_error().decode()
    e2 = eri.copy()
    e2[0, 1, 2, 3] += 1e-6
    assert not _create(lib, 4, 2, 2, h, e2)
    assert "symmetry" in lib.forte_last_error().decode()


def test_null_context_is_an_argument_error(lib):
    assert lib.forte_sigma(None, None, None, 1) == 1
    assert lib.forte_davidson(None, 1, ctypes.c_double(1e-8)) == 1
    assert lib.forte_rdms(None, None, None, None) == 1
    lib.forte_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2405_10197_gb300 as fg
    monkeypatch.setattr(fg, "_lib", None)
    monkeypatch.setattr(fg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        fg.library()


def _prototypes():
    """name -> (return type text, [parameter type texts]) from the header."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \t\*]*?)\b(forte_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        ps = [p.strip() for p in params.split(",") if p.strip()]
        if ps == ["void"]:
            ps = []
        # drop the parameter name, keep the type
        types = [re.sub(r"\b\w+$", "", p).strip() if not p.endswith("*") else p for p in ps]
        out[name] = (ret.strip(), types)
    return out


def _ctype_kind(c):
    if c in (ctypes.c_void_p, ctypes.c_char_p):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_double: "double", ctypes.c_longlong: "long long",
            ctypes.c_ulonglong: "unsigned long long"}[c]


def _decl_kind(t):
    if "*" in t:
        return "ptr"
    t = t.replace("const", "").strip()
    return t


def test_binding_signatures_match_the_header(lib):
    # a ctypes argument list that disagrees with the C prototype passes garbage silently
    protos = _prototypes()
    assert len(protos) >= len(declared_functions()) - 1
    for name, (ret, params) in protos.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, f"{name}: binding sets no argtypes"
        got = [_ctype_kind(a) for a in f.argtypes]
        want = [_decl_kind(p) for p in params]
        assert got == want, f"{name}: binding {got} vs header {want}"
        if "*" in ret:
            assert f.restype in (ctypes.c_void_p, ctypes.c_char_p), name
        elif ret.endswith("void"):
            assert f.restype is None, name
        else:
            assert f.restype is ctypes.c_int, name
