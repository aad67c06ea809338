"""Pin strength: plant plausible mistakes in a copy of the oracle (on the CPU)
and check that the pins in test_oracle_pins.py catch every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "dropped two-body term of a single replacement":
        ("if (((J >> K) & 1ULL) && K != p) v += va_so(n, eri, m, K, p, K);", ""),
    "creators of a double replacement in the wrong order":
        ("s *= op_cre(&t, o);\n    s *= op_cre(&t, m);", "s *= op_cre(&t, m);\n    s *= op_cre(&t, o);"),
    "transposed integral index (pq|rs) for <pq|rs>":
        ("return eri[(((size_t)p * n + r) * n + q) * n + s];",
         "return eri[(((size_t)p * n + q) * n + r) * n + s];"),
    "missing 1/2 on the diagonal two-body sum":
        ("e += 0.5 * va_so(n, eri, P, Q, P, Q);", "e += 1.0 * va_so(n, eri, P, Q, P, Q);"),
    "phase counts the orbital itself":
        ("for (int Q = 0; Q < P; ++Q) c += (int)((d >> Q) & 1ULL);",
         "for (int Q = 0; Q <= P; ++Q) c += (int)((d >> Q) & 1ULL);"),
    "2-RDM with r and s exchanged":
        ("s *= op_ann(&d, s_ + tg * n);\n                  if (!s) continue;\n                  s *= op_cre(&d, r + tg * n);",
         "s *= op_ann(&d, r + tg * n);\n                  if (!s) continue;\n                  s *= op_cre(&d, s_ + tg * n);"),
    "wrong sign of the one-body single element":
        ("double v = h_so(n, h, m, p);", "double v = -h_so(n, h, m, p);"),
    "3-RDM creators applied in the wrong order":
        ("s *= op_cre(&d, t + s3 * n);\n                  if (!s) continue;\n                  s *= op_cre(&d, r + s2 * n);",
         "s *= op_cre(&d, r + s2 * n);\n                  if (!s) continue;\n                  s *= op_cre(&d, t + s3 * n);"),
    "3-RDM annihilator paired with the wrong spin":
        ("s *= op_ann(&d, u + s3 * n);", "s *= op_ann(&d, u + s2 * n);"),
    "exchange integral added instead of subtracted":
        ("return v_so(n, eri, P, Q, R, S) - v_so(n, eri, P, Q, S, R);",
         "return v_so(n, eri, P, Q, R, S) + v_so(n, eri, P, Q, S, R);"),
    "occupation limit taken as strict upper bound":
        ("keep &= (tot >= gmin[g]) & (tot <= gmax[g])", "keep &= (tot >= gmin[g]) & (tot < gmax[g])", "gas.py"),
    "space boundaries shifted by one orbital":
        ("        orb = 0\n", "        orb = 1\n", "gas.py"),
    "restricted sigma without the projection of the input":
        ("Cf = np.asarray(C, dtype=np.float64).reshape(C.shape[0], -1) * keep",
         "Cf = np.asarray(C, dtype=np.float64).reshape(C.shape[0], -1)", "gas.py"),
    "spin sector with the opposite exchange sign":
        ("v[j * N + i] = parity / np.sqrt(2.0)", "v[j * N + i] = -parity / np.sqrt(2.0)", "spin.py"),
    "odd spin sector keeps the diagonal determinants":
        ("                if parity < 0:\n                    continue\n", "", "spin.py"),
    "determinant-list sigma without the double replacements":
        ("if (popc64(dets[i] ^ dets[j]) > 4) continue;", "if (popc64(dets[i] ^ dets[j]) > 2) continue;"),
    "2x2 estimate takes the upper root":
        ("return D - np.sqrt(D * D + np.asarray(V, dtype=np.float64) ** 2)",
         "return D + np.sqrt(D * D + np.asarray(V, dtype=np.float64) ** 2)", "aci.py"),
    "2x2 estimate without the half of the diagonal gap":
        ("D = 0.5 * (np.asarray(Hmm, dtype=np.float64) - E)", "D = (np.asarray(Hmm, dtype=np.float64) - E)", "aci.py"),
    "determinant diagonal stored beta-major":
        ("    d[i] = ora_hij(n, h, eri, I, I);", "    d[(i % sp.Nb) * sp.Na + i / sp.Nb] = ora_hij(n, h, eri, I, I);"),
    "model space without the reference determinants":
        ("        M = ~excl\n", "        M = ~excl & ~P\n", "aci.py"),
    "first-order space of a list without the mixed alpha-beta doubles":
        ("    for x in a1:\n        for y in b1:\n            out.add(x | (y << norb))\n", "", "aci_list.py"),
    "list coupling to the reference determinants without their coefficients":
        ("    x[len(F):] = cP\n", "    x[len(F):] = 1.0\n", "aci_list.py"),
    "list parity sector with the opposite exchange sign":
        ("            v[j] = parity / np.sqrt(2.0)\n", "            v[j] = -parity / np.sqrt(2.0)\n", "aci_list.py"),
    "list exclusion by the signed estimate":
        ("excl = aci_excluded(_mirror_max(np.abs(eps), F, norb, pair), sigma)",
         "excl = aci_excluded(_mirror_max(eps, F, norb, pair), sigma)", "aci_list.py"),
}


# the pins that can see a mistake in each file (keeps each mutation run short: the
# Davidson and adaptive-CI pins take minutes and cannot see a core Slater-Condon slip
# that the Hamiltonian, RDM and sigma pins do not see first)
PIN_FILTER = {
    "oracle_core.c": "not aci and not davidson_matches_dense and not spin_sectors and not gas",
    "gas.py": "gas",
    "spin.py": "spin",
    "aci.py": "aci",
    "aci_list.py": "",
}
# the pin file of each mutated file (test_oracle_pins.py unless named here)
PIN_FILE = {"aci_list.py": "test_oracle_aci_list.py"}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new, fname = (MUTATIONS[name] + ("oracle_core.c",))[:3]
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert old in src, f"mutation anchor no longer present in {fname}"
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    (tmp_path / "oracle" / fname).write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "synth_inputs.py"), tmp_path)
    os.makedirs(tmp_path / "tests")
    pins = PIN_FILE.get(fname, "test_oracle_pins.py")
    for f in ("conftest.py", "fock_ref.py", pins):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests")
    sel = ["-k", PIN_FILTER[fname]] if PIN_FILTER[fname] else []
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] + sel +
                       ["tests/" + pins], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake not caught: {name}\n{r.stdout[-2000:]}"
