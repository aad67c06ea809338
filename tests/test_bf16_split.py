"""The integer-only split of FP64 values into BF16 pairs (csrc/bf16_split.h), used by
the BF16x2 sigma on FP64 vectors, checked on the CPU against exact rational
arithmetic: hi is the BF16 value nearest to x (ties to even), lo the BF16 value
nearest to x - hi, and the float bits of |x| are those of the nearest binary32
value.  The header is compiled with the host compiler; no GPU is involved."""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER_DIR = os.path.join(os.path.dirname(HERE), "paper_2405_10197_gb300", "csrc")

DRIVER = r"""
#include <stdio.h>
#include "bf16_split.h"
int main() {
  unsigned long long b;
  while (scanf("%llx", &b) == 1) {
    double x;
    memcpy(&x, &b, 8);
    uint16_t h = 0, l = 0;
    uint32_t f = 0;
    const int ok = forte::bf16_split_bits(x, h, l) ? 1 : 0;
    const int okf = forte::f32_abs_bits(x, f) ? 1 : 0;
    printf("%d %04x %04x %d %08x\n", ok, h, l, okf, f);
  }
  return 0;
}
"""


def _exp2_floor(a: Fraction) -> int:
    """floor(log2(a)) for a > 0, exactly."""
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    return e


def _round_sig(v: Fraction, bits: int):
    """v rounded to `bits` significant bits, nearest, ties to even; returns (value, exponent, q)."""
    if v == 0:
        return Fraction(0), None, 0
    s = -1 if v < 0 else 1
    a = abs(v)
    e = _exp2_floor(a)
    q = a / Fraction(2) ** (e - bits + 1)  # in [2^(bits-1), 2^bits)
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    if n == 2 ** bits:
        n //= 2
        e += 1
    return s * n * Fraction(2) ** (e - bits + 1), e, n


def _bf16_bits(v: Fraction) -> int:
    """Bits of a normal BF16 value v (exactly representable)."""
    if v == 0:
        return 0
    val, e, n = _round_sig(v, 8)
    assert val == v and -126 <= e <= 127, "not a normal BF16 value"
    sign = 0x8000 if v < 0 else 0
    return sign | ((e + 127) << 7) | (n & 0x7F)


def _cases(rng):
    xs = [0.0, -0.0, 1.0, -1.0, 0.5, 3.0, 1e-30, -2.5e-20, 2.0 ** -126, 2.0 ** -117, 1.7e38, -3.0e38,
          2.0 ** 127 * 1.9999, 1.0 + 2.0 ** -8, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, 1.0 - 2.0 ** -53,
          1.0 + 2.0 ** -9 + 2.0 ** -40, -(1.0 + 2.0 ** -9), 255.0 / 256.0, 2.0 ** -120 * (1 + 2.0 ** -30),
          2.0 ** -118 + 2.0 ** -127, 2.0 ** -118 + 2.0 ** -126, -(2.0 ** -117 + 2.0 ** -126 + 2.0 ** -134)]
    # ties of hi (bit 44 of the fraction set alone) and of lo (tie at the 8th bit of the remainder)
    for _ in range(300):
        e = rng.randint(-100, 100)
        keep = rng.getrandbits(7)
        xs.append(struct.unpack("<d", struct.pack("<Q", ((e + 1023) << 52) | (keep << 45) | (1 << 44)))[0])
        sh = rng.randint(0, 36)
        rem = ((rng.getrandbits(8) | 0x80) << sh) | ((1 << (sh - 1)) if sh else 0)
        rem &= (1 << 45) - 1
        xs.append(struct.unpack("<d", struct.pack("<Q", (rng.getrandbits(1) << 63) | ((e + 1023) << 52)
                                                  | (keep << 45) | rem))[0])
    for _ in range(6000):
        b = rng.getrandbits(64)
        xs.append(struct.unpack("<d", struct.pack("<Q", b))[0])  # every exponent, NaN and inf included
    for _ in range(6000):
        xs.append(rng.uniform(-1.0, 1.0) * 10.0 ** rng.randint(-35, 35))
    return xs


@pytest.fixture(scope="module")
def split_tool(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("bf16split")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True)
    return str(exe)


def test_split_matches_exact_rounding(split_tool):
    rng = random.Random(7)
    xs = _cases(rng)
    inp = "\n".join("%016x" % struct.unpack("<Q", struct.pack("<d", x))[0] for x in xs) + "\n"
    out = subprocess.run([split_tool], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    handled = 0
    for x, line in zip(xs, out):
        ok, h, l, okf, f = line.split()
        ok, okf = int(ok), int(okf)
        finite = x == x and abs(x) != float("inf")
        if not finite:
            assert ok == 0 and okf == 0, x
            continue
        X = Fraction(x)
        # the float bits of |x|
        if x == 0:
            assert okf == 1 and int(f, 16) == 0
        elif 2.0 ** -126 <= abs(x) and abs(x) < 2.0 ** 128:
            fv, fe, fn = _round_sig(abs(X), 24)
            if fe <= 127:
                assert okf == 1, x
                assert int(f, 16) == ((fe + 127) << 23) | (fn & 0x7FFFFF), x
        else:
            assert okf == 0, x
        if ok == 0:
            # refusals only where a part is not a normal BF16 number
            if x != 0 and 2.0 ** -126 <= abs(x) < 2.0 ** 127:
                hv, he, _ = _round_sig(X, 8)
                lv, le, _ = _round_sig(X - hv, 8)
                assert lv != 0 and le < -126, x
            continue
        handled += 1
        hv, he, _ = _round_sig(X, 8)
        if x == 0:
            assert int(h, 16) == (0x8000 if math.copysign(1.0, x) < 0 else 0) and int(l, 16) == 0
            continue
        assert int(h, 16) == _bf16_bits(hv), x
        lv, le, _ = _round_sig(X - hv, 8)
        assert int(l, 16) == _bf16_bits(lv), x
        # hi + lo carries 16 significant bits of x
        if x != 0:
            assert abs(X - hv - lv) <= abs(X) * Fraction(1, 2 ** 16)
    assert handled > 6000
