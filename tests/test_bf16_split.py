"""CPU test of the integer-only FP64 -> BF16 hi + lo split used by the tensor-core path
(paper_1901_05128_gb300/csrc/bf16split.h), compiled with the host C compiler and
checked against exact rational rounding (round to nearest, ties to even, 8 significant
bits, normal BF16 range)."""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1901_05128_gb300", "csrc", "bf16split.h")

DRIVER = r'''
#include <stdio.h>
#include <inttypes.h>
#include "bf16split.h"
int main(void) {
    unsigned long long u;
    while (scanf("%llx", &u) == 1) {
        double x; uint16_t hi, lo;
        memcpy(&x, &u, 8);
        bf16_split(x, &hi, &lo);
        printf("%04x %04x\n", hi, lo);
    }
    return 0;
}
'''


def _rn_bf16(fr):
    if fr == 0:
        return Fraction(0)
    s = -1 if fr < 0 else 1
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q = a / Fraction(2) ** (e - 7)
    qi = math.floor(q)
    r = q - qi
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and qi % 2 == 1):
        qi += 1
    if qi == 256:
        qi, e = 128, e + 1
    if e < -126:
        return Fraction(0)
    if e > 127:
        return None                      # overflow
    return s * qi * Fraction(2) ** (e - 7)


def _bf16_value(bits):
    s = -1 if bits >> 15 else 1
    e = (bits >> 7) & 0xFF
    m = bits & 0x7F
    if e == 0:
        return Fraction(0) if m == 0 else None
    if e == 0xFF:
        return None
    return s * (128 + m) * Fraction(2) ** (e - 127 - 7)


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("bf16")
    src = d / "drv.c"
    src.write_text(DRIVER)
    out = d / "drv"
    subprocess.run([cc, "-O2", "-std=c99", "-I", os.path.dirname(HDR), str(src), "-o", str(out)], check=True)
    return str(out)


def _values():
    rnd = random.Random(190105128)
    vals = [0.0, -0.0, 1.0, -1.0, 1.5, 3.0, 1e-30, -1e-30, 1e30, 3.0e38, 1e-38, 2.0 ** -126, 2.0 ** -130,
            1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -30, 255.5, 256.0 - 2.0 ** -6,
            1351.4378, -0.000123456789]
    for _ in range(3000):
        m = rnd.uniform(1.0, 2.0)
        e = rnd.randint(-120, 120)
        vals.append(rnd.choice([-1, 1]) * m * 2.0 ** e)
    for _ in range(500):                 # exact ties between neighbouring BF16 values
        q = rnd.randint(128, 255)
        vals.append((q + 0.5) * 2.0 ** rnd.randint(-100, 100))
    return vals


def test_split_matches_exact_rounding(exe):
    vals = _values()
    inp = "\n".join("%016x" % struct.unpack("<Q", struct.pack("<d", v))[0] for v in vals)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for v, line in zip(vals, out):
        hi, lo = (int(t, 16) for t in line.split())
        x = Fraction(v)
        h_ref = _rn_bf16(x)
        assert h_ref is not None
        assert _bf16_value(hi) == h_ref, (v, hex(hi))
        l_ref = _rn_bf16(x - h_ref) if h_ref != 0 else Fraction(0)
        assert _bf16_value(lo) == l_ref, (v, hex(lo))
        if abs(v) >= 2.0 ** -110:        # hi + lo carries 16 bits: relative error <= 2^-16
            assert abs(Fraction(v) - h_ref - l_ref) <= abs(Fraction(v)) * Fraction(1, 2 ** 16)


TF32_DRIVER = r'''
#include <stdio.h>
#include <inttypes.h>
#include "bf16split.h"
int main(void) {
    unsigned long long u;
    while (scanf("%llx", &u) == 1) {
        double x; uint32_t hi, lo;
        memcpy(&x, &u, 8);
        tf32_split(x, &hi, &lo);
        printf("%08x %08x\n", hi, lo);
    }
    return 0;
}
'''


def _rn_bits(fr, nb):
    """Round to nb significant bits (nearest, ties to even) in the normal FP32 range."""
    if fr == 0:
        return Fraction(0)
    s = -1 if fr < 0 else 1
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q = a / Fraction(2) ** (e - nb + 1)
    qi = math.floor(q)
    r = q - qi
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and qi % 2 == 1):
        qi += 1
    if qi == 2 ** nb:
        qi, e = 2 ** (nb - 1), e + 1
    if e < -126:
        return Fraction(0)
    if e > 127:
        return None
    return s * qi * Fraction(2) ** (e - nb + 1)


def _f32_value(bits):
    s = -1 if bits >> 31 else 1
    e = (bits >> 23) & 0xFF
    m = bits & 0x7FFFFF
    if e == 0:
        return Fraction(0) if m == 0 else None
    if e == 0xFF:
        return None
    return s * (2 ** 23 + m) * Fraction(2) ** (e - 127 - 23)


@pytest.fixture(scope="module")
def exe_tf32(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("tf32")
    src = d / "drv.c"
    src.write_text(TF32_DRIVER)
    out = d / "drv"
    subprocess.run([cc, "-O2", "-std=c99", "-I", os.path.dirname(HDR), str(src), "-o", str(out)], check=True)
    return str(out)


def test_tf32_split_matches_exact_rounding(exe_tf32):
    """TF32 split: 11 significant bits per part, the 13 low FP32 mantissa bits zero,
    hi + lo within 2^-22 relative (22 bits)."""
    rnd = random.Random(190105129)
    vals = _values()
    for _ in range(500):                 # exact ties between neighbouring TF32 values
        q = rnd.randint(1024, 2047)
        vals.append((q + 0.5) * 2.0 ** rnd.randint(-100, 100))
    inp = "\n".join("%016x" % struct.unpack("<Q", struct.pack("<d", v))[0] for v in vals)
    out = subprocess.run([exe_tf32], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for v, line in zip(vals, out):
        hi, lo = (int(t, 16) for t in line.split())
        assert hi & 0x1FFF == 0 and lo & 0x1FFF == 0, (v, hex(hi), hex(lo))
        x = Fraction(v)
        h_ref = _rn_bits(x, 11)
        assert h_ref is not None
        assert _f32_value(hi) == h_ref, (v, hex(hi))
        l_ref = _rn_bits(x - h_ref, 11) if h_ref != 0 else Fraction(0)
        assert _f32_value(lo) == l_ref, (v, hex(lo))
        if abs(v) >= 2.0 ** -100:
            assert abs(Fraction(v) - h_ref - l_ref) <= abs(Fraction(v)) * Fraction(1, 2 ** 22)
