"""The device operand split of the tensor-core forms (cq_split; the same code splits the
levels and the Toeplitz tiles inside cq_history_direct) against the integer-only split of
bf16split.h compiled for the host, which tests/test_bf16_split.py pins to exact rational
rounding. The device takes a faster route for 2^-74 <= |x| < 2^127 (rounding to odd at 24
bits, one exact FP64 subtraction); every bit of hi and lo must agree on random bit
patterns (all exponents, zeros, subnormals, Inf, NaN), on values near the ends of that
range, and on exact and near ties."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from paper_1901_05128_gb300 import fastcq as fc

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1901_05128_gb300", "csrc")

DRIVER = r'''
#include <stdio.h>
#include <stdlib.h>
#include "bf16split.h"
/* stdin: n doubles; stdout: n (hi, lo) pairs, BF16 (tf32 = 0) or TF32-in-FP32 bits */
int main(int argc, char **argv) {
    const int tf32 = argc > 1 && argv[1][0] == 't';
    double x;
    while (fread(&x, sizeof x, 1, stdin) == 1) {
        if (tf32) {
            uint32_t h, l;
            tf32_split(x, &h, &l);
            fwrite(&h, 4, 1, stdout);
            fwrite(&l, 4, 1, stdout);
        } else {
            uint16_t h, l;
            bf16_split(x, &h, &l);
            fwrite(&h, 2, 1, stdout);
            fwrite(&l, 2, 1, stdout);
        }
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def host_split(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("split")
    (d / "drv.c").write_text(DRIVER)
    exe = str(d / "drv")
    subprocess.run([cc, "-O2", "-std=c99", "-I", CSRC, str(d / "drv.c"), "-o", exe], check=True)

    def run(x, tf32):
        out = subprocess.run([exe, "t" if tf32 else "b"], input=np.ascontiguousarray(x, np.float64).tobytes(),
                             capture_output=True, check=True).stdout
        pairs = np.frombuffer(out, dtype=np.uint32 if tf32 else np.uint16).reshape(-1, 2)
        return pairs[:, 0], pairs[:, 1]
    return run


def _inputs():
    rng = np.random.default_rng(190105128)
    parts = [rng.integers(0, 2 ** 63, 1 << 20, dtype=np.int64).astype(np.uint64) |
             (rng.integers(0, 2, 1 << 20, dtype=np.uint64) << np.uint64(63))]          # any bit pattern
    # exponents around the fast route's ends (949 .. 1149) and FP32's (897 .. 1150)
    ex = rng.integers(880, 1170, 1 << 20).astype(np.uint64)
    man = rng.integers(0, 2 ** 52, 1 << 20, dtype=np.int64).astype(np.uint64)
    sgn = rng.integers(0, 2, 1 << 20, dtype=np.uint64) << np.uint64(63)
    parts.append(sgn | (ex << np.uint64(52)) | man)
    # sparse low bits: the sticky bit of the 24-bit rounding set or clear
    low = np.array([0, 1, 1 << 28, (1 << 29) - 1, 1 << 29], dtype=np.uint64)
    ex2 = rng.integers(940, 1160, 1 << 18).astype(np.uint64)
    top = rng.integers(0, 2 ** 23, 1 << 18, dtype=np.int64).astype(np.uint64) << np.uint64(29)
    parts.append((ex2 << np.uint64(52)) | top | low[rng.integers(0, len(low), 1 << 18)])
    bits = np.concatenate(parts)
    x = bits.view(np.float64)
    # exact ties and near ties at 8 and 11 significant bits, including ones whose remainder
    # ties again
    q8 = rng.integers(128, 256, 1 << 16) + 0.5
    q11 = rng.integers(1024, 2048, 1 << 16) + 0.5
    e = rng.integers(-70, 120, 1 << 16).astype(np.float64)
    eps = rng.choice([0.0, 2.0 ** -40, -(2.0 ** -40), 2.0 ** -9 * 1.5], 1 << 16)
    ties = np.concatenate([(q8 + eps) * 2.0 ** (e - 7), (q11 + eps) * 2.0 ** (e - 10),
                           -(q8 * (1 + 2.0 ** -9)) * 2.0 ** (e - 7)])
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, 2.0 ** -74, 2.0 ** -74 * (1 - 2.0 ** -53),
                        2.0 ** 127, 2.0 ** 127 * (1 - 2.0 ** -53), 2.0 ** 128 * (1 - 2.0 ** -9),
                        3.4e38, 2.0 ** -126, 2.0 ** -127, 5e-324])
    return np.concatenate([x, ties, special, -special])


@pytest.mark.parametrize("prec", [fc.CQ_BF16X3, fc.CQ_TF32X3])
def test_device_split_matches_host_split(host_split, prec):
    x = _inputs()
    tf32 = prec == fc.CQ_TF32X3
    xd = torch.from_numpy(x).to("cuda")
    dt = torch.int32 if tf32 else torch.int16
    hi = torch.zeros(x.size, dtype=dt, device="cuda")
    lo = torch.zeros(x.size, dtype=dt, device="cuda")
    fc.cq_split(prec, xd, hi, lo)
    udt = np.uint32 if tf32 else np.uint16
    h_dev, l_dev = hi.cpu().numpy().view(udt), lo.cpu().numpy().view(udt)
    h_ref, l_ref = host_split(x, tf32)
    bad = np.flatnonzero((h_dev != h_ref) | (l_dev != l_ref))
    assert bad.size == 0, [(float(x[i]), hex(int(h_dev[i])), hex(int(h_ref[i])), hex(int(l_dev[i])),
                            hex(int(l_ref[i]))) for i in bad[:5]]


def test_split_of_nothing():
    x = torch.zeros(0, dtype=torch.float64, device="cuda")
    fc.cq_split(fc.CQ_BF16X3, x, x, x)
