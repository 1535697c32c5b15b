"""The bit-pattern conversions of the CUDA path (csrc/bits.cuh), compiled for
the host and checked against exact arithmetic.

The keys, the fixed-point cell sums and the float32 hi/lo records are built
from float64 bit patterns with integer operations instead of float64
conversions.  Each function must equal its definition:
  * split_f32(c): hi = c rounded to float32, lo = (c - hi) rounded to float32
    (the two conversions it replaces), for random values, exact ties and
    significands that round up into the next binade;
  * quantise_unit(u, 29): floor(u 2^29) clamped to [0, 2^29 - 1], negative and
    NaN to 0, +inf to the top, on every quantisation boundary and next to it;
  * fixed_from_double(x, E): floor(x 2^E) exactly (negative and subnormal x);
  * fixed_to_double_trunc(v): |v| truncated to 53 significant bits, signed.
"""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2401_13708_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc")
    if not nvcc:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("bits") / "bits_check")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "bits_check.cu"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    def run(lines):
        out = subprocess.run([exe], input="".join(lines), capture_output=True, text=True, check=True)
        return out.stdout.split("\n")
    return run


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_dbits(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def fbits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def test_split_f32_equals_the_two_conversions(driver):
    rng = np.random.default_rng(11)
    xs = list(rng.uniform(-1.0, 1.0, 20000))
    xs += list(rng.choice([-1.0, 1.0], 20000) * 2.0 ** rng.uniform(-75, 105, 20000))
    for _ in range(5000):  # exact ties: the 29 dropped bits are 1000...0
        h = int(rng.integers(2 ** 23, 2 ** 24))
        xs.append(float(h * 2 ** 29 + 2 ** 28) * 2.0 ** int(rng.integers(-110, -40)) * float(rng.choice([-1, 1])))
    for _ in range(5000):  # just below a power of two: rounding carries into the next binade
        xs.append(float(2 ** 53 - int(rng.integers(1, 2 ** 28))) * 2.0 ** int(rng.integers(-110, -40)))
    xs += [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -60, 2.0 ** -61, -(2.0 ** -60), 2.0 ** 99, 1e-300, 5e-324]
    out = driver([f"S {dbits(x):x}\n" for x in xs])
    bad = 0
    for x, line in zip(xs, out):
        hi = np.float32(x)
        lo = np.float32(x - float(hi))
        if line.split() != [f"{fbits(hi):08x}", f"{fbits(lo):08x}"]:
            bad += 1
    assert bad == 0


def test_quantise_is_the_clamped_floor(driver):
    rng = np.random.default_rng(12)
    us = list(rng.random(20000))
    k = rng.integers(0, 2 ** 29, 5000)
    us += [float(v) * 2.0 ** -29 for v in k]                           # on a boundary
    us += [np.nextafter(float(v) * 2.0 ** -29, -1.0) for v in k[k > 0]]  # just below one
    us += list(2.0 ** -rng.uniform(0, 1080, 5000))
    us += [0.0, -0.0, 1.0, 1.0 - 2.0 ** -53, 2.0, -1e-300, 5e-324, math.inf, -math.inf, math.nan, 1e300]
    out = driver([f"Q {dbits(u):x} 29\n" for u in us])
    top = 2 ** 29 - 1
    bad = 0
    for u, line in zip(us, out):
        if math.isnan(u) or u < 0 or (u == 0.0):
            want = 0
        elif math.isinf(u):
            want = top
        else:
            want = min(top, math.floor(Fraction(u) * 2 ** 29))
        bad += int(line) != want
    assert bad == 0


def test_fixed_point_is_the_exact_floor_and_back(driver):
    rng = np.random.default_rng(13)
    cases = []
    for _ in range(20000):
        kind = rng.random()
        if kind < 0.3:
            x = float(rng.uniform(-2e4, 2e4))
        elif kind < 0.6:
            x = float(rng.choice([-1, 1]) * 10 ** rng.uniform(-40, 4))
        elif kind < 0.7:
            x = float(rng.choice([-1, 1]) * 5e-324 * int(rng.integers(1, 1000)))
        else:
            x = float(rng.choice([-1, 1]) * rng.random() * 2.0 ** int(rng.integers(-80, 15)))
        E = int(rng.integers(60, 111))
        if abs(x) * 2.0 ** E < 2.0 ** 125:
            cases.append((x, E))
    cases += [(0.0, 100), (-0.0, 100), (-0.5, 0), (0.5, 0), (-1e-300, 100), (1e-300, 100)]
    out = driver([f"F {dbits(x):x} {E}\n" for x, E in cases])
    vals = []
    bad = 0
    for (x, E), line in zip(cases, out):
        v = int(line, 16)
        v = v - 2 ** 128 if v >= 2 ** 127 else v
        bad += v != math.floor(Fraction(x) * 2 ** E)
        vals.append(v)
    assert bad == 0
    vals += [1, -1, 2 ** 53 - 1, 2 ** 53 + 1, -(2 ** 124) - 12345, 2 ** 64 + 7, 2 ** 126 - 1]
    out = driver([f"T {v % 2 ** 128:032x}\n" for v in vals])
    for v, line in zip(vals, out):
        a = abs(v)
        t = a.bit_length()
        tr = (a >> (t - 53)) << (t - 53) if t > 53 else a
        want = 0.0 if v == 0 else (float(tr) if v > 0 else -float(tr))
        bad += from_dbits(int(line, 16)) != want
    assert bad == 0
