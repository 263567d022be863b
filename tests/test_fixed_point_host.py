"""The exact arithmetic of the gradient products, compiled for the CPU and checked
against rational arithmetic (no GPU, no oracle).

The product kernels never round a sum (reading P1): each w = r (FP64) x y (FP32)
is formed exactly from the two significands, put in two-limb fixed point at a
power-of-two scale (integer part + 40 fraction bits, truncated), summed in
integers, and rounded once to FP32 and FP64.  The same header the kernels
include is built here into a small host program (tests/host/fixed_point.cu);
every result is compared with Fraction arithmetic: w bit for bit, the fixed
point as the truncation it is defined to be, and both roundings as the
correctly rounded (nearest, ties to even) value, subnormals and overflow
included.
"""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INT_MIN = -(2 ** 31)


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fx") / "fixed_point")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1810_03063_b300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "fixed_point.cu"), "-o", exe],
                   check=True, capture_output=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return [l.split() for l in out.stdout.splitlines()]
    return run


def d_bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def f_bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def bits_d(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def bits_f(b):
    return struct.unpack("<f", struct.pack("<I", b))[0]


def rounded_bits(exact, P, emin, emax, ebits):
    """Bit pattern of `exact` rounded to nearest even in a binary format with P-bit
    significands, minimum normal exponent emin, maximum exponent emax."""
    sign = 1 if exact < 0 else 0
    a = abs(exact)
    total = 1 + ebits + (P - 1)
    if a == 0:
        return sign << (total - 1)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    q = max(e, emin) - (P - 1)                     # weight of the last significand bit
    scaled = a / Fraction(2) ** q
    n = scaled.numerator // scaled.denominator
    rem = scaled - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    if n == 0:
        return sign << (total - 1)
    if n >= 2 ** P:                                # carry into the next binade
        n //= 2
        q += 1
    e_last = q + P - 1
    if e_last > emax:
        return (sign << (total - 1)) | (((1 << ebits) - 1) << (P - 1))   # infinity
    if n < 2 ** (P - 1):                           # subnormal
        return (sign << (total - 1)) | n
    field = e_last - emin + 1
    return (sign << (total - 1)) | (field << (P - 1)) | (n - 2 ** (P - 1))


def random_double(rng):
    k = rng.random()
    if k < 0.5:
        x = rng.random() * 10 ** rng.uniform(-6, 0)      # range weights, r / Z
    elif k < 0.7:
        x = rng.random() * 2.0 ** rng.randint(-1070, -1000)   # subnormal or nearly
    elif k < 0.75:
        x = 0.0
    else:
        x = rng.uniform(-4, 4)
    return x


def random_float(rng):
    k = rng.random()
    if k < 0.5:
        x = rng.random()                                 # a strategy entry
    elif k < 0.7:
        x = rng.random() * 2.0 ** rng.randint(-149, -120)     # FP32 subnormal range
    elif k < 0.75:
        x = 0.0
    else:
        x = rng.uniform(-3, 3) * 2.0 ** rng.randint(-60, 10)
    return struct.unpack("<f", struct.pack("<f", x))[0]


def test_w_is_the_exact_product(host):
    rng = random.Random(1810030630)
    cases = [(random_double(rng), random_float(rng)) for _ in range(4000)]
    cases += [(1.0, 1.0), (2.0 ** -1074, 2.0 ** -149), (-0.0, 1.0), (1.0 - 2.0 ** -53, 1.0 - 2.0 ** -24)]
    res = host([f"w {d_bits(r)} {f_bits(y)}" for r, y in cases])
    for (r, y), (hi, lo, E, lg, neg) in zip(cases, res):
        exact = Fraction(r) * Fraction(y)
        P = (int(hi) << 64) | int(lo)
        got = Fraction(P) * Fraction(2) ** int(E)
        assert got == abs(exact), (r, y)
        if exact == 0:
            assert int(lg) == INT_MIN
        else:
            assert int(neg) == (1 if exact < 0 else 0)
            assert Fraction(2) ** int(lg) <= abs(exact) < Fraction(2) ** (int(lg) + 1)


def test_scale_bound_is_the_binade_or_one_more(host):
    """The column scale of FP32 inputs comes from lg_bound: floor(log2 |r y|) or that plus
    one (never less, or the fixed point could overflow), INT_MIN for a zero product."""
    rng = random.Random(3)
    cases = [(random_double(rng), random_float(rng)) for _ in range(4000)]
    cases += [(1.0, 1.0), (1.9999999999999998, 1.9999999), (2.0 ** -1074, 2.0 ** -149), (0.0, 1.0), (1.0, 0.0)]
    res = host([f"l {d_bits(r)} {f_bits(y)}" for r, y in cases])
    for (r, y), (lg,) in zip(cases, res):
        w = abs(Fraction(r) * Fraction(y))
        if w == 0:
            assert int(lg) == INT_MIN
            continue
        e = w.numerator.bit_length() - w.denominator.bit_length()
        while Fraction(2) ** e > w:
            e -= 1
        while Fraction(2) ** (e + 1) <= w:
            e += 1
        assert int(lg) in (e, e + 1), (r, y, lg, e)


def test_w_with_fp64_y_is_the_rounded_product(host):
    rng = random.Random(7)
    cases = [(random_double(rng), random_double(rng)) for _ in range(2000)]
    res = host([f"W {d_bits(r)} {d_bits(y)}" for r, y in cases])
    for (r, y), (hi, lo, E, lg, neg) in zip(cases, res):
        w = r * y                                        # one IEEE rounding, as on the device
        P = (int(hi) << 64) | int(lo)
        assert Fraction(P) * Fraction(2) ** int(E) == abs(Fraction(w))


def test_fixed_point_is_the_truncation_at_40_fraction_bits(host):
    rng = random.Random(11)
    cases = []
    for _ in range(4000):
        r, y = random_double(rng), random_float(rng)
        w = Fraction(r) * Fraction(y)
        if w == 0:
            cases.append((r, y, rng.randint(-20, 200)))
            continue
        lg = math.floor(math.log2(abs(w))) if abs(w) > 2 ** -1000 else None
        if lg is None:                                   # log2 of a tiny Fraction: exact way
            lg = w.numerator.bit_length() - w.denominator.bit_length()
            while Fraction(2) ** lg > abs(w):
                lg -= 1
            while Fraction(2) ** (lg + 1) <= abs(w):
                lg += 1
        ex = 47 - lg - rng.randint(0, 110)               # the column's scale, or a smaller one
        cases.append((r, y, ex))
    res = host([f"x {d_bits(r)} {f_bits(y)} {ex}" for r, y, ex in cases])
    for (r, y, ex), (v0, v1) in zip(cases, res):
        w = Fraction(r) * Fraction(y)
        t = abs(w) * Fraction(2) ** (ex + 40)
        mag = t.numerator // t.denominator               # truncation toward zero of |w|
        expect = -mag if w < 0 else mag
        assert (int(v0) << 40) + int(v1) == expect, (r, y, ex)
        assert abs(int(v1)) < 2 ** 40 and (int(v0) == 0 or int(v1) == 0 or (int(v0) < 0) == (int(v1) < 0))


def conversion_cases(rng):
    cases = []
    for _ in range(12000):
        k = rng.random()
        if k < 0.4:
            v0 = rng.randint(-(1 << 59), 1 << 59)
        elif k < 0.7:
            v0 = rng.randint(-(1 << 20), 1 << 20)
        else:
            v0 = rng.choice([0, 1, -1, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, -(1 << 58), (1 << 24) - 1,
                             (1 << 24) + 1, (1 << 62) - 1])
        v1 = rng.randint(-(1 << 51), 1 << 51) if rng.random() < 0.5 else rng.randint(-(1 << 40), 1 << 40)
        if rng.random() < 0.05:
            v1 = 0
        r = rng.random()
        ex = rng.randint(-1200, 1200) if r < 0.2 else rng.randint(-60, 200) if r < 0.8 else rng.randint(60, 260)
        cases.append((v0, v1, ex))
    for _ in range(3000):             # exact ties at both precisions, and a unit off them
        P = rng.choice([24, 53])      # (the deciding bit then lies far below the significand)
        m = rng.randint(1 << (P - 1), (1 << P) - 1)
        N = (((m << 1) | 1) << rng.randint(0, 100 - (P + 1))) + rng.choice([0, 0, 1, -1])   # |v0| < 2^60
        if rng.random() < 0.5:
            N = -N
        v0 = N >> 40
        cases.append((v0, N - (v0 << 40), rng.randint(-50, 50)))
    return cases


def test_both_roundings_are_correct(host):
    """Sums of fixed-point values (limbs of either sign, fraction limb outside [0, 2^40))
    rounded to FP32 and FP64: nearest, ties to even, subnormals, overflow to infinity."""
    cases = conversion_cases(random.Random(2))
    res = host([f"c {v0} {v1} {ex}" for v0, v1, ex in cases])
    n_sub = n_tie = 0
    for (v0, v1, ex), (b64, b32) in zip(cases, res):
        exact = Fraction((v0 << 40) + v1) / Fraction(2) ** (40 + ex)
        assert int(b64) == rounded_bits(exact, 53, -1022, 1023, 11), (v0, v1, ex)
        assert int(b32) == rounded_bits(exact, 24, -126, 127, 8), (v0, v1, ex)
        n_sub += exact != 0 and abs(exact) < Fraction(2) ** -126
    assert n_sub > 100          # the subnormal FP32 path was exercised
