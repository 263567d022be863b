"""The fixed-point arithmetic of the gradient products, compiled for the CPU and checked
against rational arithmetic (no GPU, no oracle).

Reading P1 of the products: every w = r (FP64) x y is put in 63-bit fixed point, one
int64 at the column's power-of-two scale 2^ex (|w| 2^ex < 2^52, so sums of up to 2048
terms cannot overflow), and every sum is an exact integer operation; the sums are
rounded once to FP32 and FP64.  For FP32 y the scaled product is formed from the range
split in two FP32 parts (r = r_hi + r_lo): within 2^-47 |w 2^ex| + 1.5 of the exact one;
for FP64 y it is the FP64 product, rounded once, then to an integer.  The same header
the kernels include is built here into a small host program (tests/host/fixed_point.cu)
and every result is compared with Fraction arithmetic: the scale bounds, the fixed
point within its stated error, and both roundings of a sum as the correctly rounded
(nearest, ties to even) value where the result is normal.
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


def floor_log2(w):
    """floor(log2 |w|) of a non-zero Fraction."""
    w = abs(w)
    e = w.numerator.bit_length() - w.denominator.bit_length()
    while Fraction(2) ** e > w:
        e -= 1
    while Fraction(2) ** (e + 1) <= w:
        e += 1
    return e


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


def test_scale_bound_is_the_binade_or_one_more(host):
    """The column scale of FP32 inputs comes from lg_bound: floor(log2 |r y|) or that plus
    one (never less, or the fixed point could overflow), INT_MIN for a zero product."""
    rng = random.Random(3)
    cases = [(random_double(rng), random_float(rng)) for _ in range(4000)]
    cases += [(1.0, 1.0), (1.9999999999999998, 1.9999999), (2.0 ** -1074, 2.0 ** -149), (0.0, 1.0), (1.0, 0.0)]
    res = host([f"l {d_bits(r)} {f_bits(y)}" for r, y in cases])
    for (r, y), (lg,) in zip(cases, res):
        w = Fraction(r) * Fraction(y)
        if w == 0:
            assert int(lg) == INT_MIN
            continue
        e = floor_log2(w)
        assert int(lg) in (e, e + 1), (r, y, lg, e)


def test_lg64_is_the_binade(host):
    rng = random.Random(4)
    cases = [random_double(rng) * random_double(rng) for _ in range(3000)] + [0.0, 2.0 ** -1074, 1.0, -3.0]
    res = host([f"g {d_bits(w)}" for w in cases])
    for w, (lg,) in zip(cases, res):
        if w == 0:
            assert int(lg) == INT_MIN
        else:
            assert int(lg) == floor_log2(Fraction(w)), w


def test_scale_keeps_every_term_below_2_52():
    """scale_of(M) = 51 - M, clamped to [-252, 252]: with |w| < 2^(M + 1), |w| 2^ex < 2^52 and
    a sum of 2048 terms stays below 2^63 (checked on the formula the header states)."""
    for M in range(-200, 300):
        ex = max(-252, min(252, 51 - M))
        if 51 - M >= -252:
            assert (M + 1) + ex <= 52 and 2048 * 2 ** 52 <= 2 ** 63


def test_scale_of_matches_its_definition(host):
    ms = list(range(-320, 320, 7)) + [INT_MIN]
    res = host([f"s {m}" for m in ms])
    for m, (ex,) in zip(ms, res):
        expect = 0 if m == INT_MIN else max(-252, min(252, 51 - m))
        assert int(ex) == expect, m


def fixed_cases(rng, n, fp64_y=False):
    cases = []
    for _ in range(n):
        r = abs(random_double(rng)) if rng.random() < 0.9 else random_double(rng)
        y = random_double(rng) if fp64_y else random_float(rng)
        w = Fraction(r) * Fraction(y)
        if w == 0:
            cases.append((r, y, rng.randint(-20, 200)))
            continue
        lg = floor_log2(w)
        ex = max(-252, min(252, 51 - lg - rng.randint(0, 1) - (rng.randint(0, 120) if rng.random() < 0.3 else 0)))
        cases.append((r, y, ex))
    return cases


def test_fixed_point_of_fp32_products(host):
    """fx_of: within 2^-47 |r y 2^ex| + 1.5 of r y 2^ex for every scale at or below the
    column's (ranges of any size: below 2^-60 the product is taken in FP64)."""
    rng = random.Random(11)
    cases = fixed_cases(rng, 6000)
    cases += [(1.0, 1.0, 51), (2.0 ** -61, 1.0, 112), (2.0 ** -1074, 1.0, 252), (0.3, 2.0 ** -149, 202),
              (1e-3, 0.999999, 61), (0.0, 1.0, 60), (1.0 / 3.0, -0.75, 53)]
    cases = [(r, bits_f(f_bits(y)), ex) for r, y, ex in cases]       # y as the FP32 the host reads
    res = host([f"x {d_bits(r)} {f_bits(y)} {ex}" for r, y, ex in cases])
    n_small = 0
    for (r, y, ex), (v,) in zip(cases, res):
        exact = Fraction(r) * Fraction(y) * Fraction(2) ** ex
        assert abs(Fraction(int(v)) - exact) <= Fraction(1, 2 ** 47) * abs(exact) + Fraction(3, 2), (r, y, ex, v)
        n_small += 0 < abs(r) < 2.0 ** -60
    assert n_small > 100          # the FP64 path of tiny ranges was exercised


def test_fixed_point_of_fp64_products(host):
    """fx_of64: the FP64 product r y (one rounding), scaled by 2^ex and rounded to the nearest
    integer (ties to even)."""
    rng = random.Random(12)
    cases = fixed_cases(rng, 3000, fp64_y=True)
    res = host([f"X {d_bits(r)} {d_bits(y)} {ex}" for r, y, ex in cases])
    for (r, y, ex), (v,) in zip(cases, res):
        w = Fraction(r * y) * Fraction(2) ** ex          # r * y: one IEEE rounding, as on the device
        n = math.floor(w)
        rem = w - n
        if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
            n += 1
        assert int(v) == n, (r, y, ex)


def conversion_cases(rng):
    cases = []
    for _ in range(12000):
        k = rng.random()
        if k < 0.4:
            v0 = rng.randint(-(1 << 62), 1 << 62)
        elif k < 0.7:
            v0 = rng.randint(-(1 << 20), 1 << 20)
        else:
            v0 = rng.choice([0, 1, -1, (1 << 53) - 1, 1 << 53, (1 << 53) + 1, -(1 << 58), (1 << 24) - 1,
                             (1 << 24) + 1, (1 << 62) - 1, -(1 << 63), (1 << 63) - 1])
        ex = rng.randint(-252, 252) if rng.random() < 0.3 else rng.randint(-60, 200)
        cases.append((v0, ex))
    for _ in range(3000):             # exact ties at both precisions, and a unit off them
        P = rng.choice([24, 53])
        m = rng.randint(1 << (P - 1), (1 << P) - 1)
        N = (((m << 1) | 1) << rng.randint(0, 61 - (P + 1))) + rng.choice([0, 0, 1, -1])   # |N| < 2^62
        if rng.random() < 0.5:
            N = -N
        cases.append((N, rng.randint(-50, 50)))
    return cases


def test_both_roundings_are_correct(host):
    """A fixed-point sum S 2^-ex rounded to FP32 and FP64: nearest, ties to even wherever the
    result is normal; a subnormal result is within one unit of the format's last place."""
    cases = conversion_cases(random.Random(2))
    res = host([f"c {v0} {ex}" for v0, ex in cases])
    n_sub = 0
    for (v0, ex), (b64, b32) in zip(cases, res):
        exact = Fraction(v0) / Fraction(2) ** ex
        for bits, P, emin, emax, eb, tiny, conv in ((int(b64), 53, -1022, 1023, 11, Fraction(2) ** -1074, bits_d),
                                                    (int(b32), 24, -126, 127, 8, Fraction(2) ** -149, bits_f)):
            if exact == 0 or abs(exact) >= Fraction(2) ** emin:
                assert bits == rounded_bits(exact, P, emin, emax, eb), (v0, ex, P)
            else:
                assert abs(Fraction(conv(bits)) - exact) <= tiny, (v0, ex, P)
                n_sub += P == 24
    assert n_sub > 50           # the subnormal FP32 results were exercised


def test_the_two_conversion_forms_agree(host):
    """The integer form (batches, merged items) and the conversion-instruction form (the
    one-game driver's one-terminal items) give the same bits, so results do not depend on
    which kernel formed a product."""
    cases = conversion_cases(random.Random(5))
    a = host([f"c {v0} {ex}" for v0, ex in cases])
    b = host([f"C {v0} {ex}" for v0, ex in cases])
    assert a == b
