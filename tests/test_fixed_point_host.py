"""Host build of the fixed-point helpers behind LBM_FP64_FIXED, against exact arithmetic.

The kernel's 64-bit fixed-point conversions, products and compile-time shell constants are
`__host__ __device__`; `tests/native/fixed_point_host.cu` compiles them for the CPU and
this test checks them with Python's exact integers and fractions: conversions round to
nearest (ties away from zero in magnitude), products keep the floor of the high 64 bits,
and every shell constant is the correctly rounded value of its definition from the
library's own float64 weights and lattice scale.
"""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

from paper_1703_04594_gb300 import lbm
from tests.gpu_util import ensure_built

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "fixed_point_host.cu")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    assert os.path.exists(nvcc), "nvcc is required to build the host probe"
    exe = str(tmp_path_factory.mktemp("fx") / "fixed_point_host")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-o", exe, SRC], check=True,
                   capture_output=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split("\n")[:-1]
    return run


def bits(v: float) -> str:
    return format(struct.unpack("<Q", struct.pack("<d", v))[0], "x")


def from_bits(h: str) -> float:
    return struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0]


def round_half_away(q: Fraction) -> int:
    n = abs(q)
    r = int(n) + (1 if n - int(n) >= Fraction(1, 2) else 0)
    return r if q >= 0 else -r


def test_shell_constants_are_exact(probe):
    ensure_built()
    c, w, vx, vy = lbm.model()
    c2 = c * c                                      # the float64 product the kernel uses
    shells = sorted({vx[i] ** 2 + vy[i] ** 2 for i in range(37)})
    w_of = {vx[i] ** 2 + vy[i] ** 2: w[i] for i in range(37)}
    rows = [list(map(int, line.split())) for line in probe(["const"])]
    for s, e, cw, cq, cq2, cw6 in rows:
        v2 = shells[s]
        ws = Fraction(w_of[v2])
        assert Fraction(1, 2) <= ws * 2 ** e < 1                   # w_s 2^e_s in [0.5, 1)
        assert cw == round_half_away(ws * 2 ** (e + 63))
        assert cw6 == round_half_away(ws * 2 ** (e + 64) / 6)
        if s == 0:
            continue
        q = Fraction(c2 * v2)                                      # float64 q_s = c^2 |v|^2
        assert cq == round_half_away(ws * q * 2 ** (e + 59))
        assert abs(cq2 - ws * q * q * 2 ** (e + 55)) <= 1          # one intermediate rounding


def test_double_to_fixed_rounds_to_nearest(probe):
    rng = random.Random(7)
    cases = [(0.0, 60), (-0.0, 60), (1.0, 62), (0.2, 60), (-0.2, 60), (7.999999, 58), (2.0 ** -40, 58),
             (3.0 * 2.0 ** -61, 60), (2.5 * 2.0 ** -60, 60), (-2.5 * 2.0 ** -60, 60), (5e-324, 62)]
    for _ in range(400):
        k = rng.randint(56, 69)
        mag = 2.0 ** rng.uniform(-30, 3 + 58 - k)                  # |v| 2^k < 2^62
        cases.append((rng.choice([-1, 1]) * mag, k))
    out = probe([f"from {bits(v)} {k}" for v, k in cases])
    for (v, k), got in zip(cases, out):
        assert int(got) == round_half_away(Fraction(v) * 2 ** k), (v, k)


def to_double_half_away(X: int, k: int) -> float:
    """X 2^-k rounded to 53 significant bits, ties away from zero in magnitude."""
    if X == 0:
        return 0.0
    q = Fraction(abs(X), 2 ** k)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    m = round_half_away(q / Fraction(2) ** (e - 52))               # 53-bit significand
    v = float(Fraction(m) * Fraction(2) ** (e - 52))
    return v if X > 0 else -v


def test_fixed_to_double_rounds_to_nearest(probe):
    rng = random.Random(8)
    cases = [(1, 58), (-1, 58), (2 ** 62, 60), ((1 << 62) - 1, 60), (-(1 << 62) + 1, 62), ((1 << 53) + 1, 58),
             ((1 << 54) + 2, 58), (((1 << 53) - 1) << 10 | (1 << 9), 64)]    # a tie that carries
    for _ in range(400):
        X = rng.randint(1, (1 << rng.randint(1, 62)) - 1) * rng.choice([-1, 1])
        cases.append((X, rng.randint(56, 70)))
    out = probe([f"to {X} {k}" for X, k in cases])
    for (X, k), got in zip(cases, out):
        assert from_bits(got) == to_double_half_away(X, k), (X, k)


def test_products_keep_the_floor_of_the_high_half(probe):
    rng = random.Random(9)
    lim = 1 << 63
    su = [(-1, 1), (-(1 << 63), (1 << 63) - 1), ((1 << 63) - 1, (1 << 63) - 1), (-5, 7), (0, 12345)]
    ss = [(-(1 << 63), -(1 << 63)), (-1, -1), ((1 << 63) - 1, -(1 << 63)), (-3, 5)]
    uu = [((1 << 64) - 1, (1 << 64) - 1), (1 << 63, 2), (12345, 67890)]
    for _ in range(300):
        su.append((rng.randrange(-lim, lim), rng.randrange(0, lim)))
        ss.append((rng.randrange(-lim, lim), rng.randrange(-lim, lim)))
        uu.append((rng.randrange(0, 1 << 64), rng.randrange(0, 1 << 64)))
    out = probe([f"mulsu {a} {b}" for a, b in su] + [f"mul {a} {b}" for a, b in ss] +
                [f"umul {a} {b}" for a, b in uu])
    want = [(a * b) >> 64 for a, b in su + ss + uu]                # Python >> floors
    assert [int(x) for x in out] == want



def test_approximate_products_are_0_to_2_below_the_floor(probe):
    """The relaxation loop's products drop the low partial product and the carries of the
    low halves: the result is floor(a b / 2^64) minus 0, 1 or 2.  For random operands the
    deficit is the floor of U1 + U2 + U3 with U1, U2 uniform on [0, 1) and U3 the product of
    two such: 3/4 on average (the re-centring offsets rest on that mean)."""
    rng = random.Random(13)
    lim = 1 << 63
    m32 = (1 << 32) - 1
    uu = [((1 << 64) - 1, (1 << 64) - 1), (m32, m32), ((m32 << 32) | m32, 1 << 32), (0, 5), (1 << 63, 3)]
    ss = [(-(1 << 63), -(1 << 63)), (-1, -1), ((1 << 63) - 1, -(1 << 63)), (-3, 5)]
    su = [(-1, 1), (-(1 << 63), (1 << 63) - 1), (-5, 7), (0, 12345)]
    for _ in range(2000):
        uu.append((rng.randrange(0, 1 << 64), rng.randrange(0, 1 << 64)))
        ss.append((rng.randrange(-lim, lim), rng.randrange(-lim, lim)))
        su.append((rng.randrange(-lim, lim), rng.randrange(0, lim)))
    out = probe([f"uapx {a} {b}" for a, b in uu] + [f"sapx {a} {b}" for a, b in ss] +
                [f"suapx {a} {b}" for a, b in su])
    got = [int(x) for x in out]
    deficits = [((a * b) >> 64) - g for (a, b), g in zip(uu + ss + su, got)]
    assert all(d in (0, 1, 2) for d in deficits)
    rand = deficits[5:2005]                                       # the random unsigned cases
    assert abs(sum(rand) / len(rand) - 0.75) < 0.05


def test_exponent_lowering_conversion_keeps_zero_and_rounds_to_nearest(probe):
    """fx_to_double_dp_pos: X 2^-k as the round-to-nearest float64 of X with its exponent
    lowered by k, and 0 for X = 0 (no test for zero: the unsigned min on the exponent
    word), for the kernels' formats k = 56 and 58 + e_s (60..69) and signed X."""
    rng = random.Random(17)
    cases = [(0, 56), (0, 69), (1, 60), (-1, 60), ((1 << 63) - 1, 69), (-(1 << 63), 58), (3, 56)]
    for _ in range(500):
        X = rng.randint(1, (1 << rng.randint(1, 63)) - 1) * rng.choice([-1, 1])
        cases.append((X, rng.choice([56, 60, 61, 62, 64, 65, 66, 67, 69])))
    out = probe([f"top {X} {k}" for X, k in cases])
    for (X, k), got in zip(cases, out):
        want = 0.0 if X == 0 else float(X) * 2.0 ** -k      # float(X) rounds to nearest
        assert from_bits(got) == want and bits(from_bits(got)) == bits(want), (X, k)


def test_exact_input_conversion_and_its_range(probe):
    """fx_exact_shift / fx_from_double_shifted: a population f with 2^-7 <= f 2^e < 8 is
    flagged in range and converted to exactly f 2^(59 + e) (an integer there); zero,
    negative, tiny, large and non-finite values are flagged out of range."""
    rng = random.Random(19)
    cases = []
    for e in (2, 3, 4, 6, 7, 9, 11):
        for v in (2.0 ** -7, 8.0 - 2.0 ** -50, 1.0, 0.5 + 2.0 ** -52):
            cases.append((v * 2.0 ** -e, e))
        for v in (0.0, -0.0, -1.0, 8.0, 2.0 ** -7 - 2.0 ** -60, 1e-300, 5e-324, float("inf"), float("nan")):
            cases.append((v * 2.0 ** -e if v == v and abs(v) != float("inf") else v, e))
        for _ in range(100):
            cases.append((rng.uniform(0.0, 9.0) * 2.0 ** (-e - rng.choice([0, 0, 0, 4, 8])), e))
    out = probe([f"exact {bits(v)} {e}" for v, e in cases])
    for (v, e), line in zip(cases, out):
        flag, q = (int(x) for x in line.split())
        inside = v == v and Fraction(1, 128) <= Fraction(v) * 2 ** e < 8 if v == v and abs(v) != float("inf") else False
        assert flag == int(inside), (v, e)
        if inside:
            assert Fraction(q) == Fraction(v) * 2 ** (59 + e), (v, e)


def test_fix_to_double_rn_is_the_correctly_rounded_conversion(probe):
    """fix_to_double_rn(X, k), the float64 step's conversion of its fixed-point moment sums,
    is (double)X * 2^-k rounded to nearest even: against Python's correctly rounded
    float(X) scaled by math.ldexp, on random magnitudes, exact ties (odd and even
    significands), carries into the exponent, zero and the int64 extremes, for the
    scales the kernels use (52 for the moment sums, -825 .. 974 for the adjoint's block
    fixed point)."""
    import math
    rng = random.Random(7)
    xs = [0, 1, -1, 2 ** 52, 2 ** 53 - 1, 2 ** 53 + 1, 2 ** 53 + 3, 2 ** 63 - 1, -(2 ** 63 - 1), -(2 ** 63),
          2 ** 63 - 2 ** 10, (2 ** 53 - 1) * 2 ** 10 + 2 ** 9]
    for _ in range(2000):
        xs.append(rng.getrandbits(rng.randint(1, 63)) * rng.choice([1, -1]))
        b = rng.randint(54, 63)
        x = rng.getrandbits(b) | (1 << (b - 1))
        sh = b - 53
        xs.append(((x >> sh << sh) | (1 << (sh - 1))) * rng.choice([1, -1]))   # a tie
    cases = [(x, k) for x in xs for k in (0, 52, 56, -825, 974)]
    got = probe([f"rn {x} {k}" for x, k in cases])
    for (x, k), g in zip(cases, got):
        want = math.ldexp(float(x), -k)
        assert from_bits(g) == want and (want != 0 or g == "0"), (x, k, g, want)


def test_pow2_scale_is_the_exact_product(probe):
    """pow2_scale(v, k) = v * 2^k bit for bit for normal v and normal results; zeros,
    subnormals, infinities and NaNs come back unchanged; results below the normal range
    become zero with v's sign."""
    import math
    rng = random.Random(8)
    vs = [rng.uniform(-3.0, 3.0) * 10.0 ** rng.randint(-30, 30) for _ in range(3000)]
    cases = [(v, k) for v in vs for k in (-52, -3, -2, -1, 1)]
    got = probe([f"p2 {bits(v)} {k}" for v, k in cases])
    for (v, k), g in zip(cases, got):
        assert from_bits(g) == math.ldexp(v, k), (v, k, g)
    special = [0.0, -0.0, 5e-324, -1e-310, float("inf"), float("-inf")]
    got = probe([f"p2 {bits(v)} -2" for v in special])
    for v, g in zip(special, got):
        assert g == bits(v), (v, g)
    nan = probe([f"p2 {bits(float('nan'))} 3"])[0]
    assert math.isnan(from_bits(nan))
    tiny = 2.0 ** -1020
    assert from_bits(probe([f"p2 {bits(tiny)} -5"])[0]) == 0.0
    assert probe([f"p2 {bits(-tiny)} -5"])[0] == bits(-0.0)
