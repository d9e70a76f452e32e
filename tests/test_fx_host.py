"""Host check of the block fixed-point arithmetic of the complex128 kernels
(paper_2311_01512_gb300/csrc/qs_fx.cuh) against exact rational arithmetic.

The header's host path (the same code the kernels run, with the integer
multiply-adds in 64-bit C++ arithmetic) is driven by tests/host/fx_check.cpp.
For every dot product y = sum_k x_k m_k, K <= 4, the result must satisfy

    |fx(y) - y| <= 2^-53 |y| + 2^-55 max|x_k| max|m_k|

and for 4 < K <= 8 (two accumulators, the two-target gate's rows)

    |fx(y) - y| <= 2^-53 |y| + 2^-54 max|x_k| max|m_k|

(plus the flush of subnormal inputs and outputs), every fixed-point constant
must be m rounded to nearest on its group's grid, and on random unitary gate
rows (one and two targets) the fixed-point results must be on average at least
as accurate as IEEE FP64 evaluation with fused multiply-adds.  CPU only."""

import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U = Fraction(1, 2 ** 53)
TINY = 2.0 ** -1022


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_bits(u):
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def bexp(x):
    return (bits(x) >> 52) & 0x7FF


@pytest.fixture(scope="module")
def fx_exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path_factory.mktemp("fx") / "fx_check"
    src = os.path.join(ROOT, "tests", "host", "fx_check.cpp")
    inc = os.path.join(ROOT, "paper_2311_01512_gb300", "csrc")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", inc, src, "-o", str(exe)], check=True)
    return str(exe)


def run_cases(exe, cases):
    lines = []
    for xs, ms in cases:
        lines.append(" ".join([str(len(xs))] + ["%016x" % bits(v) for v in xs] + ["%016x" % bits(v) for v in ms]))
    res = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    out = []
    for line in res.stdout.split("\n"):
        if line.strip():
            parts = line.split()
            out.append((from_bits(int(parts[0], 16)), [int(v) for v in parts[1:]]))
    assert len(out) == len(cases)
    return out


def fma(a, b, c):
    """IEEE fused multiply-add, rounded once (Fraction -> float rounds to nearest even)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def check_case(xs, ms, y, consts):
    exact = sum(Fraction(x) * Fraction(m) for x, m in zip(xs, ms))
    X = max(abs(Fraction(x)) for x in xs)
    M = max(abs(Fraction(m)) for m in ms)
    # flushed subnormal inputs contribute their whole product to the error
    flushed = sum(abs(Fraction(x) * Fraction(m)) for x, m in zip(xs, ms) if x != 0 and bexp(x) == 0)
    flushed += sum(abs(Fraction(x) * Fraction(m)) for x, m in zip(xs, ms) if m != 0 and bexp(m) == 0)
    second = Fraction(1, 2 ** 55) if len(xs) <= 4 else Fraction(1, 2 ** 54)
    bound = U * abs(exact) + second * X * M + flushed + Fraction(TINY)
    err = abs(Fraction(y) - exact)
    assert err <= bound, (xs, ms, y, float(exact), float(err), float(bound))
    # the constants: m rounded to nearest on the grid 2^(em - 1082) of its group
    em = max(bexp(m) for m in ms)
    for m, c in zip(ms, consts):
        assert abs(c) < 2 ** 60
        if bexp(m) == 0:
            assert c == 0
            continue
        grid = Fraction(2) ** (em - 1082)
        assert abs(Fraction(c) * grid - Fraction(m)) <= grid / 2, (m, c, em)
    return err, exact, X * M


def gauss_pair(rng, spread):
    return rng.gauss(0.0, 1.0) * 2.0 ** rng.randint(-spread, 0)


def random_cases(rng, n, kmin=1, kmax=4):
    cases = []
    for it in range(n):
        K = rng.randint(kmin, kmax)
        spread = (0, 3, 12, 80)[it % 4]
        scale = 2.0 ** rng.randint(-40, 40)
        xs = [gauss_pair(rng, spread) * scale for _ in range(K)]
        ms = [gauss_pair(rng, spread % 13) for _ in range(K)]
        cases.append((xs, ms))
    return cases


def edge_cases(rng):
    cases = []
    specials = [0.0, -0.0, 1.0, -1.0, 0.5, 2.0 ** -52, 1.0 + 2.0 ** -52, -(1.0 + 2.0 ** -52), 2.0 - 2.0 ** -52,
                3.0 * 2.0 ** -1070, -(2.0 ** -1030), 2.0 ** -1022, 2.0 ** 500, -(2.0 ** -500), 0.1, -1.0 / 3.0,
                math.pi, -math.e, 2.0 ** -60, 2.0 ** -59 * 3]
    for _ in range(4000):
        K = rng.randint(1, 4)
        xs = [rng.choice(specials) * (2.0 ** rng.randint(-5, 5) if rng.random() < 0.3 else 1.0) for _ in range(K)]
        ms = [rng.choice(specials[:14] + [rng.uniform(-1, 1)]) for _ in range(K)]
        # keep the products inside the normal range
        if any(abs(x) > 2.0 ** 400 for x in xs):
            ms = [m if abs(m) < 2.0 ** 100 else 1.0 for m in ms]
        cases.append((xs, ms))
    # near-total cancellation: x0 m0 + x1 m1 with m1 = -x0 m0 / x1 rounded
    for _ in range(2000):
        x0, x1, m0 = rng.gauss(0, 1), rng.gauss(0, 1), rng.gauss(0, 1)
        m1 = -x0 * m0 / x1
        cases.append(([x0, x1], [m0, m1]))
    # the largest component with all significand bits set, the others 2^-7 .. 2^-70 of it
    for d in range(0, 72):
        big = -(2.0 - 2.0 ** -52)
        small = (1.0 + 2.0 ** -52) * 2.0 ** -d
        cases.append(([big, small, -small, small], [0.25, 1.0 - 2.0 ** -53, -0.75, 0.5]))
    return cases


def unitary_rows(rng, n):
    """Rows of random 2x2 unitaries realified, on random amplitudes of a
    30-qubit-sized state (moduli near 2^-15): the one-target gate's rows."""
    cases = []
    for _ in range(n):
        a = [complex(rng.gauss(0, 1), rng.gauss(0, 1)) for _ in range(4)]
        # Gram-Schmidt on two columns: a Haar-like unitary
        c0 = a[0:2]
        nrm = math.sqrt(sum(abs(z) ** 2 for z in c0))
        c0 = [z / nrm for z in c0]
        c1 = a[2:4]
        ip = sum(z0.conjugate() * z1 for z0, z1 in zip(c0, c1))
        c1 = [z1 - ip * z0 for z0, z1 in zip(c0, c1)]
        nrm = math.sqrt(sum(abs(z) ** 2 for z in c1))
        c1 = [z / nrm for z in c1]
        m00, m10, m01, m11 = c0[0], c0[1], c1[0], c1[1]
        x = [rng.gauss(0, 1) * 2.0 ** -15 for _ in range(4)]   # (a.re, a.im, b.re, b.im)
        rows = [[m00.real, -m00.imag, m01.real, -m01.imag], [m00.imag, m00.real, m01.imag, m01.real]]
        for r in rows:
            cases.append((x, r))
    return cases


def unitary4_rows(rng, n):
    """Rows of random 4x4 unitaries realified over the eight parts of four
    amplitudes (moduli near 2^-15): the two-target gate's rows."""
    cases = []
    for _ in range(n):
        cols = []
        for _ in range(4):   # Gram-Schmidt on four Gaussian columns
            v = [complex(rng.gauss(0, 1), rng.gauss(0, 1)) for _ in range(4)]
            for c in cols:
                ip = sum(a.conjugate() * b for a, b in zip(c, v))
                v = [b - ip * a for a, b in zip(c, v)]
            nrm = math.sqrt(sum(abs(z) ** 2 for z in v))
            cols.append([z / nrm for z in v])
        x = [rng.gauss(0, 1) * 2.0 ** -15 for _ in range(8)]   # (re, im) of four amplitudes
        j = rng.randrange(4)
        u = [cols[k][j] for k in range(4)]                       # row j: u_jk
        re = [v for k in range(4) for v in (u[k].real, -u[k].imag)]
        im = [v for k in range(4) for v in (u[k].imag, u[k].real)]
        cases.append((x, re))
        cases.append((x, im))
    return cases


def test_fx_bound_random(fx_exe):
    rng = random.Random(2311015120)
    cases = random_cases(rng, 12000)
    worst = 0.0
    for (xs, ms), (y, consts) in zip(cases, run_cases(fx_exe, cases)):
        err, exact, xm = check_case(xs, ms, y, consts)
        if xm:
            worst = max(worst, float(err / xm))
    # the bound's second term alone is 2^-55 of X M; results must not sit far above 2^-53 of it
    assert worst <= 2.0 ** -52


def test_fx_bound_edges(fx_exe):
    rng = random.Random(2311015121)
    cases = edge_cases(rng)
    for (xs, ms), (y, consts) in zip(cases, run_cases(fx_exe, cases)):
        check_case(xs, ms, y, consts)


def test_fx_exact_cases(fx_exe):
    """Results that block fixed point must reproduce exactly: zero inputs, a
    single exactly representable product, sums whose exact value has at most
    53 significant bits within the grids."""
    cases = [([0.0, 0.0, 0.0, 0.0], [0.3, -0.2, 0.1, 0.5]),
             ([0.7, -0.2], [0.0, 0.0]),
             ([1.5], [0.25]),
             ([-3.0, 1.0], [0.5, 0.25]),
             ([2.0 ** -15, 2.0 ** -16, -(2.0 ** -17), 2.0 ** -18], [1.0, 1.0, 1.0, 1.0]),
             ([0.5, 0.5], [1.0, -1.0])]
    want = [0.0, 0.0, 0.375, -1.25, 2.0 ** -15 + 2.0 ** -16 - 2.0 ** -17 + 2.0 ** -18, 0.0]
    for (y, _), w in zip(run_cases(fx_exe, cases), want):
        assert y == w


def test_fx_not_less_accurate_than_fp64(fx_exe):
    """On the one-target gate's rows (random unitaries, random amplitudes) the
    mean and the 99.9th percentile of the error, in units of 2^-53 sum|x_k m_k|,
    are no larger than those of FP64 evaluated as the FP64 kernel does
    (a product, then three fused multiply-adds)."""
    rng = random.Random(2311015122)
    cases = unitary_rows(rng, 3000)
    e_fx, e_64 = [], []
    for (xs, ms), (y, consts) in zip(cases, run_cases(fx_exe, cases)):
        err, exact, _ = check_case(xs, ms, y, consts)
        s = sum(abs(Fraction(x) * Fraction(m)) for x, m in zip(xs, ms))
        y64 = ms[0] * xs[0]
        for k in range(1, 4):
            y64 = fma(ms[k], xs[k], y64)
        e_fx.append(float(err / (U * s)))
        e_64.append(float(abs(Fraction(y64) - exact) / (U * s)))
    e_fx.sort()
    e_64.sort()
    q = int(0.999 * len(e_fx))
    assert sum(e_fx) / len(e_fx) <= sum(e_64) / len(e_64)
    assert e_fx[q] <= e_64[q]


def test_fx_bound_eight_terms(fx_exe):
    """Dot products of five to eight terms, summed in two accumulators as the
    two-target gate does, within the K <= 8 bound."""
    rng = random.Random(2311015123)
    cases = random_cases(rng, 8000, 5, 8)
    for (xs, ms), (y, consts) in zip(cases, run_cases(fx_exe, cases)):
        check_case(xs, ms, y, consts)


def test_fx_eight_terms_extremes(fx_exe):
    """The largest sums eight terms can reach: every x and m with all
    significand bits set at the top of its block, all products of one sign
    (|V| within 2^11 of 2^63), and their cancelling mixtures."""
    top = 2.0 - 2.0 ** -52
    cases = []
    for sx in (1.0, -1.0):
        for sm in (1.0, -1.0):
            cases.append(([sx * top] * 8, [sm * top] * 8))
    cases.append(([top, -top] * 4, [top] * 8))
    cases.append(([top] * 7 + [2.0 ** -60], [top] * 8))
    cases.append(([top * 2.0 ** -15] * 8, [top * 2.0 ** -3] * 8))
    for (xs, ms), (y, consts) in zip(cases, run_cases(fx_exe, cases)):
        check_case(xs, ms, y, consts)
    ys = [y for y, _ in run_cases(fx_exe, cases[:4])]
    assert ys[0] == ys[3] > 0 and ys[1] == ys[2] == -ys[0]


def test_fx_two_target_rows_not_less_accurate_than_fp64(fx_exe):
    """On the two-target gate's rows (random 4x4 unitaries, random amplitudes)
    the mean and 99.9th percentile of the error, in units of 2^-53 sum|x_k m_k|,
    are no larger than those of FP64 evaluated as a product then seven fused
    multiply-adds."""
    rng = random.Random(2311015124)
    cases = unitary4_rows(rng, 1500)
    e_fx, e_64 = [], []
    for (xs, ms), (y, consts) in zip(cases, run_cases(fx_exe, cases)):
        err, exact, _ = check_case(xs, ms, y, consts)
        s = sum(abs(Fraction(x) * Fraction(m)) for x, m in zip(xs, ms))
        y64 = ms[0] * xs[0]
        for k in range(1, 8):
            y64 = fma(ms[k], xs[k], y64)
        e_fx.append(float(err / (U * s)))
        e_64.append(float(abs(Fraction(y64) - exact) / (U * s)))
    e_fx.sort()
    e_64.sort()
    q = int(0.999 * len(e_fx))
    assert sum(e_fx) / len(e_fx) <= sum(e_64) / len(e_64)
    assert e_fx[q] <= e_64[q]
