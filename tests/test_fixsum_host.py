"""The fixed-point FP64 neighbour sum of the stencil kernels (csrc/fixsum.cuh),
built for the host and checked against exact rational sums: within its
stated bound (K 2^(e_max - 1079) plus half an ulp), equal to the correctly
rounded sum when no bit is shifted out, and declining (returning false) on
NaN, infinity, tiny rows and overflow."""
import ctypes
import os
import random
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("fixsum") / "fixsum.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", os.path.join(HERE, "native", "fixsum_harness.cpp"),
                    "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.fixsum_k.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    return L


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def val(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def run(lib, xs):
    k = len(xs)
    t = (ctypes.c_uint64 * k)(*[bits(x) for x in xs])
    out = ctypes.c_uint64()
    ok = lib.fixsum_k(k, t, ctypes.byref(out))
    assert ok in (0, 1)
    return bool(ok), val(out.value)



def emax_of(xs):
    return max(max((bits(x) >> 52) & 0x7FF, 1) for x in xs)


def check(lib, xs):
    ok, got = run(lib, xs)
    exact = sum(Fraction(x) for x in xs)
    em = emax_of(xs)
    if not ok:
        return False
    bound = len(xs) * Fraction(2) ** (em - 1079) + (Fraction(abs(np.spacing(got))) / 2 if got != 0 else 0)
    assert abs(Fraction(got) - exact) <= bound, (xs, got, float(exact))
    # no bit shifted out: every term's exponent within the 4 guard bits of e_max
    if all(em - max((bits(x) >> 52) & 0x7FF, 1) <= 4 for x in xs if x != 0.0):
        assert got == float(exact), (xs, got, float(exact))
    return True


@pytest.mark.parametrize("k", [1, 6, 26, 31])
def test_random_sums_within_bound(lib, k):
    rng = random.Random(1000 + k)
    taken = 0
    for _ in range(4000):
        spread = rng.choice([0, 1, 3, 4, 10, 30, 60, 80])
        base = rng.uniform(-40, 40)
        xs = []
        for _ in range(k):
            if rng.random() < 0.15:
                xs.append(0.0)  # a masked-off term
            else:
                xs.append(rng.choice([-1, 1]) * rng.random() * 2.0 ** (base + rng.uniform(-spread, 0)))
        taken += check(lib, xs)
    assert taken == 4000


def test_exact_cancellation_and_small_exponent_spread(lib):
    x = [1.0, -1.0, 2.0 ** -30, 3.0, -3.0, 0.0]
    ok, got = run(lib, x)
    assert ok and got == 2.0 ** -30
    ok, got = run(lib, [0.5, -0.5, 0.0, 0.0, -0.0, 0.0])
    assert ok and got == 0.0 and struct.pack("<d", got) == struct.pack("<d", 0.0)
    # neighbour values of a smooth field: every exponent within the guard bits
    rng = random.Random(7)
    for _ in range(2000):
        c = rng.uniform(0.5, 1.0)
        xs = [c + rng.uniform(-0.01, 0.01) for _ in range(6)]
        ok, got = run(lib, xs)
        assert ok and got == float(sum(Fraction(v) for v in xs))


def test_ties_round_to_even(lib):
    # 2^53 + 1 is exactly halfway between two doubles: ties go to the even 2^53
    ok, got = run(lib, [2.0 ** 53, 1.0, 0.0, 0.0, 0.0, 0.0])
    assert ok and got == 2.0 ** 53
    ok, got = run(lib, [2.0 ** 53 + 2.0, 1.0, 0.0, 0.0, 0.0, 0.0])
    assert ok and got == 2.0 ** 53 + 4.0
    # rounding that carries into a new leading bit
    ok, got = run(lib, [2.0 ** 54 - 2.0, 1.0, 0.5, 0.0, 0.0, 0.0])
    assert ok and got == float(Fraction(2 ** 54 - 2) + Fraction(3, 2))


def test_declines_special_and_extreme_rows(lib):
    assert not run(lib, [1.0, float("nan"), 0.0, 0.0, 0.0, 0.0])[0]
    assert not run(lib, [float("inf"), 1.0, 0.0, 0.0, 0.0, 0.0])[0]
    assert not run(lib, [1e-300, 2e-300, 0.0, 0.0, 0.0, 5e-310])[0]  # all below 2^-966
    assert not run(lib, [1.7e308, 1.7e308, 0.0, 0.0, 0.0, 0.0])[0]  # the sum overflows
    ok, got = run(lib, [1.0, 5e-324, 0.0, 0.0, 0.0, 0.0])  # a subnormal term beside a normal one
    assert ok and got == 1.0
    ok, got = run(lib, [0.0] * 6)
    assert ok and got == 0.0


# ---------------------------------------------------------------------------
# Fixed-point dot products (the FP64 block update's P and Q columns)

@pytest.fixture(scope="module")
def dlib(lib):
    lib.fixdot_k.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.fix_align_value.argtypes = [ctypes.c_uint64, ctypes.c_int]
    lib.fix_align_value.restype = ctypes.c_int64
    lib.fix_coef_value.argtypes = [ctypes.c_uint64, ctypes.c_int]
    lib.fix_coef_value.restype = ctypes.c_int64
    return lib


def bexp(x):
    return (bits(x) >> 52) & 0x7FF


def fdot(dlib, vs, cs, E=None, Fc=None):
    k = len(vs)
    E = max(bexp(v) for v in vs) if E is None else E
    Fc = max([63] + [bexp(c) for c in cs]) if Fc is None else Fc
    out = ctypes.c_uint64()
    ok = dlib.fixdot_k(k, (ctypes.c_uint64 * k)(*[bits(v) for v in vs]),
                       (ctypes.c_uint64 * k)(*[bits(c) for c in cs]), E, Fc, ctypes.byref(out))
    assert ok in (0, 1)
    return bool(ok), val(out.value), E, Fc


def fma_chain(vs, cs):
    """K - 1 FP64 fused multiply-adds after the first product, each rounded once."""
    p = float(Fraction(vs[0]) * Fraction(cs[0]))
    for v, c in zip(vs[1:], cs[1:]):
        p = float(Fraction(v) * Fraction(c) + Fraction(p))
    return p


def test_alignment_is_truncation_and_rounding(dlib):
    """a = trunc(v 2^(1083 - E)), C = round(c 2^(1083 - Fc)), against exact
    scaling, over exponents within and far beyond the 8 guard bits."""
    rng = random.Random(7)
    for _ in range(3000):
        E = rng.randint(62, 2000)
        e = max(1, E - rng.choice([0, 1, 5, 8, 9, 30, 55, 61, 62, 63, 64, 70]))
        v = rng.choice([-1, 1]) * (1 + rng.random()) * 2.0 ** (e - 1023)
        if bexp(v) > E:
            continue
        exact = Fraction(v) * Fraction(2) ** (1083 - E)
        a = dlib.fix_align_value(bits(v), E)
        assert a == int(exact), (v, E)  # int() truncates toward zero
        assert abs(a) < 2 ** 61
        Fc = max(1023, bexp(v))
        C = dlib.fix_coef_value(bits(v), Fc)
        ex = Fraction(v) * Fraction(2) ** (1083 - Fc)
        assert abs(C - ex) <= Fraction(1, 2) and abs(C) <= 2 ** 61
    assert dlib.fix_align_value(bits(0.0), 1023) == 0 and dlib.fix_align_value(bits(-0.0), 1023) == 0
    assert dlib.fix_align_value(bits(5e-324), 62) == 0  # subnormal: below one unit


def test_dot_error_within_bound(dlib):
    """|computed - exact| <= (1 + 7K/16) 2^(E + Fc - 2102) + half an ulp, for
    rows and coefficient columns of every spread of magnitudes."""
    rng = random.Random(11)
    for _ in range(3000):
        k = rng.randint(1, 7)
        spread_v = rng.choice([0, 2, 8, 20, 60, 100])
        spread_c = rng.choice([0, 3, 10, 40])
        base = rng.uniform(-200, 200)
        vs = [rng.choice([-1, 1]) * rng.random() * 2.0 ** (base - rng.uniform(0, spread_v)) for _ in range(k)]
        cs = [rng.choice([-1, 1]) * rng.random() * 2.0 ** rng.uniform(-spread_c, 4) for _ in range(k)]
        if rng.random() < 0.1:
            cs[0] = 1.0  # the U_j term
        ok, got, E, Fc = fdot(dlib, vs, cs)
        assert ok
        exact = sum(Fraction(v) * Fraction(c) for v, c in zip(vs, cs))
        bound = (1 + Fraction(7 * k, 16)) * Fraction(2) ** (E + Fc - 2102)
        if got != 0:
            bound += Fraction(abs(np.spacing(got))) / 2
        assert abs(Fraction(got) - exact) <= bound, (vs, cs, got, float(exact))


def test_dot_exact_cases(dlib):
    """One value times a power of two is exact when the column holds only that
    coefficient (the 8 guard bits of a and C carry no bits); so are an exact
    cancellation and zero terms beside a coefficient 1."""
    rng = random.Random(3)
    for _ in range(500):
        v = rng.uniform(-1e10, 1e10)
        for c in (1.0, 2.0 ** rng.randint(-30, 30), -0.5):
            ok, got, _, _ = fdot(dlib, [v], [c])
            assert ok and got == v * c
        ok, got, _, _ = fdot(dlib, [v, -v], [1.0, 1.0])
        assert ok and got == 0.0 and math_copysign(got) > 0
        ok, got, _, _ = fdot(dlib, [v, 0.0, 0.0], [1.0, 3.0, -7.0])
        assert ok and got == v


def math_copysign(x):
    import math
    return math.copysign(1.0, x)


def test_dot_declines_outside_normal_range(dlib):
    ok, _, _, _ = fdot(dlib, [1e308, 1e308], [1.0, 1.5])  # overflow
    assert not ok
    ok, _, _, _ = fdot(dlib, [1e-300], [1e-10])  # subnormal result
    assert not ok
    ok, got, _, _ = fdot(dlib, [1e300], [1.0])
    assert ok and got == 1e300


@pytest.mark.parametrize("s", [4, 6])
def test_dot_no_less_accurate_than_fma_chain_on_krylov_rows(dlib, s):
    """On rows like the block update's (a monomial basis of the Jacobi-scaled
    7-point Laplacian, P_old and Q_old one step older, beta scaled like the
    basis), the fixed-point error is smaller than that of the FP64 FMA chain it
    replaces, in mean and in maximum (units of 2^-53 sum |v c|; measured at
    s = 4: 0.24 / 1.07 against 0.36 / 2.01, at s = 6: 0.18 / 1.71 against
    0.30 / 2.26)."""
    rng = np.random.default_rng(5)
    N = 12
    n = N ** 3

    def dinvA(v):
        V = v.reshape(N, N, N)
        out = 6 * V.copy()
        out[1:] -= V[:-1]
        out[:-1] -= V[1:]
        out[:, 1:] -= V[:, :-1]
        out[:, :-1] -= V[:, 1:]
        out[:, :, 1:] -= V[:, :, :-1]
        out[:, :, :-1] -= V[:, :, 1:]
        return (out / 6).ravel()

    U = [rng.uniform(-1, 1, n) * 1e-6]
    for _ in range(s):
        U.append(dinvA(U[-1]))
    Po = [rng.uniform(-1, 1, n) * 1.2e-6]
    for _ in range(s - 1):
        Po.append(dinvA(Po[-1]) + 0.1 * Po[-1])
    Qo = [dinvA(p) for p in Po]
    beta = np.array([[rng.normal() * 0.85 * 2.0 ** (j - l) for j in range(s)] for l in range(s)])
    errs = {"fix": [], "fma": []}
    for i in rng.choice(n, 250, replace=False):
        row = [U[c][i] for c in range(s + 1)] + [Po[l][i] for l in range(s)] + [Qo[l][i] for l in range(s)]
        E = max(bexp(v) for v in row)
        for j in range(s):
            for vs in ([U[j][i]] + [Po[l][i] for l in range(s)], [U[j + 1][i]] + [Qo[l][i] for l in range(s)]):
                cs = [1.0] + [float(beta[l, j]) for l in range(s)]
                ok, got, _, _ = fdot(dlib, vs, cs, E=E)
                assert ok
                exact = sum(Fraction(v) * Fraction(c) for v, c in zip(vs, cs))
                unit = sum(abs(Fraction(v) * Fraction(c)) for v, c in zip(vs, cs)) * Fraction(2) ** -53
                errs["fix"].append(float(abs(Fraction(got) - exact) / unit))
                errs["fma"].append(float(abs(Fraction(fma_chain(vs, cs)) - exact) / unit))
    fix, fma = np.array(errs["fix"]), np.array(errs["fma"])
    assert fix.mean() < fma.mean()
    assert fix.max() < max(fma.max(), 1.5), (fix.max(), fma.max())


def test_pack_rounds_to_nearest_even(dlib):
    """fix_pack (the one rounding of every fixed-point sum and dot product)
    against exact rounding: random magnitudes, exact ties at every position,
    carries into a new leading bit, and the normal-range limits."""
    dlib.fix_pack_value.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    rng = random.Random(17)
    cases = []
    for _ in range(3000):
        cases.append(rng.choice([-1, 1]) * rng.randrange(1, 2 ** rng.randint(1, 63)))
    for p in range(53, 63):  # ties: a 1 right below the 53 kept bits, nothing below it
        for lsb in (0, 1):
            m = ((1 << 52) | (rng.getrandbits(51) << 1) | lsb) << (p - 52)
            cases += [m | (1 << (p - 53)), -(m | (1 << (p - 53)))]
    cases += [2 ** 63 - 1, -(2 ** 63 - 1), 2 ** 53 - 1, 2 ** 54 - 1, 1, -1]
    for acc in cases:
        for e0 in (1075, 1000, 2000, 60):
            out = ctypes.c_uint64()
            ok = dlib.fix_pack_value(acc, e0, ctypes.byref(out))
            exact = Fraction(acc) * Fraction(2) ** (e0 - 1075)
            try:
                want = float(exact)  # rounds to nearest, ties to even
            except OverflowError:
                want = float("inf")
            normal = want != 0 and abs(want) != float("inf") and abs(want) >= 2.0 ** -1022
            if ok:
                assert val(out.value) == want, (acc, e0)
            else:
                assert not normal, (acc, e0, want)
    out = ctypes.c_uint64()
    assert dlib.fix_pack_value(0, 1075, ctypes.byref(out)) == 1 and out.value == 0
