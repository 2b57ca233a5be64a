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
