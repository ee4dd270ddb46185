"""Accuracy of the library's float-float arithmetic (csrc/ff.cuh), built for
the host with g++ and checked against mpmath at 200 bits.

The control-rate chain of the render keeps pitch, envelopes and phase sums in
float-float because a relative pitch error that persists integrates into
phase drift (at 4 s and 10 kHz a relative error of 1e-8 is already 4e-4
cycles). These tests bound each building block well below that: relative
errors of a few 1e-14 for exp2, expm1 and the products; absolute errors of a
few 1e-14 for log2 and sin(2 pi p); and exact modular sums for the
fixed-point phase format."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.prec = 200

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2104_12922_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("ffh") / "libffh.so")
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "ff_host_harness.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    f, pf = ctypes.c_float, ctypes.POINTER(ctypes.c_float)
    for name in ("h_exp2", "h_log2", "h_expm1", "h_sin2pi", "h_rcp", "h_frac"):
        getattr(L, name).argtypes = [f, f, pf]
    for name in ("h_div", "h_mul", "h_add"):
        getattr(L, name).argtypes = [f, f, f, f, pf]
    L.h_pow01.argtypes = [f, f, f, f, pf]
    L.h_to_fix64.argtypes = [f, f]
    L.h_to_fix64.restype = ctypes.c_ulonglong
    L.h_fix64_to_ff.argtypes = [ctypes.c_ulonglong, pf]
    return L


def split(x):
    """x (mpmath or float) -> float pair (hi, lo) and the pair's exact value."""
    x = mp.mpf(x)
    hi = np.float32(float(x))
    lo = np.float32(float(x - mp.mpf(float(hi))))
    return float(hi), float(lo), mp.mpf(float(hi)) + mp.mpf(float(lo))


def call(fn, *args):
    out = (ctypes.c_float * 2)()
    fn(*args, out)
    return mp.mpf(float(out[0])) + mp.mpf(float(out[1]))


def rel(a, b):
    return float(abs(a - b) / abs(b)) if b != 0 else float(abs(a))


def test_exp2_relative_error(lib):
    rng = np.random.default_rng(1)
    ys = list(rng.uniform(-100, 10, 400)) + list(rng.uniform(-1, 1, 400)) + \
        [0.0, 1 / 512, -1 / 512, 0.5, 127 / 256, 129 / 256, 1.5, -7.0]
    worst = 0.0
    for y in ys:
        hi, lo, yx = split(y)
        worst = max(worst, rel(call(lib.h_exp2, hi, lo), mp.power(2, yx)))
    assert worst < 4e-14, worst
    # below 2^-100 the low word is subnormal, and below 2^-126 the result is
    # flushed to 0: the error there is absolute, under 2^-126
    for y in rng.uniform(-130, -100, 50):
        hi, lo, yx = split(y)
        assert float(abs(call(lib.h_exp2, hi, lo) - mp.power(2, yx))) < 2.0 ** -126


def test_expm1_relative_error_including_tiny_arguments(lib):
    rng = np.random.default_rng(2)
    xs = list(rng.uniform(-6, 6, 300)) + list(rng.uniform(-0.4, 0.4, 300)) + \
        list(10.0 ** rng.uniform(-12, -2, 200) * rng.choice([-1, 1], 200)) + \
        [1.29e-3, -1.29e-3, 1.31e-3, -1.31e-3, 0.3466, -0.3466, 0.35, 1e-30]
    worst = 0.0
    for x in xs:
        hi, lo, xx = split(x)
        worst = max(worst, rel(call(lib.h_expm1, hi, lo), mp.expm1(xx)))
    assert worst < 4e-14, worst


def test_log2_absolute_error(lib):
    rng = np.random.default_rng(3)
    xs = list(10.0 ** rng.uniform(-35, 0, 400)) + list(rng.uniform(0.5, 1.0, 400)) + \
        [1.0, 0.5, 0.25, 1 - 1e-7, 1 - 1e-12, 1e-40, 3e-39, 0.75, 1 + 1 / 256]
    worst = 0.0
    for x in xs:
        hi, lo, xx = split(x)
        ref = mp.log(xx, 2)
        err = float(abs(call(lib.h_log2, hi, lo) - ref))
        worst = max(worst, err / max(1.0, float(abs(ref))))
    assert worst < 2e-14, worst


def test_pow01_relative_error(lib):
    rng = np.random.default_rng(4)
    worst = 0.0
    for _ in range(600):
        x = float(10.0 ** rng.uniform(-6, 0))
        a = float(rng.uniform(0.1, 6.0))
        xh, xl, xx = split(x)
        ah, al, ax = split(a)
        ref = mp.power(xx, ax)
        got = call(lib.h_pow01, xh, xl, ah, al)
        if ref > mp.mpf(2) ** -90:  # the error of log2 x is magnified by a |log2 x|
            worst = max(worst, rel(got, ref))
        else:  # the low word of the result is subnormal
            assert float(abs(got - ref)) < 2.0 ** -100
    assert worst < 1e-12, worst
    assert call(lib.h_pow01, 0.0, 0.0, 2.0, 0.0) == 0
    assert call(lib.h_pow01, 1.0, 0.0, 0.3, 0.0) == 1


def test_sin2pi_absolute_error(lib):
    rng = np.random.default_rng(5)
    ps = list(rng.uniform(0, 1, 600)) + [0.0, 0.25, 0.5, 0.75, 1 / 256, 0.125, 0.999999]
    worst = 0.0
    for p in ps:
        hi, lo, px = split(p)
        worst = max(worst, float(abs(call(lib.h_sin2pi, hi, lo) - mp.sin(2 * mp.pi * px))))
    assert worst < 2e-14, worst


def test_division_reciprocal_products_sums(lib):
    rng = np.random.default_rng(6)
    for _ in range(300):
        a, b = rng.uniform(-100, 100, 2)
        ah, al, ax = split(a)
        bh, bl, bx = split(b)
        assert rel(call(lib.h_div, ah, al, bh, bl), ax / bx) < 4e-14
        assert rel(call(lib.h_rcp, bh, bl), 1 / bx) < 4e-14
        assert rel(call(lib.h_mul, ah, al, bh, bl), ax * bx) < 4e-14
        s = ax + bx
        assert float(abs(call(lib.h_add, ah, al, bh, bl) - s)) <= 4e-14 * float(abs(ax) + abs(bx))


def test_fixed_point_phase_across_magnitudes_and_signs(lib):
    """Values from 2^-40 to 2^20 of either sign, with the low word of either
    sign: 2^32 hi below and above 2^31, negative remainders."""
    rng = np.random.default_rng(11)
    two64 = mp.mpf(2) ** 64
    for e in range(-40, 21, 3):
        for v in rng.uniform(-1.0, 1.0, 40) * 2.0 ** e:
            hi, lo, vx = split(float(v))
            for l, x in ((lo, vx), (-lo, mp.mpf(hi) - mp.mpf(lo))):
                u = lib.h_to_fix64(hi, l)
                frac = x - mp.floor(x)
                d = abs(mp.mpf(u) / two64 - frac)
                assert min(d, 1 - d) < 2.0 ** -50, (v, e, float(d))


def test_fixed_point_phase_roundtrip_and_exact_sums(lib):
    rng = np.random.default_rng(7)
    two64 = mp.mpf(2) ** 64
    acc, exact = 0, mp.mpf(0)
    for v in list(rng.uniform(-0.5, 60.0, 400)) + [0.0, 1.0, -1.0, 0.5, 2.0 ** -30, 49.99999]:
        hi, lo, vx = split(v)
        u = lib.h_to_fix64(hi, lo)
        frac = vx - mp.floor(vx)
        got = mp.mpf(u) / two64
        d = abs(got - frac)
        assert min(d, 1 - d) < 2.0 ** -50, (v, float(d))
        back = call(lib.h_fix64_to_ff, u)
        assert 0 <= back < 1 and abs(back - got) < 2.0 ** -47
        acc = (acc + u) % (1 << 64)
        exact += vx
    # the modular sum of the codes is the fractional part of the exact sum
    ef = exact - mp.floor(exact)
    d = abs(mp.mpf(acc) / two64 - ef)
    assert min(d, 1 - d) < 410 * 2.0 ** -50
