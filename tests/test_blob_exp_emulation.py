"""CPU check of the arithmetic design of the FP64 evaluator's blob Gaussian
G = 2^-(u0^2 + u1^2 + u2^2): a step-by-step emulation of its integer and
float steps (64-bit fixed-point squares, the reduction read off their bits,
the float-pair polynomial, the 117-bit table product rounded to nearest
even, and the FMA form of that product), with every float operation rounded
exactly as IEEE binary32 does, against exact rationals.  This pins the
documented error bound (< 1.05 ulp of the exact Gaussian of the given u) on
the CPU; the GPU test in test_gpu_exp.py checks the kernel itself."""
from __future__ import annotations

import math
import struct
from decimal import Decimal, getcontext
from fractions import Fraction as F

import numpy as np
import pytest

M64 = (1 << 64) - 1


def _dbits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _bitsd(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & M64))[0]


def _fbits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _bitsf(b: int) -> float:
    return struct.unpack("<f", struct.pack("<I", b & 0xFFFFFFFF))[0]


def _rn32(x: F) -> float:
    """x rounded to the nearest binary32 value, ties to even (subnormals included)."""
    if x == 0:
        return 0.0
    s = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if F(2) ** e > x:
        e -= 1
    q = F(2) ** (max(e, -126) - 23)
    t = x / q
    m = t.numerator // t.denominator
    r = t - m
    if r > F(1, 2) or (r == F(1, 2) and m % 2 == 1):
        m += 1
    return s * float(m * q)


def _add(a, b): return _rn32(F(a) + F(b))
def _sub(a, b): return _rn32(F(a) - F(b))
def _mul(a, b): return _rn32(F(a) * F(b))
def _fma(a, b, c): return _rn32(F(a) * F(b) + F(c))


LN2_HI = float.fromhex("0x1.62e4300000000p-1")
LN2_LO = float.fromhex("-0x1.05c6100000000p-29")
INV6 = float.fromhex("0x1.5555560000000p-3")
INV24 = float.fromhex("0x1.5555560000000p-5")
CULL_Q56 = 0x3A80000000000000          # 58.5 in units of 2^-56


@pytest.fixture(scope="module")
def table():
    getcontext().prec = 40
    ln2 = Decimal(2).ln()
    return [float(F((Decimal(j) / 2048 * ln2).exp())) for j in range(2048)]


def _sq_fix56(u: float):
    b = _dbits(u)
    e = (b >> 52) & 0x7FF
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    sh = e - 1015
    U = (m << min(sh, 10)) & M64 if sh >= 0 else m >> min(-sh, 63)
    H, L = U >> 32, U & 0xFFFFFFFF
    HL = H * L + (((L * L) >> 32) >> 1) + (1 << 30)
    return H * H + (HL >> 31), e


def _trunc63(x: float) -> float:
    b = _fbits(x)
    nclr = 87 - ((b >> 23) & 0xFF)
    keep = 0xFFFFFFFF if nclr <= 0 else (0 if nclr >= 24 else ~((1 << nclr) - 1) & 0xFFFFFFFF)
    return _bitsf(b & keep)


def _gauss(u, T):
    """(integer form, FMA form) of the Gaussian, or None for a negligible term."""
    q, emax = 0, 0
    for c in u:
        s, e = _sq_fix56(c)
        q += s
        emax = max(emax, e)
    assert q < 1 << 64
    if emax >= 1026 or q >= CULL_Q56:
        return None
    K = (q + (1 << 44)) >> 45
    ra = (K << 45) - q                                   # r in units of 2^-56
    vh, vl = ra >> 22, ra & ((1 << 22) - 1)
    assert -(1 << 22) <= vh <= 1 << 22
    rh = _mul(_sub(_bitsf(0x4B400000 + vh), 12582912.0), 2.0 ** -34)
    rl = _mul(_sub(_bitsf(0x4B000000 | vl), 8388608.0), 2.0 ** -56)
    k = -K
    th = _mul(rh, LN2_HI)
    tl = _fma(rl, LN2_HI, _fma(rh, LN2_LO, _fma(rh, LN2_HI, -th)))
    p2 = _mul(th, th)
    e2 = _fma(th, th, -p2)
    h = _mul(0.5, p2)
    ph = _add(th, h)
    l0 = _sub(h, _sub(ph, th))
    c34 = _mul(p2, _fma(th, INV6, _mul(p2, INV24)))
    pl = _add(l0, _add(tl, _fma(0.5, e2, _fma(th, tl, c34))))
    P = int(F(_trunc63(ph)) * 2 ** 63) + int(F(_trunc63(pl)) * 2 ** 63)
    Tj = T[k & 2047]
    # integer form: S U 2^-115 rounded to 53 bits, ties to even
    S = (_dbits(Tj) & ((1 << 52) - 1)) | (1 << 52)
    prod = S * ((1 << 63) + P)
    hi, lo = prod >> 64, prod & M64
    lz = (64 - hi.bit_length()) - 11
    mant = hi if lz == 0 else ((hi << lz) | (lo >> (64 - lz))) & M64
    rb = (lo << lz) & M64
    up = (rb >> 63) & (1 if ((rb << 1) & M64) else (mant & 1))
    g_int = _bitsd(((1023 - lz + (k >> 11)) << 52) + mant + up)
    # FMA form: RN(T + T P) in FP64, then the power-of-two scaling
    v = float(F(Tj) * F(P, 2 ** 63) + F(Tj))
    g_fp = v * 2.0 ** (k >> 11)
    return g_int, g_fp


def _points(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        mode = i % 4
        if mode == 0:
            u = rng.uniform(-7.6, 7.6, 3)
        elif mode == 1:
            u = rng.normal(0, 1, 3) * 10.0 ** rng.uniform(-12, 0.5, 3)
        else:
            d = rng.normal(0, 1, 3)
            d /= np.linalg.norm(d)
            a = rng.uniform(0, 58.5) if mode == 2 else rng.integers(0, 58 * 2048) / 2048 + rng.normal(0, 1e-9)
            u = d * math.sqrt(max(a, 0.0))
        out.append(tuple(float(c) for c in u))
    return out + [(0.0, 0.0, 0.0), (-0.0, 5e-324, 0.0), (2.0 ** -30, 2.0 ** -40, 0.0), (7.6, 0.0, 0.0),
                  (math.sqrt(58.5) * (1 - 1e-15), 0.0, 0.0), (8.0, 0.0, 0.0), (1.0, 1.0, 1.0)]


def test_emulated_blob_gaussian_error_bound(table):
    getcontext().prec = 50
    ln2 = Decimal(2).ln()
    worst, errs = 0.0, []
    for u in _points(1500, 5):
        r = _gauss(u, table)
        q = sum(F(c) ** 2 for c in u)
        if r is None:
            assert q >= F(585, 10) - F(1, 10 ** 9), u
            continue
        assert q < F(585, 10) + F(1, 10 ** 9), u
        g_int, g_fp = r
        assert _dbits(g_int) == _dbits(g_fp), u            # the two forms round alike
        ex = (-(Decimal(q.numerator) / Decimal(q.denominator)) * ln2).exp()
        err = float(abs(Decimal(g_int) - ex) / Decimal(math.ulp(float(ex))))
        errs.append(err)
        worst = max(worst, err)
    assert worst < 1.05, worst
    assert np.mean(errs) < 0.4


def test_fixed_point_squares_are_within_one_unit():
    """Each square is within 0.5 + 2^-10 units of 2^-56 of the exact u^2
    (|u| < 8: the rounding of the middle term, and below |u| = 2^-8 the
    truncation of |u| 2^60), so the sum of three is within about 1.5 units."""
    rng = np.random.default_rng(6)
    for u in np.concatenate([rng.uniform(-7.99, 7.99, 3000), 10.0 ** rng.uniform(-20, 0.9, 3000)]):
        s, e = _sq_fix56(float(u))
        assert e <= 1025
        assert abs(F(s) - F(float(u)) ** 2 * 2 ** 56) <= F(1, 2) + F(1, 2 ** 10)
