"""Write gf_dfexp_table.inc: constants of the double-float (FP32 pair) exp.

Same method as gen_exp_table.py (Tang's table-driven exp, 64-entry table) in
double-float arithmetic: ln2/64 is split into four floats L1..L4 -- L1, L2, L3
with 12 significant bits each, so that k * Li is exact for |k| < 2^12, and L4
holding the next 24 bits; 2^(j/64) and 1/6 are stored as (hi, lo) float pairs.
Every value is computed with 60-digit decimal arithmetic.
Run: python gen_dfexp_table.py > gf_dfexp_table.inc
"""
from decimal import Decimal, getcontext
import math
import struct

getcontext().prec = 60


def f32(x) -> float:
    """Round a Decimal / float to the nearest IEEE single."""
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def split_float(d: Decimal):
    hi = f32(d)
    lo = f32(d - Decimal(hi))
    return hi, lo


def trunc_bits(d: Decimal, bits: int) -> float:
    """d truncated to `bits` significant bits (exactly representable as a float)."""
    m, e = math.frexp(float(d))
    scale = 2 ** bits
    v = math.ldexp(int(Decimal(m) * scale) / scale, e)
    # correct the float(d) rounding: keep truncation of the exact decimal
    while Decimal(v) > d and d > 0:
        v = math.ldexp(int(Decimal(m) * scale - 1) / scale, e)
    return v


def fhex(x: float) -> str:
    return float.hex(x) + "f"


def main():
    L = Decimal(2).ln() / 64
    L1 = trunc_bits(L, 12)
    R = L - Decimal(L1)
    L2 = trunc_bits(R, 12)
    R = R - Decimal(L2)
    L3 = trunc_bits(R, 12)
    R = R - Decimal(L3)
    L4 = f32(R)
    inv = f32(64 / Decimal(2).ln())
    sh, sl = split_float(Decimal(1) / 6)
    print("// Generated by gen_dfexp_table.py -- constants of the double-float exp.")
    print(f"constexpr float kDfInvL = {fhex(inv)};   // 64 / ln 2")
    print(f"constexpr float kDfL1 = {fhex(L1)};   // ln2/64 = L1 + L2 + L3 + L4")
    print(f"constexpr float kDfL2 = {fhex(L2)};")
    print(f"constexpr float kDfL3 = {fhex(L3)};")
    print(f"constexpr float kDfL4 = {fhex(L4)};")
    print(f"constexpr float kDfSixthHi = {fhex(sh)};   // 1/6 = hi + lo")
    print(f"constexpr float kDfSixthLo = {fhex(sl)};")
    print("constexpr float kDfExp2Tab[128] = {   // (hi, lo) of 2^(j/64), j = 0..63")
    for j in range(64):
        h, l = split_float((Decimal(j) / 64 * Decimal(2).ln()).exp())
        print(f"    {fhex(h)}, {fhex(l)},")
    print("};")


if __name__ == "__main__":
    main()
