"""Write gf_exp_table.inc: the constants of the library's table-driven exp.

Method: P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157, with
a 256-entry table and Cody-Waite two-constant argument reduction (W. J. Cody
and W. Waite, Software Manual for the Elementary Functions, 1980):
    a = (256 m + j) ln2/256 + r,  exp(a) = 2^m * 2^(j/256) * exp(r),  |r| <= ln2/512.
Every value is computed here with 60-digit decimal arithmetic and rounded once
to the nearest double.  Run: python gen_exp_table.py > gf_exp_table.inc
"""
from decimal import Decimal, getcontext
import struct

getcontext().prec = 60


def ln2() -> Decimal:
    return Decimal(2).ln()


def to_double(d: Decimal) -> float:
    return float(d)          # correctly rounded from the decimal string


def hexf(x: float) -> str:
    return float.hex(x)


def trunc_bits(x: float, bits: int) -> float:
    """x with its significand truncated to `bits` bits (so k * x is exact for small k)."""
    m, e = __import__("math").frexp(x)
    scale = 2 ** bits
    return __import__("math").ldexp(int(m * scale) / scale, e)


def main():
    L = ln2() / 256
    hi = trunc_bits(to_double(L), 35)            # |k| < 2^18 for |a| < 709: k*hi exact
    lo = to_double(L - Decimal(hi))
    inv = to_double(256 / ln2())
    print("// Generated by gen_exp_table.py -- constants of the table-driven exp")
    print("// (Tang 1989, 256-entry table; Cody-Waite split of ln2/256).")
    print(f"constexpr double kInvLn2xN = {hexf(inv)};   // 256 / ln 2")
    print(f"constexpr double kLn2ByNHi = {hexf(hi)};   // ln2/256, 35 significant bits")
    print(f"constexpr double kLn2ByNLo = {hexf(lo)};   // ln2/256 - kLn2ByNHi")
    print("constexpr double kExp2Tab[256] = {   // 2^(j/256), correctly rounded")
    for j in range(256):
        v = to_double((Decimal(j) / 256 * ln2()).exp())
        print(f"    {hexf(v)},")
    print("};")


if __name__ == "__main__":
    main()
