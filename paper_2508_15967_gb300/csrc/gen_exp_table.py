"""Write gf_exp_table.inc: the constants of the library's table-driven exp.

Method: P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157, with
a 2048-entry table.  Natural base (the generated-medium exp), with Cody-Waite
two-constant argument reduction (W. J. Cody and W. Waite, Software Manual for
the Elementary Functions, 1980):
    a = (2048 m + j) ln2/2048 + r,  exp(a) = 2^m * 2^(j/2048) * exp(r),  |r| <= ln2/4096;
base 2 (the blob evaluator's exponential, whose reduction is exact):
    a = (2048 m + j)/2048 + r,  2^a = 2^m * 2^(j/2048) * 2^r,
    2^r - 1 = e^t - 1 = t + t^2/2 + t^3/6 + t^4/24 (+ O(t^5)),  t = r ln2,
with t formed as a float pair from ln2 = hi + lo (two floats) and the
coefficients 1/6, 1/24 as floats (their terms are below 1e-12 and 5e-17).
Every value is computed here with 60-digit decimal arithmetic and rounded once
to the nearest double (or float).  Run: python gen_exp_table.py > gf_exp_table.inc
"""
from decimal import Decimal, getcontext
import math
import struct

getcontext().prec = 60

N = 2048
HI_BITS = 31      # |k| < 2^22 for |a| < 709, so k * hi is exact


def ln2() -> Decimal:
    return Decimal(2).ln()


def to_double(d: Decimal) -> float:
    return float(d)          # correctly rounded from the decimal string


def trunc_bits(x: float, bits: int) -> float:
    """x with its significand truncated to `bits` bits (so k * x is exact for small k)."""
    m, e = math.frexp(x)
    scale = 2 ** bits
    return math.ldexp(int(m * scale) / scale, e)


def f32(x) -> float:
    """Round a Decimal / float to the nearest IEEE single."""
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def main():
    L = ln2() / N
    hi = trunc_bits(to_double(L), HI_BITS)
    lo = to_double(L - Decimal(hi))
    inv = to_double(N / ln2())
    print("// Generated by gen_exp_table.py -- constants of the table-driven exp")
    print(f"// (Tang 1989, {N}-entry table; Cody-Waite split of ln2/{N}).")
    print(f"constexpr double kInvLn2xN = {float.hex(inv)};   // {N} / ln 2")
    print(f"constexpr double kLn2ByNHi = {float.hex(hi)};   // ln2/{N}, {HI_BITS} significant bits")
    print(f"constexpr double kLn2ByNLo = {float.hex(lo)};   // ln2/{N} - kLn2ByNHi")
    L2 = ln2()
    l2h = f32(L2)
    l2l = f32(L2 - Decimal(l2h))
    print(f"constexpr float kLn2FHi = {float.hex(l2h)}f;   // ln2 = hi + lo, floats")
    print(f"constexpr float kLn2FLo = {float.hex(l2l)}f;")
    print(f"constexpr float kInv6F = {float.hex(f32(Decimal(1) / 6))}f;   // 1/6")
    print(f"constexpr float kInv24F = {float.hex(f32(Decimal(1) / 24))}f;   // 1/24")
    print(f"// 2^(j/{N}), j = 0..{N - 1}, correctly rounded (initialiser of a device array)")
    print("#define GF_EXP2_TAB_VALUES \\")
    for j in range(N):
        v = to_double((Decimal(j) / N * ln2()).exp())
        print(f"    {float.hex(v)}{',' if j < N - 1 else ''} \\")
    print("")


if __name__ == "__main__":
    main()
