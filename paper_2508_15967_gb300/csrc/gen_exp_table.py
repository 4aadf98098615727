"""Write gf_exp_table.inc: the constants of the library's table-driven exp.

Method: P. T. P. Tang, "Table-driven implementation of the exponential
function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157, with
a 2048-entry table.  Natural base (the generated-medium exp), with Cody-Waite
two-constant argument reduction (W. J. Cody and W. Waite, Software Manual for
the Elementary Functions, 1980):
    a = (2048 m + j) ln2/2048 + r,  exp(a) = 2^m * 2^(j/2048) * exp(r),  |r| <= ln2/4096;
base 2 (the blob evaluator's exponential, whose reduction is exact):
    a = (2048 m + j)/2048 + r,  2^a = 2^m * 2^(j/2048) * 2^r,
    2^r - 1 = c1 r + c2 r^2 + c3 r^3 (+ O(r^4)),  c_n = ln2^n / n!.
Every value is computed here with 60-digit decimal arithmetic and rounded once
to the nearest double.  Run: python gen_exp_table.py > gf_exp_table.inc
"""
from decimal import Decimal, getcontext
import math

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
    print(f"constexpr double kExp2C1 = {float.hex(to_double(L2))};   // ln2")
    print(f"constexpr double kExp2C2 = {float.hex(to_double(L2 ** 2 / 2))};   // ln2^2 / 2")
    print(f"constexpr double kExp2C3 = {float.hex(to_double(L2 ** 3 / 6))};   // ln2^3 / 6")
    print(f"// 2^(j/{N}), j = 0..{N - 1}, correctly rounded (initialiser of a device array)")
    print("#define GF_EXP2_TAB_VALUES \\")
    for j in range(N):
        v = to_double((Decimal(j) / N * ln2()).exp())
        print(f"    {float.hex(v)}{',' if j < N - 1 else ''} \\")
    print("")


if __name__ == "__main__":
    main()
