"""Write gf_dfexp_table.inc: constants of the double-float (FP32 pair) exp.

Tang's table-driven method (ACM TOMS 15, 1989) in base 2, as for the FP64
evaluator's exponential (gen_exp_table.py): 2^a = 2^m * 2^(j/2048) * 2^r with
an exact reduction r = a - k/2048, and 2^r - 1 = c1 r + c2 r^2 + c3 r^3.
c1 = ln2 and the table values 2^(j/2048) are stored as (hi, lo) float pairs,
hi = RN_float(v), lo = RN_float(v - hi); c2 = ln2^2/2 and c3 = ln2^3/6 as
single floats (their terms are below 1.5e-8 and 1e-12 for |r| <= 2.5e-4).
Every value is computed with 60-digit decimal arithmetic.
Run: python gen_dfexp_table.py > gf_dfexp_table.inc
"""
from decimal import Decimal, getcontext
import struct

getcontext().prec = 60

N = 2048


def f32(x) -> float:
    """Round a Decimal / float to the nearest IEEE single."""
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


def split_float(d: Decimal):
    hi = f32(d)
    lo = f32(d - Decimal(hi))
    return hi, lo


def fhex(x: float) -> str:
    return float.hex(x) + "f"


def main():
    ln2 = Decimal(2).ln()
    c1h, c1l = split_float(ln2)
    print("// Generated by gen_dfexp_table.py -- constants of the double-float base-2 exp.")
    print(f"constexpr int kDfExpN = {N};")
    print(f"constexpr float kDfC1Hi = {fhex(c1h)};   // ln2 = hi + lo")
    print(f"constexpr float kDfC1Lo = {fhex(c1l)};")
    print(f"constexpr float kDfC2 = {fhex(f32(ln2 ** 2 / 2))};   // ln2^2 / 2")
    print(f"constexpr float kDfC3 = {fhex(f32(ln2 ** 3 / 6))};   // ln2^3 / 6")
    print(f"// (hi, lo) of 2^(j/{N}), j = 0..{N - 1} (initialiser of a device array)")
    print("#define GF_DFEXP2_TAB_VALUES \\")
    for j in range(N):
        h, l = split_float((Decimal(j) / N * ln2).exp())
        print(f"    {fhex(h)}, {fhex(l)}{',' if j < N - 1 else ''} \\")
    print("")


if __name__ == "__main__":
    main()
