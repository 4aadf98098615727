"""The constant tables compiled into the CUDA library, checked on the CPU
against their mathematical definitions: the 2^(j/2048) table of the FP64 blob
exponential (correctly rounded doubles), its float-pair copy for the
double-float mode (hi = RN_float(v), lo = RN_float(v - hi)), the polynomial
and reduction constants (floats of the FP64 exponential's reduced argument), and that the committed include files are exactly
what their generator scripts print."""
from __future__ import annotations

import contextlib
import importlib.util
import io
import os
import re
import struct
from decimal import Decimal, getcontext

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2508_15967_gb300", "csrc")
HEX = r"-?0x[0-9a-fA-F]+(?:\.[0-9a-fA-F]*)?p[+-]?\d+"


def _read(name: str) -> str:
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def _generated(script: str) -> str:
    spec = importlib.util.spec_from_file_location(script[:-3], os.path.join(CSRC, script))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        mod.main()
    return buf.getvalue()


def _const(text: str, name: str) -> float:
    m = re.search(rf"constexpr (?:double|float|int) {name} = ({HEX}|\d+)f?;", text)
    assert m, name
    v = m.group(1)
    return float.fromhex(v) if v.startswith(("0x", "-0x")) else float(v)


def _f32(x) -> float:
    return struct.unpack("<f", struct.pack("<f", float(x)))[0]


@pytest.mark.parametrize("script, inc", [("gen_exp_table.py", "gf_exp_table.inc"),
                                         ("gen_dfexp_table.py", "gf_dfexp_table.inc")])
def test_include_files_are_what_the_generators_print(script, inc):
    assert _generated(script) == _read(inc)


def test_fp64_exponential_table_and_constants():
    getcontext().prec = 60
    text = _read("gf_exp_table.inc")
    values = [float.fromhex(v) for v in re.findall(HEX, text.split("GF_EXP2_TAB_VALUES")[1])]
    assert len(values) == 2048
    ln2 = Decimal(2).ln()
    for j, v in enumerate(values):
        exact = (Decimal(j) / 2048 * ln2).exp()
        assert v == float(exact), j                  # correctly rounded 2^(j/2048)
    # t = r ln2 is formed as a float pair: ln2 = hi + lo to within 2^-48 ln2;
    # the Taylor coefficients of e^t - 1 beyond t^2/2 are floats
    l2h, l2l = _const(text, "kLn2FHi"), _const(text, "kLn2FLo")
    assert l2h == _f32(ln2) and l2l == _f32(ln2 - Decimal(l2h))
    assert abs(Decimal(l2h) + Decimal(l2l) - ln2) <= Decimal(2) ** -48 * ln2
    assert _const(text, "kInv6F") == _f32(Decimal(1) / 6)
    assert _const(text, "kInv24F") == _f32(Decimal(1) / 24)
    # natural-base reduction of the generated-medium exponential: the high part
    # of ln2/2048 has few enough bits that k * hi is exact for |k| < 2^22, and
    # hi + lo is ln2/2048 to within the rounding of lo
    hi, lo = _const(text, "kLn2ByNHi"), _const(text, "kLn2ByNLo")
    num, den = hi.as_integer_ratio()                 # den a power of two, num odd
    assert num.bit_length() <= 31
    assert abs(Decimal(hi) + Decimal(lo) - ln2 / 2048) <= Decimal(2) ** -96
    assert _const(text, "kInvLn2xN") == float(2048 / ln2)


def test_double_float_exponential_table_and_constants():
    getcontext().prec = 60
    text = _read("gf_dfexp_table.inc")
    assert _const(text, "kDfExpN") == 2048
    pairs = [float.fromhex(v) for v in re.findall(HEX, text.split("GF_DFEXP2_TAB_VALUES")[1])]
    assert len(pairs) == 2 * 2048
    ln2 = Decimal(2).ln()
    for j in range(2048):
        exact = (Decimal(j) / 2048 * ln2).exp()
        hi, lo = pairs[2 * j], pairs[2 * j + 1]
        assert hi == _f32(exact) and lo == _f32(exact - Decimal(hi)), j
        assert abs(Decimal(hi) + Decimal(lo) - exact) <= Decimal(2) ** -48 * exact
    c1h, c1l = _const(text, "kDfC1Hi"), _const(text, "kDfC1Lo")
    assert c1h == _f32(ln2) and c1l == _f32(ln2 - Decimal(c1h))
    assert _const(text, "kDfC2") == _f32(ln2 ** 2 / 2)
    assert _const(text, "kDfC3") == _f32(ln2 ** 3 / 6)
