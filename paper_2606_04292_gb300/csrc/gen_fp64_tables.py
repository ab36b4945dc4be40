"""Writes fp64_tables.h: the constants of the table-driven FP64 elementary
functions in fp64math.cuh (run from this directory: python gen_fp64_tables.py).

Every value is computed in 60-digit decimal arithmetic from its definition
and rounded once to the nearest double (hi), with the remainder rounded to a
second double (lo) where a pair is kept:
  2^(j/256) and 2^(j/256) - 1 for j = -128 .. 127    (exp, expm1)
  log(1 + k/256) (k < 128), log((1 + k/256)/2) (k >= 128) and 1/(1 + k/256)
                                                    (log, log1p)
  ln 2 / 256 and ln 2 split so that a multiple by a small integer is exact.
"""
import math
from decimal import Decimal, getcontext

getcontext().prec = 60
LN2 = Decimal(2).ln()


def hx(x):
    return float(x).hex()


def pair(d):
    hi = float(d)
    lo = float(d - Decimal(hi))
    return hi, lo


def split_bits(d, bits):
    """d rounded to a double whose significand has at most `bits` bits, and
    the rounded remainder."""
    f = float(d)
    e = math.frexp(f)[1]
    hi = math.ldexp(math.floor(math.ldexp(f, bits - e)), e - bits)
    lo = float(d - Decimal(hi))
    return hi, lo


lines = ["// Generated by gen_fp64_tables.py; do not edit.  Constants of the",
         "// table-driven FP64 exp / expm1 / log / log1p of fp64math.cuh.",
         "#pragma once", "", "namespace rich {", "namespace fx {", ""]
hi, lo = split_bits(LN2 / 256, 34)  # N * hi exact for |N| < 2^19
lines += [f"constexpr double LN2_256_HI = {hx(hi)};", f"constexpr double LN2_256_LO = {hx(lo)};",
          f"constexpr double INV_LN2_256 = {hx(Decimal(256) / LN2)};"]
hi, lo = split_bits(LN2, 42)        # e * hi exact for |e| < 2^11
lines += [f"constexpr double LN2_HI = {hx(hi)};", f"constexpr double LN2_LO = {hx(lo)};", ""]
lines.append("// 2^(j/256) (hi, lo) and 2^(j/256) - 1 (hi, lo), j = -128 .. 127 at index j + 128")
lines.append("__device__ const double kExp2[256][4] = {")
for j in range(-128, 128):
    t = (LN2 * j / 256).exp()
    a, b = pair(t)
    c, d = pair(t - 1)
    lines.append(f"    {{{hx(a)}, {hx(b)}, {hx(c)}, {hx(d)}}},")
lines.append("};")
lines.append("// log(F) (hi, lo) with F = 1 + k/256 for k < 128 and F = (1 + k/256)/2 for")
lines.append("// k >= 128 (the argument is then taken as 2^(e+1) F), and 1 / (1 + k/256)")
lines.append("__device__ const double kLogF[256][3] = {")
for k in range(256):
    F = 1 + Decimal(k) / 256
    a, b = pair((F if k < 128 else F / 2).ln())
    lines.append(f"    {{{hx(a)}, {hx(b)}, {hx(1 / F)}}},")
lines.append("};")
lines += ["", "}  // namespace fx", "}  // namespace rich", ""]
with open("fp64_tables.h", "w") as f:
    f.write("\n".join(lines))
