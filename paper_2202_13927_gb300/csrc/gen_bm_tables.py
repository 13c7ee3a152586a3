"""Write vct_bm_tables.cuh: the tables of the FP64 Box-Muller transform of
vct_rng.cuh (a build-time step of the CUDA library; its output is committed,
so building the library needs neither this script nor mpmath).

Logarithm (table-driven, after P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4),
1990, with the argument reduced by a short reciprocal as in J.-M. Muller,
"Elementary Functions: Algorithms and Implementation", ch. 6): the uniform
u = 2^k m with m in [0.75, 1.5) falls in one of 256 intervals j (the 8 bits
after the leading one of its significand); c_j is the reciprocal of the
interval's centre rounded to 20 significant bits (1 exactly for the interval
just below 1), so that r = m c_j - 1 is exact in one fma (m has at most 33
significant bits) and |r| < 2^-9.  Then -ln(u) / 8 = (-k) ln2 / 8 +
ln(c_j) / 8 - ln(1 + r) / 8, the first two from tables in two parts (the
rounded value and its residual).

Angle: 2 pi u1 = 2 pi a_j + 2 pi t with a_j = (j + 1/2) / 1024 turns (j the top
10 bits of the word) and |t| < 1/2048 turn; the table holds 4 sqrt(2) sin(2 pi a_j)
and 4 sqrt(2) cos(2 pi a_j), the factor that turns (-ln u / 8) rsqrt(-ln u / 4)
into the radius sqrt(-2 ln u).

Every value is computed with 60 significant digits and rounded to the nearest
double.  Usage: python gen_bm_tables.py  (rewrites the header next to it).
"""
from __future__ import annotations

import os

import mpmath as mp

mp.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "vct_bm_tables.cuh")


def dbl(x) -> float:
    return float(mp.mpf(x))   # mpmath rounds to the nearest double


def split(x):
    hi = dbl(x)
    lo = dbl(mp.mpf(x) - mp.mpf(hi))
    return hi, lo


def short(x, bits=20):
    """x rounded to `bits` significant bits."""
    x = mp.mpf(x)
    e = int(mp.floor(mp.log(x, 2)))
    return mp.mpf(int(mp.nint(x * mp.mpf(2) ** (bits - 1 - e)))) * mp.mpf(2) ** (e - bits + 1)


def log_tables():
    c, t = [], []
    for j in range(256):
        if j < 128:   # m in [1 + j/256, 1 + (j+1)/256)
            centre = 1 + (mp.mpf(j) + mp.mpf("0.5")) / 256
        else:         # m / 2 in [(1 + j/256)/2, (1 + (j+1)/256)/2)
            centre = (1 + (mp.mpf(j) + mp.mpf("0.5")) / 256) / 2
        cj = mp.mpf(1) if j == 255 else short(1 / centre)
        c.append(dbl(cj))
        t.append(split(mp.log(cj) / 8))
    k = [split(n * mp.log(2) / 8) for n in range(34)]
    return c, t, k


N_ANGLE = 1024


def angle_table():
    s = 4 * mp.sqrt(2)
    out = []
    for j in range(N_ANGLE):
        a = 2 * mp.pi * (mp.mpf(j) + mp.mpf("0.5")) / N_ANGLE
        out.append((dbl(s * mp.sin(a)), dbl(s * mp.cos(a))))
    return out


def poly():
    # -ln(1 + r) / 8 = r (-1/8 + r (1/16 + r (-1/24 + r (1/32 + r (-1/40 + r / 48)))))
    log_c = [dbl(mp.mpf(v)) for v in ("-0.125", "0.0625", -mp.mpf(1) / 24, "0.03125", "-0.025",
                                       mp.mpf(1) / 48)]
    # angle 2 pi q 2^-33 for the odd integer q, |q| < 2^22 (|angle| < 2 pi / 2048 rad):
    # sin = q (s1 + q^2 (s3 + q^2 s5)), 1 - cos = q^2 (c2 + q^2 c4); the first terms
    # left out are below 2e-19 of the value
    b = 2 * mp.pi * mp.mpf(2) ** -33
    sin_c = [dbl(b), dbl(-b ** 3 / 6), dbl(b ** 5 / 120)]
    cos_c = [dbl(b ** 2 / 2), dbl(-b ** 4 / 24)]
    return log_c, sin_c, cos_c


def main():
    c, t, k = log_tables()
    sc = angle_table()
    log_c, sin_c, cos_c = poly()
    h = lambda v: float(v).hex()
    lines = ["// vct_bm_tables.cuh -- written by gen_bm_tables.py; do not edit.",
             "// Tables and coefficients of the FP64 Box-Muller transform in vct_rng.cuh.",
             "#pragma once", "", "namespace vct {", "namespace bm64 {", ""]
    lines.append("// reciprocals c_j (20 significant bits) of the 256 reduction intervals")
    lines.append("__device__ const double kLogC[256] = {")
    lines += ["  " + ", ".join(h(x) for x in c[i:i + 4]) + "," for i in range(0, 256, 4)]
    lines.append("};")
    lines.append("// ln(c_j) / 8 as (rounded value, residual)")
    lines.append("__device__ const double2 kLogT[256] = {")
    lines += ["  {" + h(a) + ", " + h(b) + "}," for a, b in t]
    lines.append("};")
    lines.append("// n ln2 / 8 for n = -k = 0 .. 33, as (rounded value, residual)")
    lines.append("__device__ const double2 kLogK[34] = {")
    lines += ["  {" + h(a) + ", " + h(b) + "}," for a, b in k]
    lines.append("};")
    lines.append(f"// (4 sqrt(2) sin, 4 sqrt(2) cos) of 2 pi (j + 1/2) / {N_ANGLE}")
    lines.append(f"__device__ const double2 kAngle[{N_ANGLE}] = {{")
    lines += ["  {" + h(a) + ", " + h(b) + "}," for a, b in sc]
    lines.append("};")
    lines.append("// polynomial coefficients (lowest degree first)")
    names = (("kLogP", log_c), ("kSinP", sin_c), ("kCosP", cos_c))
    for name, vals in names:
        for i, v in enumerate(vals):
            lines.append(f"constexpr double {name}{i} = {h(v)};")
    lines += ["", "}  // namespace bm64", "}  // namespace vct", ""]
    with open(OUT, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
