"""Write vct_bm_tables.cuh: the tables of the FP64 Box-Muller transform of
vct_rng.cuh (a build-time step of the CUDA library; its output is committed,
so building the library needs neither this script nor mpmath).

Logarithm (table-driven, after P. T. P. Tang, "Table-driven implementation of
the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16(4),
1990, with the argument reduced by a short reciprocal as in J.-M. Muller,
"Elementary Functions: Algorithms and Implementation", ch. 6): the uniform
u = 2^k m with m in [0.75, 1.5) falls in one of 4096 intervals j (the 12 bits
after the leading one of its significand); c_j is the reciprocal of the
interval's centre rounded to 20 significant bits (1 exactly for the interval
just below 1), so that r = m c_j - 1 is exact in one fma (m has at most 33
significant bits) and |r| < 1.01 2^-13, short enough for a degree-4 polynomial
of ln(1 + r) (the first term left out, r^5 / 5, is below 2^-54 of the result).  Then -ln(u) / 8 = (-k) ln2 / 8 +
ln(c_j) / 8 - ln(1 + r) / 8, the first two from tables in two parts (the
rounded value and its residual).

Angle: 2 pi u1 = 2 pi a_j + 2 pi t with a_j = (j + 1/2) / 4096 turns (j the top
12 bits of the word) and |t| < 1/8192 turn; the table holds 4 sqrt(2) sin(2 pi a_j)
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


N_LOG = 4096


def log_tables():
    c, t = [], []
    for j in range(N_LOG):
        if j < N_LOG // 2:   # m in [1 + j/N, 1 + (j+1)/N)
            centre = 1 + (mp.mpf(j) + mp.mpf("0.5")) / N_LOG
        else:                # m / 2 in [(1 + j/N)/2, (1 + (j+1)/N)/2)
            centre = (1 + (mp.mpf(j) + mp.mpf("0.5")) / N_LOG) / 2
        cj = mp.mpf(1) if j == N_LOG - 1 else short(1 / centre)
        c.append(dbl(cj))
        t.append(split(mp.log(cj) / 8))
    k = [split(n * mp.log(2) / 8) for n in range(34)]
    return c, t, k


N_ANGLE = 4096


def angle_table():
    s = 4 * mp.sqrt(2)
    out = []
    for j in range(N_ANGLE):
        a = 2 * mp.pi * (mp.mpf(j) + mp.mpf("0.5")) / N_ANGLE
        out.append((dbl(s * mp.sin(a)), dbl(s * mp.cos(a))))
    return out


def poly():
    # -ln(1 + r) / 8 = r (-1/8 + r (1/16 + r (-1/24 + r / 32)))
    log_c = [dbl(mp.mpf(v)) for v in ("-0.125", "0.0625", -mp.mpf(1) / 24, "0.03125")]
    # angle 2 pi q 2^-33 for the odd integer q, |q| < 2^20 (|angle| < 2 pi / 8192 rad):
    # sin = q (s1 + q^2 s3), 1 - cos = q^2 (c2 + q^2 c4); the first terms left out
    # (angle^5 / 120, angle^6 / 720) are below 3e-18 of the value
    b = 2 * mp.pi * mp.mpf(2) ** -33
    sin_c = [dbl(b), dbl(-b ** 3 / 6)]
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
    lines.append(f"// reciprocals c_j (20 significant bits) of the {N_LOG} reduction intervals")
    lines.append(f"__device__ const double kLogC[{N_LOG}] = {{")
    lines += ["  " + ", ".join(h(x) for x in c[i:i + 4]) + "," for i in range(0, N_LOG, 4)]
    lines.append("};")
    lines.append("// ln(c_j) / 8 as (rounded value, residual)")
    lines.append(f"__device__ const double2 kLogT[{N_LOG}] = {{")
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
