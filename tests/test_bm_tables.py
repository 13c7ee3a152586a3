"""The tables of the FP64 Box-Muller transform (csrc/vct_bm_tables.cuh): the
committed header is what its generator writes, and its values have the
properties the device code relies on -- checked in exact rational arithmetic,
not by re-running the generator's formulas:

* every reduction reciprocal c_j has at most 20 significant bits, so that
  r = m c_j - 1 is exact in one FP64 fma for the 33-bit significands m of the
  uniform, and |r| stays below 1.01 2^-13 over the whole interval j (the
  degree-4 logarithm polynomial's range); the interval just below 1 has c = 1;
* ln(c_j) / 8 and n ln 2 / 8 as (value, residual) pairs agree with the
  logarithm to well below an FP64 unit, and the angle table holds
  4 sqrt(2) (sin, cos) of the interval centres."""
import math
import os
import re
import subprocess
import sys
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2202_13927_gb300", "csrc")
HEADER = os.path.join(CSRC, "vct_bm_tables.cuh")


def _table(name):
    text = open(HEADER).read()
    m = re.search(r"%s\[(\d+)\] = \{(.*?)\};" % name, text, re.S)
    assert m, name
    vals = [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-fA-F.]+p[-+]?\d+", m.group(2))]
    return int(m.group(1)), vals


def _sig_bits(x: float) -> int:
    f = Fraction(x)
    n, d = f.numerator, f.denominator
    while n % 2 == 0:
        n //= 2
    return n.bit_length()


def test_reduction_reciprocals_are_short_and_keep_r_small():
    n, c = _table("kLogC")
    assert n == len(c) == 4096
    assert c[-1] == 1.0
    half = n // 2
    worst = Fraction(0)
    for j, cj in enumerate(c):
        assert _sig_bits(cj) <= 20, (j, cj)
        # the interval of significands m (j < n/2) or m / 2 (j >= n/2), ends included
        lo = 1 + Fraction(j, n)
        hi = 1 + Fraction(j + 1, n)
        if j >= half:
            lo, hi = lo / 2, hi / 2
        for m in (lo, hi):
            worst = max(worst, abs(m * Fraction(cj) - 1))
    assert worst < Fraction(101, 100) * Fraction(1, 2 ** 13), float(worst)
    # r = m c - 1 exact: 33 + 20 significant bits fit in the 53 of an FP64 value
    assert 33 + max(_sig_bits(x) for x in c) <= 53


def test_log_tables_match_the_logarithm():
    n, c = _table("kLogC")
    _, t = _table("kLogT")
    assert len(t) == 2 * n
    for j in range(0, n, 37):
        v = t[2 * j] + t[2 * j + 1]
        assert abs(v - math.log(c[j]) / 8) <= 2e-16 * max(abs(v), 1e-300) + 1e-19, j
        assert abs(t[2 * j + 1]) <= abs(t[2 * j]) * 2 ** -52 or t[2 * j] == 0.0
    nk, k = _table("kLogK")
    assert nk == 34 and len(k) == 68
    for i in range(34):
        assert abs(k[2 * i] - i * math.log(2) / 8) <= 1e-15 * max(i, 1)


def test_angle_table_holds_the_interval_centres():
    n, a = _table("kAngle")
    assert n == 4096 and len(a) == 2 * n
    s = 4 * math.sqrt(2)
    for j in range(0, n, 11):
        th = 2 * math.pi * (j + 0.5) / n
        assert abs(a[2 * j] - s * math.sin(th)) <= 4e-15 * s
        assert abs(a[2 * j + 1] - s * math.cos(th)) <= 4e-15 * s


def test_generator_writes_the_committed_header(tmp_path):
    pytest.importorskip("mpmath")
    src = open(os.path.join(CSRC, "gen_bm_tables.py")).read()
    gen = tmp_path / "gen.py"
    gen.write_text(src)
    subprocess.run([sys.executable, str(gen)], check=True, cwd=tmp_path)
    assert (tmp_path / "vct_bm_tables.cuh").read_text() == open(HEADER).read()
