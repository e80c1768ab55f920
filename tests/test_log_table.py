"""The FP64 logarithm of the transport kernels (Tang's table-driven method:
256 cells of the mantissa, ln(1 + r) to r^6) against numpy's log, with the
method's error bound: the cell table written by gen_log_table.py and the same
steps (exponent and cell from the bits, r = m / c_j - 1 by one fused
multiply-add, the series, k ln 2 added by one more) evaluated in numpy."""
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
INC = os.path.join(os.path.dirname(HERE), "paper_2503_10263_gb300", "csrc", "log_table.inc")


def _table():
    rows = []
    for line in open(INC):
        line = line.strip()
        if line.startswith("{"):
            a, b = line.strip("{},").split(",")
            rows.append((float(a), float(b)))
    return np.array(rows)


def _fma(a, b, c):
    # exact product and sum, one rounding (through Python's exact rationals)
    from fractions import Fraction
    return np.array([float(Fraction(x) * Fraction(y) + Fraction(z)) for x, y, z in
                     np.broadcast(a, b, c)])


def _log_tab(x):
    tab = _table()
    bits = x.view(np.int64)
    k = ((bits >> 52) & 0x7FF) - 1023
    j = (bits >> 44) & 0xFF
    m = ((bits & 0x000FFFFFFFFFFFFF) | 0x3FF0000000000000).view(np.float64)
    r = _fma(m, tab[j, 1], -1.0)
    p = r * (1.0 + r * (-0.5 + r * (1.0 / 3.0 + r * (-0.25 + r * (0.2 - r * (1.0 / 6.0))))))
    return _fma(k.astype(np.float64), 0.69314718055994530942, tab[j, 0] + p)


def test_table_cells():
    tab = _table()
    assert tab.shape == (256, 2)
    c = 1.0 + (np.arange(256) + 0.5) / 256.0
    np.testing.assert_allclose(tab[:, 0], np.log(c), rtol=0, atol=2e-17)
    np.testing.assert_allclose(tab[:, 1], 1.0 / c, rtol=2e-16, atol=0)


def test_log_within_bound_over_the_used_range():
    # eta in (0, 1] (optical depths), energy ratios up to 2e4 and beyond
    rng = np.random.default_rng(7)
    x = np.concatenate([
        (np.arange(1, 4001) * 2.0**-53),                 # smallest uniforms
        rng.uniform(0.0, 1.0, 20000) + 2.0**-53,
        1.0 - rng.uniform(0, 1e-6, 2000),                # near 1: tau near 0
        1.0 + rng.uniform(0, 1e-6, 2000),
        np.exp(rng.uniform(-40.0, 40.0, 20000)),
        np.array([1.0, 2.0, 0.5, 2.0**-53, 1.0 - 2.0**-53, 2e4, 1e-5, 700.0]),
    ])
    got = _log_tab(x)
    ref = np.log(x)
    err = np.abs(got - ref)
    bound = 4e-16 + 2.0 * np.spacing(np.abs(ref))
    assert np.all(err <= bound), float(np.max(err / bound))
    assert abs(got[np.nonzero(x == 1.0)[0][0]]) <= 1e-16
