"""The kernels truncate non-negative doubles with integer operations on the
bits (significand shifted by the exponent) instead of the conversion
instruction.  This is the same algorithm on the host, checked against
numpy's truncation over every binade of interest and the edge values; the
GPU parity tests then see identical tallies."""
import numpy as np


def trunc_bits(y: np.ndarray) -> np.ndarray:
    b = y.view(np.int64)
    e = (b >> 52).astype(np.int64) - 1075
    m = (b & 0x000FFFFFFFFFFFFF) | 0x0010000000000000
    out = np.zeros_like(b)
    pos = e >= 0
    mid = (e < 0) & (e >= -52)
    out[pos] = m[pos] << e[pos]
    out[mid] = m[mid] >> (-e[mid])
    return out


def floor_or_m1(x: np.ndarray) -> np.ndarray:
    return np.where(x.view(np.int64) < 0, -1, trunc_bits(np.abs(x)))


def test_trunc_matches_conversion_over_binades():
    rng = np.random.default_rng(1)
    ys = [rng.uniform(0.0, 1.0, 20000) * 2.0 ** k for k in range(-60, 62)]
    edges = np.array([0.0, 5e-324, 2.2250738585072014e-308, 0.49999999999999994, 0.5,
                      0.9999999999999999, 1.0, 1.5, 2.0 ** 52 - 0.5, 2.0 ** 52, 2.0 ** 52 + 1,
                      2.0 ** 53, 2.0 ** 53 + 2, 2.0 ** 62, 2.0 ** 63 - 1024])
    y = np.concatenate(ys + [edges])
    np.testing.assert_array_equal(trunc_bits(y), np.trunc(y).astype(np.int64))


def test_floor_or_m1():
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-3000.0, 3000.0, 100000), [0.0, -0.0, -1e-300, 1e-300]])
    want = np.where(x < 0, -1, np.floor(x)).astype(np.int64)
    want[x.view(np.int64) < 0] = -1          # -0.0 counts as negative; callers clamp at 0
    np.testing.assert_array_equal(floor_or_m1(x), want)


def u53_scaled(m: int, k: int) -> float:
    """m 2^-k from the bits (0 <= m < 2^53), as the kernels build it."""
    if m == 0:
        return 0.0
    p = m.bit_length() - 1
    b = ((1023 + p - k) << 52) | ((m << (52 - p)) & 0x000FFFFFFFFFFFFF)
    return float(np.array([b], np.int64).view(np.float64)[0])


def test_integer_to_double_from_bits():
    rng = np.random.default_rng(3)
    ms = [0, 1, 2, 3, (1 << 53) - 1, 1 << 52] + [int(x) for x in rng.integers(0, 1 << 53, 20000)]
    ms += [int(x) >> int(s) for x, s in zip(rng.integers(1, 1 << 53, 2000),
                                            rng.integers(0, 52, 2000))]
    for m in ms:
        for k in (0, 24, 53):
            assert u53_scaled(m, k) == m * 2.0 ** -k, (m, k)
