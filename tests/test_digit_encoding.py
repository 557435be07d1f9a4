"""The exact-integer encodings of the tensor-core path, checked on the CPU
against the FP8 E4M3 format definition (1 sign bit, 4 exponent bits with bias
7, 3 mantissa bits; exponent field 0 encodes the subnormals m * 2^-9):

  * the device table of the balanced base-16 digits -8..8 (kE4M3Int in the
    tensor-core source) encodes each digit exactly;
  * the int8 genotype codes 0, 1, 2, read as E4M3 bit patterns, are exactly
    g * 2^-9, so they enter the products without conversion;
  * balanced base-16 digits in [-8, 8] represent every integer below the
    fixed-point range exactly, and the digit sums of a column stay below
    2^24 (exact in FP32) while n <= 2^20.
"""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def e4m3(byte: int) -> float:
    s = -1.0 if byte & 0x80 else 1.0
    e = (byte >> 3) & 0xF
    m = byte & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return s * m * 2.0 ** -9
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def device_digit_table():
    src = open(os.path.join(ROOT, "paper_2601_02826_gb300", "csrc", "k_tc.cu")).read()
    m = re.search(r"kE4M3Int\[17\]\s*=\s*\{([^}]*)\}", src)
    assert m, "digit table not found"
    return [int(x, 16) for x in re.findall(r"0x[0-9A-Fa-f]{2}", m.group(1))]


def test_device_digit_table_encodes_minus8_to_8_exactly():
    table = device_digit_table()
    assert len(table) == 17
    assert [e4m3(b) for b in table] == [float(t) for t in range(-8, 9)]


def test_genotype_codes_are_exact_subnormals():
    assert [e4m3(g) for g in (0, 1, 2)] == [0.0, 2.0 ** -9, 2.0 ** -8]


def balanced_digits(W: int, D: int):
    """Balanced base-16 digits d_0 (most significant) .. d_{D-1} of W."""
    out = [0] * D
    for k in range(D - 1, 0, -1):
        t = ((W + 8) & 15) - 8
        out[k] = t
        W = (W - t) >> 4
    out[0] = W
    return out


def test_balanced_digits_are_exact_and_bounded():
    rng = np.random.default_rng(3)
    for D in (7, 11):
        lim = 2 ** (4 * D - 1)  # |W| < half the fixed-point range
        for W in list(rng.integers(-lim + 1, lim, 2000)) + [lim - 1, -(lim - 1), 0, 7, -8, 8]:
            W = int(W)
            d = balanced_digits(W, D)
            assert all(-8 <= t <= 8 for t in d), (W, d)
            v = 0
            for t in d:
                v = v * 16 + t
            assert v == W


def test_column_digit_sums_fit_fp32_below_2_20_samples():
    n = 2 ** 20
    worst = n * 2 * 8  # every code 2, every digit 8
    assert worst * 2.0 ** -9 == float(np.float32(worst * 2.0 ** -9))
    assert worst <= 2 ** 24
    # one more sample with the same products would leave the exact range
    assert (n + 1) * 16 > 2 ** 24
