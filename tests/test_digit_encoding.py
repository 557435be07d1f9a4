"""The exact-integer encodings of the tensor-core path, checked on the CPU
against the FP8 E4M3 format definition (1 sign bit, 4 exponent bits with bias
7, 3 mantissa bits; exponent field 0 encodes the subnormals m * 2^-9):

  * the device table of the balanced base-16 digits -8..8 (kE4M3Int in the
    tensor-core source) encodes each digit exactly;
  * the int8 genotype codes 0, 1, 2, read as E4M3 bit patterns, are exactly
    g * 2^-9, so they enter the products without conversion;
  * balanced base-16 digits in [-8, 8] represent every integer below the
    fixed-point range exactly, and the digit sums of a column stay below
    2^24 (exact in FP32) while n <= 2^20;
  * the set-up passes' 52-bit fixed point (a vector per segment rounded to
    q = hi 2^26 + lo, 0 <= lo < 2^26, with a power-of-two unit above its
    largest entry): the split is exact, the rounding is half a unit, the
    int64 sums of codes times hi and lo cannot overflow, and a power method
    that rounds its vectors this way gives the oracle's estimates.
"""
import math
import os
import re

import numpy as np

from oracle import fsqrppa as O
from paper_2601_02826_gb300 import synth

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


def fix52(w):
    """A segment's 52-bit fixed point as the set-up kernels form it: unit =
    2^(e-52) with 2^e > max |w| (e = ilogb(max) + 1), q = w / unit rounded to
    nearest (ties to even), hi = floor(q / 2^26), lo = q - hi 2^26."""
    m = float(np.max(np.abs(w))) if w.size else 0.0
    if m == 0.0:
        z = np.zeros(w.size, dtype=np.int64)
        return z, z, 0.0
    e = math.frexp(m)[1]  # m = f 2^e with 0.5 <= f < 1, so 2^e > m
    q = np.rint(np.ldexp(w, 52 - e)).astype(np.int64)
    hi = q >> 26
    return hi, q - (hi << 26), math.ldexp(1.0, e - 52)


def test_fixed_point_split_is_exact_and_rounds_by_half_a_unit():
    rng = np.random.default_rng(5)
    for w in (rng.standard_normal(5000), rng.standard_normal(3000) * 1e-7,
              np.array([1.0, -1.0, 0.5, -0.75, 2.0 ** -60, 0.0]), -rng.exponential(3.0, 1000)):
        hi, lo, unit = fix52(w)
        assert np.all((lo >= 0) & (lo < 2 ** 26)) and np.all(np.abs(hi) <= 2 ** 26)
        q = hi * 2 ** 26 + lo
        assert np.all(np.abs(q) <= 2 ** 52)
        assert np.all(np.abs(q * unit - w) <= 0.5 * unit)  # q * unit is exact in FP64


def test_fixed_point_sums_cannot_overflow_int64():
    n = 2 ** 20  # samples (column pass) or columns of a split (row pass)
    worst = n * 2 * 2 ** 26  # every code 2, |hi| or lo at its bound
    assert worst < 2 ** 53  # also exact when converted to FP64 for the combination
    assert worst < 2 ** 63


def _power_fixed(Xg, codes, a, b, max_iter, tol):
    """Algorithm of the oracle's power_lambda with the set-up kernels'
    arithmetic: u = X~_g v from (a_j v_j) in fixed point, w = X~_g^T u from u in
    fixed point, both as exact integer sums of the 0/1/2 codes."""
    pg = Xg.shape[1]
    v = np.full(pg, 1.0 / math.sqrt(pg))
    lam = 0.0
    for _ in range(max_iter):
        hi, lo, unit = fix52(a * v)
        u = unit * ((codes.T @ hi).astype(float) * 2 ** 26 + (codes.T @ lo).astype(float)) + float(b @ v)
        lam_new = float(u @ u)
        hi, lo, unit = fix52(u)
        w = a * (unit * ((codes @ hi).astype(float) * 2 ** 26 + (codes @ lo).astype(float))) + b * u.sum()
        nw = math.sqrt(float(w @ w))
        if nw == 0.0:
            return 0.0
        v = w / nw
        if abs(lam_new - lam) <= tol * lam_new:
            return lam_new
        lam = lam_new
    return lam


def test_power_method_on_fixed_point_vectors_matches_the_oracle():
    for fmt in (synth.FMT_INT8, synth.FMT_2BIT):
        w = synth.tiny_geno(103, 257, 700, c=0, fmt=fmt, G=4, taus=(0.7,))
        g = np.asarray(O.decode_stored(w.geno, w.fmt, w.n), dtype=np.int64)
        d = O.build_design(g, w.cov)
        bp = w.block_ptr()
        for it, tol in ((7, 0.0), (100, 1e-6)):
            for k in range(len(bp) - 1):
                j0, j1 = max(bp[k], 1), bp[k + 1]  # column 0 is the intercept (a = 0, b = 1)
                a = np.where(d.sd[j0:j1] > 0, 1.0 / np.where(d.sd[j0:j1] > 0, d.sd[j0:j1], 1.0), 0.0)
                b = -d.mean[j0:j1] * a
                Xg = d.Xt[:, bp[k]:bp[k + 1]]
                codes = g[j0 - 1:j1 - 1]
                if bp[k] == 0:  # the intercept column joins the block as a = 0, b = 1
                    a, b = np.r_[0.0, a], np.r_[1.0, b]
                    codes = np.vstack([np.zeros((1, w.n), dtype=np.int64), codes])
                got = _power_fixed(Xg, codes, a, b, it, tol)
                ref, _ = O.power_lambda(Xg, it, tol)
                assert abs(got - ref) <= 1e-13 * ref, (fmt, it, k, got, ref)
