"""The seeded genotype workloads follow their stated recipes (CPU only):
Bin(2, MAF) codes with MAF ~ U(0.05, 0.5); the AR(1) haplotype model of the
LD generator, whose allele correlation at lag k is the bivariate-normal
orthant formula (2/pi) arcsin(rho^k) when the threshold is the median;
missing fractions; block layouts; and the response's causal set, covariate
weights and the grid's tau x lambda axes.
"""
import math

import numpy as np

from paper_2601_02826_gb300 import synth


def test_binomial_codes_have_hardy_weinberg_frequencies():
    rng = np.random.default_rng(11)
    n = 200_000
    maf = np.array([0.05, 0.2, 0.35, 0.5])
    g = synth.binomial_genotypes(rng, n, maf)
    assert g.dtype == np.int8 and g.shape == (4, n)
    for j, m in enumerate(maf):
        expect = np.array([(1 - m) ** 2, 2 * m * (1 - m), m * m])
        got = np.bincount(g[j], minlength=3)[:3] / n
        assert np.all(np.abs(got - expect) <= 4 * np.sqrt(expect * (1 - expect) / n) + 1e-12), (m, got, expect)


def test_minor_allele_frequencies_are_uniform_on_the_stated_range():
    maf = synth._maf(np.random.default_rng(12), 100_000)
    assert maf.min() >= 0.05 and maf.max() <= 0.5
    # U(0.05, 0.5): mean 0.275, sd 0.45 / sqrt(12)
    assert abs(maf.mean() - 0.275) < 4 * (0.45 / math.sqrt(12)) / math.sqrt(maf.size)


def test_ld_generator_has_the_ar1_allele_correlation():
    rng = np.random.default_rng(13)
    n, p, rho = 40_000, 12, 0.8
    g = synth.ld_genotypes(rng, n, np.full(p, 0.5), rho).astype(np.float64)
    assert np.all(np.abs(g.mean(axis=1) - 1.0) < 0.03)  # 2 * MAF
    for lag in (1, 2, 5):
        r = np.mean([np.corrcoef(g[j], g[j + lag])[0, 1] for j in range(p - lag)])
        expect = 2.0 / math.pi * math.asin(rho ** lag)
        assert abs(r - expect) < 0.02, (lag, r, expect)


def test_missing_entries_take_the_given_fraction():
    rng = np.random.default_rng(14)
    g = synth.add_missing(rng, np.ones((50, 4000), dtype=np.int8), 0.01)
    frac = np.mean(g < 0)
    assert abs(frac - 0.01) < 4 * math.sqrt(0.01 * 0.99 / g.size)
    packed, _ = synth.pack_2bit(g)
    assert np.array_equal(synth.unpack_2bit(packed, 4000) < 0, g < 0)  # missing <-> code 3


def test_ragged_and_equal_block_layouts():
    rng = np.random.default_rng(15)
    P = 500_001
    sizes = synth.ragged_blocks(rng, P, 5000, 30000)
    assert sum(sizes) == P
    assert all(5000 <= s <= 30000 for s in sizes[:-1]) and 1 <= sizes[-1] <= 30000
    eq = synth.equal_blocks(100_006, 32)
    assert sum(eq) == 100_006 and max(eq) - min(eq) <= 1
    assert eq[:100_006 % 32] == [100_006 // 32 + 1] * (100_006 % 32)


def test_genotype_workload_response_and_weights():
    w = synth.geno_workload("t", 400, 3000, 3, synth.FMT_INT8, 50, 0.1, "normal", True, [0.5], [0.1], 4, 16)
    assert np.count_nonzero(w.beta_true) == 50
    assert abs(np.std(w.beta_true[w.beta_true != 0]) - 0.1) < 0.04
    assert w.omega[0] == 0.0 and np.all(w.omega[1:4] == 0.0) and np.all(w.omega[4:] == 1.0)
    assert np.all(np.isfinite(w.y)) and w.cov.shape == (3, 400)
    assert sum(w.block_sizes) == w.P and len(w.block_sizes) == 4


def test_grid_axes():
    w = synth.grid_int8(n=64, p=300)
    assert w.taus == [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9]
    fr = np.asarray(w.lambda_fracs)
    assert len(fr) == 20 and fr[0] == 1.0 and abs(fr[-1] - 0.01) < 1e-15
    assert np.allclose(fr[1:] / fr[:-1], 0.01 ** (1 / 19))
