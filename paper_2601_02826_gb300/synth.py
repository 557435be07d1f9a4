"""Seeded synthetic workloads for penalized quantile regression with p >> n.

This module only draws data: genotype matrices, dense covariates, responses,
feature-block partitions and quantile/penalty grids. It holds none of the
solver's arithmetic (no standardisation, no lambda_max, no step sizes), so
both the CUDA path and the CPU oracle can take their inputs from here.

Shapes follow the paper's simulation and biobank workloads (Section 7:
sparse DGP with AR(1) design; UK Biobank 30,000 x 482,502 SNPs, G = 48),
scaled to the five workloads below:

  small_dense     n=500,    p=2,000      dense N(0,1) FP64, t(3) noise, G=4
  geno_int8       n=5,000,  p=100,000    int8 Bin(2, MAF), 5 covariates, G=32
  grid_int8       n=10,000, p=500,000    int8, ragged blocks U(5k,30k)
  warm_2bit       n=20,000, p=1,000,000  2-bit packed
  biobank_2bit    n=50,000, p=2,000,000  2-bit packed with AR(1) LD
  paper_sparse    n=1,000,  p=2,000      the paper's sparse DGP (Section 7.1), dense FP64
  paper_dense     n=10,000, p=20,000     the paper's dense DGP (Section 7.2), dense FP64

Genotype storage is SNP-major (one SNP column = all samples, contiguous),
padded to a 16-byte multiple per column:
  int8: one byte per sample, values 0/1/2 (-1 = missing)
  2bit: four samples per byte, sample i in bits 2*(i%4)..2*(i%4)+1 of byte
        i//4; codes 0/1/2 = genotype, 3 = missing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2601_02826

FMT_DENSE_F64 = 0
FMT_INT8 = 1
FMT_2BIT = 2


def padded_ld(n: int, fmt: int) -> int:
    """Bytes per stored column, rounded up to a multiple of 16."""
    if fmt == FMT_DENSE_F64:
        raw = 8 * n
    elif fmt == FMT_INT8:
        raw = n
    elif fmt == FMT_2BIT:
        raw = (n + 3) // 4
    else:
        raise ValueError(f"unknown format {fmt}")
    return (raw + 15) // 16 * 16


@dataclass
class Workload:
    name: str
    n: int
    p: int                       # genotype / main feature columns
    c: int                       # dense covariate columns
    fmt: int
    geno: np.ndarray             # (p, ld) uint8/int8 rows = SNP columns, or (p, n) float64 for dense
    ld: int                      # bytes per SNP column
    cov: np.ndarray              # (c, n) float64, covariate-major (one covariate contiguous)
    y: np.ndarray                # (n,) float64
    taus: list
    block_sizes: list            # G entries summing to 1 + c + p
    omega: np.ndarray            # (1 + c + p,) penalty weights, omega[0] = 0
    lambda_fracs: list           # lambda / lambda_max grid
    beta_true: np.ndarray = field(default=None)  # (p,) effects on raw genotype scale
    recipe: str = ""

    @property
    def P(self) -> int:
        return 1 + self.c + self.p

    def block_ptr(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.block_sizes)]).astype(np.int64)


# ---------------------------------------------------------------- genotypes

def _maf(rng, p, lo=0.05, hi=0.5):
    return rng.uniform(lo, hi, size=p)


def binomial_genotypes(rng, n, maf, chunk=2048):
    """g_ij ~ Bin(2, maf_j), one uniform per entry through the Bin(2, .) CDF.

    Returns an int8 array of shape (p, n), SNP-major.
    """
    p = len(maf)
    out = np.empty((p, n), dtype=np.int8)
    for j0 in range(0, p, chunk):
        j1 = min(p, j0 + chunk)
        m = maf[j0:j1, None].astype(np.float32)
        u = rng.random((j1 - j0, n), dtype=np.float32)
        p2 = m * m                       # P(g = 2)
        p12 = 1.0 - (1.0 - m) * (1.0 - m)  # P(g >= 1)
        out[j0:j1] = (u < p2).astype(np.int8) + (u < p12).astype(np.int8)
    return out


def ld_genotypes(rng, n, maf, rho=0.8, chunk=4096):
    """Genotypes with linkage-disequilibrium-like structure.

    Each individual carries two latent Gaussian haplotype chains that follow
    an AR(1) process with correlation rho across adjacent SNPs; allele = 1
    when the latent value falls below Phi^{-1}(maf_j), genotype = sum of the
    two alleles.
    """
    from scipy.special import ndtri
    p = len(maf)
    thr = ndtri(maf).astype(np.float32)
    out = np.empty((p, n), dtype=np.int8)
    h = rng.standard_normal((2, n), dtype=np.float32)
    a = np.float32(rho)
    b = np.float32(math.sqrt(1.0 - rho * rho))
    for j0 in range(0, p, chunk):
        j1 = min(p, j0 + chunk)
        eps = rng.standard_normal((j1 - j0, 2, n), dtype=np.float32)
        for jj in range(j1 - j0):
            if j0 + jj > 0:
                h = a * h + b * eps[jj]
            out[j0 + jj] = (h[0] < thr[j0 + jj]).astype(np.int8) + (h[1] < thr[j0 + jj]).astype(np.int8)
    return out


def store_int8(g: np.ndarray) -> tuple[np.ndarray, int]:
    """SNP-major int8 genotypes (p, n) -> padded (p, ld) int8 storage."""
    p, n = g.shape
    ld = padded_ld(n, FMT_INT8)
    out = np.zeros((p, ld), dtype=np.int8)
    out[:, :n] = g
    return out, ld


def pack_2bit(g: np.ndarray) -> tuple[np.ndarray, int]:
    """SNP-major genotypes (p, n) with values 0/1/2 and -1 (missing) -> 2-bit codes.

    Sample i goes to bits 2*(i%4) of byte i//4; missing becomes code 3.
    """
    p, n = g.shape
    ld = padded_ld(n, FMT_2BIT)
    codes = np.where(g < 0, 3, g).astype(np.uint8)
    npad = 4 * ld
    full = np.zeros((p, npad), dtype=np.uint8)
    full[:, :n] = codes
    full = full.reshape(p, ld, 4)
    packed = (full[:, :, 0] | (full[:, :, 1] << 2) | (full[:, :, 2] << 4) | (full[:, :, 3] << 6)).astype(np.uint8)
    return packed, ld


def unpack_2bit(packed: np.ndarray, n: int) -> np.ndarray:
    """Inverse of pack_2bit: returns int8 (p, n) with -1 for missing."""
    p, ld = packed.shape
    b = packed.astype(np.uint8)
    codes = np.stack([(b >> (2 * k)) & 3 for k in range(4)], axis=-1).reshape(p, 4 * ld)[:, :n].astype(np.int8)
    codes[codes == 3] = -1
    return codes


def unpack_int8(stored: np.ndarray, n: int) -> np.ndarray:
    return np.ascontiguousarray(stored[:, :n])


def add_missing(rng, g: np.ndarray, frac: float) -> np.ndarray:
    """Marks a random fraction of genotype entries as missing (-1)."""
    g = g.copy()
    mask = rng.random(g.shape) < frac
    g[mask] = -1
    return g


# ------------------------------------------------------------ block layouts

def equal_blocks(P: int, G: int) -> list:
    """G contiguous blocks; the first P mod G blocks get one extra column."""
    base, extra = divmod(P, G)
    return [base + (1 if g < extra else 0) for g in range(G)]


def ragged_blocks(rng, P: int, lo: int, hi: int) -> list:
    """Block sizes drawn U(lo, hi) until they cover P; the last block takes the rest."""
    sizes = []
    left = P
    while left > 0:
        s = int(rng.integers(lo, hi + 1))
        if s >= left:
            s = left
        sizes.append(s)
        left -= s
    return sizes


# ---------------------------------------------------------------- workloads

def _dense_genotype_response(rng, g, cov, n_causal, eff_sd, noise, hetero):
    """y = G_raw beta* + C gamma_c + eps on the raw genotype scale."""
    p, n = g.shape
    causal = rng.choice(p, size=n_causal, replace=False)
    beta = np.zeros(p)
    beta[causal] = rng.normal(0.0, eff_sd, size=n_causal)
    gf = g[causal].astype(np.float64)
    gf[gf < 0] = 0.0
    lin = beta[causal] @ gf
    if cov.shape[0]:
        lin = lin + rng.normal(0.0, 0.3, size=cov.shape[0]) @ cov
    if noise == "t3":
        eps = rng.standard_t(3, size=n)
    else:
        eps = rng.standard_normal(n)
    if hetero:
        hidx = rng.choice(p, size=10, replace=False)
        gam = rng.normal(0.0, eff_sd, size=10)
        hg = g[hidx].astype(np.float64)
        hg[hg < 0] = 0.0
        eps = (1.0 + 0.5 * np.abs(gam @ hg)) * eps
    return lin + eps, beta


def small_dense(seed: int | None = None, n: int = 500, p: int = 2000, G: int = 4,
                tau: float = 0.5) -> Workload:
    """n x p i.i.d. N(0,1) FP64 design plus intercept; 10 N(0,1) effects; t(3) noise."""
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    X = rng.standard_normal((p, n))               # feature-major
    k = min(10, p)
    idx = rng.choice(p, size=k, replace=False)
    beta = np.zeros(p)
    beta[idx] = rng.standard_normal(k)
    y = beta @ X + rng.standard_t(3, size=n)
    P = 1 + p
    omega = np.ones(P)
    omega[0] = 0.0
    ld = padded_ld(n, FMT_DENSE_F64)
    Xs = np.zeros((p, ld // 8))
    Xs[:, :n] = X
    return Workload("small_dense", n, p, 0, FMT_DENSE_F64, Xs, ld,
                    np.zeros((0, n)), y, [tau], equal_blocks(P, G), omega, [0.1], beta,
                    recipe=f"X ~ N(0,1) {n}x{p} FP64, 10 effects N(0,1), eps ~ t(3), G={G}")


def geno_workload(name, n, p, c, fmt, n_causal, eff_sd, noise, hetero, taus, lambda_fracs,
                  blocks, seed, ld_rho=None, missing=0.0, penalize_cov=False):
    rng = np.random.default_rng(seed)
    maf = _maf(rng, p)
    g = ld_genotypes(rng, n, maf, ld_rho) if ld_rho else binomial_genotypes(rng, n, maf)
    if missing > 0:
        g = add_missing(rng, g, missing)
    cov = rng.standard_normal((c, n))
    y, beta = _dense_genotype_response(rng, g, cov, n_causal, eff_sd, noise, hetero)
    if fmt == FMT_INT8:
        stored, ld = store_int8(g)
    else:
        stored, ld = pack_2bit(g)
    P = 1 + c + p
    omega = np.ones(P)
    omega[0] = 0.0
    if not penalize_cov:
        omega[1:1 + c] = 0.0
    if blocks == "equal32":
        bs = equal_blocks(P, 32)
    elif isinstance(blocks, tuple) and blocks[0] == "ragged":
        bs = ragged_blocks(rng, P, blocks[1], blocks[2])
    elif isinstance(blocks, int):
        bs = equal_blocks(P, blocks)
    else:
        raise ValueError(blocks)
    recipe = (f"n={n}, p={p} {'int8' if fmt == FMT_INT8 else '2-bit'} Bin(2,MAF), MAF~U(0.05,0.5)"
              f"{', AR(1) LD rho=%.2f' % ld_rho if ld_rho else ''}; c={c} N(0,1) covariates; "
              f"{n_causal} causal N(0,{eff_sd}^2); noise {noise}{' heteroscedastic' if hetero else ''}; "
              f"G={len(bs)}")
    return Workload(name, n, p, c, fmt, stored, ld, cov, y, list(taus), bs, omega,
                    list(lambda_fracs), beta, recipe=recipe)


def geno_int8(seed=None, n=5000, p=100_000, c=5, G=32, missing=0.0):
    """Genotype-shaped precision workload: 3 quantiles at lambda = 0.1 lambda_max."""
    return geno_workload("geno_int8", n, p, c, FMT_INT8, 50, 0.1, "normal", True,
                         [0.1, 0.5, 0.9], [0.1], G, SEED_BASE + 2 if seed is None else seed,
                         missing=missing)


def grid_int8(seed=None, n=10_000, p=500_000, c=0, n_tau=9, n_lambda=20, blocks=("ragged", 5000, 30000)):
    """Batched tau x lambda grid: 9 quantiles x 20 log-spaced lambda from lambda_max to 0.01 lambda_max."""
    taus = [round(0.1 * (k + 1), 10) for k in range(n_tau)] if n_tau == 9 else list(np.linspace(0.1, 0.9, n_tau))
    fr = list(np.geomspace(1.0, 0.01, n_lambda))
    return geno_workload("grid_int8", n, p, c, FMT_INT8, 100, 0.1, "t3", False, taus, fr, blocks,
                         SEED_BASE + 3 if seed is None else seed)


def warm_2bit(seed=None, n=20_000, p=1_000_000, c=0, n_tau=9, n_lambda=30, blocks=("ragged", 5000, 30000)):
    taus = list(np.linspace(0.1, 0.9, n_tau))
    fr = list(np.geomspace(1.0, 0.01, n_lambda))
    return geno_workload("warm_2bit", n, p, c, FMT_2BIT, 200, 0.05, "t3", True, taus, fr, blocks,
                         SEED_BASE + 4 if seed is None else seed)


def biobank_2bit(seed=None, n=50_000, p=2_000_000, c=10, blocks=("ragged", 5000, 30000)):
    taus = [0.05, 0.25, 0.5, 0.75, 0.95]
    fr = list(np.geomspace(1.0, 0.01, 50))
    return geno_workload("biobank_2bit", n, p, c, FMT_2BIT, 500, 0.05, "t3", False, taus, fr, blocks,
                         SEED_BASE + 5 if seed is None else seed, ld_rho=0.8)


def _ar1_gaussian(rng, n, p, rho=0.5):
    """n draws of N(0, Sigma) with Sigma_ij = rho^|i-j| (a stationary AR(1) across the columns)."""
    X = np.empty((p, n))
    X[0] = rng.standard_normal(n)
    b = math.sqrt(1.0 - rho * rho)
    for j in range(1, p):
        X[j] = rho * X[j - 1] + b * rng.standard_normal(n)
    return X


def paper_sparse(n=1000, p=2000, seed=None, G=5, tau=0.5):
    """The sparse simulation design of the paper's Section 7.1 (eq. dgp_simulation):
    X~ ~ N(0, Sigma), Sigma_ij = 0.5^|i-j|; X_1 = Phi(X~_1), X_j = X~_j otherwise;
    Y = X_6 - X_20 + X_50 - X_100 + X_500 - X_1000 + X_p + 0.7 X_1 eps, eps ~ N(0, 1).
    Dense FP64 storage, every omega_j = 1, G = 5 equal blocks. beta_true holds
    the tau = 0.5 quantile coefficients (beta_1 = 0.7 Phi^{-1}(tau) in general)."""
    from scipy.special import ndtr
    rng = np.random.default_rng(SEED_BASE + 11 if seed is None else seed)
    X = _ar1_gaussian(rng, n, p)
    X[0] = ndtr(X[0])
    beta = np.zeros(p)
    for j, v in ((6, 1.0), (20, -1.0), (50, 1.0), (100, -1.0), (500, 1.0), (1000, -1.0), (p, 1.0)):
        if j <= p:
            beta[j - 1] += v
    y = beta @ X + 0.7 * X[0] * rng.standard_normal(n)
    P = 1 + p
    omega = np.ones(P)
    omega[0] = 0.0
    ld = padded_ld(n, FMT_DENSE_F64)
    Xs = np.zeros((p, ld // 8))
    Xs[:, :n] = X
    return Workload("paper_sparse", n, p, 0, FMT_DENSE_F64, Xs, ld, np.zeros((0, n)), y, [tau],
                    equal_blocks(P, G), omega, [0.1], beta,
                    recipe=f"Section 7.1 sparse DGP: AR(1) 0.5 Gaussian {n}x{p}, X_1 = Phi(.), "
                           f"heteroscedastic 0.7 X_1 eps; G={G}")


def paper_dense(n=10_000, p=20_000, seed=None, G=5, m1=500, m2=50, s1=0.3, s2=0.1):
    """The dense simulation design of the paper's Section 7.2: the same AR(1)
    design with X_j = Phi(X~_j) for m1 < j <= m1 + m2;
    Y = sum_{j<=m1} a_j X_j + (sum_{m1<j<=m1+m2} |b_j| X_j) eps,
    a_j ~ N(0, s1/m1), b_j ~ N(0, s2/m2), eps ~ N(0, 1)."""
    from scipy.special import ndtr
    rng = np.random.default_rng(SEED_BASE + 12 if seed is None else seed)
    X = _ar1_gaussian(rng, n, p)
    X[m1:m1 + m2] = ndtr(X[m1:m1 + m2])
    a = rng.normal(0.0, math.sqrt(s1 / m1), m1)
    b = rng.normal(0.0, math.sqrt(s2 / m2), m2)
    y = a @ X[:m1] + (np.abs(b) @ X[m1:m1 + m2]) * rng.standard_normal(n)
    beta = np.zeros(p)
    beta[:m1] = a
    P = 1 + p
    omega = np.ones(P)
    omega[0] = 0.0
    ld = padded_ld(n, FMT_DENSE_F64)
    Xs = np.zeros((p, ld // 8))
    Xs[:, :n] = X
    return Workload("paper_dense", n, p, 0, FMT_DENSE_F64, Xs, ld, np.zeros((0, n)), y, [0.1, 0.5, 0.9],
                    equal_blocks(P, G), omega, [0.1], beta,
                    recipe=f"Section 7.2 dense DGP: AR(1) 0.5 Gaussian {n}x{p}, {m1} effects N(0,{s1}/{m1}), "
                           f"{m2} scale columns Phi(.); G={G}")


def tiny_geno(seed, n, p, c=0, fmt=FMT_INT8, G=3, missing=0.0, taus=(0.5,), penalize_cov=True):
    """Small genotype problems for parity tests (several tiles plus a ragged tail)."""
    return geno_workload("tiny_geno", n, p, c, fmt, max(1, min(5, p // 4)), 0.3, "t3", True,
                         list(taus), [0.1], G, seed, missing=missing, penalize_cov=penalize_cov)


def tiny_dense(seed, n, p, G=2, tau=0.5):
    return small_dense(seed=seed, n=n, p=p, G=G, tau=tau)
