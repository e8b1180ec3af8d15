"""Seeded synthetic GWAS inputs with the shapes and distributions of the
paper's workload (245 samples x 4 covariates x 10643 SNPs, section "Results").

This module holds input generation only -- none of the method's arithmetic --
and is the one piece that the library's callers, the benchmark and the CPU
oracle's tests share.

Recipe (numpy PCG64, one seed per workload):
  X[:, 0] = 1, X[:, 1:] ~ N(0, 1)              (covariates, already normalised)
  MAF_j ~ U(0.05, 0.5),  S_ij ~ Binomial(2, MAF_j)  (genotypes kept raw in {0,1,2})
  beta_true ~ N(0, variance 0.5),  y_i ~ Bernoulli(sigmoid(x_i . beta_true))
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GwasData:
    X: np.ndarray       # n x d float64, column 0 is the intercept
    y: np.ndarray       # n float64 in {0, 1}
    S: np.ndarray       # n x k float64 in {0, 1, 2}
    beta_true: np.ndarray
    maf: np.ndarray


def make_gwas(n: int, d: int, k: int, seed: int) -> GwasData:
    """n samples, d covariates including the intercept, k SNPs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.empty((n, d))
    X[:, 0] = 1.0
    X[:, 1:] = rng.standard_normal((n, d - 1))
    maf = rng.uniform(0.05, 0.5, size=k)
    S = rng.binomial(2, maf[None, :], size=(n, k)).astype(np.float64)
    beta_true = rng.normal(0.0, np.sqrt(0.5), size=d)
    eta = X @ beta_true
    prob = 1.0 / (1.0 + np.exp(-eta))
    y = (rng.uniform(size=n) < prob).astype(np.float64)
    return GwasData(X=X, y=y, S=S, beta_true=beta_true, maf=maf)


def make_residues(rows: int, N: int, moduli, seed: int) -> np.ndarray:
    """rows x N uint64 residues, row r uniform in [0, moduli[r])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((rows, N), np.uint64)
    for r in range(rows):
        out[r] = rng.integers(0, int(moduli[r]), size=N, dtype=np.uint64)
    return out


def make_slots(M: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """M complex slot values with N(0, scale^2) real and imaginary parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * (rng.standard_normal(M) + 1j * rng.standard_normal(M))


# The workloads the tests and the benchmark run (name -> parameters).
WORKLOADS = {
    # small plain job: N = 2^13, 4 q-limbs (60 + 3 x 40 bits), 1 special prime
    "small-n64": dict(logN=13, L=4, q0_bits=60, scale_bits=40, K=1, sp_bits=60, dnum=4,
                      n=64, d=4, k=256, seed=1001, split=True),
    # paper-shaped job: N = 2^16, 24 q-limbs (60 + 23 x 45), 8 special primes, dnum 3
    "paper-n245": dict(logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60, dnum=3,
                       n=245, d=5, k=10643, seed=1002, split=False),
    # kernel microbench: 64 ciphertexts x 2 polys x 24 limbs at N = 2^16
    "ntt-ks-micro": dict(logN=16, L=24, q0_bits=60, scale_bits=45, K=8, sp_bits=60, dnum=3,
                         n_ct=64, seed=1003),
}
