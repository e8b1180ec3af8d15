"""O2 -- plaintext FP64 of the paper's approximated semi-parallel GWAS.

TEST INFRASTRUCTURE ONLY.  Follows, step by step and in plain numpy float64:
  Alg. 9  (Homomorphic LogReg): beta0 = 0; p = sigma7(X beta);
          g = X^T (y - p); beta <- beta - 4 (X^T X)^-1 g          (eq. updateBeta
          with the Bohning-Lindsay Hessian, eq. hessianApprox)
  eq. sigma7 exactly as printed (degree-7 polynomial in x/8)
  Alg. 11 preamble: w = p(1 - p) with p the last p computed inside the loop;
          w^-1 = inverseSlots(w) (Alg. 10: guess 3, three Newton steps -- NOT 1/w);
          z = X beta + w^-1 (y - p)                                      (eq. z)
  eq. M:  M = I - X (X^T X)^-1 X^T;  S' = M S (eq. Sprime);  z' = M z (eq. zprime)
  eq. estSNPeffect / estSNPerror:
          b' = (w z')^T S' / colSum(w S'^2);  err' = 1 / colSum(w S'^2)
  denominators through the complex-slot route of eqs. z-square .. S-odd
  (pairs of SNPs as x + iy; x^2 = Re(z zbar + z^2)/2, y^2 = Re(z zbar - z^2)/2).
The p-value is a reading (the paper compares p-values but does not define
them): SE = sqrt(err'), Wald statistic b'/SE, two-sided normal tail.
"""
from __future__ import annotations

import math

import numpy as np

# eq. sigma7 coefficients of (x/8)^1, ^3, ^5, ^7 and the constant term
SIGMA7_C0 = 0.5
SIGMA7_C = (-1.73496, 4.19407, -5.43402, 2.50739)


def sigma7(x):
    """eq. sigma7: 0.5 - 1.73496 (x/8) + 4.19407 (x/8)^3 - 5.43402 (x/8)^5 + 2.50739 (x/8)^7."""
    u = np.asarray(x, dtype=np.float64) / 8.0
    return (SIGMA7_C0 + SIGMA7_C[0] * u + SIGMA7_C[1] * u ** 3 + SIGMA7_C[2] * u ** 5
            + SIGMA7_C[3] * u ** 7)


def inverse_slots(w, guess=3.0, iters=3):
    """Alg. 10: Newton iteration for 1/w started at 3, three steps."""
    g = np.full_like(np.asarray(w, dtype=np.float64), guess)
    for _ in range(iters):
        g = g * (2.0 - w * g)
    return g


def xtx_inv(X):
    """Client pre-processing (section "Hessian Matrix Approximation"): (X^T X)^-1."""
    return np.linalg.inv(X.T @ X)


def hom_logreg(X, y, A, kappa, corrected=False, sigmoid=None):
    """Alg. 9 in FP64.  Returns (beta_kappa, p_last) where p_last is the p
    computed in the last iteration (from beta_(kappa-1)).

    corrected=True mirrors both sign slips of the printed formulas (sigma
    evaluated at -X beta, update beta + 4 A g); in exact arithmetic this gives
    beta_corrected = -beta_literal with identical p.
    sigmoid overrides sigma7 (e.g. the exact logistic function)."""
    f = sigma7 if sigmoid is None else sigmoid
    beta = np.zeros(X.shape[1])
    p = None
    for _ in range(kappa):
        xb = X @ beta
        p = f(-xb) if corrected else f(xb)
        g = X.T @ (y - p)
        beta = beta + 4.0 * (A @ g) if corrected else beta - 4.0 * (A @ g)
    return beta, p


def semi_parallel_fp64(X, y, S, kappa, corrected=False, A=None):
    """The approximated semi-parallel GWAS of Alg. 11 in FP64.

    X: n x d (column 0 = 1), y: n, S: n x k.  Returns a dict with b, err, num,
    den, pval and the intermediate vectors."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    S = np.asarray(S, np.float64)
    n, k = S.shape
    if A is None:
        A = xtx_inv(X)
    beta, p = hom_logreg(X, y, A, kappa, corrected=corrected)
    w = p * (1.0 - p)
    winv = inverse_slots(w)
    z = X @ beta + winv * (y - p)
    M = np.eye(n) - X @ A @ X.T
    zp = M @ z
    Sp = M @ S
    num = (w * zp) @ Sp
    den = complex_route_den(Sp, w)
    b = num / den
    err = 1.0 / den
    return dict(beta=beta, p=p, w=w, winv=winv, z=z, M=M, zp=zp, Sp=Sp, num=num, den=den,
                b=b, err=err, pval=wald_pvalue(b, err), A=A)


def complex_route_den(Sp, w):
    """colSum(w S'^2) computed as in eqs. S-even / S-odd: columns (2c, 2c+1)
    packed as x + iy; denEven = (WSC + WSS)/2, denOdd = (WSC - WSS)/2 with
    WSS = (w S') S', WSC = (w S') conj(S'); real parts are the two sums."""
    n, k = Sp.shape
    kk = k + (k % 2)
    P = np.zeros((n, kk))
    P[:, :k] = Sp
    Z = P[:, 0::2] + 1j * P[:, 1::2]
    WS = w[:, None] * Z
    WSS = (WS * Z).sum(axis=0)
    WSC = (WS * np.conj(Z)).sum(axis=0)
    den = np.empty(kk)
    den[0::2] = np.real(0.5 * (WSC + WSS))
    den[1::2] = np.real(0.5 * (WSC - WSS))
    return den[:k]


def wald_pvalue(b, err):
    """Reading of the paper's p-values: two-sided normal tail of b / sqrt(err)."""
    b = np.asarray(b, np.float64)
    se = np.sqrt(np.asarray(err, np.float64))
    zs = np.abs(b / se)
    return np.array([math.erfc(v / math.sqrt(2.0)) for v in zs])


def neglog10p(b, err):
    return -np.log10(np.maximum(wald_pvalue(b, err), 1e-300))
