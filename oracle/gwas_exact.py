"""O3 -- exact references (sanity, reported, not parity).

TEST INFRASTRUCTURE ONLY.
  (i)  the original semi-parallel GWAS (eqs. z, Str, ztr, SNPeffect, SNPerror)
       with the exact sigmoid (eq. sigmoid), Newton-Raphson to convergence
       (eqs. updateBeta, grad, hessian with W = diag(p(1-p))) and the
       W-weighted projection;
  (ii) brute force: one logistic regression per SNP on [X, s_j], Newton to
       convergence, coefficient of s_j and its standard error.
"""
from __future__ import annotations

import numpy as np


def sigmoid(x):
    """eq. sigmoid: 1 / (1 + exp(-x))."""
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def newton_logreg(X, y, iters=100, tol=1e-13):
    """Maximum-likelihood logistic regression by Newton-Raphson:
    beta <- beta + (X^T W X)^-1 X^T (y - p) (the ascent direction of the
    log-likelihood; eq. updateBeta with H the negated Hessian)."""
    beta = np.zeros(X.shape[1])
    for _ in range(iters):
        p = sigmoid(X @ beta)
        W = p * (1.0 - p)
        H = X.T @ (W[:, None] * X)
        step = np.linalg.solve(H, X.T @ (y - p))
        beta = beta + step
        if np.max(np.abs(step)) < tol:
            break
    return beta


def semi_parallel_exact(X, y, S):
    """Sikorska et al.'s semi-parallel GWAS (section "Semi-Parallel GWAS with
    Homomorphic Encryption", eqs. z .. SNPerror)."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    S = np.asarray(S, np.float64)
    beta = newton_logreg(X, y)
    p = sigmoid(X @ beta)
    w = p * (1.0 - p)
    z = X @ beta + (y - p) / w
    XtWX_inv = np.linalg.inv(X.T @ (w[:, None] * X))
    Sst = S - X @ (XtWX_inv @ (X.T @ (w[:, None] * S)))
    zst = z - X @ (XtWX_inv @ (X.T @ (w * z)))
    den = (w[:, None] * Sst ** 2).sum(axis=0)
    b = ((w * zst) @ Sst) / den
    err = 1.0 / den
    return dict(beta=beta, b=b, err=err)


def per_snp_logreg(X, y, S):
    """Brute force: for each SNP j fit [X, s_j] and return the SNP coefficient
    and its variance (inverse Fisher information)."""
    X = np.asarray(X, np.float64)
    S = np.asarray(S, np.float64)
    k = S.shape[1]
    b = np.zeros(k)
    var = np.zeros(k)
    for j in range(k):
        Z = np.concatenate([X, S[:, j:j + 1]], axis=1)
        beta = newton_logreg(Z, y)
        p = sigmoid(Z @ beta)
        W = p * (1.0 - p)
        info = Z.T @ (W[:, None] * Z)
        b[j] = beta[-1]
        var[j] = np.linalg.inv(info)[-1, -1]
    return dict(b=b, err=var)
