"""Prior probabilities P from the seeds (Sec. IV-A: a Gaussian fitted to the seed intensities of
each region).  Oracle, FP64.  Test infrastructure only.

For label k with seed intensities v: mu_k = mean(v), sigma_k = max(std(v), sigma_floor)
(maximum-likelihood, ddof = 0).  p^k(x) is proportional to N(J(x); mu_k, sigma_k) and each row
of P is normalized to sum to 1 (P is a matrix of probabilities, Sec. II-A), computed with the
log-sum-exp shift.  The constant 1/sqrt(2 pi) cancels in the normalization.
"""
from __future__ import annotations

import numpy as np

SIGMA_FLOOR = 1e-3


def gaussian_fit(J, seed_idx, seed_lab, n_labels, sigma_floor=SIGMA_FLOOR):
    J = np.asarray(J, dtype=np.float64)
    mu = np.zeros(n_labels)
    sig = np.zeros(n_labels)
    for k in range(n_labels):
        v = J[seed_idx[seed_lab == k]]
        if v.size == 0:
            raise ValueError(f"label {k} has no seed")
        mu[k] = v.mean()
        sig[k] = max(np.sqrt(np.mean((v - mu[k]) ** 2)), sigma_floor)
    return mu, sig


def gaussian_priors(J, seed_idx, seed_lab, n_labels, sigma_floor=SIGMA_FLOOR):
    J = np.asarray(J, dtype=np.float64)
    mu, sig = gaussian_fit(J, seed_idx, seed_lab, n_labels, sigma_floor)
    logp = -0.5 * ((J[:, None] - mu[None, :]) / sig[None, :]) ** 2 - np.log(sig)[None, :]
    logp -= logp.max(axis=1, keepdims=True)
    P = np.exp(logp)
    return P / P.sum(axis=1, keepdims=True)
