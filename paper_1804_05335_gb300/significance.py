"""Significance of plane powers and harmonic sums (host side, for candidates).

A plane value of pure noise is exponential with the row's mean from
fdas_noise_means (even columns: full bins; odd columns: half bins), so a
power P has the single-trial false-alarm probability exp(-P / mean).  A
harmonic sum adds H such values with nearly equal means; its tail is taken
from the gamma distribution with the same mean and variance (shape
(sum m)^2 / sum m^2, scale sum m^2 / sum m), exact when the means are equal.
Significances are returned as log probabilities and as equivalent one-sided
Gaussian sigmas.
"""
from __future__ import annotations

import math
from statistics import NormalDist

import numpy as np
import torch

from . import fdas_noise_means, fdas_num_templates


def noise_means(p) -> np.ndarray:
    """(K, 2) array: mean noise power of even and odd columns of each row."""
    K = fdas_num_templates(p)
    m = torch.empty(2 * K, dtype=torch.float32, device="cuda")
    fdas_noise_means(p, m)
    return m.view(K, 2).cpu().numpy().astype(np.float64)


def sigma_from_logp(logp: float) -> float:
    """One-sided Gaussian sigma whose tail probability is exp(logp)."""
    if logp > -700.0:
        p = math.exp(logp)
        return 0.0 if p >= 0.5 else -NormalDist().inv_cdf(p)
    # far tail: solve log Q(s) = logp with log Q(s) ~ -s^2/2 - log(s sqrt(2 pi))
    s = math.sqrt(-2.0 * logp)
    for _ in range(20):
        s = math.sqrt(max(-2.0 * logp - 2.0 * math.log(s * math.sqrt(2.0 * math.pi)), 1.0))
    return s


def point_significance(power, mean):
    """(log false-alarm probability, sigma) of single plane values."""
    logp = -np.asarray(power, np.float64) / np.asarray(mean, np.float64)
    return logp, np.array([sigma_from_logp(float(v)) for v in np.atleast_1d(logp)])


def harmonic_significance(total, means):
    """(log false-alarm probability, sigma) of a harmonic sum `total` of
    values with noise means `means` (one per harmonic)."""
    from scipy.special import gammaincc, gammaln   # host-side statistics only
    m = np.asarray(means, np.float64)
    k = m.sum() ** 2 / (m * m).sum()
    theta = (m * m).sum() / m.sum()
    x = float(total) / theta
    q = gammaincc(k, x)
    if q > 0.0:
        logp = math.log(q)
    else:   # far tail: Q(k, x) ~ x^(k-1) e^-x / Gamma(k)
        logp = (k - 1.0) * math.log(x) - x - gammaln(k)
    return logp, sigma_from_logp(logp)
