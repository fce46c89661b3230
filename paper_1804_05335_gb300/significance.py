"""Significance of plane powers and harmonic sums (host side, for candidates).

A plane value of pure noise is exponential with the row's mean from
fdas_noise_means (even columns: full bins; odd columns: half bins), so a
power P has the single-trial false-alarm probability exp(-P / mean).  A
harmonic sum adds H such values whose means differ slightly from row to row;
its tail P(X_1 + ... + X_H > x) is computed exactly (up to FP64 rounding) by
uniformisation: the sum is the time to pass H exponential phases in turn, so
with Lambda = the largest rate 1/m_i,
  P(sum > x) = sum_n Poisson(n; Lambda x) * P(fewer than H phases passed
               after n uniformised events),
a series of non-negative terms with no cancellation, carried in log scale so
that far tails do not underflow.  Equal means give the Erlang tail.  The
paper leaves these statistics open (Section 5.2).  Significances are returned
as log probabilities and as equivalent one-sided Gaussian sigmas.
"""
from __future__ import annotations

import math

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
    """One-sided Gaussian sigma whose upper-tail probability is exp(logp)
    (0 when that probability is at least 1/2): -Phi^{-1}(exp(logp)), taken
    from the log-domain inverse normal CDF so that far tails keep full
    precision."""
    from scipy.special import ndtri_exp   # host-side statistics only
    if logp >= math.log(0.5):
        return 0.0
    return float(-ndtri_exp(float(logp)))


def point_significance(power, mean):
    """(log false-alarm probability, sigma) of single plane values."""
    logp = -np.asarray(power, np.float64) / np.asarray(mean, np.float64)
    return logp, np.array([sigma_from_logp(float(v)) for v in np.atleast_1d(logp)])


def exp_sum_log_tail(x: float, means) -> float:
    """log P(X_1 + ... + X_H > x) for independent exponentials with `means`."""
    m = np.asarray(means, np.float64).ravel()
    if m.size == 0 or np.any(m <= 0.0):
        raise ValueError("means must be positive")
    if x <= 0.0:
        return 0.0
    rate = 1.0 / m
    lam = float(rate.max())
    p = rate / lam                       # per-event advance probability of each phase
    mu = lam * float(x)                  # Poisson mean of the uniformised events
    H = m.size
    # phase occupation after n events, scaled by exp(-log_scale); phase H absorbs
    a = np.zeros(H)
    a[0] = 1.0
    log_scale = 0.0
    n_max = int(mu + 12.0 * math.sqrt(mu) + 60.0)
    log_pois = -mu                       # log Poisson(0; mu)
    terms = []
    for n in range(n_max + 1):
        s = float(a.sum())
        if s <= 0.0:
            break                        # absorbed with certainty
        terms.append(log_pois + log_scale + math.log(s))
        # next event: stay with 1 - p_i, advance with p_i
        adv = a * p
        a = a - adv
        a[1:] += adv[:-1]
        top = float(a.max())
        if top <= 0.0:
            break
        a /= top
        log_scale += math.log(top)
        log_pois += math.log(mu) - math.log(n + 1)
    t = np.asarray(terms)
    hi = float(t.max())
    return hi + math.log(float(np.exp(t - hi).sum()))


def harmonic_significance(total, means):
    """(log false-alarm probability, sigma) of a harmonic sum `total` of
    values with noise means `means` (one per harmonic)."""
    logp = exp_sum_log_tail(float(total), means)
    return logp, sigma_from_logp(logp)
