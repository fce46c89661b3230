"""The host-side significance conversion (paper_1804_05335_gb300.significance)
against the oracle's arbitrary-precision definitions: the exact tail of a sum
of exponentials with unequal means and the one-sided Gaussian sigma of a log
tail probability.  The paper leaves these statistics open (Section 5.2)."""
import math

import numpy as np
import pytest

import oracle.fdas_oracle as O

pytest.importorskip("mpmath")
S = pytest.importorskip("paper_1804_05335_gb300.significance")


@pytest.mark.parametrize("x,means", [
    (5.0, [1.0, 1.0]),
    (5.0, [1.0, 1.0001, 0.9999]),
    (30.0, [1.0, 1.02, 0.98, 1.01, 1.2, 0.9, 1.1, 1.05]),
    (400.0, [1.0, 1.001, 1.002, 1.003, 1.2337, 1.234, 1.2338, 1.2339]),
    (2000.0, [1.0, 1.1]),
    (0.5, [1.0, 2.0]),
    (12.0, [1.4]),
    (60.0, [0.9983, 0.9991, 1.0004, 1.0012]),
])
def test_harmonic_tail_matches_oracle(x, means):
    got = S.exp_sum_log_tail(x, means)
    ref = O.exp_sum_log_tail(x, means)
    assert abs(got / ref - 1.0) < 1e-9, (got, ref)
    logp, sig = S.harmonic_significance(x, means)
    assert logp == got
    assert abs(sig - O.sigma_of_log_tail(ref)) < 1e-9 * max(1.0, sig)


@pytest.mark.parametrize("logp", [-0.7, -1.8410216450092634, -15.065, -40.0, -700.0, -701.0,
                                  -1000.0, -5000.0, -1e5])
def test_sigma_matches_oracle(logp):
    got = S.sigma_from_logp(logp)
    ref = O.sigma_of_log_tail(logp)
    assert abs(got - ref) < 1e-9 * max(1.0, ref), (got, ref)


def test_point_significance_is_the_exponential_tail():
    logp, sig = S.point_significance([20.0, 2.0], [1.0, 1.2337])
    assert np.allclose(logp, [-20.0, -2.0 / 1.2337], rtol=0, atol=1e-15)
    assert abs(sig[0] - O.sigma_of_log_tail(-20.0)) < 1e-9 * sig[0]


def test_tail_edge_cases():
    assert S.exp_sum_log_tail(0.0, [1.0, 2.0]) == 0.0
    assert S.exp_sum_log_tail(-3.0, [1.0]) == 0.0
    with pytest.raises(ValueError):
        S.exp_sum_log_tail(1.0, [1.0, 0.0])
    assert S.sigma_from_logp(math.log(0.5)) == 0.0
