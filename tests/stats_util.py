"""Statistical comparisons of shower samples (used by the mixed-precision
and serving tests; validated on the CPU by tests/test_stats_power.py)."""
import numpy as np
from scipy import stats


def profile_test(h1, h2, group=5):
    """Two-sample Hotelling T^2 test of the mean longitudinal profile.

    Deposits in neighbouring layers are strongly correlated (one shower
    fills many layers), so layers are summed in groups of `group` and the
    mean vectors are compared with the pooled covariance; T^2 maps to an F
    distribution with (p, n1 + n2 - p - 1) degrees of freedom."""
    g1 = h1.reshape(len(h1), -1, group).sum(2)
    g2 = h2.reshape(len(h2), -1, group).sum(2)
    keep = (g1.var(0) > 0) & (g2.var(0) > 0)
    g1, g2 = g1[:, keep], g2[:, keep]
    n1, n2, p = len(g1), len(g2), g1.shape[1]
    S = ((n1 - 1) * np.cov(g1, rowvar=False) + (n2 - 1) * np.cov(g2, rowvar=False)) / (n1 + n2 - 2)
    d = g1.mean(0) - g2.mean(0)
    t2 = n1 * n2 / (n1 + n2) * d @ np.linalg.solve(S, d)
    f = (n1 + n2 - p - 1) / (p * (n1 + n2 - 2)) * t2
    return t2, p, stats.f.sf(f, p, n1 + n2 - p - 1)


def mean_test(a, b):
    """Welch z of the difference of two sample means."""
    d = a.mean() - b.mean()
    se = np.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
    return d, se
