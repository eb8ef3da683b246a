"""BLER confidence intervals (oracle; test infrastructure only).

The paper reports no BLER numbers (its figures are not available as numbers)
and names no interval; this build uses the Wilson score interval at 95 %
(z = 1.959964) and, when SciPy is present, Clopper-Pearson alongside.
"""
from __future__ import annotations

import math

Z95 = 1.959963984540054


def wilson(k: int, n: int, z: float = Z95):
    """Wilson score interval (lo, hi) for k failures out of n."""
    if n == 0:
        return 0.0, 1.0
    p = k / n
    den = 1.0 + z * z / n
    centre = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return max(0.0, centre - half), min(1.0, centre + half)


def clopper_pearson(k: int, n: int, alpha: float = 0.05):
    from scipy.stats import beta
    lo = 0.0 if k == 0 else float(beta.ppf(alpha / 2, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - alpha / 2, k + 1, n - k))
    return lo, hi
