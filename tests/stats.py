"""Statistical comparison helpers shared by the tests."""
from __future__ import annotations

import math

import numpy as np


def stats(sum_, sumsq, n):
    sum_ = np.asarray(sum_, dtype=np.float64)
    sumsq = np.asarray(sumsq, dtype=np.float64)
    mean = sum_ / n
    var = np.maximum(sumsq / n - mean * mean, 0.0)
    return mean, np.sqrt(var / max(n - 1, 1))


def compare_tallies(m1, e1, m2, e2, frac_3sigma=0.99, max_sigma=5.0, p_min=1e-3):
    """Per-bin agreement of two independent estimates of the same expectation.

    Pass: at least `frac_3sigma` of the bins where either side is non-empty lie
    within 3 combined standard errors, none beyond `max_sigma`, and the
    chi-square over those bins has an upper-tail p-value >= p_min."""
    m1, e1, m2, e2 = map(lambda a: np.asarray(a, dtype=np.float64), (m1, e1, m2, e2))
    sig = np.sqrt(e1 * e1 + e2 * e2)
    nz = (m1 != 0) | (m2 != 0)
    both = nz & (sig > 0)
    z = np.zeros_like(m1)
    z[both] = (m1[both] - m2[both]) / sig[both]
    # a bin non-empty on one side only, with no error estimate, is a hard failure
    lonely = nz & (sig == 0) & (m1 != m2)
    nb = int(both.sum())
    within = float((np.abs(z[both]) <= 3.0).mean()) if nb else 1.0
    worst = float(np.abs(z[both]).max()) if nb else 0.0
    chi2 = float((z[both] ** 2).sum())
    p = chi2_sf(chi2, nb) if nb else 1.0
    ok = (within >= frac_3sigma) and (worst <= max_sigma) and (p >= p_min) and not lonely.any()
    return ok, {"bins": nb, "within3": within, "worst": worst, "chi2": chi2, "p": p,
                "lonely": int(lonely.sum())}


def compare_tallies_unequal(m1, e1, n1, m2, e2, n2, min_count=100.0, max_sigma=5.5, **kw):
    """compare_tallies for samples of very different sizes (n1 >> n2).

    Under the hypothesis that both estimate the same means, the per-history
    variance of a bin is best estimated from the larger sample; the smaller
    sample's standard error is taken from it (e1 sqrt(n1/n2)) instead of its
    own count, whose downward fluctuations would shrink its error and inflate
    the deviation.  A bin whose expected count in the smaller sample (mean x
    n2, unit weights) is below min_count is far from Gaussian there, so such
    bins are merged into one aggregate bin before the comparison; the
    well-populated bins are compared one by one, none beyond max_sigma (5.5:
    the Poisson tail of a 100-count bin is heavier than the Gaussian one)."""
    m1, e1, m2, e2 = map(lambda a: np.asarray(a, dtype=np.float64), (m1, e1, m2, e2))
    if n1 < n2:
        return compare_tallies_unequal(m2, e2, n2, m1, e1, n1, min_count, max_sigma, **kw)
    e2p = e1 * math.sqrt(n1 / n2)
    big = np.abs(m1) * n2 >= min_count
    rest = ~big
    M1 = np.concatenate([m1[big], [m1[rest].sum()]])
    E1 = np.concatenate([e1[big], [math.sqrt((e1[rest] ** 2).sum())]])
    M2 = np.concatenate([m2[big], [m2[rest].sum()]])
    E2 = np.concatenate([e2p[big], [math.sqrt((e2p[rest] ** 2).sum())]])
    ok, info = compare_tallies(M1, E1, M2, E2, max_sigma=max_sigma, **kw)
    info["merged_bins"] = int(rest.sum())
    return ok, info


def chi2_sf(x, k):
    """Upper tail of the chi-square distribution (Wilson-Hilferty for large k)."""
    try:
        from scipy.stats import chi2
        return float(chi2.sf(x, k))
    except Exception:  # pragma: no cover - scipy missing on some boxes
        if k <= 0:
            return 1.0
        z = ((x / k) ** (1 / 3) - (1 - 2 / (9 * k))) / math.sqrt(2 / (9 * k))
        return 0.5 * math.erfc(z / math.sqrt(2))
