"""Statistical comparison of sampled neighbour counts with exact probabilities.

chisq_pvalue: Pearson chi-square over the neighbour bins, bins with expected
    count < 5 merged (smallest first); zero-probability bins must be empty.
tv_distance:  total-variation distance over at most `nbins` bins of about
    equal probability formed in neighbour order.  With n draws the TV of a
    perfect sampler over k bins is about 0.5 * sqrt(2 k / (pi n)), so 25 bins
    at 4e6 draws sit near 1e-3, below the 2e-3 bound.
"""
import numpy as np
from scipy import stats


def chisq_pvalue(counts, probs, min_expected=5.0):
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    assert counts.shape == probs.shape
    zero = probs <= 0
    assert counts[zero].sum() == 0, f"{int(counts[zero].sum())} draws landed on zero-probability neighbours"
    c, p = counts[~zero], probs[~zero]
    n = c.sum()
    e = p / p.sum() * n
    order = np.argsort(e, kind="stable")
    obs, exp, ao, ae = [], [], 0.0, 0.0
    for i in order:
        ao += c[i]
        ae += e[i]
        if ae >= min_expected:
            obs.append(ao)
            exp.append(ae)
            ao = ae = 0.0
    if ae > 0:
        if obs:
            obs[-1] += ao
            exp[-1] += ae
        else:
            obs.append(ao)
            exp.append(ae)
    if len(obs) < 2:
        return 1.0
    return float(stats.chisquare(obs, exp).pvalue)


def tv_distance(counts, probs, nbins=25):
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    f = counts / counts.sum()
    p = probs / probs.sum()
    if len(p) > nbins:
        mid = np.cumsum(p) - p / 2
        b = np.minimum((mid * nbins).astype(np.int64), nbins - 1)
        f = np.bincount(b, weights=f, minlength=nbins)
        p = np.bincount(b, weights=p, minlength=nbins)
    return 0.5 * float(np.abs(f - p).sum())
