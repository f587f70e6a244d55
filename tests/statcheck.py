"""Statistical comparison of sampled neighbour counts with exact probabilities.

chisq_pvalue: Pearson chi-square over the neighbour bins, bins with expected
    count < 5 merged (smallest first); zero-probability bins must be empty.
tv_distance:  total-variation distance over at most `nbins` bins of about
    equal probability formed in neighbour order.  With n draws the TV of a
    perfect sampler over k bins is about 0.5 * sqrt(2 k / (pi n)), so 25 bins
    at 4e6 draws sit near 1e-3, below the 2e-3 bound.
assert_follows: the per-state acceptance rule built on the two.
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


# Per-state acceptance: chi-square p > P_MIN and TV < TV_MAX, the levels the
# fast samplers are held to.  Each parity run checks several hundred states,
# so a correct sampler would miss p > 0.01 somewhere in most runs; a state
# whose first sample misses either bound is therefore drawn once more with
# fresh seeds and that second, independent sample must meet both.  A correct
# sampler then fails a state with probability about 1e-4, while a biased one
# (p ~ 0 at these draw counts) fails both samples.
P_MIN = 0.01
TV_MAX = 2e-3

# (what, first p, first TV, redrawn) of every state checked in this process
RECORD = []


def assert_follows(draw, probs, what, ndraws=None, tv_max=TV_MAX, p_min=P_MIN):
    """draw(k) returns the k-th independent sample of neighbour counts
    (k = 0, then k = 1 if the first misses a bound)."""
    probs = np.asarray(probs, dtype=np.float64)
    for k in (0, 1):
        counts = np.asarray(draw(k))
        if ndraws is not None:
            assert counts.sum() == ndraws, (what, int(counts.sum()), ndraws)
        pv, tv = chisq_pvalue(counts, probs), tv_distance(counts, probs)
        ok = pv > p_min and tv < tv_max
        if k == 0:
            RECORD.append((str(what), pv, tv, not ok))
        if ok:
            return
    raise AssertionError(f"{what}: chi-square p = {pv:.3g}, TV = {tv:.3g} "
                         f"(bounds p > {p_min}, TV < {tv_max}) on the first and the redrawn sample")


def assert_pvalue_follows(pvalue, what, p_min=P_MIN):
    """The same rule for a statistic with no TV part (whole-walk path
    frequencies): pvalue(k) is the chi-square p of the k-th independent
    sample."""
    for k in (0, 1):
        pv = float(pvalue(k))
        if k == 0:
            RECORD.append((str(what), pv, float("nan"), not pv > p_min))
        if pv > p_min:
            return
    raise AssertionError(f"{what}: chi-square p = {pv:.3g} (bound p > {p_min}) on the first and the redrawn sample")


def summary():
    """One line on the states checked so far, or None."""
    if not RECORD:
        return None
    ps = np.array([r[1] for r in RECORD])
    tvs = [r[2] for r in RECORD if r[2] == r[2]]
    redrawn = sum(r[3] for r in RECORD)
    tv = f", TV max {max(tvs):.3g}" if tvs else ""
    return (f"distribution checks: {len(RECORD)} states, first-sample p min {ps.min():.3g} / median "
            f"{np.median(ps):.3g}{tv}, redrawn {redrawn} "
            f"({redrawn / len(RECORD):.2%}; ~{P_MIN:.0%}+ expected by chance)")
