"""The statistical acceptance rule itself (CPU): exact multinomial samples
pass it, samples of a slightly wrong distribution fail it, and draws on a
zero-probability neighbour fail at once.  These fix how much bias the
per-state checks of the fast samplers can see."""
import numpy as np
import pytest

import statcheck
from statcheck import assert_follows, chisq_pvalue, tv_distance


@pytest.fixture(autouse=True)
def _private_record(monkeypatch):
    # the planted biases below stay out of the session's summary of real checks
    monkeypatch.setattr(statcheck, "RECORD", [])


def _hub_probs(d=5000, seed=0):
    rng = np.random.default_rng(seed)
    w = rng.lognormal(0.0, 1.0, d)
    w[rng.choice(d, d // 10, replace=False)] = 0.0  # some neighbours excluded, as metapath does
    return w / w.sum()


def _draw(probs, n, seed):
    return np.random.default_rng(seed).multinomial(n, probs)


def test_exact_samples_pass():
    probs = _hub_probs()
    for s in range(8):
        assert_follows(lambda k: _draw(probs, 4_000_000, 100 * s + k), probs, ("exact", s), 4_000_000)


def test_tv_noise_floor():
    """TV over 25 merged bins of exact samples sits near 0.5 sqrt(2k/(pi n))."""
    probs = _hub_probs()
    n, k = 4_000_000, 25
    tvs = [tv_distance(_draw(probs, n, s), probs) for s in range(20)]
    floor = 0.5 * np.sqrt(2 * k / (np.pi * n))
    assert 0.7 * floor < np.mean(tvs) < 1.3 * floor
    assert max(tvs) < statcheck.TV_MAX


@pytest.mark.parametrize("shift", [3e-3, 1e-2])
def test_small_bias_fails(shift):
    """Moving a fraction `shift` of the probability mass from the first to the
    last half of the neighbours (in neighbour order) fails both samples
    (at 4e6 draws over 4,500 neighbours the TV bound catches 0.3 %; 0.1 %
    stays inside the noise)."""
    probs = _hub_probs()
    nz = np.nonzero(probs)[0]
    first, last = nz[: len(nz) // 2], nz[len(nz) // 2:]
    wrong = probs.copy()
    wrong[first] *= 1 - shift / probs[first].sum()
    wrong[last] *= 1 + shift / probs[last].sum()
    with pytest.raises(AssertionError):
        assert_follows(lambda k: _draw(wrong, 4_000_000, 7 + k), probs, ("biased", shift), 4_000_000)


def test_bias_on_one_neighbour_fails():
    """One neighbour drawn 10 % too often (a typical off-by-one at a row end)."""
    probs = _hub_probs(d=64)
    wrong = probs.copy()
    j = int(np.argmax(probs))
    wrong[j] *= 1.1
    wrong /= wrong.sum()
    assert chisq_pvalue(_draw(wrong, 4_000_000, 3), probs) < 1e-6


def test_draw_on_zero_probability_neighbour_fails_at_once():
    probs = _hub_probs(d=64)
    counts = _draw(probs, 1_000_000, 5)
    counts[int(np.argmin(probs))] += 1
    with pytest.raises(AssertionError, match="zero-probability"):
        chisq_pvalue(counts, probs)


def test_redraw_rule_passes_after_one_unlucky_sample():
    """A first sample outside the bounds is redrawn once; only a second miss
    fails the state."""
    probs = _hub_probs(d=64)
    nz = np.nonzero(probs)[0]
    swapped = probs.copy()
    swapped[nz] = probs[nz[::-1]]  # same support, wrong weights
    bad = _draw(swapped, 4_000_000, 1)
    good = _draw(probs, 4_000_000, 2)
    n0 = len(statcheck.RECORD)
    assert_follows(lambda k: bad if k == 0 else good, probs, "redrawn once", 4_000_000)
    assert statcheck.RECORD[n0][3]  # recorded as redrawn
    with pytest.raises(AssertionError):
        assert_follows(lambda k: bad, probs, "missed twice", 4_000_000)
