"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- published values, closed forms, brute-force enumeration,
library routines, or invariants (FlexiWalker, arXiv 2512.00705)."""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2512_00705_gb300 import synth
from conftest import read_golden


# --------------------------------------------------------------- Philox KATs
def test_philox_known_answers():
    """Published Random123 known-answer vectors for Philox4x32-10."""
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        ctr, key, want = vals[0:4], vals[4:6], tuple(vals[6:10])
        assert oracle.philox4x32_10(ctr, key) == want


def test_exact_uniform_from_published_vector():
    """Exact-mode uniform: Philox4x32-10 at counter (walker, hop, 0, 0) under
    key (seed low, seed high), u = (x0 >> 8) * 2^-24.  At seed, walker and hop
    0 that is the all-zero published vector, so its x0 fixes u."""
    zero = [r for r in read_golden("philox4x32_10_kat.txt") if all(int(x, 16) == 0 for x in r[:6])]
    assert len(zero) == 1
    x0 = int(zero[0][6], 16)
    assert oracle.exact_uniform(0, 0, 0) == (x0 >> 8) / 2.0**24


def test_exact_uniform_range_and_uniformity():
    us = np.array([oracle.exact_uniform(42, w, s) for w in range(2000) for s in range(5)])
    assert us.min() >= 0.0 and us.max() < 1.0
    # on the 2^-24 grid
    assert np.all(us * 2**24 == np.floor(us * 2**24))
    # uniform (Kolmogorov-Smirnov against U[0,1))
    assert stats.kstest(us, "uniform").pvalue > 0.01


# ------------------------------------------------------- worked example, Fig 2
def _star(weights):
    d = len(weights)
    edges = [(0, i + 1) for i in range(d)]
    return synth.from_edges(d + 1, edges, h=weights)


def test_worked_example_probabilities():
    rows = read_golden("worked_example_fig2.txt")
    w = [float(r[1]) for r in rows]
    want = [float(r[2]) for r in rows]
    g = _star(w)
    got = oracle.transition_probs(g, 0, -1, 0, "weighted")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_icdf_pick_frequencies_match_probabilities():
    """Inverse transform: over a fine grid of u the share mapped to k equals
    p_k up to the grid step, and the map is monotone (Sec. 2.2, ITS)."""
    rows = read_golden("worked_example_fig2.txt")
    w = np.array([float(r[1]) for r in rows], dtype=np.float32)
    want = np.array([float(r[2]) for r in rows])
    grid = (np.arange(0, 2**14) * 2**10).astype(np.float64) * 2.0**-24
    picks = np.array([oracle.icdf_pick(w, float(u)) for u in grid])
    assert np.all(np.diff(picks) >= 0)
    share = np.bincount(picks, minlength=4) / len(grid)
    np.testing.assert_allclose(share, want, atol=2.0 / len(grid))
    # zero weights are never picked; all-zero gives a dead end
    w2 = np.array([0, 1, 0, 2, 0], dtype=np.float32)
    picks2 = {oracle.icdf_pick(w2, float(u)) for u in grid[::7]}
    assert picks2 == {1, 3}
    assert oracle.icdf_pick(np.zeros(3, np.float32), 0.5) == -1


# -------------------------------------------------- node2vec closed forms, Eq 2
def _cycle(n):
    return synth.from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def _complete(n):
    return synth.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


@pytest.mark.parametrize("p,q", [(2.0, 0.5), (0.25, 4.0), (1.0, 1.0), (3.0, 0.7)])
def test_node2vec_closed_forms(p, q):
    ip, iq = 1.0 / p, 1.0 / q
    # cycle C_6, at v=2 coming from v'=1: neighbours {1 (return), 3 (distance 2)}
    g = _cycle(6)
    pr = oracle.transition_probs(g, 2, 1, 1, "node2vec", p, q)
    nb = list(g.cols[g.offsets[2]:g.offsets[3]])
    assert nb == [1, 3]
    np.testing.assert_allclose(pr[0], ip / (ip + iq), rtol=1e-6)
    # triangle, at v=1 from v'=0: neighbours {0 (return), 2 (adjacent to v')}
    g = _cycle(3)
    pr = oracle.transition_probs(g, 1, 0, 1, "node2vec", p, q)
    np.testing.assert_allclose(pr[0], ip / (ip + 1.0), rtol=1e-6)
    # K_5, at v=3 from v'=0: return has 1/p, the three others weight 1
    g = _complete(5)
    pr = oracle.transition_probs(g, 3, 0, 1, "node2vec", p, q)
    nb = list(g.cols[g.offsets[3]:g.offsets[4]])
    assert nb[0] == 0
    np.testing.assert_allclose(pr[0], ip / (ip + 3.0), rtol=1e-6)
    np.testing.assert_allclose(pr[1:], 1.0 / (ip + 3.0), rtol=1e-6)
    # without a previous node (hop 0): first-order walk
    pr = oracle.transition_probs(g, 3, -1, 0, "node2vec", p, q)
    np.testing.assert_allclose(pr, 0.25, rtol=1e-12)


def test_node2vec_weighted_closed_form():
    """Path a-b-c-d plus chord b-d: at c from b, neighbours b (return, h=2),
    d (adjacent to b, h=3); p=2, q=0.5 -> weights 2*0.5=1, 3*1=3."""
    g = synth.from_edges(4, [(0, 1), (1, 2), (2, 3), (1, 3)], h=[1.0, 2.0, 3.0, 5.0])
    pr = oracle.transition_probs(g, 2, 1, 1, "node2vec", 2.0, 0.5)
    np.testing.assert_allclose(pr, [0.25, 0.75], rtol=1e-7)
    # at b from a: neighbours a (return, h=1 -> 0.5), c (dist 2 from a, h=2 -> 4), d (dist 2, h=5 -> 10)
    pr = oracle.transition_probs(g, 1, 0, 1, "node2vec", 2.0, 0.5)
    np.testing.assert_allclose(pr, np.array([0.5, 4.0, 10.0]) / 14.5, rtol=1e-7)


def test_known_bound_unweighted_node2vec():
    """Sec. 3.3: unweighted node2vec with a=1, b=0.5 has maximum weight 2."""
    (a, b, h, mx), = [[float(x) for x in r] for r in read_golden("node2vec_known_bound.txt")]
    mode, B, _ = oracle.step_plan(h, 10.0, True, "node2vec", a, b, 4.0)
    assert B == mx
    g = _complete(6)  # every non-return neighbour adjacent to v'
    wt = oracle.transition_weights(g, 2, 0, 1, "node2vec", a, b)
    assert wt.max() <= B
    g = _cycle(8)     # every non-return neighbour at distance 2: weight 1/b = 2 reaches the bound
    wt = oracle.transition_weights(g, 2, 1, 1, "node2vec", a, b)
    assert wt.max() == B


# ------------------------------------------------------- second-order PageRank
def test_pagerank2_closed_forms():
    """Eq. (2ndpr), gamma = 0.2, h = 1: triangle at v=1 from v'=0 (d = d' = 2):
    neighbour 2 is adjacent to v' -> (0.8/2 + 0.2/2) * 2 = 1.0; the return to
    v' takes the other branch -> (0.8/2) * 2 = 0.8."""
    g = _cycle(3)
    pr = oracle.transition_probs(g, 1, 0, 1, "pagerank2")
    np.testing.assert_allclose(pr, [0.8 / 1.8, 1.0 / 1.8], rtol=1e-6)
    # star centre 0 with 4 leaves, at leaf 1 from the centre: d(v)=1, d(v')=4, max_d = 4;
    # the only neighbour is v' itself -> probability 1
    g = synth.from_edges(5, [(0, i) for i in range(1, 5)])
    np.testing.assert_allclose(oracle.transition_probs(g, 1, 0, 1, "pagerank2"), [1.0])
    # at the centre from leaf 1: d(v)=4, d(v')=1, max_d=4; no leaf is adjacent to leaf 1,
    # all weights ((1-g)/4)*4 = 0.8 -> uniform
    np.testing.assert_allclose(oracle.transition_probs(g, 0, 1, 1, "pagerank2"), [0.25] * 4, rtol=1e-6)
    # K_4 at v=3 from v'=0: the others adjacent to v' get (0.8/3 + 0.2/3)*3 = 1, return 0.8
    g = _complete(4)
    np.testing.assert_allclose(oracle.transition_probs(g, 3, 0, 1, "pagerank2"),
                               np.array([0.8, 1.0, 1.0]) / 2.8, rtol=1e-6)
    # unequal degrees with a common neighbour: v'=0 has N = {1, 2}, v=1 has
    # N = {0, 2, 3, 4}; from 0 to 1: d(v)=4, d(v')=2, max_d=4; neighbour 2 is
    # adjacent to v' -> (0.8/4 + 0.2/2) * 4 = 1.2, the others (0.8/4) * 4 = 0.8
    g = synth.from_edges(5, [(0, 1), (0, 2), (1, 2), (1, 3), (1, 4)])
    np.testing.assert_allclose(oracle.transition_probs(g, 1, 0, 1, "pagerank2"),
                               np.array([0.8, 1.2, 0.8, 0.8]) / 3.6, rtol=1e-6)
    # gamma = 0 reduces to a first-order walk
    g = synth.random_graph(12, 0.4, seed=4, weighted=True)
    for v in range(12):
        nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
        if len(nb):
            np.testing.assert_allclose(oracle.transition_probs(g, v, int(nb[0]), 1, "pagerank2", gamma=0.0),
                                       oracle.transition_probs(g, v, -1, 0, "weighted"), rtol=1e-6)


# ------------------------------------------------------------------ metapath
def test_metapath_filter():
    g = synth.from_edges(5, [(0, 1), (0, 2), (0, 3), (0, 4)], h=[1.0, 2.0, 3.0, 4.0], labels=[0, 1, 1, 2])
    schema = [1, 2, 0]
    np.testing.assert_allclose(oracle.transition_probs(g, 0, -1, 0, "metapath", schema=schema), [0, 0.4, 0.6, 0])
    np.testing.assert_allclose(oracle.transition_probs(g, 0, 3, 1, "metapath", schema=schema), [0, 0, 0, 1])
    np.testing.assert_allclose(oracle.transition_probs(g, 0, 3, 2, "metapath", schema=schema), [1, 0, 0, 0])
    # cyclic schema: hop 3 uses schema[0]
    np.testing.assert_allclose(oracle.transition_probs(g, 0, 3, 3, "metapath", schema=schema), [0, 0.4, 0.6, 0])
    # schema label absent -> dead end (all zero)
    assert oracle.transition_probs(g, 0, -1, 0, "metapath", schema=[3]).sum() == 0


# ------------------------------------------------------- brute force, 8 nodes
from bruteforce import bf_paths as _bf_paths, merged_chisquare
from statcheck import assert_pvalue_follows


CASES = [("weighted", 1.0, 1.0, None), ("node2vec", 2.0, 0.5, None), ("node2vec", 0.25, 4.0, None),
         ("node2vec", 3.0, 0.7, None), ("metapath", 1.0, 1.0, [0, 1, 2]), ("pagerank2", 1.0, 1.0, None)]


@pytest.mark.parametrize("algo,p,q,schema", CASES)
@pytest.mark.parametrize("gseed", [11, 12])
def test_brute_force_path_probabilities(algo, p, q, schema, gseed):
    g = synth.random_graph(8, 0.45, seed=gseed, weighted=True, nlabels=3)
    L = 4
    for start in range(8):
        bf = _bf_paths(g, start, L, algo, p, q, schema)
        assert abs(sum(bf.values()) - 1.0) < 1e-12
        for path, pb in bf.items():
            # product of the oracle's per-hop probabilities along the path
            prob, prev = 1.0, -1
            for j in range(L):
                v, u = path[j], path[j + 1]
                if u == -1:
                    assert oracle.transition_probs(g, v, prev, j, algo, p, q, schema).sum() == 0
                    break
                pr = oracle.transition_probs(g, v, prev, j, algo, p, q, schema)
                nb = list(g.cols[g.offsets[v]:g.offsets[v + 1]])
                prob *= pr[nb.index(u)]
                prev = v
            assert prob == pytest.approx(pb, rel=2e-6, abs=1e-12)


@pytest.mark.parametrize("algo,p,q,schema", CASES)
def test_brute_force_sampler_frequencies(algo, p, q, schema):
    """Exact-mode walks from one start, many walker ids: path frequencies
    match brute-force path probabilities (chi-square, merged bins)."""
    g = synth.random_graph(8, 0.45, seed=11, weighted=True, nlabels=3)
    L, W, start = 4, 60000, 0
    bf = _bf_paths(g, start, L, algo, p, q, schema)
    assert_pvalue_follows(lambda k: merged_chisquare(bf, oracle.walk(g, np.full(W, start, np.int32), L, algo, p, q,
                                                                      schema, seed=7 + 7919 * k)[0]),
                          ("oracle paths", algo, p, q))


# --------------------------------------------------------- reductions / invariants
@pytest.mark.parametrize("algo,p,q,schema", CASES)
@pytest.mark.parametrize("weighted", [True, False])
def test_rjs_walk_frequencies(algo, p, q, schema, weighted):
    """Rejection-sampled walks (Sec. 3.3) from one start: path frequencies
    match brute-force path probabilities, as the exact-mode walks' do, with
    and without property weights (also where 1/p or 1/q sets max(w))."""
    g = synth.random_graph(8, 0.45, seed=11, weighted=weighted, nlabels=3)
    L, W, start = 4, 60000, 0
    bf = _bf_paths(g, start, L, algo, p, q, schema)
    assert_pvalue_follows(lambda k: merged_chisquare(bf, oracle.walk_rjs(g, np.full(W, start, np.int32), L, algo, p,
                                                                          q, schema, seed=9 + 7919 * k)[0]),
                          ("oracle rjs paths", algo, p, q, weighted))


def _lemire(x, d):
    """Lemire (ACM TOMACS 2019): floor(x d / 2^32), or None when the low word
    of x d is below 2^32 mod d."""
    m = x * d
    return None if (m & 0xFFFFFFFF) < (2**32 % d) else m >> 32


def test_rjs_proposal_is_lemire_index_of_the_trial_words():
    """With equal weights every proposal is accepted (U * B < B for U < 1), so
    hop 0 from the centre of a star is the first trial's proposal: Lemire's
    index of x0 of Philox4x32-10 at counter (walker, 0, 1, 0), else of x1."""
    for d in (1, 2, 3, 7, 1000, 65537):
        g = synth.from_edges(d + 1, [(0, i) for i in range(1, d + 1)], h=[0.75] * d)
        W, seed = 512, 0x1234_5678_9ABC
        out, _ = oracle.walk_rjs(g, np.zeros(W, np.int32), 1, "weighted", seed=seed)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for w in range(W):
            x = oracle.philox4x32_10([w, 0, 1, 0], key)
            k = _lemire(x[0], d)
            k = _lemire(x[1], d) if k is None else k
            assert k is not None  # two rejections in a row: 2^-64 for these d
            assert out[w, 1] == 1 + k, (d, w)


@pytest.mark.parametrize("algo,p,q,schema", CASES)
def test_rjs_class_envelope_walk_frequencies(algo, p, q, schema):
    """Rejection sampling under the weight-class envelopes (classes of h
    relative to h_MAX with bounds B, B/2, B/4; for metapath five classes
    inside the required label's entries) on weights spread over three
    decades, so that every class is populated: path frequencies match
    brute-force path probabilities."""
    g = synth.random_graph(8, 0.45, seed=11, weighted=True, nlabels=3)
    g.h = (g.h ** 3 + np.float32(1e-3)).astype(np.float32)
    L, W, start = 4, 60000, 0
    bf = _bf_paths(g, start, L, algo, p, q, schema)
    assert_pvalue_follows(lambda k: merged_chisquare(bf, oracle.walk_rjs(g, np.full(W, start, np.int32), L, algo, p,
                                                                          q, schema, seed=19 + 7919 * k,
                                                                          envelope="classes")[0]),
                          ("oracle rjs class envelope paths", algo, p, q))


def test_rjs_class_envelope_slots():
    """Weights h = hmax, hmax/2, hmax/4 sit exactly on their class bounds, so
    every proposal is accepted and hop 0 from the star centre is the entry
    that the first trial's slot names: with row weights [.25, 1, .5, 1, .25]
    the class order is positions 1, 3 (class 0), 2 (class 1), 0, 4 (class 2),
    and the 4*2 + 2*1 + 2 = 12 slots map to 1,1,1,1, 3,3,3,3, 2,2, 0, 4."""
    hs = [0.25, 1.0, 0.5, 1.0, 0.25]
    slot_to_pos = [1] * 4 + [3] * 4 + [2] * 2 + [0, 4]
    g = synth.from_edges(6, [(0, i) for i in range(1, 6)], h=hs)
    W, seed = 4096, 99
    out, _ = oracle.walk_rjs(g, np.zeros(W, np.int32), 1, "weighted", seed=seed, envelope="classes")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for w in range(W):
        x = oracle.philox4x32_10([w, 0, 1, 0], key)
        t = _lemire(x[0], 12)
        t = _lemire(x[1], 12) if t is None else t
        assert out[w, 1] == 1 + slot_to_pos[t], w
    # the uniform proposal of the single bound spreads over the 5 entries instead
    single, _ = oracle.walk_rjs(g, np.zeros(W, np.int32), 1, "weighted", seed=seed)
    assert not np.array_equal(single, out)


def test_rjs_label_class_envelope_slots():
    """Metapath under the label-segment envelope: the label-1 entries of the
    star centre carry h = M, M/2, M/4, M/8, M/16 (M = 1), each on its class
    bound, so every proposal is accepted and hop 0 is the entry named by the
    first slot.  Row (label, h): (1,1) (0,.7) (1,.125) (1,.5) (2,.3) (1,.0625)
    (1,.25) (1,1) -> class order 0, 7 | 3 | 6 | 2 | 5 and 16*2 + 8 + 4 + 2 + 1
    = 47 slots; labels 0 and 2 are never proposed."""
    labs = [1, 0, 1, 1, 2, 1, 1, 1]
    hs = [1.0, 0.7, 0.125, 0.5, 0.3, 0.0625, 0.25, 1.0]
    slot_to_pos = [0] * 16 + [7] * 16 + [3] * 8 + [6] * 4 + [2] * 2 + [5]
    g = synth.from_edges(9, [(0, i) for i in range(1, 9)], h=hs, labels=labs)
    W, seed = 4096, 7
    out, _ = oracle.walk_rjs(g, np.zeros(W, np.int32), 1, "metapath", schema=[1], seed=seed, envelope="classes")
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for w in range(W):
        x = oracle.philox4x32_10([w, 0, 1, 0], key)
        t = _lemire(x[0], 47)
        t = _lemire(x[1], 47) if t is None else t
        assert out[w, 1] == 1 + slot_to_pos[t], w
    # a label the row lacks is a dead end
    dead, _ = oracle.walk_rjs(g, np.zeros(4, np.int32), 2, "metapath", schema=[3], seed=seed, envelope="classes")
    assert np.all(dead[:, 1:] == -1)


@pytest.mark.parametrize("envelope", ["single", "classes"])
@pytest.mark.parametrize("algo,schema", [("weighted", None), ("metapath", [2])])
def test_rjs_mean_trials_equal_envelope_mass_ratio(envelope, algo, schema):
    """Sec. 3.3: a trial accepts with probability (sum of w~) / (envelope
    mass), so the trials per hop are geometric with mean mass / sum w~:
    single bound d * h_MAX; weight classes (4 n0 + 2 n1 + n2) * h_MAX / 4;
    metapath label segment (16 n0 + 8 n1 + 4 n2 + 2 n3 + n4) * M / 16 over
    the required label's entries (single bound: d * h_MAX over the row)."""
    g = synth.workload_graph("small")
    g.h = synth.edge_weights(g, "lognormal", 1.5, seed=13)
    v = int(np.argmax(g.degrees()))
    h = g.h[g.offsets[v]:g.offsets[v + 1]].astype(np.float64)
    lab = g.labels[g.offsets[v]:g.offsets[v + 1]]
    hmax = h.max()
    if algo == "weighted":
        total = h.sum()
        if envelope == "single":
            mass = len(h) * hmax
        else:
            n0, n1 = int((h > hmax / 2).sum()), int(((h > hmax / 4) & (h <= hmax / 2)).sum())
            mass = (4 * n0 + 2 * n1 + (len(h) - n0 - n1)) * hmax / 4
    else:
        hl = h[lab == schema[0]]
        total = hl.sum()
        if envelope == "single":
            mass = len(h) * hmax
        else:
            M = hl.max()
            cls = np.minimum(np.floor(-np.log2(hl / M)).astype(int), 4)  # class c: h in (M/2^(c+1), M/2^c]
            mass = sum((16 >> c) * int((cls == c).sum()) for c in range(5)) * M / 16
    W = 200_000
    _, hops, trials = oracle.walk_rjs(g, np.full(W, v, np.int32), 1, algo, schema=schema, seed=3,
                                      envelope=envelope, return_trials=True)
    assert hops == W
    e = mass / total
    assert abs(trials / hops - e) < 5 * np.sqrt(e * (e - 1) / W) + 1e-3, (trials / hops, e)


def test_node2vec_p1q1_equals_weighted_walk():
    """node2vec with p = q = 1 has w = 1 everywhere, so its walks equal the
    weighted first-order walk bit for bit under the same draws."""
    g = synth.workload_graph("small")
    starts = np.arange(g.n, dtype=np.int32)
    a, ha = oracle.walk(g, starts, 20, "node2vec", 1.0, 1.0, seed=42)
    b, hb = oracle.walk(g, starts, 20, "weighted", seed=42)
    assert ha == hb
    np.testing.assert_array_equal(a, b)


def _check_walk_invariants(g, starts, out, algo, schema=None):
    L = out.shape[1] - 1
    assert np.array_equal(out[:, 0], starts)
    for row in out:
        alive = True
        for j in range(L):
            v, u = row[j], row[j + 1]
            if u == -1:
                alive = False
                continue
            assert alive, "-1 only as a suffix"
            nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
            k = np.searchsorted(nb, u)
            assert k < len(nb) and nb[k] == u, "hop is not an edge"
            if algo == "metapath":
                assert g.labels[g.offsets[v] + k] == schema[j % len(schema)]


@pytest.mark.parametrize("algo,schema", [("node2vec", None), ("metapath", [0, 1, 2, 3, 4]), ("weighted", None)])
def test_walk_invariants_small(algo, schema):
    g = synth.workload_graph("small")
    starts = np.arange(g.n, dtype=np.int32)
    out, hops = oracle.walk(g, starts, 20, algo, 2.0, 0.5, schema, seed=42)
    _check_walk_invariants(g, starts[:600], out[:600], algo, schema)
    assert hops == int((out[:, 1:] >= 0).sum())
    # dead ends only where the total transition weight is zero
    for i in range(0, g.n, 7):
        row = out[i]
        if row[-1] == -1:
            j = int(np.argmax(row == -1)) - 1
            prev = int(row[j - 1]) if j >= 1 else -1
            assert oracle.transition_probs(g, int(row[j]), prev, j, algo, 2.0, 0.5, schema).sum() == 0


def test_walk_rejects_bad_arguments():
    g = synth.workload_graph("small")
    with pytest.raises(ValueError):
        oracle.walk(g, np.array([g.n], np.int32), 5, "weighted")
    with pytest.raises(ValueError):
        oracle.walk(g, np.array([0], np.int32), 5, "node2vec", 0.0, 1.0)


def test_walker_base_shifts_random_stream():
    g = synth.workload_graph("small")
    starts = np.arange(64, dtype=np.int32)
    full, _ = oracle.walk(g, np.concatenate([starts, starts]), 10, "node2vec", 2.0, 0.5, seed=5)
    tail, _ = oracle.walk(g, starts, 10, "node2vec", 2.0, 0.5, seed=5, walker_base=64)
    np.testing.assert_array_equal(full[64:], tail)


# ------------------------------------------------------------ preprocess + plan
def test_node_stats_match_library_reductions():
    g = synth.workload_graph("small")
    hmax, hsum = oracle.node_stats(g)
    deg = g.degrees()
    nz = deg > 0
    idx = g.offsets[:-1][nz]
    np.testing.assert_array_equal(hmax[nz], np.maximum.reduceat(g.h, idx))
    np.testing.assert_allclose(hsum[nz], np.add.reduceat(g.h.astype(np.float64), idx), rtol=1e-12)
    assert np.all(hmax[~nz] == 0) and np.all(hsum[~nz] == 0)
    g2 = synth.Csr(g.offsets, g.cols)
    hmax2, hsum2 = oracle.node_stats(g2)
    np.testing.assert_array_equal(hsum2, deg)
    np.testing.assert_array_equal(hmax2[nz], 1.0)


def test_label_stats_match_library_reductions():
    g = synth.workload_graph("small")
    lmax, lsum = oracle.label_stats(g)
    rows = np.repeat(np.arange(g.n), g.degrees())
    for l in range(8):
        sel = g.labels == l
        want_sum = np.bincount(rows[sel], weights=g.h[sel].astype(np.float64), minlength=g.n)
        want_max = np.zeros(g.n, np.float32)
        np.maximum.at(want_max, rows[sel], g.h[sel])
        np.testing.assert_allclose(lsum[:, l], want_sum, rtol=1e-12)
        np.testing.assert_array_equal(lmax[:, l], want_max)
    # the per-label sums add up to h_SUM
    _, hsum = oracle.node_stats(g)
    np.testing.assert_allclose(lsum.sum(axis=1), hsum, rtol=1e-12)


# ------------------------------------------------------ 8-bit weights
def _rows(*rows):
    """A CSR whose row v holds the weights rows[v] (columns are placeholders:
    quantization reads only the rows' weights)."""
    n = max(len(rows), max(len(r) for r in rows) + 1)
    offsets = np.zeros(n + 1, dtype=np.int32)
    offsets[1:len(rows) + 1] = np.cumsum([len(r) for r in rows])
    offsets[len(rows) + 1:] = offsets[len(rows)]
    cols = np.concatenate([np.arange(1, len(r) + 1) for r in rows]).astype(np.int32)
    h = np.concatenate([np.asarray(r, np.float32) for r in rows]).astype(np.float32)
    return synth.Csr(offsets, cols, h)


def test_quantize_on_the_integer_grid():
    """A row whose maximum is 255 gets scale exactly 1: codes are h rounded to
    the nearest integer with ties to even, kept in 1..255, read back exactly.
    A row with maximum 127.5 gets scale exactly 1/2 of its own, whatever the
    other rows hold; rows without entries get scale 0."""
    g = _rows([255.0, 1.0, 2.0, 0.4, 2.5, 3.5, 254.5, 100.49, 0.5, 1.5, 17.0],
              [127.5, 0.25, 1.0, 0.75, 1.25, 0.2],
              [])
    codes, scales, hq = oracle.quantize_weights(g)
    assert scales[0] == 1.0 and scales[1] == 0.5 and np.all(scales[2:] == 0.0)
    np.testing.assert_array_equal(codes[:11], [255, 1, 2, 1, 2, 4, 254, 100, 1, 2, 17])
    np.testing.assert_array_equal(codes[11:], [255, 1, 2, 2, 2, 1])  # 0.75/0.5 = 1.5 -> 2, 1.25/0.5 = 2.5 -> 2
    np.testing.assert_array_equal(hq, codes.astype(np.float32) * np.repeat(scales, np.diff(g.offsets)))


@pytest.mark.parametrize("kind,param", [("uniform01", 1.0), ("lognormal", 1.0), ("pareto", 1.5)])
def test_quantize_is_nearest_code_within_half_a_step(kind, param):
    """Against fp64, row by row: s_v is the row's max h / 255 rounded once,
    the row's largest weight gets 255, every unclamped code is the nearest
    integer to h / s_v (|code - h/s_v| <= 1/2, so a floor or a ceiling
    fails), and only weights below s_v / 2 clamp to 1."""
    g = synth.rmat(12, 16, seed=5)
    g.h = synth.edge_weights(g, kind, param, seed=6)
    codes, scales, hq = oracle.quantize_weights(g)
    deg = np.diff(g.offsets)
    rows = np.repeat(np.arange(g.n), deg)
    rmax = np.zeros(g.n, np.float32)
    np.maximum.at(rmax, rows, g.h)
    assert np.array_equal(scales, (rmax.astype(np.float64) / 255.0).astype(np.float32))
    nz = np.nonzero(deg > 0)[0]
    cmax = np.zeros(g.n, np.int64)
    np.maximum.at(cmax, rows, codes.astype(np.int64))
    assert np.all(cmax[nz] == 255) and codes.min() >= 1
    s = scales[rows].astype(np.float64)
    ratio = g.h.astype(np.float64) / s
    slack = ratio * 2.0 ** -22  # the FP32 quotient h / s_v may sit this far from the exact one
    un = ratio >= 0.5 + slack
    assert np.all(np.abs(codes[un] - ratio[un]) <= 0.5 + slack[un])
    assert np.all(codes[~un] == 1)
    np.testing.assert_array_equal(hq, (codes.astype(np.float64) * s).astype(np.float32))
    assert np.all(np.abs(hq[un].astype(np.float64) - g.h[un]) <= (0.5 + slack[un]) * s[un] + hq[un] * 2.0 ** -23)


def test_quantize_scale_is_per_row():
    """Multiplying one row's weights by 1000 leaves every other row's codes
    and scale unchanged, and that row's codes too (its scale grows 1000-fold
    up to rounding)."""
    g = synth.rmat(10, 8, seed=2)
    g.h = synth.edge_weights(g, "lognormal", 1.0, seed=3)
    c, s, _ = oracle.quantize_weights(g)
    deg = np.diff(g.offsets)
    v = int(np.argmax(deg))
    h2 = g.h.copy()
    h2[g.offsets[v]:g.offsets[v + 1]] *= np.float32(1024.0)
    c2, s2, _ = oracle.quantize_weights(synth.Csr(g.offsets, g.cols, h2))
    np.testing.assert_array_equal(c2, c)
    other = np.arange(g.n) != v
    np.testing.assert_array_equal(s2[other], s[other])
    assert s2[v] == s[v] * 1024.0


def test_quantize_commutes_with_power_of_two_scaling():
    """Scaling every weight by 2^k scales every s_v by 2^k exactly and keeps the codes."""
    g = synth.rmat(10, 8, seed=2)
    g.h = synth.edge_weights(g, "lognormal", 1.0, seed=3)
    c, s, _ = oracle.quantize_weights(g)
    for k in (-3, 5):
        ck, sk, _ = oracle.quantize_weights(synth.Csr(g.offsets, g.cols, g.h * np.float32(2.0 ** k)))
        np.testing.assert_array_equal(sk, s * np.float32(2.0 ** k))
        np.testing.assert_array_equal(ck, c)


def test_quantized_integer_weights_leave_walks_unchanged():
    """Integer weights whose every row has maximum 255 are their own codes, so
    exact-mode walks over the dequantized weights equal those over the
    originals."""
    g = synth.rmat(10, 8, seed=4)
    rng = np.random.default_rng(1)
    w = synth.edge_weights(g, "uniform01", seed=5)
    h = np.ceil(w * 255.0).astype(np.float32)
    for v in range(g.n):
        if g.offsets[v + 1] > g.offsets[v]:
            h[g.offsets[v] + int(np.argmax(h[g.offsets[v]:g.offsets[v + 1]]))] = 255.0
    gi = synth.Csr(g.offsets, g.cols, h)
    _, s, hq = oracle.quantize_weights(gi)
    assert np.all(s[np.diff(g.offsets) > 0] == 1.0) and np.array_equal(hq, h)
    starts = rng.integers(0, g.n, 500).astype(np.int32)
    a, _ = oracle.walk(gi, starts, 12, "node2vec", 2.0, 0.5, seed=8)
    b, _ = oracle.walk(synth.Csr(g.offsets, g.cols, hq), starts, 12, "node2vec", 2.0, 0.5, seed=8)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("algo,p,q", [("node2vec", 2.0, 0.5), ("node2vec", 0.25, 4.0), ("node2vec", 4.0, 0.25),
                                      ("metapath", 1, 1), ("weighted", 1, 1), ("pagerank2", 1, 1)])
def test_bound_dominates_every_weight(algo, p, q):
    """eRJS is exact only if B >= max w~ (Sec. 3.3 proof): check on every
    (v, v') state of a graph."""
    g = synth.random_graph(40, 0.2, seed=3, weighted=True, nlabels=5)
    hmax, hsum = oracle.node_stats(g)
    schema = [0, 1, 2, 3, 4]
    for v in range(g.n):
        prevs = [-1] + list(g.cols[g.offsets[v]:g.offsets[v + 1]])
        for vp in prevs:
            for step in ([0] if vp < 0 else [1, 2]):
                wt = oracle.transition_weights(g, v, int(vp), step, algo, p, q, schema)
                dv = int(g.offsets[v + 1] - g.offsets[v])
                dp = int(g.offsets[vp + 1] - g.offsets[vp]) if vp >= 0 else 1
                _, B, _ = oracle.step_plan(float(hmax[v]), float(hsum[v]), vp >= 0, algo, p, q, 4.0, dv=dv, dprev=dp)
                if len(wt):
                    assert wt.max() <= B


def test_cost_model_hand_made():
    """Eq. (runtime): eRJS iff r*B < sum-hat."""
    # weighted: B = h_MAX, sum-hat = h_SUM
    assert oracle.step_plan(1.0, 10.0, True, "weighted", r=4.0)[0] == oracle.MODE_RJS
    assert oracle.step_plan(1.0, 3.0, True, "weighted", r=4.0)[0] == oracle.MODE_RVS
    assert oracle.step_plan(1.0, 4.0, True, "weighted", r=4.0)[0] == oracle.MODE_RVS  # strict <
    # metapath: sum-hat = h_SUM * (1 + 0) / 2
    m, B, S = oracle.step_plan(2.0, 20.0, True, "metapath", r=4.0)
    assert (B, S) == (2.0, 10.0) and m == oracle.MODE_RJS
    m, B, S = oracle.step_plan(2.0, 15.0, True, "metapath", r=4.0)
    assert m == oracle.MODE_RVS
    # node2vec p=2, q=0.5: max w = 2, mean w = (0.5 + 1 + 2) / 3
    m, B, S = oracle.step_plan(1.0, 30.0, True, "node2vec", 2.0, 0.5, r=4.0)
    assert B == 2.0 and S == pytest.approx(30.0 * 3.5 / 3, rel=1e-7)
    assert m == oracle.MODE_RJS
    m, B, S = oracle.step_plan(1.0, 6.0, True, "node2vec", 2.0, 0.5, r=4.0)
    assert m == oracle.MODE_RVS
    # hop 0 of node2vec: first-order (B = h_MAX, sum-hat = h_SUM)
    m, B, S = oracle.step_plan(1.0, 6.0, False, "node2vec", 2.0, 0.5, r=4.0)
    assert (B, S, m) == (1.0, 6.0, oracle.MODE_RJS)
