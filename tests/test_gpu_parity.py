"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Exact mode must equal the oracle's walks bit for bit; the fast modes (eRJS,
eRVS with and without jumps, cost-model auto) must reproduce the oracle's
exact per-step distributions (per state: chi-square p > 0.01 and TV < 2e-3
over 25 merged bins at >= 2e6 draws, with one redraw on fresh seeds, see
statcheck.assert_follows) and keep the walk invariants."""
import numpy as np
import pytest

import oracle
from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth
from bruteforce import bf_paths, merged_chisquare
from statcheck import assert_follows, assert_pvalue_follows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALGOS = [("node2vec", 2.0, 0.5, None), ("node2vec", 0.25, 4.0, None), ("node2vec", 4.0, 0.25, None),
         ("node2vec", 1.0, 1.0, None), ("metapath", 1.0, 1.0, [0, 1, 2, 3, 4]), ("weighted", 1.0, 1.0, None),
         ("pagerank2", 1.0, 1.0, None)]


@pytest.fixture(scope="module")
def small():
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    yield g, G
    G.close()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ------------------------------------------------------------ exact mode
@pytest.mark.parametrize("algo,p,q,schema", ALGOS)
def test_exact_mode_bit_identical_small(small, algo, p, q, schema):
    g, G = small
    starts = np.arange(g.n, dtype=np.int32)
    out = G.walk(_cuda(starts), 20, algo, p=p, q=q, schema=schema, mode="exact", seed=42).cpu().numpy()
    ref, hops = oracle.walk(g, starts, 20, algo, p, q, schema, seed=42)
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"
    G.check()


@pytest.mark.parametrize("W,L,base", [(4093, 20, 0), (31, 7, 1000), (1, 1, 5), (257, 0, 0), (0, 5, 0)])
def test_exact_mode_ragged_sizes(small, W, L, base):
    g, G = small
    starts = synth.random_starts(g.n, W, seed=W + 1)
    if W == 0:
        out = torch.empty((0, L + 1), dtype=torch.int32, device="cuda")
        G.walk(_cuda(starts), L, "node2vec", p=2.0, q=0.5, mode="exact", out=out)
        return
    out = G.walk(_cuda(starts), L, "node2vec", p=2.0, q=0.5, mode="exact", seed=7, walker_base=base).cpu().numpy()
    ref, _ = oracle.walk(g, starts, L, "node2vec", 2.0, 0.5, seed=7, walker_base=base)
    assert np.array_equal(out, ref)


def test_exact_mode_unweighted(small):
    g, G = small
    starts = np.arange(g.n, dtype=np.int32)
    out = G.walk(_cuda(starts), 15, "node2vec", p=1.0, q=0.5, mode="exact", seed=3,
                 flags=fw.FLAG_UNWEIGHTED).cpu().numpy()
    ref, _ = oracle.walk(synth.Csr(g.offsets, g.cols), starts, 15, "node2vec", 1.0, 0.5, seed=3)
    assert np.array_equal(out, ref)
    # a graph created without weights gives the same walks
    G2 = fw.Graph(offsets=g.offsets, cols=g.cols)
    out2 = G2.walk(_cuda(starts), 15, "node2vec", p=1.0, q=0.5, mode="exact", seed=3).cpu().numpy()
    G2.close()
    assert np.array_equal(out2, ref)


# ------------------------------------------------- eRJS with the paper's bound
RJS_ALGOS = [("node2vec", 2.0, 0.5), ("node2vec", 0.25, 4.0), ("node2vec", 4.0, 0.25), ("node2vec", 1.0, 1.0),
             ("weighted", 1.0, 1.0), ("pagerank2", 1.0, 1.0)]
NO_HANDOFF = 1 << 30  # a trial budget no step reaches: every hop stays in eRJS


@pytest.mark.parametrize("algo,p,q", RJS_ALGOS)
@pytest.mark.parametrize("unweighted", [False, True])
def test_plain_rjs_walks_bit_identical_to_oracle_rjs(small, algo, p, q, unweighted):
    """eRJS with the single bound B = max(w) h_MAX[v] and the uniform proposal
    of Sec. 3.3 (FW_FLAG_PLAIN_RJS), every step kept in eRJS: the kernel
    draws the oracle's proposals and uniforms trial by trial, so its rows
    equal the oracle's rejection-sampled walks bit for bit (the squeeze tests,
    the Bloom pre-check and the row search only shorten the work)."""
    g, G = small
    W, L = 4093, 20
    starts = synth.random_starts(g.n, W, seed=17)
    flags = fw.FLAG_PLAIN_RJS | (fw.FLAG_UNWEIGHTED if unweighted else 0)
    out = G.walk(_cuda(starts), L, algo, p=p, q=q, mode="rjs", flags=flags, rjs_cap=NO_HANDOFF, seed=42,
                 walker_base=11).cpu().numpy()
    ref, _ = oracle.walk_rjs(synth.Csr(g.offsets, g.cols) if unweighted else g, starts, L, algo, p, q, seed=42,
                             walker_base=11)
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"


@pytest.mark.parametrize("algo,p,q,schema", [("weighted", 1.0, 1.0, None), ("node2vec", 1.0, 1.0, None),
                                             ("node2vec", 4.0, 0.25, None), ("node2vec", 2.0, 0.5, None),
                                             ("metapath", 1.0, 1.0, [0, 1, 2, 3, 4]), ("metapath", 1.0, 1.0, [3])])
@pytest.mark.parametrize("weights", ["uniform01", "lognormal"])
def test_class_envelope_rjs_walks_bit_identical_to_oracle_rjs(algo, p, q, schema, weights):
    """eRJS under the weight-class envelopes (the default for weighted graphs;
    these settings use no split proposal; metapath samples inside the
    label-grouped view), every step kept in eRJS: the class-ordered records,
    the packed class counts and the slot map give the oracle's proposals
    trial by trial, so the rows are bit-identical."""
    g = synth.workload_graph("small")
    if weights == "lognormal":
        g.h = synth.edge_weights(g, "lognormal", 1.5, seed=13)
    G = fw.Graph(g)
    W, L = 4093, 20
    starts = synth.random_starts(g.n, W, seed=23)
    out = G.walk(_cuda(starts), L, algo, p=p, q=q, schema=schema, mode="rjs", rjs_cap=NO_HANDOFF, seed=42,
                 walker_base=5).cpu().numpy()
    G.close()
    ref, _ = oracle.walk_rjs(g, starts, L, algo, p, q, schema, seed=42, walker_base=5, envelope="classes")
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"


def test_graph_from_device_arrays(small):
    g, _ = small
    G = fw.Graph(offsets=_cuda(g.offsets), cols=_cuda(g.cols), weights=_cuda(g.h), labels=_cuda(g.labels))
    starts = np.arange(0, g.n, 3, dtype=np.int32)
    out = G.walk(_cuda(starts), 10, "metapath", schema=[0, 1, 2, 3, 4], mode="exact", seed=9).cpu().numpy()
    ref, _ = oracle.walk(g, starts, 10, "metapath", schema=[0, 1, 2, 3, 4], seed=9)
    assert np.array_equal(out, ref)
    G.close()


def test_device_csr_validation():
    g = synth.from_edges(4, [(0, 1), (1, 2), (2, 3)])
    cols = g.cols.copy()
    cols[1], cols[2] = cols[2], cols[1]  # row 1 no longer sorted
    with pytest.raises(fw.FlexiWalkError) as e:
        fw.Graph(offsets=_cuda(g.offsets), cols=_cuda(cols))
    assert e.value.status == -2
    bad_w = np.ones(g.e, np.float32)
    bad_w[0] = 0.0
    with pytest.raises(fw.FlexiWalkError) as e:
        fw.Graph(offsets=_cuda(g.offsets), cols=_cuda(g.cols), weights=_cuda(bad_w))
    assert e.value.status == -2


def test_bad_start_is_reported(small):
    g, G = small
    starts = np.array([0, g.n + 5, 1], dtype=np.int32)
    out = G.walk(_cuda(starts), 4, "weighted", mode="exact").cpu().numpy()
    assert np.all(out[1] == -1)
    with pytest.raises(fw.FlexiWalkError) as e:
        G.check()
    assert e.value.status == -6
    G.check()  # cleared


def test_walk_host_matches_device(small):
    g, G = small
    starts = np.arange(g.n, dtype=np.int32)
    a = G.walk_host(starts, 12, "node2vec", p=2.0, q=0.5, mode="auto", seed=11)
    b = G.walk(_cuda(starts), 12, "node2vec", p=2.0, q=0.5, mode="auto", seed=11).cpu().numpy()
    assert np.array_equal(a, b)


# ------------------------------------------------------------ preprocessing / plan
def test_label_stats_parity(small):
    g, G = small
    st = G.label_stats().cpu().numpy()
    lmax, lsum = oracle.label_stats(g)
    assert np.array_equal(st[:, :, 0], lmax)
    np.testing.assert_allclose(st[:, :, 1], lsum, rtol=2e-6, atol=1e-6)


def test_node_stats_parity(small):
    g, G = small
    hmax, hsum = G.node_stats()
    rmax, rsum = oracle.node_stats(g)
    assert np.array_equal(hmax.cpu().numpy(), rmax)
    np.testing.assert_allclose(hsum.cpu().numpy(), rsum, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("algo,p,q", [("node2vec", 2.0, 0.5), ("node2vec", 0.25, 4.0), ("metapath", 1, 1),
                                      ("weighted", 1, 1), ("pagerank2", 1, 1)])
def test_step_plan_parity(small, algo, p, q):
    g, G = small
    deg = g.degrees()
    v = np.arange(g.n, dtype=np.int32)
    vp = np.where((v % 2 == 1) & (deg > 0), g.cols[np.minimum(g.offsets[:-1], g.e - 1)], -1).astype(np.int32)
    r = 4.0
    m, B, S = G.step_plan(_cuda(v), _cuda(vp), algo, p=p, q=q, schema=[0, 1, 2, 3, 4], cost_ratio=r)
    m, B, S = m.cpu().numpy(), B.cpu().numpy(), S.cpu().numpy()
    rmax, rsum = oracle.node_stats(g)
    ghmax, ghsum = [t.cpu().numpy() for t in G.node_stats()]
    for i in range(g.n):
        dv, dp = int(deg[i]), (int(deg[vp[i]]) if vp[i] >= 0 else 1)
        if algo == "pagerank2" and vp[i] >= 0 and dv == 0:
            continue
        om, oB, oS = oracle.step_plan(float(ghmax[i]), float(ghsum[i]), vp[i] >= 0, algo, p, q, r, dv=dv, dprev=dp)
        assert B[i] == oB and S[i] == oS and m[i] == om, i
        # and against the oracle's own fp64 sums, away from the decision boundary
        om2, oB2, oS2 = oracle.step_plan(float(rmax[i]), float(rsum[i]), vp[i] >= 0, algo, p, q, r, dv=dv, dprev=dp)
        assert oB2 == B[i]
        if abs(r * oB2 - oS2) > 1e-4 * max(1.0, oS2):
            assert om2 == m[i]


# ------------------------------------------------------------ fast-mode distributions
def _states(g):
    """(v, v_prev, step) states covering degrees 1, 2, ~4, ~32, ~300, max,
    each with no v', with the highest-degree neighbour as v', and (d > 4)
    with the lowest-degree neighbour as v' (short N(v'): second-order
    PageRank then splits the common neighbours off)."""
    deg = g.degrees()
    out = []
    for target in [1, 2, 4, 32, 300, int(deg.max())]:
        v = int(np.argmin(np.abs(deg - target) + (deg == 0) * 10**9))
        nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
        hub_prev = int(nb[np.argmax(deg[nb])])
        out.append((v, -1, 0))
        out.append((v, hub_prev, 1))
        if target > 4:
            out.append((v, int(nb[np.argmin(deg[nb])]), 1))
    return out


@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("rvs", 0), ("rvs", fw.FLAG_RVS_NOJUMP), ("auto", 0), ("random", 0),
                                        ("degree", 0)])
@pytest.mark.parametrize("algo,p,q,schema", [("node2vec", 2.0, 0.5, None), ("node2vec", 0.25, 4.0, None),
                                             ("node2vec", 2.0, 4.0, None),
                                             ("metapath", 1.0, 1.0, [0, 1, 2, 3, 4]), ("weighted", 1.0, 1.0, None),
                                             ("pagerank2", 1.0, 1.0, None)])
def test_fast_mode_distributions(small, mode, flags, algo, p, q, schema):
    g, G = small
    ndraws = 4_000_000
    for (v, vp, step) in _states(g):
        probs = oracle.transition_probs(g, v, vp, step, algo, p, q, schema)
        draw = lambda k: G.sample_hist(v, vp, step, algo, ndraws, p=p, q=q, schema=schema, mode=mode, flags=flags,
                                       seed=1234 + v + 7919 * k).cpu().numpy()
        if probs.sum() == 0:
            assert draw(0).sum() == 0
            continue
        assert_follows(draw, probs, (algo, p, q, mode, flags, v, vp, step), ndraws)


@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("rvs", 0), ("rvs", fw.FLAG_RVS_NOJUMP), ("auto", 0),
                                        ("rjs", fw.FLAG_NO_GROUPS), ("rvs", fw.FLAG_NO_GROUPS)])
def test_metapath_every_label_distributions(small, mode, flags):
    """Metapath inside each label's segment of the label-grouped view (and
    over whole rows with FW_FLAG_NO_GROUPS): for every required label 0..4 at
    the states of _states, the draws follow the oracle's probabilities."""
    g, G = small
    ndraws = 2_000_000
    for (v, vp, step) in _states(g)[::2]:
        for lab in range(5):
            probs = oracle.transition_probs(g, v, -1, step, "metapath", schema=[lab])
            draw = lambda k: G.sample_hist(v, -1, step, "metapath", ndraws, schema=[lab], mode=mode, flags=flags,
                                           seed=77 + v + lab + 7919 * k).cpu().numpy()
            if probs.sum() == 0:
                assert draw(0).sum() == 0
                continue
            assert_follows(draw, probs, ("metapath", mode, flags, v, lab), ndraws)


@pytest.mark.parametrize("algo,p,q", [("weighted", 1.0, 1.0), ("node2vec", 0.25, 4.0), ("node2vec", 4.0, 0.25),
                                      ("node2vec", 2.0, 4.0), ("pagerank2", 1.0, 1.0)])
def test_weight_class_envelopes_with_skewed_weights(algo, p, q):
    """eRJS with the weight-class envelope (default) and with the paper's
    uniform proposal (FW_FLAG_PLAIN_RJS) on lognormal(0, 1.5) weights, where
    every class is well populated and the split proposals' mixture weights
    depend on the class counts: both follow the oracle's probabilities."""
    g = synth.workload_graph("small")
    g.h = synth.edge_weights(g, "lognormal", 1.5, seed=13)
    G = fw.Graph(g)
    for (v, vp, step) in _states(g):
        probs = oracle.transition_probs(g, v, vp, step, algo, p, q)
        for flags in (0, fw.FLAG_PLAIN_RJS):
            draw = lambda k: G.sample_hist(v, vp, step, algo, 2_000_000, p=p, q=q, mode="rjs", flags=flags,
                                           seed=31 + v + flags + 7919 * k).cpu().numpy()
            assert_follows(draw, probs, (algo, p, q, flags, v, vp), 2_000_000)
    G.close()


@pytest.mark.parametrize("algo,p,q", [("node2vec", 0.25, 4.0), ("node2vec", 4.0, 0.25), ("pagerank2", 1.0, 1.0),
                                      ("weighted", 1.0, 1.0)])
@pytest.mark.parametrize("how", ["flag", "no-weights"])
def test_unweighted_fast_mode_distributions(small, algo, p, q, how):
    """h = 1, either by FW_FLAG_UNWEIGHTED on the weighted graph or on a
    graph created without weights (no weight classes, no class-ordered
    records): eRJS and the cost model against the oracle's unweighted
    probabilities."""
    g, G = small
    gu = synth.Csr(g.offsets, g.cols)
    if how == "flag":
        Gx, flags = G, fw.FLAG_UNWEIGHTED
    else:
        Gx, flags = fw.Graph(gu), 0
    for (v, vp, step) in _states(g)[::2]:
        probs = oracle.transition_probs(gu, v, vp, step, algo, p, q)
        for mode in ("rjs", "auto"):
            draw = lambda k: Gx.sample_hist(v, vp, step, algo, 2_000_000, p=p, q=q, mode=mode, flags=flags,
                                            seed=51 + v + 7919 * k).cpu().numpy()
            assert_follows(draw, probs, (algo, p, q, how, mode, v, vp), 2_000_000)
    if how != "flag":
        Gx.close()


def test_worked_example_distribution():
    """Fig. 2: weights {3,2,4,1} -> {0.3,0.2,0.4,0.1} for every mode."""
    g = synth.from_edges(5, [(0, 1), (0, 2), (0, 3), (0, 4)], h=[3.0, 2.0, 4.0, 1.0])
    G = fw.Graph(g)
    for mode in ["rjs", "rvs", "auto", "exact"]:
        counts = G.sample_hist(0, -1, 0, "weighted", 4_000_000, mode=mode, seed=99).cpu().numpy()
        f = counts / counts.sum()
        assert np.abs(f - [0.3, 0.2, 0.4, 0.1]).max() < 1.5e-3, (mode, f)
    G.close()


def test_rjs_bound_invariance(small):
    """Sec. 3.3: the accepted distribution does not depend on the bound; a
    10x looser cost ratio only changes the choice, and a trial cap of 1
    (almost every step handed to eRVS) keeps the distribution too."""
    g, G = small
    deg = g.degrees()
    v = int(np.argmax(deg))
    probs = oracle.transition_probs(g, v, -1, 0, "weighted")
    for cap in [1, 2, 1000]:
        draw = lambda k: G.sample_hist(v, -1, 0, "weighted", 4_000_000, mode="rjs", rjs_cap=cap,
                                       seed=5 + 7919 * k).cpu().numpy()
        assert_follows(draw, probs, ("rjs cap", cap), 4_000_000)


def test_dead_end_states(small):
    g, G = small
    deg = g.degrees()
    iso = int(np.argmax(deg == 0))
    for mode in ["rjs", "rvs", "auto", "exact"]:
        c = G.sample_hist(iso, -1, 0, "weighted", 1000, mode=mode).cpu().numpy()
        assert c.sum() == 0
    # metapath state with no matching label: every mode ends the walk
    for v in range(g.n):
        if 0 < deg[v] <= 6 and oracle.transition_probs(g, v, -1, 0, "metapath", schema=[4]).sum() == 0:
            for mode in ["rjs", "rvs", "auto", "exact"]:
                c = G.sample_hist(v, -1, 0, "metapath", 5000, schema=[4], mode=mode).cpu().numpy()
                assert c.sum() == 0
            break


# ------------------------------------------------------------ invariants / determinism
def _invariants(g, starts, out, algo, schema=None, check_dead=True, p=1.0, q=1.0):
    L = out.shape[1] - 1
    assert np.array_equal(out[:, 0], starts)
    n = np.int64(g.n)
    keys = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets)) * n + g.cols
    alive = out[:, 1:] >= 0
    # -1 only as a suffix
    assert np.all(alive[:, :-1] | ~alive[:, 1:])
    v = out[:, :-1].astype(np.int64)
    u = out[:, 1:].astype(np.int64)
    q_ = (v * n + u)[alive]
    pos = np.searchsorted(keys, q_)
    assert np.all(pos < len(keys)) and np.all(keys[np.minimum(pos, len(keys) - 1)] == q_), "hop is not an edge"
    if algo == "metapath":
        lab = g.labels[pos]
        hop = np.broadcast_to(np.arange(L), alive.shape)[alive]
        assert np.all(lab == np.asarray(schema)[hop % len(schema)])
    if check_dead:
        dead = np.nonzero(~alive.all(axis=1))[0][:200]
        for r in dead:
            j = int(np.argmin(alive[r]))
            prev = int(out[r, j - 1]) if j >= 1 else -1
            assert oracle.transition_probs(g, int(out[r, j]), prev, j, algo, p, q, schema).sum() == 0


@pytest.mark.parametrize("algo,p,q,schema", ALGOS)
@pytest.mark.parametrize("mode", ["auto", "rjs", "rvs"])
def test_fast_walk_invariants_small(small, algo, p, q, schema, mode):
    g, G = small
    starts = np.arange(g.n, dtype=np.int32)
    out = G.walk(_cuda(starts), 20, algo, p=p, q=q, schema=schema, mode=mode, seed=5).cpu().numpy()
    _invariants(g, starts, out, algo, schema, p=p, q=q)
    again = G.walk(_cuda(starts), 20, algo, p=p, q=q, schema=schema, mode=mode, seed=5).cpu().numpy()
    assert np.array_equal(out, again), "fast modes must be deterministic for a fixed seed"


def test_counters(small):
    g, G = small
    starts = np.arange(g.n, dtype=np.int32)
    G.reset_counters()
    out = G.walk(_cuda(starts), 20, "node2vec", p=2.0, q=0.5, flags=fw.FLAG_COUNTERS, seed=5)
    c = G.counters()
    o = out.cpu().numpy()
    assert c["hops"] == int((o[:, 1:] >= 0).sum())
    assert c["rjs_steps"] + c["rvs_steps"] == c["hops"]
    assert c["dead_ends"] == int((o[:, -1] < 0).sum())
    plain = G.walk(_cuda(starts), 20, "node2vec", p=2.0, q=0.5, seed=5).cpu().numpy()
    assert np.array_equal(o, plain), "counting build must not change the walks"


@pytest.mark.parametrize("algo,p,q,envelope", [("node2vec", 2.0, 0.5, "single"), ("node2vec", 0.25, 4.0, "single"),
                                               ("node2vec", 4.0, 0.25, "single"), ("weighted", 1.0, 1.0, "single"),
                                               ("node2vec", 1.0, 1.0, "classes"), ("node2vec", 4.0, 0.25, "classes"),
                                               ("node2vec", 2.0, 0.5, "classes"), ("weighted", 1.0, 1.0, "classes")])
def test_counters_match_oracle_trials_and_byte_model(small, algo, p, q, envelope):
    """The counting build's trial counter equals the oracle's count of
    rejection trials (void Lemire draws included) on walks that are
    bit-identical to the oracle's, and its byte counter equals the byte
    model recomputed here from those trials: 32 B for each walker's first
    node record (later ones ride in the accepted trial's edge record), 32 B
    per trial (one edge record; a trial whose two Lemire draws both fall in
    the rejection zone reads nothing, about 1e-12 per trial at these
    degrees), 32 B per membership probe (the GPU's probe count) and 4 B per
    row entry written."""
    g, G = small
    W, L = 4093, 20
    starts = synth.random_starts(g.n, W, seed=17)
    flags = fw.FLAG_COUNTERS | (fw.FLAG_PLAIN_RJS if envelope == "single" else 0)
    G.reset_counters()
    out = G.walk(_cuda(starts), L, algo, p=p, q=q, mode="rjs", flags=flags, rjs_cap=NO_HANDOFF, seed=42,
                 walker_base=11).cpu().numpy()
    c = G.counters()
    ref, hops, trials = oracle.walk_rjs(g, starts, L, algo, p, q, seed=42, walker_base=11, envelope=envelope,
                                        return_trials=True)
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"
    assert c["hops"] == hops
    assert c["rjs_trials"] == trials, (c["rjs_trials"], trials)
    assert c["rvs_steps"] == 0 and c["handoffs"] == 0 and c["rjs_steps"] == hops
    if algo == "weighted" or (p == 1.0 and q == 1.0):
        assert c["probes"] == 0
    model = 32 * W + 32 * trials + 32 * c["probes"] + 4 * hops
    assert c["bytes"] == model, (c["bytes"], model)


# ------------------------------------------------------------ whole-walk distributions
def _asymmetric(g, seed):
    """Same structure, an independent weight on each direction of every edge."""
    rng = np.random.default_rng(seed)
    return synth.Csr(g.offsets, g.cols, (1.0 - rng.random(g.e)).astype(np.float32), g.labels)


WALK_CASES = [("node2vec", 0.25, 4.0, None), ("node2vec", 2.0, 0.5, None), ("node2vec", 4.0, 0.25, None),
              ("node2vec", 2.0, 4.0, None),
              ("metapath", 1.0, 1.0, [0, 1, 2]), ("weighted", 1.0, 1.0, None), ("pagerank2", 1.0, 1.0, None)]


@pytest.mark.parametrize("graph", ["sparse", "sparse-asym", "dense"])
@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("rjs", fw.FLAG_PLAIN_RJS), ("rvs", 0), ("auto", 0),
                                        ("auto", fw.FLAG_PAPER_SUM), ("auto", fw.FLAG_NO_GROUPS)])
@pytest.mark.parametrize("algo,p,q,schema", WALK_CASES)
def test_fast_walk_path_distribution(graph, mode, flags, algo, p, q, schema):
    """GPU walks from one start, many walker ids: frequencies of whole paths
    match brute-force path probabilities (chi-square, merged bins).  This
    covers the walk-only paths: edge records carried between steps, the
    split return edge fed by the arriving edge (symmetric weights) or by a
    search (asymmetric), and warp-level eRVS (dense graph)."""
    if graph == "dense":
        g = synth.random_graph(24, 0.85, seed=21, weighted=True, nlabels=3)
        L = 3
    else:
        g = synth.random_graph(8, 0.45, seed=11, weighted=True, nlabels=3)
        L = 4
        if graph == "sparse-asym":
            g = _asymmetric(g, 3)
    G = fw.Graph(g)
    assert G.info["symmetric"] == (0 if graph == "sparse-asym" else 1)
    W, start = 300_000, 0
    starts = torch.full((W,), start, dtype=torch.int32, device="cuda")
    bf = bf_paths(g, start, L, algo, p, q, schema)
    assert_pvalue_follows(lambda k: merged_chisquare(bf, G.walk(starts, L, algo, p=p, q=q, schema=schema, mode=mode,
                                                                 flags=flags, seed=17 + 7919 * k).cpu().numpy()),
                          (graph, algo, p, q, mode, flags))
    G.close()


@pytest.mark.parametrize("gamma", [0.2, 0.8])
@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("auto", 0), ("rjs", fw.FLAG_PLAIN_RJS)])
def test_pagerank2_common_neighbour_split_paths(gamma, mode, flags):
    """A hub whose leaves have short rows: stepping from a leaf v' onto the
    hub v gives w1 / w2 = 1 + gamma/(1-gamma) * d(v)/d(v') > 2, where eRJS
    splits the common neighbours off (FLAG_PLAIN_RJS: the plain bound).
    Whole 4-hop path frequencies against brute force."""
    edges = [(0, k) for k in range(1, 10)] + [(1, 2), (2, 3), (4, 5), (6, 7), (7, 8), (8, 9), (1, 10), (10, 11)]
    g = synth.from_edges(12, edges, h=[0.25 + 0.07 * i for i in range(len(edges))])
    G = fw.Graph(g)
    W, L = 400_000, 4
    bf = bf_paths(g, 1, L, "pagerank2", 1.0, 1.0, None, gamma=gamma)
    starts = torch.full((W,), 1, dtype=torch.int32, device="cuda")
    assert_pvalue_follows(lambda k: merged_chisquare(bf, G.walk(starts, L, "pagerank2", gamma=gamma, mode=mode,
                                                                 flags=flags, seed=29 + 7919 * k).cpu().numpy()),
                          ("pagerank2 split", gamma, mode, flags))
    G.close()
