"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: R-MAT s22 (4,194,304 walkers x 80 hops, node2vec) and R-MAT
s23 (metapath, 2M starts).  Exact mode and eRJS under the paper's single
bound: sampled blocks of rows against the oracle, which computes them walker
by walker.  Fast modes: invariants on sampled rows, and per-state
distributions at the largest hubs."""
import numpy as np
import pytest

import oracle
from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth
from statcheck import assert_follows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PQ = [(1.0, 1.0), (4.0, 0.25), (0.25, 4.0)]


@pytest.fixture(scope="module")
def s22():
    g = synth.workload_graph("s22")
    G = fw.Graph(g)
    yield g, G
    G.close()


def _blocks(n, nblocks, size, seed):
    rng = np.random.default_rng(seed)
    return sorted(int(x) for x in rng.choice(n // size, nblocks, replace=False) * size)


@pytest.mark.parametrize("p,q", PQ)
def test_exact_mode_full_s22_sampled_rows(s22, p, q):
    """All 4,194,304 walkers x 80 hops in exact mode; six contiguous 64-row
    blocks and a seeded random subset of 65,536 walkers (all 80 hops) equal
    the oracle's rows, which it computes walker by walker."""
    g, G = s22
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    out = G.walk(starts, 80, "node2vec", p=p, q=q, mode="exact", seed=42)
    for b in _blocks(g.n, 6, 64, seed=int(p * 100 + q)):
        sub = np.arange(b, b + 64, dtype=np.int32)
        ref, _ = oracle.walk(g, sub, 80, "node2vec", p, q, seed=42, walker_base=b)
        got = out[b:b + 64].cpu().numpy()
        assert np.array_equal(got, ref), f"block {b}: {(got != ref).any(axis=1).sum()} rows differ"
    sub = np.sort(np.random.default_rng(44).choice(g.n, 65_536, replace=False)).astype(np.int32)
    ref, _ = oracle.walk_ids(g, sub, sub.astype(np.uint32), 80, "node2vec", p, q, seed=42)
    got = out[torch.from_numpy(sub).cuda().long()].cpu().numpy()
    assert np.array_equal(got, ref), f"{(got != ref).any(axis=1).sum()} of 65,536 sampled rows differ"


@pytest.mark.parametrize("p,q,envelope", [(1.0, 1.0, "single"), (4.0, 0.25, "single"), (0.25, 4.0, "single"),
                                          (1.0, 1.0, "classes"), (4.0, 0.25, "classes")])
def test_rjs_full_s22_sampled_rows(s22, p, q, envelope):
    """The bench's launch with every hop in eRJS (no hand-off), under the
    paper's single bound (FW_FLAG_PLAIN_RJS) and under the weight-class
    envelope (the default; (0.25, 4) would add split proposals): sampled
    64-row blocks equal the oracle's rejection-sampled walks bit for bit."""
    g, G = s22
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    flags = fw.FLAG_PLAIN_RJS if envelope == "single" else 0
    out = G.walk(starts, 80, "node2vec", p=p, q=q, mode="rjs", flags=flags, rjs_cap=1 << 30, seed=42)
    for b in _blocks(g.n, 4, 64, seed=int(p * 100 + q) + 1):
        sub = np.arange(b, b + 64, dtype=np.int32)
        ref, _ = oracle.walk_rjs(g, sub, 80, "node2vec", p, q, seed=42, walker_base=b, envelope=envelope)
        got = out[b:b + 64].cpu().numpy()
        assert np.array_equal(got, ref), f"block {b}: {(got != ref).any(axis=1).sum()} rows differ"


def _edge_keys(g):
    return np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets)) * np.int64(g.n) + g.cols


@pytest.mark.parametrize("p,q", PQ)
def test_fast_mode_full_s22_invariants(s22, p, q):
    """The bench's walk (cost-model mode, one walker per node, 80 hops):
    every hop of 100,000 sampled rows is an edge, -1 only as a suffix, and
    only isolated start nodes end early (h > 0, so node2vec has no other
    dead end)."""
    g, G = s22
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    out = G.walk(starts, 80, "node2vec", p=p, q=q, mode="auto", seed=42)
    rows = np.sort(np.random.default_rng(3).choice(g.n, 100_000, replace=False))
    o = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(o[:, 0], rows)
    alive = o[:, 1:] >= 0
    assert np.all(alive[:, :-1] | ~alive[:, 1:])
    deg = g.degrees()
    assert np.array_equal(~alive[:, 0], deg[rows] == 0)
    assert np.all(alive[deg[rows] > 0])
    keys = _edge_keys(g)
    q_ = (o[:, :-1].astype(np.int64) * np.int64(g.n) + o[:, 1:])[alive]
    pos = np.searchsorted(keys, q_)
    assert np.all(keys[np.minimum(pos, len(keys) - 1)] == q_)


@pytest.mark.parametrize("p,q", PQ)
def test_bench_walk_identical_without_row_filters(s22, p, q):
    """The bench's launch with and without the Bloom pre-check: equal rows."""
    g, G = s22
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    a = G.walk(starts, 80, "node2vec", p=p, q=q, mode="auto", seed=42)
    b = G.walk(starts, 80, "node2vec", p=p, q=q, mode="auto", seed=42, flags=fw.FLAG_NO_BLOOM)
    assert torch.equal(a, b)


@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("auto", 0), ("rvs", 0), ("rvs", fw.FLAG_RVS_NOJUMP)])
def test_hub_distributions_s22(s22, mode, flags):
    """The largest hub (d = 162,957): weighted and node2vec from a low-degree
    v', and node2vec at a low-degree node whose v' is the hub, 4e6 draws in
    every mode (the jump-less eRVS scans the whole hub row per draw)."""
    g, G = s22
    ndraws = 4_000_000
    deg = g.degrees()
    hub = int(np.argmax(deg))
    nb = g.cols[g.offsets[hub]:g.offsets[hub + 1]]
    small_prev = int(nb[np.argmin(deg[nb])])
    states = [(hub, -1, 0, "weighted", 1.0, 1.0), (hub, small_prev, 1, "node2vec", 2.0, 0.5),
              (hub, small_prev, 1, "node2vec", 0.25, 4.0), (small_prev, hub, 1, "node2vec", 4.0, 0.25),
              (hub, small_prev, 1, "pagerank2", 1.0, 1.0), (small_prev, hub, 1, "pagerank2", 1.0, 1.0)]
    for (v, vp, step, algo, p, q) in states:
        probs = oracle.transition_probs(g, v, vp, step, algo, p, q)
        draw = lambda k: G.sample_hist(v, vp, step, algo, ndraws, p=p, q=q, mode=mode, flags=flags,
                                       seed=77 + v + 7919 * k).cpu().numpy()
        assert_follows(draw, probs, (mode, flags, v, vp, algo, p, q), ndraws)


@pytest.mark.parametrize("algo,p,q,flags", [("weighted", 1.0, 1.0, 0), ("node2vec", 2.0, 0.5, 0),
                                             ("node2vec", 0.25, 4.0, fw.FLAG_RVS_NOJUMP)])
def test_hub_steps_same_rows_shared_or_alone(s22, algo, p, q, flags):
    """eRVS steps at the largest hub (d = 162,957, above the 32,768-entry threshold)
    are scanned in fixed chunks from a phase-1 reference.  In a small launch
    with forced eRVS, idle warps of a block help scan them (or the owning
    warp scans alone when the block's task slots are taken); with
    FW_FLAG_NO_HUB_SHARE every step stays on its warp, as in big launches.
    4,096 walkers starting at the hub give the same rows either way, and the
    first 16 walked one per launch give the same rows again."""
    g, G = s22
    hub = int(np.argmax(g.degrees()))
    W, L = 4096, 3
    starts = torch.full((W,), hub, dtype=torch.int32, device="cuda")
    kw = dict(p=p, q=q, mode="rvs", seed=91)
    shared = G.walk(starts, L, algo, flags=flags, **kw).cpu().numpy()
    alone = G.walk(starts, L, algo, flags=flags | fw.FLAG_NO_HUB_SHARE, **kw).cpu().numpy()
    assert np.all(shared[:, 1] >= 0)
    assert np.array_equal(shared, alone), f"{(shared != alone).any(axis=1).sum()} rows differ"
    for i in range(16):
        one = G.walk(starts[i:i + 1], L, algo, walker_base=i, flags=flags, **kw).cpu().numpy()
        assert np.array_equal(one[0], shared[i]), i
    G.check()


def test_hub_sharing_shortens_small_hub_walks(s22):
    """32 walkers from the largest hub, 10 hops of forced eRVS: with the
    block's idle warps helping, the launch takes well under the time of
    every hub step on its own warp (same rows)."""
    g, G = s22
    hub = int(np.argmax(g.degrees()))
    starts = torch.full((32,), hub, dtype=torch.int32, device="cuda")

    def timed(flags):
        out = G.walk(starts, 10, "node2vec", mode="rvs", seed=5, flags=flags)
        ts = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            G.walk(starts, 10, "node2vec", mode="rvs", seed=5, flags=flags, out=out)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts), out.cpu().numpy()

    t_shared, rows_shared = timed(0)
    t_alone, rows_alone = timed(fw.FLAG_NO_HUB_SHARE)
    assert np.array_equal(rows_shared, rows_alone)
    assert t_shared < 0.6 * t_alone, (t_shared, t_alone)


@pytest.fixture(scope="module")
def s23():
    g = synth.workload_graph("s23_meta")
    G = fw.Graph(g)
    yield g, G
    G.close()


@pytest.mark.parametrize("mode,flags,hub_too", [("rjs", 0, True), ("auto", 0, True), ("rjs", fw.FLAG_NO_GROUPS, True),
                                                 ("rvs", 0, False)])
def test_hub_label_distributions_s23(s23, mode, flags, hub_too):
    """Metapath at the largest hub of R-MAT s23 (lognormal(0,1) weights, where
    the five weight classes of a label segment matter most) and at a node of
    degree ~1000, for every required label: the label-grouped sampler (and the
    whole-row sampler) against the oracle, 4e6 draws.  eRVS-only runs at the
    smaller node alone (a hub scan per draw would take minutes)."""
    g, G = s23
    deg = g.degrees()
    hub = int(np.argmax(deg))
    mid = int(np.argmin(np.abs(deg - 1000)))
    for v in ((hub, mid) if hub_too else (mid,)):
        for lab in range(5):
            probs = oracle.transition_probs(g, v, -1, 0, "metapath", schema=[lab])
            draw = lambda k: G.sample_hist(v, -1, 0, "metapath", 4_000_000, schema=[lab], mode=mode, flags=flags,
                                           seed=91 + v + lab + 7919 * k).cpu().numpy()
            assert_follows(draw, probs, ("metapath", mode, flags, v, lab), 4_000_000)


def test_rjs_full_s23_metapath_sampled_rows(s23):
    """The metapath bench's launch (2M starts, schema 0-4) with every hop in
    eRJS inside the label-grouped view (five weight classes per label
    segment, lognormal weights), no hand-off: sampled 128-row blocks equal
    the oracle's rejection-sampled walks bit for bit."""
    g, G = s23
    starts_h = synth.random_starts(g.n, 2_000_000, seed=43)
    schema = [0, 1, 2, 3, 4]
    out = G.walk(torch.from_numpy(starts_h).cuda(), 40, "metapath", schema=schema, mode="rjs", rjs_cap=1 << 30,
                 seed=42)
    for b in _blocks(len(starts_h), 4, 128, seed=7):
        ref, _ = oracle.walk_rjs(g, starts_h[b:b + 128], 40, "metapath", schema=schema, seed=42, walker_base=b,
                                 envelope="classes")
        got = out[b:b + 128].cpu().numpy()
        assert np.array_equal(got, ref), f"block {b}: {(got != ref).any(axis=1).sum()} rows differ"


def test_exact_mode_full_s23_metapath_sampled_rows(s23):
    g, G = s23
    starts_h = synth.random_starts(g.n, 2_000_000, seed=43)
    starts = torch.from_numpy(starts_h).cuda()
    schema = [0, 1, 2, 3, 4]
    for L in (5, 40):
        out = G.walk(starts, L, "metapath", schema=schema, mode="exact", seed=42)
        for b in _blocks(len(starts_h), 4, 128, seed=L):
            ref, _ = oracle.walk(g, starts_h[b:b + 128], L, "metapath", schema=schema, seed=42, walker_base=b)
            assert np.array_equal(out[b:b + 128].cpu().numpy(), ref)
        fast = G.walk(starts, L, "metapath", schema=schema, mode="auto", seed=42)
        rows = np.random.default_rng(L).choice(len(starts_h), 20_000, replace=False)
        o = fast[torch.from_numpy(rows).cuda()].cpu().numpy()
        alive = o[:, 1:] >= 0
        assert np.all(alive[:, :-1] | ~alive[:, 1:])
        keys = _edge_keys(g)
        q_ = (o[:, :-1].astype(np.int64) * np.int64(g.n) + o[:, 1:])[alive]
        pos = np.minimum(np.searchsorted(keys, q_), len(keys) - 1)
        assert np.all(keys[pos] == q_)
        hop = np.broadcast_to(np.arange(L), alive.shape)[alive]
        assert np.all(g.labels[pos] == np.asarray(schema)[hop % 5])
