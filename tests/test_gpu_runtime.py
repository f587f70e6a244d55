"""GPU tests of the runtime around the samplers: the profiled cost ratio
(Sec. 5.1), its cache, that no runtime choice changes the walks'
distribution, batches and the serving loop."""
import ctypes
import os
import time

import numpy as np
import pytest

import oracle
from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth
from bruteforce import bf_paths, merged_chisquare
from statcheck import assert_pvalue_follows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    yield g, G
    G.close()


@pytest.mark.parametrize("algo,p,q,schema", [("node2vec", 2.0, 0.5, None), ("metapath", 1.0, 1.0, [0, 1, 2, 3, 4]),
                                             ("weighted", 1.0, 1.0, None), ("pagerank2", 1.0, 1.0, None)])
def test_autotune_profiling_installs_a_ratio(small, algo, p, q, schema, tmp_path):
    g, G = small
    cache = str(tmp_path / "ratios.txt")
    r = G.autotune(algo, p=p, q=q, schema=schema, method=0, cache_path=cache)
    assert np.isfinite(r) and 0.01 < r < 1000.0
    assert G.info["cost_ratios"][fw.ALGO[algo]] == pytest.approx(r)
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and f"{G.info['fingerprint']:016x}" in lines[0]
    # a cache hit returns the stored value without measuring
    with open(cache, "w") as f:
        f.write(lines[0].rsplit("r=", 1)[0] + "r=123.5\n")
    assert G.autotune(algo, p=p, q=q, schema=schema, method=0, cache_path=cache) == pytest.approx(123.5)
    # another (p, q), other sampler flags, or another gamma miss and append
    G.autotune(algo, p=p * 2, q=q, schema=schema, method=0, cache_path=cache)
    assert len(open(cache).read().splitlines()) == 2
    G.autotune(algo, p=p, q=q, schema=schema, flags=fw.FLAG_UNWEIGHTED, method=0, cache_path=cache)
    assert len(open(cache).read().splitlines()) == 3
    G.autotune(algo, p=p, q=q, schema=schema, gamma=0.5, method=0, cache_path=cache)
    assert len(open(cache).read().splitlines()) == 4
    # every algorithm keeps its own ratio
    G.set_cost_ratio(4.0)
    G.autotune(algo, p=p, q=q, schema=schema, method=0)
    others = [a for a in range(4) if a != fw.ALGO[algo]]
    assert all(G.info["cost_ratios"][a] == 4.0 for a in others)
    G.set_cost_ratio(4.0)


def test_autotune_sweep_picks_from_the_ladder(small):
    g, G = small
    r = G.autotune("node2vec", p=2.0, q=0.5, method=1)
    assert r in [0.125, 0.25, 0.5, 1, 2, 4, 8, 16, 32, 64]
    G.set_cost_ratio(4.0)


def test_autotune_shape_installs_and_caches_the_launch_shape(small, tmp_path):
    """Method 2 tunes r and the launch shape, installs them for the algorithm
    alone, and a cache hit restores all four without measuring."""
    g, G = small
    cache = str(tmp_path / "shape.txt")
    r = G.autotune("node2vec", p=0.5, q=2.0, method=2, cache_path=cache)
    info = G.info
    a = fw.ALGO["node2vec"]
    assert r in [0.125, 0.25, 0.5, 1, 2, 4, 8, 16, 32, 64]
    assert info["lane_max_degrees"][a] in (1, 4, 8, 16, 32, 64)
    assert info["rjs_batches"][a] in (1, 2, 3, 4, 6)
    assert info["trial_budgets"][a] in (0.25, 0.5, 1.0, 2.0, 4.0)
    others = [x for x in range(4) if x != a]
    assert all(info["lane_max_degrees"][x] == 8 and info["rjs_batches"][x] == 2 for x in others)
    line = open(cache).read().splitlines()[0]
    assert "method=2" in line and "lane=" in line and "batch=" in line and "budget=" in line
    with open(cache, "w") as f:
        f.write(line.rsplit("r=", 1)[0] + "r=16 lane=32 batch=3 budget=0.5\n")
    assert G.autotune("node2vec", p=0.5, q=2.0, method=2, cache_path=cache) == pytest.approx(16.0)
    info = G.info
    assert (info["lane_max_degrees"][a], info["rjs_batches"][a], info["trial_budgets"][a]) == (32, 3, 0.5)
    # the shape reaches the walks: an explicit shape in fw_params equals the installed one
    starts = torch.from_numpy(np.arange(g.n, dtype=np.int32)).cuda()
    x1 = G.walk(starts, 20, "node2vec", p=0.5, q=2.0, seed=4)
    x2 = G.walk(starts, 20, "node2vec", p=0.5, q=2.0, seed=4, cost_ratio=16.0, lane_max_degree=32, rjs_batch=3,
                trial_budget=0.5)
    assert torch.equal(x1, x2)
    # back to the defaults for the module's other tests
    with open(cache, "w") as f:
        f.write(line.rsplit("r=", 1)[0] + "r=4 lane=8 batch=2 budget=1\n")
    G.autotune("node2vec", p=0.5, q=2.0, method=2, cache_path=cache)
    G.set_cost_ratio(4.0)


@pytest.mark.parametrize("algo,p,q", [("node2vec", 0.25, 4.0), ("node2vec", 4.0, 0.25), ("weighted", 1.0, 1.0),
                                      ("pagerank2", 1.0, 1.0)])
def test_rjs_batch_leaves_rows_unchanged(small, algo, p, q):
    """Trial t of a step always draws counter t: how many trials a lane runs
    between two warp ballots changes no row."""
    g, G = small
    starts = torch.from_numpy(np.tile(np.arange(g.n, dtype=np.int32), 2)).cuda()
    ref = G.walk(starts, 25, algo, p=p, q=q, mode="auto", seed=8, rjs_batch=2)
    for batch in (1, 3, 6, 16):
        assert torch.equal(G.walk(starts, 25, algo, p=p, q=q, mode="auto", seed=8, rjs_batch=batch), ref), batch


@pytest.mark.parametrize("shape", [dict(lane_max_degree=1), dict(lane_max_degree=64), dict(trial_budget=0.25),
                                   dict(trial_budget=4.0, rjs_batch=6)])
def test_launch_shape_never_changes_the_distribution(shape):
    """Where eRVS steps run (lane or warp) and when eRJS hands a step over
    only change which sampler draws it: whole-path frequencies still match
    brute-force path probabilities."""
    g = synth.random_graph(24, 0.85, seed=21, weighted=True, nlabels=3)
    G = fw.Graph(g)
    W, L = 300_000, 3
    starts = torch.zeros(W, dtype=torch.int32, device="cuda")
    bf = bf_paths(g, 0, L, "node2vec", 0.5, 2.0, None)
    assert_pvalue_follows(lambda k: merged_chisquare(bf, G.walk(starts, L, "node2vec", p=0.5, q=2.0, mode="auto",
                                                                 cost_ratio=1.0, seed=13 + 7919 * k,
                                                                 **shape).cpu().numpy()), ("shape", shape))
    G.close()


def test_launch_shape_out_of_range_is_refused(small):
    g, G = small
    starts = torch.zeros(8, dtype=torch.int32, device="cuda")
    for bad in (dict(lane_max_degree=65), dict(rjs_batch=17), dict(trial_budget=float("inf"))):
        with pytest.raises(fw.FlexiWalkError) as e:
            G.walk(starts, 3, "weighted", **bad)
        assert e.value.status == -1


def test_fingerprint_tracks_the_graph(small):
    g, G = small
    G2 = fw.Graph(g)
    assert G2.info["fingerprint"] == G.info["fingerprint"]
    # the fingerprint hashes 4096 evenly spaced entries: change one of them
    h2 = g.h.copy()
    h2[(g.e - 1) * 2048 // 4095] *= 0.5
    G3 = fw.Graph(synth.Csr(g.offsets, g.cols, h2, g.labels))
    assert G3.info["fingerprint"] != G.info["fingerprint"]
    G2.close()
    G3.close()


@pytest.mark.parametrize("ratio", [0.01, 4.0, 1000.0])
def test_cost_ratio_never_changes_the_distribution(ratio):
    """Eq. (runtime) only picks a sampler; extreme ratios (all eRVS, all
    eRJS) give the same path distribution."""
    g = synth.random_graph(8, 0.45, seed=11, weighted=True, nlabels=3)
    G = fw.Graph(g)
    W, L = 300_000, 4
    starts = torch.zeros(W, dtype=torch.int32, device="cuda")
    bf = bf_paths(g, 0, L, "node2vec", 0.5, 2.0, None)
    assert_pvalue_follows(lambda k: merged_chisquare(bf, G.walk(starts, L, "node2vec", p=0.5, q=2.0, mode="auto",
                                                                 cost_ratio=ratio, seed=3 + 7919 * k).cpu().numpy()),
                          ("cost ratio", ratio))
    G.close()


# ------------------------------------------------------------ batching
def _mixed_jobs(g, count, seed, max_walkers=3000, max_length=30):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        algo = ["node2vec", "metapath", "weighted", "pagerank2"][i % 4]
        w = int(rng.integers(1, max_walkers))
        spec = dict(starts=synth.random_starts(g.n, w, seed=seed * 100 + i), length=int(rng.integers(0, max_length)),
                    algo=algo, mode=["auto", "rjs", "rvs", "exact"][int(rng.integers(0, 4))],
                    seed=int(rng.integers(1, 1 << 40)), walker_base=int(rng.integers(0, 1000)))
        if algo == "node2vec":
            spec["p"], spec["q"] = float(rng.choice([0.25, 0.5, 1, 2, 4])), float(rng.choice([0.25, 0.5, 1, 2, 4]))
        if algo == "metapath":
            spec["schema"] = [0, 1, 2, 3, 4]
        specs.append(spec)
    return specs


def _kw(spec):
    return {k: spec[k] for k in ("p", "q", "schema", "mode", "seed", "walker_base") if k in spec}


@pytest.mark.parametrize("count", [10, 70])
def test_batch_rows_equal_separate_walks(small, count):
    """A job's rows in a batch equal its rows from its own fw_walk."""
    g, G = small
    specs = _mixed_jobs(g, count, seed=count)
    jobs, outs = [], []
    for sp in specs:
        st = torch.from_numpy(sp["starts"]).cuda()
        out = torch.full((st.numel(), sp["length"] + 1), -7, dtype=torch.int32, device="cuda")
        sp["_st"] = st
        outs.append(out)
        jobs.append(fw.make_job(st, sp["length"], sp["algo"], out, **_kw(sp)))
    fw.fw_walk_batch(G.handle, jobs)
    for sp, out in zip(specs, outs):
        alone = G.walk(sp["_st"], sp["length"], sp["algo"], **_kw(sp))
        assert torch.equal(out, alone), sp["algo"]


def test_batch_plan_replays(small):
    g, G = small
    specs = _mixed_jobs(g, 12, seed=5)
    jobs, outs, sts = [], [], []
    for sp in specs:
        st = torch.from_numpy(sp["starts"]).cuda()
        out = torch.empty((st.numel(), sp["length"] + 1), dtype=torch.int32, device="cuda")
        sts.append(st)
        outs.append(out)
        jobs.append(fw.make_job(st, sp["length"], sp["algo"], out, **_kw(sp)))
    plan = fw.BatchPlan(G, jobs)
    n0 = fw.fw_launch_count()
    plan.launch()
    torch.cuda.synchronize()
    # one graph launch holding one walk kernel per algorithm present
    assert fw.fw_launch_count() - n0 == len({sp["algo"] for sp in specs})
    first = [o.clone() for o in outs]
    for sp, st, o in zip(specs, sts, first):
        assert torch.equal(o, G.walk(st, sp["length"], sp["algo"], **_kw(sp)))
    # new start contents, same buffers: the replay follows them
    for st in sts:
        st.copy_(torch.randint(0, g.n, st.shape, dtype=torch.int32, device="cuda"))
    plan.launch()
    torch.cuda.synchronize()
    for sp, st, o in zip(specs, sts, outs):
        assert torch.equal(o, G.walk(st, sp["length"], sp["algo"], **_kw(sp)))
    plan.close()


# ------------------------------------------------------------ serving
@pytest.mark.parametrize("large_query_steps", [None, 0, 5000])
def test_server_results_equal_alone_in_a_concurrent_mix(small, large_query_steps):
    """Queries submitted from several threads while others run on the GPU
    give exactly the rows of fw_walk_host alone (0 differing entries), with
    the default size classes, with one class, and with most queries large
    (their own waves, admitted after the small ones)."""
    import threading
    g, G = small
    srv = fw.Server(G, mem_budget=64 << 20, max_waves=3, max_jobs_per_wave=16, large_query_steps=large_query_steps)
    specs = _mixed_jobs(g, 160, seed=9, max_walkers=5000)
    outs = [np.full((len(sp["starts"]), sp["length"] + 1), -7, dtype=np.int32) for sp in specs]
    tickets = [None] * len(specs)

    def client(k):
        for i in range(k, len(specs), 4):
            sp = specs[i]
            tickets[i] = srv.submit(sp["starts"], sp["length"], sp["algo"], outs[i], **_kw(sp))

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    [t.start() for t in th]
    [t.join() for t in th]
    lat = [srv.wait(t, timeout=60.0) for t in tickets]
    assert all(x >= 0 for x in lat)
    st = srv.stats()
    assert st["completed"] == len(specs) and st["failed"] == 0 and st["pending"] == 0
    assert st["peak_device_bytes"] <= 64 << 20
    srv.close()
    for sp, out in zip(specs, outs):
        alone = G.walk_host(sp["starts"], sp["length"], sp["algo"], **_kw(sp))
        assert np.array_equal(out, alone)


def test_server_burst_merges_queries_into_overlapping_waves(small):
    """A burst of 400 queries submitted in one call: waves merge several
    queries (queries_per_wave > 1) and overlap on the device
    (peak_inflight_waves > 1); every query's rows equal fw_walk_host's
    alone, the batched poll releases every ticket once, and the device's hop
    count equals the hops in the rows.  Queries of up to 40,000 walkers x
    up to 90 hops keep each wave's device work longer than its launch."""
    g, G = small
    srv = fw.Server(G, mem_budget=2 << 30, max_waves=6, max_jobs_per_wave=32)
    specs = _mixed_jobs(g, 400, seed=21, max_walkers=40000, max_length=90)
    outs = [np.full((len(sp["starts"]), sp["length"] + 1), -7, dtype=np.int32) for sp in specs]
    qs = (fw.fw_job * len(specs))(*[fw.make_host_query(sp["starts"], sp["length"], sp["algo"], o, **_kw(sp))
                                     for sp, o in zip(specs, outs)])
    tickets = srv.submit_many(qs)
    assert len(set(tickets.tolist())) == len(specs)
    pending = tickets.copy()
    deadline = time.time() + 120.0
    while len(pending) and time.time() < deadline:
        done, lat, st = srv.poll_many(pending)
        assert np.all(st[done == 1] == 0)
        assert np.all(lat[done == 1] >= 0)
        pending = pending[done == 0]
    assert len(pending) == 0, "queries did not finish"
    d2, _, st2 = srv.poll_many(tickets[:3])  # released tickets are unknown now
    assert np.all(d2 == 1) and np.all(st2 == -1)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(specs) and stats["failed"] == 0
    assert stats["queries_per_wave"] > 1.0, stats
    assert stats["peak_inflight_waves"] > 1, stats
    hops = sum(int((o[:, 1:] >= 0).sum()) for o in outs)
    assert stats["walker_steps"] == hops
    for sp, out in zip(specs, outs):
        assert np.array_equal(out, G.walk_host(sp["starts"], sp["length"], sp["algo"], **_kw(sp)))


def test_server_merges_copies_of_back_to_back_buffers(small):
    """Queries whose starts and rows are consecutive slices of one pinned
    pool: their copies merge (fewer copies than two per query) and every
    query's rows still equal fw_walk_host's alone.  The budget is not a
    multiple of 256 bytes (it is rounded down, so every staged buffer stays
    4-byte aligned)."""
    g, G = small
    specs = _mixed_jobs(g, 120, seed=33, max_walkers=3000, max_length=40)
    n_in = sum(len(sp["starts"]) for sp in specs)
    n_out = sum(len(sp["starts"]) * (sp["length"] + 1) for sp in specs)
    pool_in = torch.empty(n_in, dtype=torch.int32).pin_memory().numpy()
    pool_out = torch.empty(n_out, dtype=torch.int32).pin_memory().numpy()
    pool_out[:] = -7
    outs, qs, a, b = [], [], 0, 0
    for sp in specs:
        w, L = len(sp["starts"]), sp["length"]
        pool_in[a:a + w] = sp["starts"]
        o = pool_out[b:b + w * (L + 1)].reshape(w, L + 1)
        qs.append(fw.make_host_query(pool_in[a:a + w], L, sp["algo"], o, **_kw(sp)))
        outs.append(o)
        a += w
        b += w * (L + 1)
    srv = fw.Server(G, mem_budget=(256 << 20) + 37, max_waves=4, max_jobs_per_wave=32)
    tickets = srv.submit_many((fw.fw_job * len(qs))(*qs))
    for t in tickets:
        srv.wait(int(t), timeout=60.0)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(specs) and stats["failed"] == 0
    assert stats["copies"] < 2 * len(specs), stats
    for sp, out in zip(specs, outs):
        assert np.array_equal(out, G.walk_host(sp["starts"], sp["length"], sp["algo"], **_kw(sp)))


def test_server_submit_many_stops_at_the_first_bad_query(small):
    g, G = small
    srv = fw.Server(G, mem_budget=16 << 20, max_waves=2)
    good = [np.arange(50, dtype=np.int32) for _ in range(3)]
    bad = np.array([0, g.n], dtype=np.int32)
    outs = [np.empty((50, 6), np.int32) for _ in range(3)] + [np.empty((2, 6), np.int32)]
    qs = (fw.fw_job * 4)(*([fw.make_host_query(st, 5, "weighted", o) for st, o in zip(good[:2], outs[:2])] +
                            [fw.make_host_query(bad, 5, "weighted", outs[3]),
                             fw.make_host_query(good[2], 5, "weighted", outs[2])]))
    tickets = np.zeros(4, dtype=np.uint64)
    n = ctypes.c_int32()
    st = fw.lib().fw_server_submit_many(srv.handle, ctypes.cast(qs, ctypes.c_void_p), 4, tickets.ctypes.data,
                                        ctypes.byref(n))
    assert st == -1 and n.value == 2 and b"query 2" in fw.lib().fw_last_error()
    for t in tickets[:2]:
        srv.wait(int(t), timeout=30.0)
    srv.close()


def test_server_errors_and_timeouts(small):
    g, G = small
    with pytest.raises(fw.FlexiWalkError) as e:
        fw.Server(G, mem_budget=1 << 20, max_waves=2, large_query_steps=-1)
    assert e.value.status == -1
    srv = fw.Server(G, mem_budget=1 << 20, max_waves=2)
    big = np.zeros(1 << 17, dtype=np.int32)                 # 2^17 walkers x 11 entries > 1 MiB
    with pytest.raises(fw.FlexiWalkError) as e:
        srv.submit(big, 10, "weighted", np.empty((big.shape[0], 11), np.int32))
    assert e.value.status == -3
    bad = np.array([0, g.n], dtype=np.int32)
    with pytest.raises(fw.FlexiWalkError) as e:
        srv.submit(bad, 3, "weighted", np.empty((2, 4), np.int32))
    assert e.value.status == -1
    with pytest.raises(fw.FlexiWalkError):
        srv.submit(np.zeros(4, np.int32), 3, "node2vec", np.empty((4, 4), np.int32), p=0.0)
    starts = np.arange(4000, dtype=np.int32) % g.n
    out = np.empty((4000, 31), np.int32)
    t = srv.submit(starts, 30, "node2vec", out, p=2.0, q=0.5)
    try:
        srv.wait(t, timeout=0.0)
        timed_out = False
    except fw.FlexiWalkError as err:
        assert err.status == -5
        timed_out = True
    if timed_out:
        srv.wait(t, timeout=30.0)
    with pytest.raises(fw.FlexiWalkError):
        srv.wait(t, timeout=1.0)  # released after collection
    # destroy drains queries never waited for
    outs = []
    for i in range(20):
        o = np.full((100, 6), -7, np.int32)
        outs.append(o)
        srv.submit(np.arange(100, dtype=np.int32), 5, "weighted", o, seed=i)
    srv.close()
    for i, o in enumerate(outs):
        assert np.array_equal(o, G.walk_host(np.arange(100, dtype=np.int32), 5, "weighted", seed=i))


def test_sharded_walks_reassemble_to_the_single_walk(small):
    """Queries spread over 3 'GPUs' by the start-node hash (Sec. 5.6), each
    shard walked with its global indices as stream ids: the reassembled rows
    equal one walk over all queries, in every mode."""
    from paper_2512_00705_gb300 import sharding
    g, G = small
    starts = np.tile(np.arange(g.n, dtype=np.int32), 2)
    for mode in ["auto", "rjs", "rvs", "exact"]:
        full = G.walk(torch.from_numpy(starts).cuda(), 15, "node2vec", p=0.5, q=2.0, mode=mode, seed=9).cpu().numpy()
        parts = []
        for r in range(3):
            idx = sharding.shard(starts, r, 3)
            rows = G.walk_ids(torch.from_numpy(starts[idx]).cuda(), torch.from_numpy(idx.astype(np.int32)).cuda(), 15,
                              "node2vec", p=0.5, q=2.0, mode=mode, seed=9).cpu().numpy()
            parts.append((idx, rows))
        assert np.array_equal(sharding.assemble(parts, len(starts), 16), full), mode


@pytest.mark.parametrize("algo,p,q,schema,base", [("node2vec", 0.25, 4.0, None, 0),
                                                  ("metapath", 1.0, 1.0, [0, 1, 2, 3, 4], 77)])
def test_chunked_host_walk_equals_device_walk(small, algo, p, q, schema, base):
    """fw_walk_host splits rows of >= 128 MiB into chunks walked on two
    streams and copied out on a third: 3.2M walkers x 21 entries (269 MB, 4
    chunks, ragged: 3.2M is not a multiple of 4 * 256) must give exactly the
    rows of one device walk, in pinned and in pageable host memory."""
    g, G = small
    W, L = 3_200_003, 20
    starts = synth.random_starts(g.n, W, seed=31)
    want = G.walk(torch.from_numpy(starts).cuda(), L, algo, p=p, q=q, schema=schema, mode="auto", seed=9,
                  walker_base=base).cpu().numpy()
    pinned_in = torch.from_numpy(starts).pin_memory().numpy()
    pinned_out = torch.empty((W, L + 1), dtype=torch.int32).pin_memory().numpy()
    for st_h, out in [(pinned_in, pinned_out), (starts, np.full((W, L + 1), -7, dtype=np.int32))]:
        got = G.walk_host(st_h, L, algo, p=p, q=q, schema=schema, mode="auto", seed=9, walker_base=base, out=out)
        assert np.array_equal(got, want), f"{(got != want).any(axis=1).sum()} rows differ"


def test_gather_ceiling_probe():
    """fw_gather_ceiling: a positive, finite rate of random 32-byte gathers
    that does not exceed one gather per SM clock cycle."""
    table = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rate = fw.fw_gather_ceiling(table)
    props = torch.cuda.get_device_properties(0)
    assert np.isfinite(rate) and rate > 1e8
    assert rate < props.multi_processor_count * 2.5e9
