"""8-bit property weights (low-precision weights, named in Sec. 6.2 as an
extension): a resident graph switched to weight codes must sample exactly as
the oracle does over the oracle's own dequantized weights -- bit-identical
walks in exact mode, matching per-step and whole-path distributions in the
fast modes -- with every derived structure rebuilt from the new weights."""
import numpy as np
import pytest

import oracle
from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth
from bruteforce import bf_paths, merged_chisquare
from statcheck import assert_follows, assert_pvalue_follows, chisq_pvalue

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALGOS = [("node2vec", 2.0, 0.5, None), ("node2vec", 0.25, 4.0, None), ("metapath", 1.0, 1.0, [0, 1, 2, 3, 4]),
         ("weighted", 1.0, 1.0, None), ("pagerank2", 1.0, 1.0, None)]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _skewed_small():
    """s12 R-MAT with lognormal(0, 1.25) weights: with one scale per graph
    about two fifths of them would fall below half a code step; with a
    scale per row far fewer do."""
    g = synth.workload_graph("small")
    g.h = synth.edge_weights(g, "lognormal", 1.25, seed=12)
    return g


@pytest.fixture(scope="module")
def quantized():
    g = _skewed_small()
    G = fw.Graph(g)
    fp0 = G.info["fingerprint"]
    bytes0 = G.info["device_bytes"]
    s = G.quantize_weights()
    codes, scales, hq = oracle.quantize_weights(g)
    gq = synth.Csr(g.offsets, g.cols, hq, g.labels)
    yield g, gq, G, dict(scale=s, scales_ref=scales, fp0=fp0, bytes0=bytes0, codes=codes)
    G.close()


def test_scale_and_graph_info(quantized):
    g, gq, G, m = quantized
    scales = G.weight_scales().cpu().numpy()
    assert np.array_equal(scales, m["scales_ref"])            # bit-exact FP32 scale of every row
    assert m["scale"] == float(m["scales_ref"].max())
    assert G.info["weight_scale"] == m["scale"]
    assert G.info["fingerprint"] != m["fp0"]                  # autotune caches keyed apart
    assert G.info["device_bytes"] == m["bytes0"] + g.e + 4 * g.n  # one byte per weight, one scale per node
    assert G.info["symmetric"] == 0                           # mirrored entries are coded against two scales
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    cmax = np.zeros(g.n, np.int64)
    np.maximum.at(cmax, rows, m["codes"].astype(np.int64))
    assert np.all(cmax[np.diff(g.offsets) > 0] == 255)        # every row keeps its largest weight at 255
    assert 0 < (m["codes"] == 1).mean() < 0.15                # the clamp occurs (about 2 in 5 with one scale per graph)
    assert G.quantize_weights() == m["scale"]                 # a second call is a no-op


def test_weight_scales_before_quantization_is_refused():
    g = synth.random_graph(8, 0.5, seed=2, weighted=True)
    G = fw.Graph(g)
    with pytest.raises(fw.FlexiWalkError) as e:
        G.weight_scales()
    assert e.value.status == -8
    G.close()


def test_derived_statistics_follow_the_codes(quantized):
    g, gq, G, _ = quantized
    hmax, hsum = G.node_stats()
    rmax, rsum = oracle.node_stats(gq)
    assert np.array_equal(hmax.cpu().numpy(), rmax)
    np.testing.assert_allclose(hsum.cpu().numpy(), rsum, rtol=2e-6, atol=1e-6)
    st = G.label_stats().cpu().numpy()
    lmax, lsum = oracle.label_stats(gq)
    assert np.array_equal(st[:, :, 0], lmax)
    np.testing.assert_allclose(st[:, :, 1], lsum, rtol=2e-6, atol=1e-6)


@pytest.mark.parametrize("algo,p,q,schema", ALGOS)
def test_exact_mode_bit_identical(quantized, algo, p, q, schema):
    g, gq, G, _ = quantized
    starts = np.arange(g.n, dtype=np.int32)
    out = G.walk(_cuda(starts), 20, algo, p=p, q=q, schema=schema, mode="exact", seed=42).cpu().numpy()
    ref, _ = oracle.walk(gq, starts, 20, algo, p, q, schema, seed=42)
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"
    G.check()


@pytest.mark.parametrize("W,L,base", [(4093, 13, 7), (33, 3, 0), (1, 40, 9)])
def test_exact_mode_ragged(quantized, W, L, base):
    g, gq, G, _ = quantized
    starts = synth.random_starts(g.n, W, seed=W)
    out = G.walk(_cuda(starts), L, "node2vec", p=0.5, q=2.0, mode="exact", seed=3, walker_base=base).cpu().numpy()
    ref, _ = oracle.walk(gq, starts, L, "node2vec", 0.5, 2.0, seed=3, walker_base=base)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("rvs", 0), ("rvs", fw.FLAG_RVS_NOJUMP), ("auto", 0)])
@pytest.mark.parametrize("algo,p,q,schema", ALGOS[:4])
def test_fast_mode_distributions(quantized, mode, flags, algo, p, q, schema):
    """Per-step distributions at nodes of degree ~1 .. max equal the oracle's
    over the dequantized weights."""
    g, gq, G, _ = quantized
    deg = g.degrees()
    ndraws = 4_000_000
    for target in [2, 32, 300, int(deg.max())]:
        v = int(np.argmin(np.abs(deg - target) + (deg == 0) * 10**9))
        nb = g.cols[g.offsets[v]:g.offsets[v + 1]]
        for vp, step in [(-1, 0), (int(nb[np.argmax(deg[nb])]), 1)]:
            probs = oracle.transition_probs(gq, v, vp, step, algo, p, q, schema)
            draw = lambda k: G.sample_hist(v, vp, step, algo, ndraws, p=p, q=q, schema=schema, mode=mode,
                                           flags=flags, seed=555 + v + 7919 * k).cpu().numpy()
            if probs.sum() == 0:
                assert draw(0).sum() == 0
                continue
            assert_follows(draw, probs, (algo, p, q, mode, flags, v, vp), ndraws)


@pytest.mark.parametrize("mode", ["rjs", "rvs", "auto"])
@pytest.mark.parametrize("algo,p,q,schema", [("node2vec", 0.25, 4.0, None), ("metapath", 1.0, 1.0, [0, 1, 2]),
                                             ("pagerank2", 1.0, 1.0, None)])
def test_fast_walk_path_distribution(mode, algo, p, q, schema):
    """Whole 4-hop paths on a tiny graph whose weights span three decades."""
    g = synth.random_graph(8, 0.45, seed=11, weighted=True, nlabels=3)
    g.h = (g.h ** 3 + np.float32(1e-3)).astype(np.float32)
    _, _, hq = oracle.quantize_weights(g)
    gq = synth.Csr(g.offsets, g.cols, hq, g.labels)
    G = fw.Graph(g)
    G.quantize_weights()
    W, L = 300_000, 4
    bf = bf_paths(gq, 0, L, algo, p, q, schema)
    starts = torch.zeros(W, dtype=torch.int32, device="cuda")
    assert_pvalue_follows(lambda k: merged_chisquare(bf, G.walk(starts, L, algo, p=p, q=q, schema=schema, mode=mode,
                                                                 seed=23 + 7919 * k).cpu().numpy()),
                          ("quantized paths", algo, p, q, mode))
    G.close()


def test_unweighted_graph_is_refused():
    g = synth.random_graph(8, 0.5, seed=1, weighted=False)
    G = fw.Graph(g)
    with pytest.raises(fw.FlexiWalkError) as e:
        G.quantize_weights()
    assert e.value.status == -8
    G.close()


@pytest.mark.parametrize("alpha", [1.0, 2.0, 3.0])
def test_skewed_weights_keep_their_distribution(alpha):
    """Pareto(alpha) weights, alpha <= 3, on the s12 structure: with a scale
    per row every dequantized weight lies within s_v = h_MAX[v] / 255 of the
    original (half a step when rounded, under s_v when clamped), so the
    first-order distribution at v moves by at most
    TV <= sum_k |h'_k - h_k| / sum_k h_k <= d_v s_v / h_SUM[v]; the oracle's
    dequantized probabilities meet that bound at every node, and at the
    hubs (most skewed rows) the GPU's draws follow the dequantized
    probabilities in every fast mode."""
    g = synth.workload_graph("small")
    g.h = synth.edge_weights(g, "pareto", alpha, seed=14)
    codes, scales, hq = oracle.quantize_weights(g)
    gq = synth.Csr(g.offsets, g.cols, hq, g.labels)
    deg = g.degrees()
    worst = 0.0
    for v in np.nonzero(deg > 0)[0]:
        sl = slice(g.offsets[v], g.offsets[v + 1])
        p = g.h[sl].astype(np.float64) / g.h[sl].astype(np.float64).sum()
        pq = hq[sl].astype(np.float64) / hq[sl].astype(np.float64).sum()
        tv = 0.5 * np.abs(p - pq).sum()
        bound = deg[v] * float(scales[v]) / g.h[sl].astype(np.float64).sum()
        assert tv <= bound * (1 + 1e-6) + 1e-12, (v, tv, bound)
        worst = max(worst, tv)
    G = fw.Graph(g)
    G.quantize_weights()
    for v in np.argsort(deg)[-3:]:
        probs = oracle.transition_probs(gq, int(v), -1, 0, "weighted")
        for mode in ("rjs", "rvs", "auto"):
            draw = lambda k: G.sample_hist(int(v), -1, 0, "weighted", 2_000_000, mode=mode,
                                           seed=71 + int(v) + 7919 * k).cpu().numpy()
            assert_follows(draw, probs, ("pareto", alpha, mode, int(v)), 2_000_000)
    G.close()
