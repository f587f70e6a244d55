"""The per-row Bloom filters are a pre-check in front of the exact search of
N(v'): they may skip a search, never change its answer.  So every walk, in
every mode, must be bit-identical with and without them, while the counted
membership probes drop."""
import numpy as np
import pytest

from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("node2vec", 2.0, 0.5), ("node2vec", 0.25, 4.0), ("node2vec", 4.0, 0.25), ("pagerank2", 1.0, 1.0)]


@pytest.fixture(scope="module")
def small():
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    yield g, G
    G.close()


@pytest.mark.parametrize("algo,p,q", CASES)
@pytest.mark.parametrize("mode", ["auto", "rjs", "rvs", "exact"])
def test_walks_identical_without_filters(small, algo, p, q, mode):
    g, G = small
    starts = torch.from_numpy(np.tile(np.arange(g.n, dtype=np.int32), 4)).cuda()
    a = G.walk(starts, 30, algo, p=p, q=q, mode=mode, seed=11)
    b = G.walk(starts, 30, algo, p=p, q=q, mode=mode, seed=11, flags=fw.FLAG_NO_BLOOM)
    assert torch.equal(a, b)


def test_filters_cut_membership_probes(small):
    g, G = small
    starts = torch.from_numpy(np.tile(np.arange(g.n, dtype=np.int32), 4)).cuda()
    probes = []
    for flags in (fw.FLAG_COUNTERS, fw.FLAG_COUNTERS | fw.FLAG_NO_BLOOM):
        G.reset_counters()
        G.walk(starts, 30, "node2vec", p=0.25, q=4.0, mode="rjs", seed=11, flags=flags)
        probes.append(G.counters()["probes"])
    assert probes[0] < 0.75 * probes[1], probes


def test_filter_bytes_in_graph_info(small):
    g, G = small
    # 32 bytes per 256-bit block: one block per 32 row entries plus one per node
    assert G.info["device_bytes"] >= 32 * (g.e // 32 + g.n + 1)
