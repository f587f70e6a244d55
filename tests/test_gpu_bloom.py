"""The per-row membership tables and Bloom filters stand in for the search
of N(v'): the table (the default) replaces it with an exact hash lookup,
the filter (without tables) may skip a search; neither may change an
answer.  So every walk, in every mode,
must be bit-identical with and without them (and with either alone), while
the counted membership probes drop."""
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
    for flags in (fw.FLAG_NO_BLOOM, fw.FLAG_NO_TABLE, fw.FLAG_NO_BLOOM | fw.FLAG_NO_TABLE):
        b = G.walk(starts, 30, algo, p=p, q=q, mode=mode, seed=11, flags=flags)
        assert torch.equal(a, b), flags


def test_filters_cut_membership_probes(small):
    g, G = small
    starts = torch.from_numpy(np.tile(np.arange(g.n, dtype=np.int32), 4)).cuda()
    probes = {}
    for flags in (0, fw.FLAG_NO_TABLE, fw.FLAG_NO_BLOOM, fw.FLAG_NO_BLOOM | fw.FLAG_NO_TABLE):
        G.reset_counters()
        G.walk(starts, 30, "node2vec", p=0.25, q=4.0, mode="rjs", seed=11, flags=flags | fw.FLAG_COUNTERS)
        probes[flags] = G.counters()["probes"]
    search = probes[fw.FLAG_NO_BLOOM | fw.FLAG_NO_TABLE]
    assert probes[fw.FLAG_NO_TABLE] < 0.75 * search, probes          # filter, then search
    assert probes[0] < 0.75 * probes[fw.FLAG_NO_TABLE], probes       # the table (the default)
    assert probes[fw.FLAG_NO_BLOOM] == probes[0], probes             # the filter is not consulted beside it


def test_table_lookup_is_exact_on_every_row_entry():
    """Every (row, id) pair of a graph whose hubs fill their tables unevenly
    is found, and ids next to them are not: exact-mode second-order
    PageRank consults N(v') for every neighbour of v, so its walks equal
    the search-only walks on a graph of long rows."""
    g = synth.rmat(11, 48, 0.7, 0.1, 0.1, seed=9)
    g.h = synth.edge_weights(g, "uniform01", seed=4)
    G = fw.Graph(g)
    starts = torch.from_numpy(np.tile(np.arange(g.n, dtype=np.int32), 2)).cuda()
    for algo, p, q in (("pagerank2", 1.0, 1.0), ("node2vec", 0.5, 2.0)):
        a = G.walk(starts, 16, algo, p=p, q=q, mode="exact", seed=5, flags=fw.FLAG_NO_BLOOM)
        b = G.walk(starts, 16, algo, p=p, q=q, mode="exact", seed=5, flags=fw.FLAG_NO_BLOOM | fw.FLAG_NO_TABLE)
        assert torch.equal(a, b), algo
    G.close()


def test_filter_bytes_in_graph_info(small):
    g, G = small
    # filters: 32 bytes per 256-bit block, one block per 32 row entries plus one per node;
    # tables: 32 bytes per 8-slot bucket, one bucket per 4 row entries plus one per node
    assert G.info["device_bytes"] >= 32 * (g.e // 32 + g.n + 1) + 32 * (g.e // 4 + g.n + 1)
