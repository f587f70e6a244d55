"""GPU parity for metapath configurations off the common path: edge labels
of 8 and above (the per-label statistics and the label-grouped view are then
not built, so metapath plans by the Sec. 4.2 rule, B = h_MAX and
sum estimate h_SUM / 2, and samples over whole rows) and schemas of length
7 and 16 (the longest the C ABI accepts), against the CPU oracle through the
C ABI: exact mode bit for bit, eRJS with the paper's bound bit for bit,
the fast modes in distribution, and the walk invariants."""
import numpy as np
import pytest

import oracle
from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth
from statcheck import assert_follows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEMA7_HI = [0, 9, 8, 3, 1, 7, 2]           # labels >= 8 inside a 7-long schema
SCHEMA16_HI = [9, 0, 1, 8, 2, 3, 9, 4, 5, 6, 7, 8, 0, 9, 1, 2]
SCHEMA7 = [4, 0, 3, 1, 1, 2, 0]              # labels < 8 (label-grouped view)
SCHEMA16 = [0, 1, 2, 3, 4, 4, 3, 2, 1, 0, 2, 2, 4, 1, 3, 0]


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ten_labels():
    """R-MAT s12 with labels uniform in {0..9}: a label >= 8 occurs."""
    g = synth.workload_graph("small")
    g.labels = synth.edge_labels(g, 10, seed=31)
    assert int(g.labels.max()) >= 8
    G = fw.Graph(g)
    yield g, G
    G.close()


def _invariants(g, starts, out, schema):
    L = out.shape[1] - 1
    assert np.array_equal(out[:, 0], starts)
    alive = out[:, 1:] >= 0
    assert np.all(alive[:, :-1] | ~alive[:, 1:]), "-1 only as a suffix"
    n = np.int64(g.n)
    keys = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets)) * n + g.cols
    q = (out[:, :-1].astype(np.int64) * n + out[:, 1:])[alive]
    pos = np.searchsorted(keys, q)
    assert np.all(keys[np.minimum(pos, len(keys) - 1)] == q), "hop is not an edge"
    hop = np.broadcast_to(np.arange(L), alive.shape)[alive]
    assert np.all(g.labels[pos] == np.asarray(schema)[hop % len(schema)]), "label off the schema"
    for r in np.nonzero(~alive.all(axis=1))[0][:300]:   # a dead end only where no neighbour has the label
        j = int(np.argmin(alive[r]))
        assert oracle.transition_probs(g, int(out[r, j]), -1, j, "metapath", schema=schema).sum() == 0


def test_labels_ten_switch_off_label_statistics(ten_labels):
    _, G = ten_labels
    with pytest.raises(fw.FlexiWalkError) as e:
        G.label_stats()
    assert e.value.status == -8  # FW_ERR_UNSUPPORTED: statistics not built with a label >= 8


@pytest.mark.parametrize("schema", [SCHEMA7_HI, SCHEMA16_HI, [9]])
def test_exact_mode_labels_ten_bit_identical(ten_labels, schema):
    g, G = ten_labels
    starts = np.arange(g.n, dtype=np.int32)
    L = 40
    out = G.walk(_cuda(starts), L, "metapath", schema=schema, mode="exact", seed=42).cpu().numpy()
    ref, _ = oracle.walk(g, starts, L, "metapath", schema=schema, seed=42)
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"


@pytest.mark.parametrize("schema", [SCHEMA7, SCHEMA16])
def test_exact_mode_long_schemas_bit_identical(schema):
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    starts = synth.random_starts(g.n, 3001, seed=8)
    L = 37  # more hops than two passes over a 16-long schema, ragged
    out = G.walk(_cuda(starts), L, "metapath", schema=schema, mode="exact", seed=3, walker_base=9).cpu().numpy()
    G.close()
    ref, _ = oracle.walk(g, starts, L, "metapath", schema=schema, seed=3, walker_base=9)
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"


@pytest.mark.parametrize("schema", [SCHEMA7, SCHEMA16, [2]])
def test_label_group_rjs_long_schemas_bit_identical(schema):
    """eRJS inside the label-grouped view with 7- and 16-long schemas (every
    step kept in eRJS): rows equal the oracle's label-segment walks."""
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    starts = synth.random_starts(g.n, 4093, seed=19)
    L = 33
    out = G.walk(_cuda(starts), L, "metapath", schema=schema, mode="rjs", rjs_cap=1 << 30, seed=42,
                 walker_base=3).cpu().numpy()
    G.close()
    ref, _ = oracle.walk_rjs(g, starts, L, "metapath", schema=schema, seed=42, walker_base=3, envelope="classes")
    assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"


def test_plain_rjs_labels_ten_bit_identical():
    """Labels >= 8, the paper's single bound B = h_MAX over the whole row
    (FW_FLAG_PLAIN_RJS): on a dense graph with h in [0.5, 1] no step with a
    matching label exhausts 2^16 trials (acceptance >= 1/(2d) per trial),
    and a step without one runs the budget out and the eRVS hand-off finds
    the dead end the oracle reports, so rows are bit-identical."""
    g = synth.random_graph(40, 0.55, seed=5, weighted=True, nlabels=10)
    rng = np.random.default_rng(6)
    # one weight per undirected edge in [0.5, 1], mirrored
    n = g.n
    wm = np.triu(0.5 + 0.5 * (1.0 - rng.random((n, n))), 1)
    wm = wm + wm.T
    rows = np.repeat(np.arange(n), np.diff(g.offsets))
    g.h = wm[rows, g.cols].astype(np.float32)
    G = fw.Graph(g)
    starts = synth.random_starts(n, 6000, seed=12)
    for schema in (SCHEMA7_HI, SCHEMA16_HI):
        out = G.walk(_cuda(starts), 24, "metapath", schema=schema, mode="rjs", flags=fw.FLAG_PLAIN_RJS,
                     rjs_cap=1 << 16, seed=7, walker_base=2).cpu().numpy()
        ref, _ = oracle.walk_rjs(g, starts, 24, "metapath", schema=schema, seed=7, walker_base=2)
        assert np.array_equal(out, ref), f"{(out != ref).any(axis=1).sum()} rows differ"
        assert (ref[:, -1] < 0).any(), "the case should include dead ends"
    G.close()


@pytest.mark.parametrize("mode,flags", [("rjs", 0), ("rvs", 0), ("rvs", fw.FLAG_RVS_NOJUMP), ("auto", 0),
                                        ("rjs", fw.FLAG_PLAIN_RJS)])
def test_labels_ten_distributions(ten_labels, mode, flags):
    """Per-step draws at states of degree 1 .. max for required labels 9, 8
    and 2 (step index into SCHEMA7_HI) follow the oracle's probabilities;
    states without the label must give no draw."""
    g, G = ten_labels
    deg = g.degrees()
    ndraws = 2_000_000
    for target in [2, 32, 300, int(deg.max())]:
        v = int(np.argmin(np.abs(deg - target) + (deg == 0) * 10**9))
        for step in (1, 2, 6):  # SCHEMA7_HI[1] = 9, [2] = 8, [6] = 2
            probs = oracle.transition_probs(g, v, -1, step, "metapath", schema=SCHEMA7_HI)
            draw = lambda k: G.sample_hist(v, -1, step, "metapath", ndraws, schema=SCHEMA7_HI, mode=mode,
                                           flags=flags, seed=88 + v + step + 7919 * k).cpu().numpy()
            if probs.sum() == 0:
                assert draw(0).sum() == 0
                continue
            assert_follows(draw, probs, ("labels>=8", mode, flags, v, step), ndraws)


@pytest.mark.parametrize("schema", [SCHEMA16, SCHEMA16_HI])
@pytest.mark.parametrize("mode", ["rjs", "rvs", "auto"])
def test_long_schema_distributions(ten_labels, schema, mode):
    """Step 13 of a 16-long schema (labels < 8 on the grouped path, labels
    up to 9 on the whole-row path) follows the oracle's probabilities."""
    g10, G10 = ten_labels
    if schema is SCHEMA16:
        g = synth.workload_graph("small")
        G = fw.Graph(g)
    else:
        g, G = g10, G10
    deg = g.degrees()
    step = 13
    for target in [4, 300, int(deg.max())]:
        v = int(np.argmin(np.abs(deg - target) + (deg == 0) * 10**9))
        probs = oracle.transition_probs(g, v, -1, step, "metapath", schema=schema)
        draw = lambda k: G.sample_hist(v, -1, step, "metapath", 2_000_000, schema=schema, mode=mode,
                                       seed=61 + v + 7919 * k).cpu().numpy()
        if probs.sum() == 0:
            assert draw(0).sum() == 0
            continue
        assert_follows(draw, probs, ("schema16", schema[step], mode, v), 2_000_000)
    if schema is SCHEMA16:
        G.close()


@pytest.mark.parametrize("schema", [SCHEMA7_HI, SCHEMA16_HI])
@pytest.mark.parametrize("mode", ["auto", "rjs", "rvs"])
def test_labels_ten_walk_invariants(ten_labels, schema, mode):
    g, G = ten_labels
    starts = np.arange(g.n, dtype=np.int32)
    out = G.walk(_cuda(starts), 30, "metapath", schema=schema, mode=mode, seed=5).cpu().numpy()
    _invariants(g, starts, out, schema)
    again = G.walk(_cuda(starts), 30, "metapath", schema=schema, mode=mode, seed=5).cpu().numpy()
    assert np.array_equal(out, again)
