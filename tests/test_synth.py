"""The seeded synthetic inputs every test and the bench use: R-MAT graphs
are valid symmetric CSR (rows sorted, no self-loops or duplicates), the same
seed gives the same graph, weights and labels are mirrored per undirected
edge and fall in their stated ranges, and the R-MAT skew shows in the degrees."""
import numpy as np
import pytest

from paper_2512_00705_gb300 import synth


@pytest.fixture(scope="module")
def g10():
    return synth.rmat(10, 16, seed=1)


def _mirror_index(g):
    """Position of entry (u, v)'s mirror (v, u) for every entry."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    keys = rows * g.n + g.cols
    mirror = g.cols.astype(np.int64) * g.n + rows
    pos = np.searchsorted(keys, mirror)
    assert np.all(keys[pos] == mirror), "some entry has no mirror"
    return pos


def test_rmat_is_valid_symmetric_csr(g10):
    g = g10
    assert g.n == 1024 and g.offsets[0] == 0 and g.offsets[-1] == g.e
    assert np.all(np.diff(g.offsets) >= 0)
    rows = np.repeat(np.arange(g.n), np.diff(g.offsets))
    assert np.all((g.cols >= 0) & (g.cols < g.n))
    assert not np.any(g.cols == rows), "self-loop"
    same_row = rows[1:] == rows[:-1]
    assert np.all(g.cols[1:][same_row] > g.cols[:-1][same_row]), "rows not strictly ascending"
    _mirror_index(g)
    assert g.e <= 2 * 16 * 1024


def test_rmat_is_seeded(g10):
    again = synth.rmat(10, 16, seed=1)
    other = synth.rmat(10, 16, seed=2)
    assert np.array_equal(again.offsets, g10.offsets) and np.array_equal(again.cols, g10.cols)
    assert not (np.array_equal(other.offsets, g10.offsets) and np.array_equal(other.cols, g10.cols))


def test_rmat_degrees_are_skewed(g10):
    d = g10.degrees()
    # a = 0.57 concentrates edges: the largest degree is far above the mean
    assert d.max() > 8 * d.mean()


@pytest.mark.parametrize("kind,param,lo,hi", [("uniform01", 1.0, 0.0, 1.0), ("uniform15", 1.0, 1.0, 5.0),
                                              ("lognormal", 1.0, 0.0, np.inf), ("pareto", 1.5, 1.0, np.inf)])
def test_edge_weights_ranges_and_mirrors(g10, kind, param, lo, hi):
    h = synth.edge_weights(g10, kind, param, seed=2)
    assert h.dtype == np.float32 and h.shape == (g10.e,)
    assert np.all(h > lo) if kind == "uniform01" else np.all(h >= lo)
    assert np.all(h <= hi) if kind == "uniform01" else np.all(h < hi)
    assert np.array_equal(h, h[_mirror_index(g10)])
    assert np.array_equal(h, synth.edge_weights(g10, kind, param, seed=2))


def test_edge_labels_range_and_mirrors(g10):
    lab = synth.edge_labels(g10, 5, seed=3)
    assert lab.dtype == np.uint8 and np.all(lab < 5)
    assert np.array_equal(lab, lab[_mirror_index(g10)])
    assert set(np.unique(lab).tolist()) == {0, 1, 2, 3, 4}


def test_random_starts_seeded_and_in_range():
    a = synth.random_starts(1000, 5000, seed=7)
    assert a.dtype == np.int32 and np.all((a >= 0) & (a < 1000))
    assert np.array_equal(a, synth.random_starts(1000, 5000, seed=7))
    assert not np.array_equal(a, synth.random_starts(1000, 5000, seed=8))


def test_from_edges_builds_sorted_symmetric_rows():
    g = synth.from_edges(4, [(0, 2), (2, 1), (3, 0)], h=[1.0, 2.0, 3.0], labels=[1, 2, 3])
    assert g.offsets.tolist() == [0, 2, 3, 5, 6]
    assert g.cols.tolist() == [2, 3, 2, 0, 1, 0]
    assert g.h.tolist() == [1.0, 3.0, 2.0, 1.0, 2.0, 3.0]
    assert g.labels.tolist() == [1, 3, 2, 1, 2, 3]
    with pytest.raises(ValueError):
        synth.from_edges(2, [(1, 1)])
