"""Seeded synthetic inputs for dynamic random walks.

R-MAT graphs as sorted, symmetric int32 CSR with per-undirected-edge property
weights and labels, plus walker start sets.  This module is input generation
only: it holds none of the walk method's arithmetic, so the GPU path and the
CPU oracle can both be fed from it.

The compiled part (``rmat.c``) is built by ``build()``; it is plain C with
OpenMP and gives identical output on x86-64 and AArch64 and for any thread
count.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmat.c")
_SO = os.path.join(_HERE, "_build", "libfwsynth.so")
_lock = threading.Lock()
_lib = None

WEIGHT_KINDS = {"uniform01": 0, "lognormal": 1, "pareto": 2, "uniform15": 3}


def build(force: bool = False) -> str:
    """Compile rmat.c into a shared library next to it; returns its path."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                   check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32, i64, u64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p
            lib.fws_rmat_build.argtypes = [i32, i32, dbl, dbl, dbl, u64, i32, i32, ctypes.POINTER(vp),
                                           ctypes.POINTER(i32), ctypes.POINTER(i64)]
            lib.fws_rmat_build.restype = ctypes.c_int
            lib.fws_rmat_copy.argtypes = [vp, vp, vp]
            lib.fws_rmat_copy.restype = ctypes.c_int
            lib.fws_rmat_free.argtypes = [vp]
            lib.fws_rmat_free.restype = None
            lib.fws_edge_weights.argtypes = [vp, vp, i32, i32, dbl, u64, vp, i32]
            lib.fws_edge_weights.restype = ctypes.c_int
            lib.fws_edge_labels.argtypes = [vp, vp, i32, i32, u64, vp, i32]
            lib.fws_edge_labels.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclasses.dataclass
class Csr:
    """A graph in CSR form: offsets int32[n+1], cols int32[e] (rows sorted
    ascending), optional property weights h float32[e] and labels uint8[e]."""
    offsets: np.ndarray
    cols: np.ndarray
    h: Optional[np.ndarray] = None
    labels: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def e(self) -> int:
        return int(self.cols.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True, threads: int = 0) -> Csr:
    """Undirected R-MAT graph: 2^scale nodes, edge_factor * 2^scale generated
    edges, symmetrised, self-loops and duplicates removed, rows sorted."""
    lib = _load()
    h = ctypes.c_void_p()
    n = ctypes.c_int32()
    e = ctypes.c_int64()
    rc = lib.fws_rmat_build(scale, edge_factor, a, b, c, seed, int(permute), threads,
                            ctypes.byref(h), ctypes.byref(n), ctypes.byref(e))
    if rc != 0:
        raise RuntimeError(f"fws_rmat_build failed with code {rc}")
    try:
        offsets = np.empty(n.value + 1, dtype=np.int32)
        cols = np.empty(e.value, dtype=np.int32)
        lib.fws_rmat_copy(h, offsets.ctypes.data, cols.ctypes.data)
    finally:
        lib.fws_rmat_free(h)
    return Csr(offsets, cols)


def edge_weights(g: Csr, kind: str = "uniform01", param: float = 1.0, seed: int = 2,
                 threads: int = 0) -> np.ndarray:
    """One property weight per undirected edge (mirrored entries equal).
    kinds: uniform01 -> (0,1]; uniform15 -> [1,5); lognormal -> exp(param*Z);
    pareto -> classical Pareto with x_m = 1 and shape param."""
    lib = _load()
    out = np.empty(g.e, dtype=np.float32)
    rc = lib.fws_edge_weights(g.offsets.ctypes.data, g.cols.ctypes.data, g.n, WEIGHT_KINDS[kind],
                              float(param), seed, out.ctypes.data, threads)
    if rc != 0:
        raise ValueError("fws_edge_weights: bad arguments")
    return out


def degree_weights(g: Csr) -> np.ndarray:
    """Degree-based property weights: h(v, u) = d(u), the target's degree
    (not symmetric: h(v, u) != h(u, v) in general)."""
    return g.degrees()[g.cols].astype(np.float32)


def edge_labels(g: Csr, nlabels: int = 5, seed: int = 3, threads: int = 0) -> np.ndarray:
    """One label in {0..nlabels-1} per undirected edge (mirrored entries equal)."""
    lib = _load()
    out = np.empty(g.e, dtype=np.uint8)
    rc = lib.fws_edge_labels(g.offsets.ctypes.data, g.cols.ctypes.data, g.n, nlabels, seed,
                             out.ctypes.data, threads)
    if rc != 0:
        raise ValueError("fws_edge_labels: bad arguments")
    return out


def random_starts(n: int, count: int, seed: int) -> np.ndarray:
    """`count` start nodes uniform over [0, n) (numpy PCG64, platform independent)."""
    return np.random.default_rng(seed).integers(0, n, size=count, dtype=np.int64).astype(np.int32)


def random_graph(n: int, p_edge: float, seed: int, weighted: bool = True, nlabels: int = 0) -> Csr:
    """Small Erdos-Renyi style undirected graph (no self-loops) for tests."""
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < p_edge
    m = np.triu(m, 1)
    m = m | m.T
    rows = [np.nonzero(m[i])[0].astype(np.int32) for i in range(n)]
    offsets = np.zeros(n + 1, dtype=np.int32)
    offsets[1:] = np.cumsum([len(r) for r in rows])
    cols = np.concatenate(rows).astype(np.int32) if offsets[-1] > 0 else np.zeros(0, np.int32)
    g = Csr(offsets, cols)
    if weighted:
        wm = np.triu(1.0 - rng.random((n, n)), 1)
        wm = (wm + wm.T).astype(np.float32)
        g.h = np.concatenate([wm[i, rows[i]] for i in range(n)]).astype(np.float32) if g.e else np.zeros(0, np.float32)
    if nlabels:
        lm = np.triu(rng.integers(0, nlabels, (n, n)), 1)
        lm = lm + lm.T
        g.labels = np.concatenate([lm[i, rows[i]] for i in range(n)]).astype(np.uint8) if g.e else np.zeros(0, np.uint8)
    return g


def from_edges(n: int, edges, h=None, labels=None) -> Csr:
    """Symmetric CSR from an undirected edge list [(u, v), ...]; optional
    per-edge weight and label lists in the same order as `edges`."""
    adj = [dict() for _ in range(n)]
    for i, (u, v) in enumerate(edges):
        if u == v:
            raise ValueError("self-loop")
        attr = (1.0 if h is None else float(h[i]), 0 if labels is None else int(labels[i]))
        adj[u][v] = attr
        adj[v][u] = attr
    offsets = np.zeros(n + 1, dtype=np.int32)
    cols, hs, ls = [], [], []
    for u in range(n):
        for v in sorted(adj[u]):
            cols.append(v)
            hs.append(adj[u][v][0])
            ls.append(adj[u][v][1])
        offsets[u + 1] = len(cols)
    g = Csr(offsets, np.asarray(cols, dtype=np.int32))
    if h is not None:
        g.h = np.asarray(hs, dtype=np.float32)
    if labels is not None:
        g.labels = np.asarray(ls, dtype=np.uint8)
    return g


# Workload recipes (sizes and distributions of the paper's evaluation,
# Sec. 5.1, on R-MAT stand-ins for its real graphs).
def workload_graph(name: str, threads: int = 0) -> Csr:
    """Graphs of the named workloads:
      small   : R-MAT s12 ef16 (.57,.19,.19), h ~ U(0,1]
      s22     : R-MAT s22 ef16 (.57,.19,.19), h ~ U(0,1], labels U{0..4}
      s23_meta: R-MAT s23 ef16 (.57,.19,.19), h ~ lognormal(0,1), labels U{0..4}
      s24_skew: R-MAT s24 ef24 (.7,.1,.1),   h ~ U(0,1], labels U{0..4}
    Generator seed 1, weight seed 2, label seed 3."""
    if name == "small":
        g = rmat(12, 16, 0.57, 0.19, 0.19, seed=1, threads=threads)
        g.h = edge_weights(g, "uniform01", seed=2, threads=threads)
        g.labels = edge_labels(g, 5, seed=3, threads=threads)
    elif name == "s22":
        g = rmat(22, 16, 0.57, 0.19, 0.19, seed=1, threads=threads)
        g.h = edge_weights(g, "uniform01", seed=2, threads=threads)
        g.labels = edge_labels(g, 5, seed=3, threads=threads)
    elif name == "s23_meta":
        g = rmat(23, 16, 0.57, 0.19, 0.19, seed=1, threads=threads)
        g.h = edge_weights(g, "lognormal", 1.0, seed=2, threads=threads)
        g.labels = edge_labels(g, 5, seed=3, threads=threads)
    elif name == "s24_skew":
        g = rmat(24, 24, 0.7, 0.1, 0.1, seed=1, threads=threads)
        g.h = edge_weights(g, "uniform01", seed=2, threads=threads)
        g.labels = edge_labels(g, 5, seed=3, threads=threads)
    else:
        raise KeyError(name)
    return g
