"""CPU oracle for dynamic random walks -- TEST INFRASTRUCTURE.

Only the test-suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  The GPU library never links or calls it, and it
shares no code with the GPU path.

It wraps ``fw_oracle.c`` (plain C, fp64 probabilities, FP32 inverse-CDF
sampling, its own Philox4x32-10), compiled here with gcc and
``-ffp-contract=off``.  Functions (paper sections in each docstring):

  philox4x32_10         Salmon et al., SC'11
  exact_uniform         exact-mode uniform for (seed, walker, hop)
  transition_weights    Eq. (prob) with Eq. (node2vec) / MetaPath rule / Eq. (2ndpr), FP32
  transition_probs      Eq. (prob), fp64
  icdf_pick             Sec. 2.2 inverse transform sampling, FP32
  walk                  full exact-mode walks
  walk_rjs              walks drawn hop by hop by rejection sampling (Sec. 3.3)
                        with the bound B = max(w) * h_MAX[v]
  node_stats            h_MAX / h_SUM preprocessing, Sec. 4.2
  step_plan             bound (Sec. 3.3) + sum estimate (Eq. sum_estimation)
                        + cost-model choice (Eq. runtime)
  label_stats           per-node, per-label max / sum of h (labels < 8)
  quantize_weights      8-bit weight codes with one scale per node (Sec. 6.2
                        names low-precision weights as an extension)

Graph arguments are any object with ``offsets``, ``cols``, ``h`` (or None)
and ``labels`` (or None) numpy attributes.

If the environment variable ``FW_ORACLE_LIB`` names a shared library, that
prebuilt library is loaded instead of building ``fw_oracle.c``; the mutation
tests use it to run the pins against copies of the oracle with a planted
mistake.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fw_oracle.c")
_SO = os.path.join(_HERE, "_build", "libfw_oracle.so")
_lock = threading.Lock()
_lib = None

WEIGHTED, NODE2VEC, METAPATH, PAGERANK2 = 0, 1, 2, 3
MODE_RJS, MODE_RVS = 1, 2
ALGOS = {"weighted": WEIGHTED, "node2vec": NODE2VEC, "metapath": METAPATH, "pagerank2": PAGERANK2}

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            so = os.environ.get("FW_ORACLE_LIB") or build()
            L = ctypes.CDLL(so)
            vp, i32, i64, u32, u64, f32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_float)
            L.or_philox4x32_10.argtypes = [vp, vp, vp]
            L.or_philox4x32_10.restype = None
            L.or_exact_uniform.argtypes = [u64, u32, u32]
            L.or_exact_uniform.restype = f32
            L.or_recip.argtypes = [f32]
            L.or_recip.restype = f32
            wargs = [vp, vp, vp, vp, i32, i32, i32, i32, i32, f32, f32, f32, vp, i32, vp]
            L.or_transition_weights.argtypes = wargs
            L.or_transition_weights.restype = i64
            L.or_transition_probs.argtypes = wargs
            L.or_transition_probs.restype = i64
            L.or_icdf_pick.argtypes = [vp, i64, f32]
            L.or_icdf_pick.restype = i64
            L.or_walk.argtypes = [vp, vp, vp, vp, i32, vp, i32, i32, i32, f32, f32, f32, vp, i32, u64, u32, vp, i32]
            L.or_walk.restype = i64
            L.or_walk_ids.argtypes = [vp, vp, vp, vp, i32, vp, vp, i32, i32, i32, f32, f32, f32, vp, i32, u64, vp,
                                      i32]
            L.or_walk_ids.restype = i64
            L.or_walk_rjs.argtypes = [vp, vp, vp, vp, i32, vp, i32, i32, i32, f32, f32, f32, vp, i32, u64, u32, i32, vp,
                                      i32, vp]
            L.or_walk_rjs.restype = i64
            L.or_node_stats.argtypes = [vp, vp, i32, vp, vp]
            L.or_node_stats.restype = ctypes.c_int
            L.or_step_plan.argtypes = [f32, f32, i32, i32, i32, i32, f32, f32, f32, f32, vp, vp]
            L.or_step_plan.restype = ctypes.c_int
            L.or_label_stats.argtypes = [vp, vp, vp, i32, vp, vp]
            L.or_label_stats.restype = ctypes.c_int
            L.or_quantize_weights.argtypes = [vp, i32, vp, vp, vp, vp]
            L.or_quantize_weights.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _graph_args(g):
    offsets = np.ascontiguousarray(g.offsets, dtype=np.int32)
    cols = np.ascontiguousarray(g.cols, dtype=np.int32)
    h = None if getattr(g, "h", None) is None else np.ascontiguousarray(g.h, dtype=np.float32)
    labels = None if getattr(g, "labels", None) is None else np.ascontiguousarray(g.labels, dtype=np.uint8)
    return offsets, cols, h, labels


def _schema_arr(schema):
    if schema is None or len(schema) == 0:
        return None, 0
    s = np.ascontiguousarray(np.asarray(schema, dtype=np.uint8))
    return s, int(s.shape[0])


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: ctr 4 x uint32, key 2 x uint32 -> 4 x uint32."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return tuple(int(x) for x in out)


def exact_uniform(seed: int, walker: int, hop: int) -> float:
    return float(_load().or_exact_uniform(seed, walker, hop))


def recip(p: float) -> float:
    return float(_load().or_recip(p))


def transition_weights(g, v, vprev, step, algo, p=1.0, q=1.0, schema=None, gamma=0.2):
    """FP32 transition weights of v's neighbours in CSR order."""
    L = _load()
    offsets, cols, h, labels = _graph_args(g)
    s, slen = _schema_arr(schema)
    a = ALGOS.get(algo, algo)
    d = L.or_transition_weights(_ptr(offsets), _ptr(cols), _ptr(h), _ptr(labels), offsets.shape[0] - 1,
                                v, vprev, step, a, p, q, gamma, _ptr(s), slen, None)
    if d < 0:
        raise ValueError("or_transition_weights: bad arguments")
    wt = np.zeros(d, dtype=np.float32)
    L.or_transition_weights(_ptr(offsets), _ptr(cols), _ptr(h), _ptr(labels), offsets.shape[0] - 1,
                            v, vprev, step, a, p, q, gamma, _ptr(s), slen, _ptr(wt))
    return wt


def transition_probs(g, v, vprev, step, algo, p=1.0, q=1.0, schema=None, gamma=0.2):
    """fp64 transition probabilities of v's neighbours in CSR order."""
    L = _load()
    offsets, cols, h, labels = _graph_args(g)
    s, slen = _schema_arr(schema)
    a = ALGOS.get(algo, algo)
    d = int(offsets[v + 1] - offsets[v]) if 0 <= v < offsets.shape[0] - 1 else 0
    pr = np.zeros(max(d, 1), dtype=np.float64)
    r = L.or_transition_probs(_ptr(offsets), _ptr(cols), _ptr(h), _ptr(labels), offsets.shape[0] - 1,
                              v, vprev, step, a, p, q, gamma, _ptr(s), slen, _ptr(pr))
    if r < 0:
        raise ValueError("or_transition_probs: bad arguments")
    return pr[:d]


def icdf_pick(wt, u: float) -> int:
    w = np.ascontiguousarray(wt, dtype=np.float32)
    return int(_load().or_icdf_pick(_ptr(w), w.shape[0], u))


def walk(g, starts, length, algo, p=1.0, q=1.0, schema=None, seed=42, walker_base=0, threads=0, gamma=0.2):
    """Exact-mode walks: returns (out int32[W][L+1], hops)."""
    L = _load()
    offsets, cols, h, labels = _graph_args(g)
    st = np.ascontiguousarray(starts, dtype=np.int32)
    s, slen = _schema_arr(schema)
    out = np.empty((st.shape[0], length + 1), dtype=np.int32)
    hops = L.or_walk(_ptr(offsets), _ptr(cols), _ptr(h), _ptr(labels), offsets.shape[0] - 1, _ptr(st),
                     st.shape[0], length, ALGOS.get(algo, algo), p, q, gamma, _ptr(s), slen, seed, walker_base,
                     _ptr(out), threads)
    if hops < 0:
        raise ValueError("or_walk: bad arguments")
    return out, int(hops)


def walk_rjs(g, starts, length, algo, p=1.0, q=1.0, schema=None, seed=42, walker_base=0, threads=0, gamma=0.2,
             envelope="single", return_trials=False):
    """Walks whose every hop is drawn by rejection sampling against
    B = max(w) * h_MAX[v] (Sec. 3.3), trial t of hop j of walker i using
    Philox4x32-10 counter (i, j, 1, t): an index by Lemire's method from x0
    (else x1, else no proposal) and U = (x2 >> 8) * 2^-24.  envelope
    "single": the paper's uniform proposal; "classes": the weight-class
    slots of or_walk_rjs (weighted graphs), for metapath the five classes
    inside the required label's entries.  Returns (out int32[W][L+1], hops),
    and the number of trials of all hops (void ones included) as a third
    element with return_trials."""
    L = _load()
    offsets, cols, h, labels = _graph_args(g)
    st = np.ascontiguousarray(starts, dtype=np.int32)
    s, slen = _schema_arr(schema)
    out = np.empty((st.shape[0], length + 1), dtype=np.int32)
    trials = ctypes.c_int64(0)
    hops = L.or_walk_rjs(_ptr(offsets), _ptr(cols), _ptr(h), _ptr(labels), offsets.shape[0] - 1, _ptr(st),
                         st.shape[0], length, ALGOS.get(algo, algo), p, q, gamma, _ptr(s), slen, seed, walker_base,
                         {"single": 0, "classes": 1}[envelope], _ptr(out), threads, ctypes.byref(trials))
    if hops < 0:
        raise ValueError("or_walk_rjs: bad arguments")
    return (out, int(hops), int(trials.value)) if return_trials else (out, int(hops))


def walk_ids(g, starts, ids, length, algo, p=1.0, q=1.0, schema=None, seed=42, threads=0, gamma=0.2):
    """Exact-mode walks with an explicit random-stream id per walker."""
    L = _load()
    offsets, cols, h, labels = _graph_args(g)
    st = np.ascontiguousarray(starts, dtype=np.int32)
    wi = np.ascontiguousarray(ids, dtype=np.uint32)
    assert wi.shape == st.shape
    s, slen = _schema_arr(schema)
    out = np.empty((st.shape[0], length + 1), dtype=np.int32)
    hops = L.or_walk_ids(_ptr(offsets), _ptr(cols), _ptr(h), _ptr(labels), offsets.shape[0] - 1, _ptr(st), _ptr(wi),
                         st.shape[0], length, ALGOS.get(algo, algo), p, q, gamma, _ptr(s), slen, seed, _ptr(out),
                         threads)
    if hops < 0:
        raise ValueError("or_walk_ids: bad arguments")
    return out, int(hops)


def node_stats(g):
    """(h_MAX float32[n], h_SUM float64[n])."""
    offsets, _, h, _ = _graph_args(g)
    n = offsets.shape[0] - 1
    hmax = np.zeros(n, dtype=np.float32)
    hsum = np.zeros(n, dtype=np.float64)
    _load().or_node_stats(_ptr(offsets), _ptr(h), n, _ptr(hmax), _ptr(hsum))
    return hmax, hsum


def step_plan(hmax, hsum, has_prev, algo, p=1.0, q=1.0, r=4.0, dv=1, dprev=1, gamma=0.2):
    """(mode, B, sum_hat) for one walker step; mode MODE_RJS or MODE_RVS.
    dv / dprev (degrees of v and v') matter for second-order PageRank only."""
    B = ctypes.c_float()
    S = ctypes.c_float()
    m = _load().or_step_plan(hmax, hsum, int(bool(has_prev)), int(dv), int(dprev), ALGOS.get(algo, algo), p, q, gamma,
                             r, ctypes.addressof(B), ctypes.addressof(S))
    if m < 0:
        raise ValueError("or_step_plan: bad arguments")
    return m, B.value, S.value


def label_stats(g):
    """(max float32[n][8], sum float64[n][8]) of h per node and label."""
    offsets, _, h, labels = _graph_args(g)
    n = offsets.shape[0] - 1
    lmax = np.zeros((n, 8), dtype=np.float32)
    lsum = np.zeros((n, 8), dtype=np.float64)
    if _load().or_label_stats(_ptr(offsets), _ptr(h), _ptr(labels), n, _ptr(lmax), _ptr(lsum)) != 0:
        raise ValueError("labels missing or >= 8")
    return lmax, lsum


def quantize_weights(g):
    """(codes uint8[e], scales float32[n], dequantized float32[e]) of the
    graph's property weights, one scale per node (its row's maximum / 255)."""
    offsets, _, h, _ = _graph_args(g)
    n = offsets.shape[0] - 1
    e = int(offsets[-1])
    codes = np.zeros(e, dtype=np.uint8)
    scales = np.zeros(n, dtype=np.float32)
    hq = np.zeros(e, dtype=np.float32)
    if _load().or_quantize_weights(_ptr(offsets), n, _ptr(h), _ptr(codes), _ptr(scales), _ptr(hq)) != 0:
        raise ValueError("or_quantize_weights: bad arguments")
    return codes, scales, hq
