"""Thin Python binding of the C ABI in include/flexiwalk.h (argument
marshalling only).  Every step of the walk runs in the CUDA library; torch
supplies device memory and streams.  If the library is missing the calls
raise -- there is no fallback.

Functions carry the C names (fw_graph_create, fw_walk, ...); `Graph` wraps a
handle for convenience.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import _build

ALGO = {"weighted": 0, "node2vec": 1, "metapath": 2, "pagerank2": 3}
MODE = {"auto": 0, "rjs": 1, "rvs": 2, "exact": 3, "random": 4, "degree": 5}
FLAG_RVS_NOJUMP, FLAG_COUNTERS, FLAG_UNWEIGHTED, FLAG_PLAIN_RJS, FLAG_PAPER_SUM, FLAG_NO_BLOOM = 1, 2, 4, 8, 16, 32
FLAG_NO_GROUPS, FLAG_NO_TABLE, FLAG_NO_HUB_SHARE = 64, 128, 256
PTR_HOST, PTR_DEVICE = 0, 1
STATUS = {0: "FW_OK", -1: "FW_ERR_ARG", -2: "FW_ERR_CSR", -3: "FW_ERR_OOM", -4: "FW_ERR_CUDA",
          -5: "FW_ERR_TIMEOUT", -6: "FW_ERR_DEVICE_CHECK", -7: "FW_ERR_BUSY", -8: "FW_ERR_UNSUPPORTED"}


class FlexiWalkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class fw_params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_float), ("q", ctypes.c_float), ("schema", ctypes.c_uint8 * 16),
                ("schema_len", ctypes.c_int32), ("mode", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("cost_ratio", ctypes.c_float), ("rjs_cap", ctypes.c_int32), ("walker_base", ctypes.c_uint32),
                ("gamma", ctypes.c_float), ("lane_max_degree", ctypes.c_int32), ("rjs_batch", ctypes.c_int32),
                ("trial_budget", ctypes.c_float)]


class fw_graph_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("e", ctypes.c_int64), ("max_degree", ctypes.c_int32),
                ("has_weights", ctypes.c_int32), ("has_labels", ctypes.c_int32), ("cost_ratio", ctypes.c_float),
                ("preprocess_ms", ctypes.c_double), ("device_bytes", ctypes.c_size_t), ("symmetric", ctypes.c_int32),
                ("cost_ratios", ctypes.c_float * 4), ("fingerprint", ctypes.c_uint64),
                ("weight_scale", ctypes.c_float), ("lane_max_degrees", ctypes.c_int32 * 4),
                ("rjs_batches", ctypes.c_int32 * 4), ("trial_budgets", ctypes.c_float * 4)]


class fw_job(ctypes.Structure):
    _fields_ = [("starts", ctypes.c_void_p), ("num_walkers", ctypes.c_int32), ("len", ctypes.c_int32),
                ("algo", ctypes.c_int32), ("params", fw_params), ("seed", ctypes.c_uint64), ("out", ctypes.c_void_p)]


class fw_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_waves", ctypes.c_int32), ("max_jobs_per_wave", ctypes.c_int32),
                ("large_query_steps", ctypes.c_int64)]


class fw_server_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("waves", ctypes.c_uint64), ("queries_per_wave", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("peak_device_bytes", ctypes.c_size_t), ("peak_inflight_waves", ctypes.c_int32),
                ("walker_steps", ctypes.c_uint64),
                ("queue_p50_ms", ctypes.c_double), ("queue_p99_ms", ctypes.c_double),
                ("wave_p50_ms", ctypes.c_double), ("wave_p99_ms", ctypes.c_double),
                ("enqueue_ms_per_wave", ctypes.c_double), ("copies", ctypes.c_uint64)]


COUNTER_FIELDS = ["hops", "rjs_steps", "rvs_steps", "exact_steps", "handoffs", "rjs_trials", "rvs_items",
                  "rvs_keys", "probes", "dead_ends", "bytes"]


class fw_counters(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in COUNTER_FIELDS]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    """The built library; FLEXIWALK_LIB overrides it (e.g. to compare builds)."""
    return os.environ.get("FLEXIWALK_LIB") or _build.LIB


def lib() -> ctypes.CDLL:
    """Load libflexiwalk.so (built by __graft_entry__.build()).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} missing (run __graft_entry__.build())")
            L = ctypes.CDLL(path)
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            P = ctypes.POINTER
            sig = {
                "fw_params_default": (None, [P(fw_params)]),
                "fw_graph_create": (ctypes.c_int, [vp, vp, vp, vp, i32, i64, i32, vp, P(vp)]),
                "fw_graph_destroy": (ctypes.c_int, [vp]),
                "fw_graph_info": (ctypes.c_int, [vp, P(fw_graph_info_t)]),
                "fw_graph_node_stats": (ctypes.c_int, [vp, vp, vp, vp]),
                "fw_graph_set_cost_ratio": (ctypes.c_int, [vp, ctypes.c_float]),
                "fw_graph_label_stats": (ctypes.c_int, [vp, vp, vp]),
                "fw_graph_quantize_weights": (ctypes.c_int, [vp, P(ctypes.c_float), vp]),
                "fw_graph_weight_scales": (ctypes.c_int, [vp, vp, vp]),
                "fw_autotune": (ctypes.c_int, [vp, i32, P(fw_params), i32, ctypes.c_char_p, P(ctypes.c_float), vp]),
                "fw_walk": (ctypes.c_int, [vp, vp, i32, i32, i32, P(fw_params), u64, vp, vp]),
                "fw_walk_host": (ctypes.c_int, [vp, vp, i32, i32, i32, P(fw_params), u64, vp, vp]),
                "fw_walk_ids": (ctypes.c_int, [vp, vp, vp, i32, i32, i32, P(fw_params), u64, vp, vp]),
                "fw_sample_hist": (ctypes.c_int, [vp, i32, i32, i32, i32, P(fw_params), u64, i64, vp, vp]),
                "fw_step_plan": (ctypes.c_int, [vp, vp, vp, i32, i32, P(fw_params), vp, vp, vp, vp]),
                "fw_counters_read": (ctypes.c_int, [vp, P(fw_counters), vp]),
                "fw_counters_reset": (ctypes.c_int, [vp, vp]),
                "fw_graph_check": (ctypes.c_int, [vp, vp]),
                "fw_walk_batch": (ctypes.c_int, [vp, P(fw_job), i32, vp]),
                "fw_batch_plan_create": (ctypes.c_int, [vp, P(fw_job), i32, P(vp)]),
                "fw_batch_plan_launch": (ctypes.c_int, [vp, vp]),
                "fw_batch_plan_destroy": (ctypes.c_int, [vp]),
                "fw_walk_host_noalloc": (ctypes.c_int, [vp, vp, i32, i32, i32, P(fw_params), u64, vp, vp]),
                "fw_server_config_default": (None, [P(fw_server_config)]),
                "fw_server_create": (ctypes.c_int, [vp, P(fw_server_config), P(vp)]),
                "fw_server_submit": (ctypes.c_int, [vp, vp, i32, i32, i32, P(fw_params), u64, vp,
                                                     P(ctypes.c_uint64)]),
                "fw_server_submit_many": (ctypes.c_int, [vp, vp, i32, vp, P(i32)]),
                "fw_server_poll_many": (ctypes.c_int, [vp, vp, i32, vp, vp, vp]),
                "fw_server_poll": (ctypes.c_int, [vp, ctypes.c_uint64, P(i32), P(ctypes.c_double)]),
                "fw_server_wait": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_double, P(ctypes.c_double)]),
                "fw_server_stats": (ctypes.c_int, [vp, P(fw_server_stats_t)]),
                "fw_server_destroy": (ctypes.c_int, [vp]),
                "fw_gather_ceiling": (ctypes.c_int, [vp, u64, P(ctypes.c_double), vp]),
                "fw_launch_count": (ctypes.c_uint64, []),
                "fw_last_error": (ctypes.c_char_p, []),
                "fw_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise FlexiWalkError(status, lib().fw_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(p: float = 1.0, q: float = 1.0, schema: Optional[Sequence[int]] = None, mode="auto", flags: int = 0,
                cost_ratio: float = 0.0, rjs_cap: int = 0, walker_base: int = 0, gamma: float = 0.2,
                lane_max_degree: int = 0, rjs_batch: int = 0, trial_budget: float = 0.0) -> fw_params:
    prm = fw_params()
    lib().fw_params_default(ctypes.byref(prm))
    prm.p, prm.q = float(p), float(q)
    prm.gamma = float(gamma)
    if schema is not None:
        s = list(schema)
        if not 1 <= len(s) <= 16:
            raise ValueError("schema length must be 1..16")
        for i, x in enumerate(s):
            prm.schema[i] = int(x)
        prm.schema_len = len(s)
    prm.mode = MODE[mode] if isinstance(mode, str) else int(mode)
    prm.flags = int(flags)
    prm.cost_ratio = float(cost_ratio)
    prm.rjs_cap = int(rjs_cap)
    prm.walker_base = int(walker_base)
    prm.lane_max_degree = int(lane_max_degree)
    prm.rjs_batch = int(rjs_batch)
    prm.trial_budget = float(trial_budget)
    return prm


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def fw_graph_create(offsets, cols, weights=None, labels=None, stream=None) -> int:
    """Arrays may be numpy (host) or torch CUDA tensors (device); all of one kind."""
    is_np = isinstance(offsets, np.ndarray)
    if is_np:
        offsets = np.ascontiguousarray(offsets, dtype=np.int32)
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        weights = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        labels = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
        n, e = offsets.shape[0] - 1, cols.shape[0]
        kind = PTR_HOST
    else:
        n, e = offsets.numel() - 1, cols.numel()
        kind = PTR_DEVICE
    h = ctypes.c_void_p()
    _check(lib().fw_graph_create(_ptr(offsets), _ptr(cols), _ptr(weights), _ptr(labels), n, e, kind,
                                 _stream_ptr(stream) if kind == PTR_DEVICE or stream is not None else None,
                                 ctypes.byref(h)))
    return h.value


def fw_graph_destroy(handle: int):
    _check(lib().fw_graph_destroy(handle))


def fw_graph_info(handle: int) -> dict:
    info = fw_graph_info_t()
    _check(lib().fw_graph_info(handle, ctypes.byref(info)))
    d = {f: getattr(info, f) for f, _ in fw_graph_info_t._fields_}
    for k in ("cost_ratios", "lane_max_degrees", "rjs_batches", "trial_budgets"):
        d[k] = list(d[k])
    return d


def fw_walk(handle: int, starts, length: int, algo, params: fw_params, seed: int, out, stream=None):
    """starts: CUDA int32 [W]; out: CUDA int32 [W, length+1]."""
    _check(lib().fw_walk(handle, _ptr(starts), starts.numel(), length, ALGO.get(algo, algo), ctypes.byref(params),
                         seed, _ptr(out), _stream_ptr(stream)))


def fw_walk_ids(handle: int, starts, walker_ids, length: int, algo, params: fw_params, seed: int, out, stream=None):
    """starts: CUDA int32 [W]; walker_ids: CUDA int32/uint32 [W]; out: CUDA int32 [W, length+1]."""
    _check(lib().fw_walk_ids(handle, _ptr(starts), _ptr(walker_ids), starts.numel(), length, ALGO.get(algo, algo),
                             ctypes.byref(params), seed, _ptr(out), _stream_ptr(stream)))


def fw_gather_ceiling(table, stream=None) -> float:
    """Random 32-byte gathers per second over `table` (a CUDA tensor of a
    power-of-two size >= 64 MiB, overwritten); synchronises the stream."""
    rate = ctypes.c_double()
    _check(lib().fw_gather_ceiling(_ptr(table), table.numel() * table.element_size(), ctypes.byref(rate),
                                   _stream_ptr(stream)))
    return rate.value


def fw_walk_host(handle: int, starts: np.ndarray, length: int, algo, params: fw_params, seed: int, out: np.ndarray,
                 stream=None):
    """starts / out are host buffers (numpy or pinned torch CPU tensors)."""
    n = starts.shape[0] if isinstance(starts, np.ndarray) else starts.numel()
    _check(lib().fw_walk_host(handle, _ptr(starts), n, length, ALGO.get(algo, algo), ctypes.byref(params), seed,
                              _ptr(out), _stream_ptr(stream)))


def fw_sample_hist(handle: int, v: int, v_prev: int, step: int, algo, params: fw_params, seed: int, ndraws: int,
                   counts, stream=None):
    _check(lib().fw_sample_hist(handle, v, v_prev, step, ALGO.get(algo, algo), ctypes.byref(params), seed, ndraws,
                                _ptr(counts), _stream_ptr(stream)))


def fw_step_plan(handle: int, v, v_prev, algo, params: fw_params, bound, sum_hat, mode, stream=None):
    _check(lib().fw_step_plan(handle, _ptr(v), _ptr(v_prev), v.numel(), ALGO.get(algo, algo), ctypes.byref(params),
                              _ptr(bound), _ptr(sum_hat), _ptr(mode), _stream_ptr(stream)))


def fw_graph_node_stats(handle: int, hmax, hsum, stream=None):
    _check(lib().fw_graph_node_stats(handle, _ptr(hmax), _ptr(hsum), _stream_ptr(stream)))


def fw_graph_set_cost_ratio(handle: int, ratio: float):
    _check(lib().fw_graph_set_cost_ratio(handle, float(ratio)))


def fw_autotune(handle: int, algo, params: fw_params, method: int = 0, cache_path: Optional[str] = None,
                stream=None) -> float:
    r = ctypes.c_float()
    _check(lib().fw_autotune(handle, ALGO.get(algo, algo), ctypes.byref(params), method,
                             None if cache_path is None else os.fsencode(cache_path), ctypes.byref(r),
                             _stream_ptr(stream)))
    return float(r.value)


def fw_counters_read(handle: int, stream=None) -> dict:
    c = fw_counters()
    _check(lib().fw_counters_read(handle, ctypes.byref(c), _stream_ptr(stream)))
    return {f: int(getattr(c, f)) for f in COUNTER_FIELDS}


def fw_counters_reset(handle: int, stream=None):
    _check(lib().fw_counters_reset(handle, _stream_ptr(stream)))


def fw_graph_check(handle: int, stream=None):
    _check(lib().fw_graph_check(handle, _stream_ptr(stream)))


def fw_launch_count() -> int:
    return int(lib().fw_launch_count())


class Graph:
    """A device-resident graph: CSR int32 offsets / cols, optional FP32
    property weights h and uint8 labels."""

    def __init__(self, csr=None, *, offsets=None, cols=None, weights=None, labels=None, stream=None):
        if csr is not None:
            offsets, cols = csr.offsets, csr.cols
            weights, labels = getattr(csr, "h", None), getattr(csr, "labels", None)
        self._off = np.asarray(offsets) if isinstance(offsets, np.ndarray) else offsets.cpu().numpy()
        self.handle = fw_graph_create(offsets, cols, weights, labels, stream)
        self.info = fw_graph_info(self.handle)
        self.n, self.e = self.info["n"], self.info["e"]

    def close(self):
        if self.handle:
            fw_graph_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def walk(self, starts, length: int, algo="node2vec", *, p=1.0, q=1.0, schema=None, mode="auto", seed=42,
             flags=0, cost_ratio=0.0, rjs_cap=0, walker_base=0, gamma=0.2, out=None, stream=None, **shape):
        """shape: lane_max_degree / rjs_batch / trial_budget of fw_params (0: the graph's tuned value)."""
        import torch
        if out is None:
            out = torch.empty((starts.numel(), length + 1), dtype=torch.int32, device=starts.device)
        prm = make_params(p, q, schema, mode, flags, cost_ratio, rjs_cap, walker_base, gamma, **shape)
        fw_walk(self.handle, starts, length, algo, prm, seed, out, stream)
        return out

    def walk_ids(self, starts, walker_ids, length: int, algo="node2vec", *, p=1.0, q=1.0, schema=None, mode="auto",
                 seed=42, flags=0, cost_ratio=0.0, rjs_cap=0, gamma=0.2, out=None, stream=None, **shape):
        import torch
        if out is None:
            out = torch.empty((starts.numel(), length + 1), dtype=torch.int32, device=starts.device)
        prm = make_params(p, q, schema, mode, flags, cost_ratio, rjs_cap, 0, gamma, **shape)
        fw_walk_ids(self.handle, starts, walker_ids, length, algo, prm, seed, out, stream)
        return out

    def walk_host(self, starts, length: int, algo="node2vec", *, p=1.0, q=1.0, schema=None, mode="auto", seed=42,
                  flags=0, cost_ratio=0.0, rjs_cap=0, walker_base=0, gamma=0.2, out=None, stream=None, **shape):
        if out is None:
            out = np.empty((len(starts), length + 1), dtype=np.int32)
        prm = make_params(p, q, schema, mode, flags, cost_ratio, rjs_cap, walker_base, gamma, **shape)
        fw_walk_host(self.handle, starts, length, algo, prm, seed, out, stream)
        return out

    def sample_hist(self, v: int, v_prev: int, step: int, algo="node2vec", ndraws: int = 1_000_000, *, p=1.0, q=1.0,
                    schema=None, mode="auto", seed=42, flags=0, cost_ratio=0.0, rjs_cap=0, walker_base=0,
                    gamma=0.2, stream=None, **shape):
        import torch
        d = self.degree(v)
        counts = torch.zeros(max(d, 1), dtype=torch.int64, device="cuda")
        prm = make_params(p, q, schema, mode, flags, cost_ratio, rjs_cap, walker_base, gamma, **shape)
        fw_sample_hist(self.handle, v, v_prev, step, algo, prm, seed, ndraws, counts, stream)
        return counts[:d]

    def step_plan(self, v, v_prev, algo="node2vec", *, p=1.0, q=1.0, schema=None, cost_ratio=0.0, gamma=0.2,
                  stream=None):
        """(mode, B, sum_hat) for states (v[i], v_prev[i]); v_prev[i] = -1: no previous node."""
        import torch
        bound = torch.empty(v.numel(), dtype=torch.float32, device=v.device)
        s = torch.empty_like(bound)
        m = torch.empty(v.numel(), dtype=torch.int32, device=v.device)
        prm = make_params(p, q, schema, "auto", 0, cost_ratio, 0, 0, gamma)
        fw_step_plan(self.handle, v, v_prev, algo, prm, bound, s, m, stream)
        return m, bound, s

    def node_stats(self, stream=None):
        import torch
        hmax = torch.empty(self.n, dtype=torch.float32, device="cuda")
        hsum = torch.empty_like(hmax)
        fw_graph_node_stats(self.handle, hmax, hsum, stream)
        return hmax, hsum

    def label_stats(self, stream=None):
        """Per-label node statistics as a CUDA float32 tensor [n, 8, 2] (max, sum)."""
        import torch
        out = torch.empty((self.n, 8, 2), dtype=torch.float32, device="cuda")
        _check(lib().fw_graph_label_stats(self.handle, _ptr(out), _stream_ptr(stream)))
        return out

    def counters(self, stream=None) -> dict:
        return fw_counters_read(self.handle, stream)

    def reset_counters(self, stream=None):
        fw_counters_reset(self.handle, stream)

    def check(self, stream=None):
        fw_graph_check(self.handle, stream)

    def autotune(self, algo="node2vec", *, p=1.0, q=1.0, schema=None, gamma=0.2, flags=0, method=0,
                 cache_path=None, stream=None):
        r = fw_autotune(self.handle, algo, make_params(p, q, schema, flags=flags, gamma=gamma), method, cache_path,
                        stream)
        self.info = fw_graph_info(self.handle)
        return r

    def set_cost_ratio(self, r: float):
        fw_graph_set_cost_ratio(self.handle, r)
        self.info = fw_graph_info(self.handle)

    def quantize_weights(self, stream=None) -> float:
        """Switch the graph to 8-bit weight codes (code * the scale of the
        row's node); returns the largest per-node scale."""
        s = ctypes.c_float()
        _check(lib().fw_graph_quantize_weights(self.handle, ctypes.byref(s), _stream_ptr(stream)))
        self.info = fw_graph_info(self.handle)
        return float(s.value)

    def weight_scales(self, stream=None):
        """Per-node scales of the 8-bit codes as a CUDA float32 tensor [n]."""
        import torch
        out = torch.empty(max(self.n, 1), dtype=torch.float32, device="cuda")
        _check(lib().fw_graph_weight_scales(self.handle, _ptr(out), _stream_ptr(stream)))
        return out[:self.n]

    def degree(self, v: int) -> int:
        return int(self._off[v + 1] - self._off[v])


# ---------------------------------------------------------------- batching
def make_job(starts, length: int, algo, out, *, p=1.0, q=1.0, schema=None, mode="auto", seed=42, flags=0,
             cost_ratio=0.0, rjs_cap=0, walker_base=0, gamma=0.2, **shape) -> fw_job:
    """One batch entry; starts / out are CUDA tensors that must outlive the launch."""
    j = fw_job()
    j.starts = _ptr(starts)
    j.num_walkers = starts.numel()
    j.len = length
    j.algo = ALGO.get(algo, algo)
    j.params = make_params(p, q, schema, mode, flags, cost_ratio, rjs_cap, walker_base, gamma, **shape)
    j.seed = seed
    j.out = _ptr(out)
    return j


def make_host_query(starts: np.ndarray, length: int, algo, out: np.ndarray, *, p=1.0, q=1.0, schema=None,
                    mode="auto", seed=42, flags=0, walker_base=0, gamma=0.2) -> fw_job:
    """One query for Server.submit_many: starts / out are host numpy arrays
    (int32[W], int32[W][length+1]) that must outlive the query."""
    j = fw_job()
    j.starts = starts.ctypes.data
    j.num_walkers = starts.shape[0]
    j.len = length
    j.algo = ALGO.get(algo, algo)
    j.params = make_params(p, q, schema, mode, flags, 0.0, 0, walker_base, gamma)
    j.seed = seed
    j.out = out.ctypes.data
    return j


def fw_walk_batch(handle: int, jobs, stream=None):
    arr = (fw_job * len(jobs))(*jobs)
    _check(lib().fw_walk_batch(handle, arr, len(jobs), _stream_ptr(stream)))


class BatchPlan:
    """A batch captured once into a CUDA graph and replayed by launch()."""

    def __init__(self, graph: "Graph", jobs):
        self._jobs = (fw_job * len(jobs))(*jobs)
        h = ctypes.c_void_p()
        _check(lib().fw_batch_plan_create(graph.handle, self._jobs, len(jobs), ctypes.byref(h)))
        self.handle = h.value

    def launch(self, stream=None):
        _check(lib().fw_batch_plan_launch(self.handle, _stream_ptr(stream)))

    def close(self):
        if self.handle:
            _check(lib().fw_batch_plan_destroy(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving
class Server:
    """Continuous-batching walk server over a resident Graph (C ABI fw_server_*)."""

    def __init__(self, graph: "Graph", mem_budget: int = 1 << 30, max_waves: int = 4, max_jobs_per_wave: int = 64,
                 large_query_steps: Optional[int] = None):
        cfg = fw_server_config()
        lib().fw_server_config_default(ctypes.byref(cfg))
        cfg.mem_budget, cfg.max_waves, cfg.max_jobs_per_wave = mem_budget, max_waves, max_jobs_per_wave
        if large_query_steps is not None:
            cfg.large_query_steps = large_query_steps
        h = ctypes.c_void_p()
        _check(lib().fw_server_create(graph.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self.graph = graph

    def submit(self, starts, length: int, algo, out, *, p=1.0, q=1.0, schema=None, mode="auto", seed=42, flags=0,
               walker_base=0, gamma=0.2) -> int:
        """starts / out: host buffers (numpy or pinned torch CPU tensors) kept alive until collected."""
        n = starts.shape[0] if isinstance(starts, np.ndarray) else starts.numel()
        prm = make_params(p, q, schema, mode, flags, 0.0, 0, walker_base, gamma)
        t = ctypes.c_uint64()
        _check(lib().fw_server_submit(self.handle, _ptr(starts), n, length, ALGO.get(algo, algo), ctypes.byref(prm),
                                      seed, _ptr(out), ctypes.byref(t)))
        return int(t.value)

    def submit_many(self, jobs) -> np.ndarray:
        """Queue many queries in one call: `jobs` is a ctypes array of fw_job
        (make_host_query) whose buffers stay alive until collected; returns
        the tickets (uint64 numpy array)."""
        n = len(jobs)
        tickets = np.zeros(n, dtype=np.uint64)
        done = ctypes.c_int32()
        _check(lib().fw_server_submit_many(self.handle, ctypes.cast(jobs, ctypes.c_void_p), n,
                                           tickets.ctypes.data, ctypes.byref(done)))
        return tickets

    def poll_many(self, tickets: np.ndarray):
        """(done int32[n], latency_ms float64[n], status int32[n]) for the
        tickets; finished ones are released."""
        t = np.ascontiguousarray(tickets, dtype=np.uint64)
        done = np.zeros(t.shape[0], dtype=np.int32)
        lat = np.zeros(t.shape[0], dtype=np.float64)
        st = np.zeros(t.shape[0], dtype=np.int32)
        _check(lib().fw_server_poll_many(self.handle, t.ctypes.data, t.shape[0], done.ctypes.data, lat.ctypes.data,
                                         st.ctypes.data))
        return done, lat, st

    def poll(self, ticket: int):
        """None while running, else the latency in ms (the ticket is released)."""
        done = ctypes.c_int32()
        lat = ctypes.c_double()
        _check(lib().fw_server_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(lat)))
        return float(lat.value) if done.value else None

    def wait(self, ticket: int, timeout: float = 60.0) -> float:
        lat = ctypes.c_double()
        _check(lib().fw_server_wait(self.handle, ticket, timeout, ctypes.byref(lat)))
        return float(lat.value)

    def stats(self) -> dict:
        st = fw_server_stats_t()
        _check(lib().fw_server_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in fw_server_stats_t._fields_}

    def close(self):
        if self.handle:
            _check(lib().fw_server_destroy(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
