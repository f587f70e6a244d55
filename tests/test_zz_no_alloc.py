"""fw_walk_host_noalloc -- the host-buffer walk for callers that cannot
allocate device memory (their own pool owns the GPU, or allocation is
forbidden after start-up) -- must return exactly the rows of fw_walk_host,
call after call, although every call reuses the same fixed device array."""
import ctypes

import numpy as np
import pytest

from paper_2512_00705_gb300 import flexiwalk as fw
from paper_2512_00705_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc():
    fn = fw.lib().fw_walk_host_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   ctypes.POINTER(fw.fw_params), ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def test_noalloc_walk_matches_walk_host_on_consecutive_calls():
    fn = _noalloc()
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    stream = torch.cuda.current_stream().cuda_stream
    calls = [  # (walkers, length, algo, params, seed): the second call is smaller,
               # so stale rows of the first would show up in its output
        (np.arange(g.n, dtype=np.int32), 20, "node2vec", fw.make_params(2.0, 0.5, mode="auto"), 42),
        (synth.random_starts(g.n, 777, seed=5), 9, "metapath",
         fw.make_params(schema=[0, 1, 2, 3, 4], mode="rvs", walker_base=123), 7),
    ]
    for starts, length, algo, prm, seed in calls:
        want = np.empty((starts.shape[0], length + 1), dtype=np.int32)
        fw.fw_walk_host(G.handle, starts, length, algo, prm, seed, want, stream)
        got = np.full_like(want, -7)
        st = fn(G.handle, starts.ctypes.data, starts.shape[0], length, fw.ALGO[algo], ctypes.byref(prm), seed,
                got.ctypes.data, stream)
        assert st == 0, fw.lib().fw_last_error()
        np.testing.assert_array_equal(got, want)
    G.close()


def test_noalloc_walk_rejects_requests_beyond_its_array():
    fn = _noalloc()
    g = synth.workload_graph("small")
    G = fw.Graph(g)
    starts = np.zeros(1 << 20, dtype=np.int32)           # 1 Mi walkers x 11 entries > 16 MiB
    out = np.empty((starts.shape[0], 11), dtype=np.int32)
    prm = fw.make_params()
    st = fn(G.handle, starts.ctypes.data, starts.shape[0], 10, 0, ctypes.byref(prm), 1, out.ctypes.data,
            torch.cuda.current_stream().cuda_stream)
    assert st == -1
    assert b"16" in fw.lib().fw_last_error() or b"at most" in fw.lib().fw_last_error()
    G.close()
