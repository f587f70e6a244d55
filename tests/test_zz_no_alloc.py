"""fw_walk_host_noalloc -- the host-buffer walk for callers that cannot
allocate device memory (their own pool owns the GPU, or allocation is
forbidden after start-up) -- must return exactly the rows of fw_walk_host,
call after call, although every call reuses the same fixed device array,
and it must not allocate: neither device memory (cudaMalloc, which would
show in the device's free bytes) nor the default stream-ordered pool
(cudaMallocAsync, which would raise the pool's used-memory high-water
mark)."""
import ctypes

import numpy as np
import pytest

import oracle
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
    assert b"at most" in fw.lib().fw_last_error()
    G.close()


CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8  # CUmemPool_attribute in cuda.h


def _pool_high_water():
    """(read, reset) of the used-memory high-water mark of the current device's
    default stream-ordered pool, through the driver API (the library links its
    own static runtime, but the default pool is the driver's)."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0

    def read():
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value

    def reset():
        z = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(z)) == 0

    return read, reset


def test_noalloc_walk_allocates_nothing():
    """Warm up once on one graph (loads the library's module, which holds the
    fixed array, and the walk kernels), then walk a freshly created graph
    twice with different shapes: the device's free bytes and the default
    pool's high-water mark stay where they were, and the rows equal the
    oracle's exact-mode walks.  The second call is larger than the first and
    close to the array's limit, so staging it anywhere else would take about
    14 MB of fresh device memory."""
    fn = _noalloc()
    stream = torch.cuda.current_stream().cuda_stream
    g = synth.workload_graph("small")
    calls = [(synth.random_starts(g.n, 5000, seed=41), 20, fw.make_params(2.0, 0.5, mode="exact"), 42),
             (synth.random_starts(g.n, 160_000, seed=42), 21, fw.make_params(0.25, 4.0, mode="exact",
                                                                               walker_base=77), 9)]
    warm = fw.Graph(synth.rmat(9, 8, seed=3))
    for starts, length, prm, seed in calls:
        st = np.ascontiguousarray(starts % warm.n, dtype=np.int32)
        out = np.empty((st.shape[0], length + 1), dtype=np.int32)
        assert fn(warm.handle, st.ctypes.data, st.shape[0], length, fw.ALGO["node2vec"], ctypes.byref(prm), seed,
                  out.ctypes.data, stream) == 0, fw.lib().fw_last_error()
    warm.close()
    G = fw.Graph(g)  # fresh graph: its host-walk staging has never been allocated
    torch.cuda.synchronize()
    read_high, reset_high = _pool_high_water()
    reset_high()
    free0 = torch.cuda.mem_get_info()[0]
    high0 = read_high()
    for starts, length, prm, seed in calls:
        got = np.full((starts.shape[0], length + 1), -7, dtype=np.int32)
        st = fn(G.handle, starts.ctypes.data, starts.shape[0], length, fw.ALGO["node2vec"], ctypes.byref(prm), seed,
                got.ctypes.data, stream)
        assert st == 0, fw.lib().fw_last_error()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed: the call allocated"
        assert read_high() == high0, "the default stream-ordered pool was used: the call allocated"
        ref, _ = oracle.walk(g, starts, length, "node2vec", prm.p, prm.q, seed=seed, walker_base=prm.walker_base)
        np.testing.assert_array_equal(got, ref)
    G.close()


def test_noalloc_rejects_sizes_whose_product_wraps():
    """num_walkers = len = INT32_MAX: 4 * W * (L + 1) wraps a 64-bit size to
    0; the call must still see that the request does not fit (it returns
    before touching the buffers, which are never read here)."""
    fn = _noalloc()
    g = synth.rmat(8, 8, seed=2)
    G = fw.Graph(g)
    dummy = np.zeros(1, dtype=np.int32)
    prm = fw.make_params()
    big = 2**31 - 1
    st = fn(G.handle, dummy.ctypes.data, big, big, 0, ctypes.byref(prm), 1, dummy.ctypes.data,
            torch.cuda.current_stream().cuda_stream)
    assert st == -1, fw.lib().fw_last_error()
    assert b"does not fit" in fw.lib().fw_last_error()
    G.close()
