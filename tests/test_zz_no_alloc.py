"""sd_query_noalloc, the query entry point that allocates no device memory.

It exists for callers that own a fixed device-memory budget and must not let
a library call cudaMalloc while they run (an allocation there could block on
the device or fail part-way). This file is named to be collected last, so a
run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from _metrics import assert_parity

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_sd_query_on_two_calls():
    from paper_2108_10480_gb300 import SmoothDistance, _native
    lib = _native.lib()
    V, F = synth.icosphere(4)
    V = synth.perturb_radial(V, 0.01, 5)
    q = torch.from_numpy(synth.shell_queries(20000, seed=6)).cuda()
    M = q.shape[0]
    sd = SmoothDistance(tris=(V, F), alpha=200.0, beta=0.5, device="cuda:0")
    ref_v, ref_g = sd.query(q)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        v = torch.full((M,), float("nan"), device="cuda")
        g = torch.full((M, 3), float("nan"), device="cuda")
        rc = lib.sd_query_noalloc(sd.handle, _p(q), M, _p(v), _p(g), stream)
        assert rc == 0, lib.sd_status_str(rc)
        torch.cuda.synchronize()
        assert_parity(v.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64),
                      ref_v.cpu().numpy().astype(np.float64), ref_g.cpu().numpy().astype(np.float64),
                      200.0, None, f"noalloc call {call}")
    assert sd.status() == 0


def test_noalloc_rejects_more_than_its_limit():
    from paper_2108_10480_gb300 import SmoothDistance, _native
    lib = _native.lib()
    sd = SmoothDistance(points=synth.points_on_sphere(64, 0.0, 0), alpha=10.0, beta=0.5, device="cuda:0")
    q = torch.zeros(262145, 3, device="cuda")
    v = torch.empty(262145, device="cuda")
    rc = lib.sd_query_noalloc(sd.handle, _p(q), q.shape[0], _p(v), None, None)
    assert rc == 6   # SD_ERR_TOO_LARGE


def _pool_used_high(dev=0):
    """(current, high-water) bytes of the device's default memory pool,
    where stream-ordered allocations (cudaMallocAsync) come from; the
    high-water mark is reset to the current use first."""
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    cur, zero = ctypes.c_uint64(0), ctypes.c_uint64(0)
    USED_CURRENT, USED_HIGH = 7, 8        # cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh
    assert rt.cudaMemPoolGetAttribute(pool, USED_CURRENT, ctypes.byref(cur)) == 0

    def high():
        h = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(h)) == 0
        return h.value
    assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    return cur.value, high


def test_noalloc_at_its_limit_against_the_oracle_without_allocating():
    """M = 262,144, the documented maximum, where the sort's look-back words
    and tile counters sit at the end of the static array: sampled outputs
    against the FP64 oracle, and the default memory pool's high-water mark
    unchanged across two calls (the library's other entry points allocate
    from that pool)."""
    from paper_2108_10480_gb300 import SmoothDistance, _native
    lib = _native.lib()
    V, F = synth.icosphere(4)
    V = synth.perturb_radial(V, 0.01, 5)
    qn = synth.shell_queries(262144, seed=8)
    q = torch.from_numpy(qn).cuda()
    M = q.shape[0]
    sd = SmoothDistance(tris=(V, F), alpha=200.0, beta=0.5, device="cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    v = torch.empty(M, device="cuda")
    g = torch.empty(M, 3, device="cuda")
    torch.cuda.synchronize()
    used, high = _pool_used_high()
    for _ in range(2):
        assert lib.sd_query_noalloc(sd.handle, _p(q), M, _p(v), _p(g), stream) == 0
    torch.cuda.synchronize()
    assert high() == used
    idx = np.random.default_rng(3).choice(M, 3000, replace=False)
    sc = oracle.Scene(tri_V=V, tri_F=F)
    sc.build_tree(1)
    bv, bg, _, _ = sc.bh(qn[idx], 200.0, 0.5)
    assert_parity(v.cpu().numpy().astype(np.float64)[idx], g.cpu().numpy().astype(np.float64)[idx], bv, bg, 200.0,
                  None, "noalloc M=262144")
    assert sd.status() == 0


@pytest.mark.parametrize("M", [1, 2])
def test_noalloc_tiny_batches_value_only(M):
    """M = 1 (no sort: the query is its own order) and M = 2, without a
    gradient output: the values equal sd_query's value-only path."""
    from paper_2108_10480_gb300 import SmoothDistance, _native
    lib = _native.lib()
    V, F = synth.icosphere(3)
    sd = SmoothDistance(tris=(V, F), alpha=50.0, beta=0.5, device="cuda:0")
    q = torch.tensor([[0.1, 1.05, -0.2], [0.7, -0.3, 0.2]][:M], device="cuda")
    ref, _ = sd.query(q, grad=False)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        v = torch.full((M,), float("nan"), device="cuda")
        assert lib.sd_query_noalloc(sd.handle, _p(q), M, _p(v), None, stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(v, ref)
