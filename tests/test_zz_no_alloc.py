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
