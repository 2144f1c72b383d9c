"""The library's bounded device-side waits, made to run out on purpose in a
test-only build of libsd (never the product default):

* SD_SORT_SPIN_LIMIT = -1: every tile of every radix-sort pass but the first
  gives up its decoupled look-back at once and counts its digit prefix
  directly from the keys. The build's Morton sort and the query order must
  still be exact: the tree equals the oracle's bit for bit and the order
  equals the product library's.
* SD_TC_WAIT_LIMIT = 0: the tcgen05 kernel's first mbarrier wait of every
  warp group runs out. The call must return, every output row must be NaN
  (the group drains its committed GEMM, issues nothing more and frees its
  tensor memory), and the product library must run normally afterwards on
  the same device.

Nothing here can fault or hang: the waits end after a bounded number of
polls, the sort's fallback reads only keys of earlier tiles of the same
pass, and the drained tile writes only its own rows.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

DEFINES = ("SD_SORT_SPIN_LIMIT=-1", "SD_TC_WAIT_LIMIT=0")


@pytest.fixture(scope="module")
def waits_lib():
    from paper_2108_10480_gb300 import _native, build_ext
    path = build_ext.build(tag="waits", defines=DEFINES)
    L = ctypes.CDLL(path)
    for name, (res, args) in _native.SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_sort_look_back_fallback_is_exact(waits_lib):
    from paper_2108_10480_gb300 import SmoothDistance, _native
    L = waits_lib
    V, F = synth.icosphere(4)
    V = synth.perturb_radial(V, 0.01, 2)
    Vt, Ft = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    g = _native.SdGeometry()
    g.tris = _native.SdTris(_p(Vt), V.shape[0], _p(Ft), F.shape[0])
    bo = _native.SdBuildOpts()
    L.sd_default_build_opts(ctypes.byref(bo))
    tree = ctypes.c_void_p()
    assert L.sd_build(ctypes.byref(g), 100.0, 0.5, ctypes.byref(bo), _stream(), ctypes.byref(tree)) == 0
    info = _native.SdTreeInfo()
    assert L.sd_tree_get_info(tree, ctypes.byref(info)) == 0
    n, nb = info.n_prims, info.n_buckets
    codes = np.zeros(n, np.uint64)
    srt = np.zeros(n, np.int32)
    left = np.zeros(nb - 1, np.int32)
    right = np.zeros(nb - 1, np.int32)
    view = _native.SdTreeView()
    view.codes = ctypes.c_void_p(codes.ctypes.data)
    view.sorted = ctypes.c_void_p(srt.ctypes.data)
    view.left = ctypes.c_void_p(left.ctypes.data)
    view.right = ctypes.c_void_p(right.ctypes.data)
    assert L.sd_tree_export(tree, ctypes.byref(view)) == 0
    o = oracle.Scene(tri_V=V, tri_F=F).build_tree(1)
    assert np.array_equal(codes, o["codes"]) and np.array_equal(srt.astype(np.int64), o["sorted"])
    assert np.array_equal(left, o["left"]) and np.array_equal(right, o["right"])
    # the query order (24-bit Hilbert keys, three passes over 80 tiles)
    q = torch.from_numpy(synth.shell_queries(81_920, seed=4)).cuda()
    order = torch.empty(q.shape[0], dtype=torch.int32, device="cuda")
    assert L.sd_query_order(tree, _p(q), q.shape[0], _p(order), _stream()) == 0
    assert L.sd_query_status(tree, _stream()) == 0
    ref = SmoothDistance(tris=(V, F), alpha=100.0, beta=0.5, device="cuda:0").query_order(q)
    torch.cuda.synchronize()
    assert torch.equal(order, ref)
    L.sd_free(tree)


def test_tensor_core_wait_runs_out_and_returns(waits_lib):
    from paper_2108_10480_gb300.surrogate import Surrogate
    L = waits_lib
    sur = Surrogate((-2.0, -2.0, -2.0), (2.0, 2.0, 2.0), seed=1, device="cuda:0")
    x = torch.rand(3000, 3, device="cuda") * 4.0 - 2.0
    y = torch.zeros(3000, device="cuda")
    dy = torch.zeros(3000, 3, device="cuda")
    fr = np.ascontiguousarray(sur.frame, np.float32)       # host float[7]
    rc = L.sd_mlp_forward(_p(sur.params), ctypes.c_void_p(fr.ctypes.data), _p(x), x.shape[0], _p(y), _p(dy),
                          _stream())
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.isnan(y).all() and torch.isnan(dy).all()
    # the product library on the same device afterwards
    y2, dy2 = sur.forward(x)
    torch.cuda.synchronize()
    assert torch.isfinite(y2).all() and torch.isfinite(dy2).all()
