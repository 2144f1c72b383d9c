"""GPU build (sd_build) against the oracle: Morton codes, sorted order, radix
tree topology, node and leaf AABBs, counts and weight parameters, bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(**kw):
    from paper_2108_10480_gb300 import SmoothDistance
    return SmoothDistance(device="cuda:0", **kw)


def _scene(name):
    if name == "points":
        P = synth.points_on_sphere(4096, 0.005, 0)
        return dict(points=P), oracle.Scene(points=P)
    if name == "dup_points":
        p = synth.points_on_sphere(300, 0.0, 1)
        P = np.concatenate([p, p, p[:77]])
        return dict(points=P), oracle.Scene(points=P)
    if name == "tris":
        V, F = synth.icosphere(4)
        V = synth.perturb_radial(V, 0.01, 2)
        return dict(tris=(V, F)), oracle.Scene(tri_V=V, tri_F=F)
    if name == "mixed":
        V, F = synth.icosphere(3)
        Ve, E = synth.tiny_mesh("polyline")
        P = synth.points_on_sphere(500, 0.02, 3) * 1.4
        return (dict(points=P, edges=(Ve, E), tris=(V, F)),
                oracle.Scene(points=P, edge_V=Ve, edge_E=E, tri_V=V, tri_F=F))
    if name in ("points_cap", "points_cap1"):
        # 131,072 primitives fill 128 sort tiles of 1,024 keys exactly; one
        # more adds a tile that holds a single key
        P = synth.points_on_sphere(131_072 + (name == "points_cap1"), 0.005, 5)
        return dict(points=P), oracle.Scene(points=P)
    if name == "ico6":
        c = synth.config2(m=16)
        return dict(tris=(c["V"], c["F"])), oracle.Scene(tri_V=c["V"], tri_F=c["F"])
    raise KeyError(name)


@pytest.mark.parametrize("name", ["points", "dup_points", "tris", "mixed", "ico6", "points_cap", "points_cap1"])
@pytest.mark.parametrize("L", [1, 4, 7])
def test_build_bit_exact(name, L):
    kw, sc = _scene(name)
    sd = _gpu(alpha=100.0, beta=0.5, leaf_size=L, **kw)
    g = sd.export()
    o = sc.build_tree(L)
    info = sd.info()
    assert g["nb"] == o["nb"]
    assert np.array_equal(np.array(info["scene_lo"], np.float32), o["scene_box"][:3])
    assert np.array_equal(np.array(info["scene_hi"], np.float32), o["scene_box"][3:])
    assert np.array_equal(g["codes"], o["codes"])
    assert np.array_equal(g["sorted"].astype(np.int64), o["sorted"])
    assert np.array_equal(g["left"], o["left"]) and np.array_equal(g["right"], o["right"])
    assert np.array_equal(g["node_lo"], o["node_lo"]) and np.array_equal(g["node_hi"], o["node_hi"])
    assert np.array_equal(g["node_count"].astype(np.int64), o["node_count"])
    assert np.array_equal(g["leaf_lo"], o["leaf_lo"]) and np.array_equal(g["leaf_hi"], o["leaf_hi"])
    assert np.array_equal(g["leaf_count"].astype(np.int64), o["leaf_count"])
    params, kind, iso = sc.prim_params()
    assert np.array_equal(g["params"], params.astype(np.float32))
    assert info["A_E"] == sc.A_E and info["A_T"] == sc.A_T


@pytest.mark.parametrize("name", ["tris", "ico6", "points_cap1"])
def test_build_bit_exact_largest_leaf(name):
    """L = 1024, the largest leaf size: 5, 80 and 129 buckets (a single
    block of bucket runs, a wide root)."""
    test_build_bit_exact(name, 1024)


def test_build_errors_are_reported():
    from paper_2108_10480_gb300 import SdError
    P = synth.points_on_sphere(100, 0.0, 0)
    P[17, 1] = np.nan
    with pytest.raises(SdError) as e:
        _gpu(points=P, alpha=10.0, beta=0.5)
    assert e.value.code == 4
    V, F = synth.icosphere(1)
    F = F.copy()
    F[3, 2] = V.shape[0]
    with pytest.raises(SdError) as e:
        _gpu(tris=(V, F), alpha=10.0, beta=0.5)
    assert e.value.code == 5


def test_single_primitive_and_empty():
    sd = _gpu(points=np.array([[0.1, 0.2, 0.3]], np.float32), alpha=10.0, beta=0.5)
    g = sd.export()
    assert g["nb"] == 1 and g["left"].size == 0
    v, gr = sd.query(torch.tensor([[0.1, 0.2, 1.3]], device="cuda"))
    assert abs(v.item() - 1.0) < 1e-6
    e = _gpu(alpha=10.0, beta=0.5)
    v, gr = e.query(torch.zeros(5, 3, device="cuda"))
    assert torch.isinf(v).all() and (gr == 0).all()


def test_order_on_a_second_stream():
    """After a deferred-check build, sd_query_order on another stream waits
    for the build's scene box only; joined back, the query gives exactly the
    single-stream results."""
    V, F = synth.icosphere(4)
    q = torch.from_numpy(synth.shell_queries(50000, seed=5)).cuda()
    a = _gpu(tris=(V, F), alpha=200.0, beta=0.5, check=False)
    oa = a.query_order(q)
    va, ga = a.query(q, order=oa)
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    fork, join = torch.cuda.Event(), torch.cuda.Event()
    for _ in range(3):
        fork.record(main)
        b = _gpu(tris=(V, F), alpha=200.0, beta=0.5, check=False)
        side.wait_event(fork)
        ob = b.query_order(q, stream=side)
        join.record(side)
        main.wait_event(join)
        vb, gb = b.query(q, order=ob)
        assert torch.equal(oa, ob) and torch.equal(va, vb) and torch.equal(ga, gb)
        assert b.status() == 0


def test_deferred_checks():
    """check=False enqueues the same build without waiting: identical tree,
    identical query results, and invalid input reported by status()."""
    V, F = synth.icosphere(3)
    q = torch.from_numpy(synth.uniform_box(5000, [-1.5] * 3, [1.5] * 3, 3)).cuda()
    a = _gpu(tris=(V, F), alpha=50.0, beta=0.5)
    b = _gpu(tris=(V, F), alpha=50.0, beta=0.5, check=False)
    va, ga = a.query(q)
    vb, gb = b.query(q)
    assert b.status() == 0
    assert torch.equal(va, vb) and torch.equal(ga, gb)
    assert a.info() == b.info()
    F2 = F.copy()
    F2[3, 2] = V.shape[0]
    c = _gpu(tris=(V, F2), alpha=10.0, beta=0.5, check=False)
    assert c.status() == 5
    P = synth.points_on_sphere(100, 0.0, 0)
    P[17, 1] = np.nan
    d = _gpu(points=P, alpha=10.0, beta=0.5, check=False)
    assert d.status() == 4
    assert d.status() == 0          # reading the status clears it
