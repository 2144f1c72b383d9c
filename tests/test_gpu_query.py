"""GPU smooth distance and gradient (sd_query / sd_query_brute) against the
FP64 oracle, element by element, on seeded inputs; Barnes-Hut work counts
bit-exact; edge cases."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _metrics import assert_parity

pytestmark = pytest.mark.gpu


def _gpu(**kw):
    from paper_2108_10480_gb300 import SmoothDistance
    return SmoothDistance(device="cuda:0", **kw)


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def _np(x):
    return x.detach().cpu().numpy().astype(np.float64)


# ---------------------------------------------------------------- points (config 1)
@pytest.mark.parametrize("L", [1, 4])
def test_points_config1(L):
    c = synth.config1()
    alpha = c["alpha"]
    sd = _gpu(points=c["points"], alpha=alpha, beta=0.5, leaf_size=L)
    sc = oracle.Scene(points=c["points"])
    sc.build_tree(L)
    q = c["queries"]
    rv, rg, dmin = sc.brute(q, alpha)
    v, g = sd.query_brute(_t(q))
    assert_parity(_np(v), _np(g), rv, rg, alpha, dmin, "brute")
    bv, bg, bc, _ = sc.bh(q, alpha, 0.5)
    v, g, cnt = sd.query(_t(q), counts=True)
    assert_parity(_np(v), _np(g), bv, bg, alpha, dmin, "bh")
    assert np.array_equal(cnt.cpu().numpy(), bc)
    assert sd.status() == 0


# ---------------------------------------------------------------- triangles
@pytest.fixture(scope="module")
def ico4():
    V, F = synth.icosphere(4)
    V = synth.perturb_radial(V, 0.01, 1)
    sc = oracle.Scene(tri_V=V, tri_F=F)
    q = synth.shell_queries(2048, seed=2)
    return V, F, sc, q


@pytest.mark.parametrize("alpha", [50.0, 200.0, 1000.0])
def test_triangles_brute(ico4, alpha):
    V, F, sc, q = ico4
    sd = _gpu(tris=(V, F), alpha=alpha, beta=0.0)
    rv, rg, dmin = sc.brute(q, alpha)
    v, g = sd.query_brute(_t(q))
    assert_parity(_np(v), _np(g), rv, rg, alpha, dmin, f"brute a={alpha}")
    # beta = 0 traversal is exact: it equals the brute force (Sec. 3.5)
    v0, g0 = sd.query(_t(q))
    assert_parity(_np(v0), _np(g0), rv, rg, alpha, dmin, f"beta0 a={alpha}")


@pytest.mark.parametrize("alpha", [50.0, 200.0, 1000.0])
@pytest.mark.parametrize("beta", [0.25, 0.5, 1.0])
@pytest.mark.parametrize("L", [1, 4])
def test_triangles_bh(ico4, alpha, beta, L):
    V, F, sc, q = ico4
    sd = _gpu(tris=(V, F), alpha=alpha, beta=beta, leaf_size=L)
    sc.build_tree(L)
    bv, bg, bc, _ = sc.bh(q, alpha, beta)
    v, g, cnt = sd.query(_t(q), counts=True)
    assert np.array_equal(cnt.cpu().numpy(), bc)
    assert_parity(_np(v), _np(g), bv, bg, alpha, None, f"bh a={alpha} b={beta} L={L}")


def test_largest_leaf_size(ico4):
    """L = 1024, the largest leaf the build accepts: five buckets over the
    5,120 triangles, so every opened leaf queues up to 1,024 primitives per
    lane. Work counts bit-exact, values and gradients within the parity
    bound."""
    V, F, sc, q = ico4
    sd = _gpu(tris=(V, F), alpha=200.0, beta=0.5, leaf_size=1024)
    assert sd.info()["n_buckets"] == 5
    sc.build_tree(1024)
    bv, bg, bc, _ = sc.bh(q, 200.0, 0.5)
    sc.build_tree(1)
    v, g, cnt = sd.query(_t(q), counts=True)
    assert np.array_equal(cnt.cpu().numpy(), bc)
    assert_parity(_np(v), _np(g), bv, bg, 200.0, None, "bh L=1024")


@pytest.fixture(scope="module")
def ico6():
    c = synth.config2()
    sc = oracle.Scene(tri_V=c["V"], tri_F=c["F"])
    sc.build_tree(1)
    return c, sc


@pytest.mark.parametrize("alpha", [50.0, 200.0, 1000.0])
@pytest.mark.parametrize("beta", [0.25, 0.5, 1.0])
def test_triangles_full_size_sampled(ico6, alpha, beta):
    """Level-6 icosphere (81,920 triangles), all 262,144 queries of the
    benchmark workload traversed in the benchmark's launch configuration
    (Hilbert order from sd_query_order, persistent grid) at every (alpha,
    beta) cell; 3,000 sampled outputs per cell against the oracle (the
    same sample everywhere, 70 % of it in the shell), plus the work counts
    of every sampled query."""
    c, sc = ico6
    sd = _gpu(tris=(c["V"], c["F"]), alpha=alpha, beta=beta)
    q = _t(c["queries"])
    v, g, cnt = sd.query(q, counts=True, order=sd.query_order(q))
    idx = np.random.default_rng(0).choice(c["queries"].shape[0], 3000, replace=False)
    bv, bg, bc, _ = sc.bh(c["queries"][idx], alpha, beta)
    assert_parity(_np(v)[idx], _np(g)[idx], bv, bg, alpha, None, f"config2 sampled a={alpha} b={beta}")
    assert np.array_equal(cnt.cpu().numpy()[idx], bc)
    assert sd.status() == 0


def test_street_points_full_size_sampled():
    """Plain point queries on the street workload: the 100,002 vertices of
    the posed body (placed in fp32 exactly as the GPU places them) against
    2,000,000 lidar points + 50,000 wire segments, alpha 50, beta 0.5, through
    sd_query; 3,000 sampled outputs and their work counts against the
    oracle."""
    from oracle import pose as PO
    s = synth.config3_scene()
    b = synth.config3_body()
    X = PO.place(b["V0"], np.concatenate([b["theta"], b["p"]]), "f32")
    sd = _gpu(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5)
    v, g, cnt = sd.query(_t(X), counts=True)
    assert sd.status() == 0
    idx = np.random.default_rng(1).choice(X.shape[0], 3000, replace=False)
    sc = oracle.Scene(points=s["points"], edge_V=s["wire_V"], edge_E=s["wire_E"])
    sc.build_tree(1)
    bv, bg, bc, _ = sc.bh(X[idx], 50.0, 0.5)
    assert_parity(_np(v)[idx], _np(g)[idx], bv, bg, 50.0, None, "street sampled")
    assert np.array_equal(cnt.cpu().numpy()[idx], bc)


# ---------------------------------------------------------------- edges / mixed / options
def test_edges_and_mixed():
    Ve, E = synth.tiny_mesh("polyline")
    V, F = synth.icosphere(3)
    P = synth.points_on_sphere(700, 0.02, 3) * 1.4
    q = synth.uniform_box(1500, -1.6, 1.6, 4)
    for kw, sc in [
        (dict(edges=(Ve, E)), oracle.Scene(edge_V=Ve, edge_E=E)),
        (dict(points=P, edges=(Ve, E), tris=(V, F)), oracle.Scene(points=P, edge_V=Ve, edge_E=E, tri_V=V, tri_F=F)),
    ]:
        for L in (1, 3):
            sd = _gpu(alpha=60.0, beta=0.5, leaf_size=L, **kw)
            sc.build_tree(L)
            rv, rg, dmin = sc.brute(q, 60.0)
            v, g = sd.query_brute(_t(q))
            assert_parity(_np(v), _np(g), rv, rg, 60.0, dmin, "brute " + ",".join(kw))
            bv, bg, bc, _ = sc.bh(q, 60.0, 0.5)
            v, g, cnt = sd.query(_t(q), counts=True)
            assert_parity(_np(v), _np(g), bv, bg, 60.0, dmin, "bh " + ",".join(kw))
            assert np.array_equal(cnt.cpu().numpy(), bc)


@pytest.mark.parametrize("opt", ["atten", "metric", "unit"])
def test_weight_options(ico4, opt):
    V, F, sc, q = ico4
    alpha = 100.0
    kw = dict(atten=dict(alpha_u=400.0), metric=dict(paper_metric=True), unit=dict(weights="unit"))[opt]
    okw = dict(atten=dict(alpha_u=400.0), metric=dict(paper_metric=True), unit=dict(unit=True))[opt]
    sd = _gpu(tris=(V, F), alpha=alpha, beta=0.5, **kw)
    rv, rg, dmin = sc.brute(q, alpha, **okw)
    v, g = sd.query_brute(_t(q))
    assert_parity(_np(v), _np(g), rv, rg, alpha, dmin, opt)
    sc.build_tree(1)
    bv, bg, _, _ = sc.bh(q, alpha, 0.5, **okw)
    v, g = sd.query(_t(q))
    assert_parity(_np(v), _np(g), bv, bg, alpha, None, opt + " bh")


# ---------------------------------------------------------------- edge cases
def test_order_value_only_and_ragged_sizes(ico4):
    V, F, sc, q = ico4
    sd = _gpu(tris=(V, F), alpha=200.0, beta=0.5)
    v1, g1 = sd.query(_t(q), sort=True)
    v2, g2 = sd.query(_t(q), sort=False)
    v3, _ = sd.query(_t(q), grad=False)
    # the same terms are summed whatever the traversal order; only the
    # summation order (which queries share a warp) changes the rounding
    assert_parity(_np(v2), _np(g2), _np(v1), _np(g1), 200.0, None, "order")
    assert torch.allclose(v1, v3, rtol=2e-6, atol=1e-7)
    # a fixed order and launch shape gives bitwise identical results
    v4, g4 = sd.query(_t(q), sort=True)
    assert torch.equal(v1, v4) and torch.equal(g1, g4)
    for m in (0, 1, 31, 33, 1000):
        vm, gm = sd.query(_t(q[:m]), sort=False)
        assert vm.shape == (m,)
        if m:
            assert_parity(_np(vm), _np(gm), _np(v2[:m]), _np(g2[:m]), 200.0, None, f"m={m}")
    for b in (32, 64, 256):
        vb, gb = sd.query(_t(q), block=b)
        assert torch.equal(vb, v1) and torch.equal(gb, g1)


def test_nonfinite_query_sets_status(ico4):
    V, F, sc, q = ico4
    sd = _gpu(tris=(V, F), alpha=200.0, beta=0.5)
    qq = q[:64].copy()
    qq[5, 0] = np.nan
    qq[9, 2] = np.inf
    v, g = sd.query(_t(qq))
    assert sd.status() == 4
    assert sd.status() == 0            # cleared by the read
    vn = _np(v)
    assert np.isnan(vn[5]) and np.isnan(vn[9]) and np.isfinite(np.delete(vn, [5, 9])).all()


def test_degenerate_geometry_and_contact():
    # coincident points, zero-length edges, zero-area triangles; queries on
    # the geometry (d = 0) and far away
    P = np.array([[0, 0, 0], [0, 0, 0], [1, 0, 0]], np.float32)
    Ve = np.array([[0, 1, 0], [0, 1, 0], [1, 1, 0]], np.float32)
    E = np.array([[0, 1], [1, 2]], np.int32)
    Vt = np.array([[0, 0, 1], [1, 0, 1], [2, 0, 1], [0, 1, 1]], np.float32)
    Ft = np.array([[0, 1, 2], [0, 1, 3]], np.int32)
    q = np.array([[0, 0, 0], [0.5, 1, 0], [0.2, 0.2, 1], [30, -20, 10], [0.3, 0.4, 0.5]], np.float32)
    sc = oracle.Scene(points=P, edge_V=Ve, edge_E=E, tri_V=Vt, tri_F=Ft)
    sd = _gpu(points=P, edges=(Ve, E), tris=(Vt, Ft), alpha=20.0, beta=0.0)
    rv, rg, dmin = sc.brute(q, 20.0)
    v, g = sd.query_brute(_t(q))
    assert_parity(_np(v), _np(g), rv, rg, 20.0, dmin, "degenerate")
    v, g = sd.query(_t(q))
    assert_parity(_np(v), _np(g), rv, rg, 20.0, dmin, "degenerate bh")


def test_query_order_is_a_hilbert_walk():
    """sd_query_order on the centres of an aligned 16^3 block of its 256^3
    grid: a permutation in which consecutive queries are face neighbours
    (the Hilbert curve covers every aligned block contiguously), and the
    traversal result is independent of the order up to summation order."""
    from paper_2108_10480_gb300 import SmoothDistance
    P = np.array([[0.0, 0.0, 0.0], [256.0, 256.0, 256.0]], np.float32)
    sd = SmoothDistance(points=P, alpha=1.0, beta=0.5, device="cuda:0")
    g = np.stack(np.meshgrid(*[np.arange(32, 48)] * 3, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(0)
    g = g[rng.permutation(len(g))]
    q = torch.from_numpy((g + 0.5).astype(np.float32)).cuda()
    order = sd.query_order(q).cpu().numpy()
    assert np.array_equal(np.sort(order), np.arange(len(g)))
    walk = g[order]
    step = np.abs(np.diff(walk, axis=0))
    assert np.all(step.sum(1) == 1)
    v0, g0 = sd.query(q, sort=False)
    v1, g1 = sd.query(q)
    assert torch.allclose(v0, v1, rtol=1e-6) and torch.allclose(g0, g1, rtol=1e-5, atol=1e-7)
