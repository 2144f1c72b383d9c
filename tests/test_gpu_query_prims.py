"""Edge and triangle queries (sd_query_prims) and the query-mesh objective
(sd_mesh_reduce) against the FP64 oracle: exact evaluation at beta = 0,
Barnes-Hut with identical node decisions, point primitives equal to point
queries, and the per-vertex gradients of Eq. dlse_full."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _metrics import assert_parity
from oracle import mesh as OMesh

pytestmark = pytest.mark.gpu


def _data(kind):
    V, F = synth.icosphere(3)
    Vl, El = synth.tiny_mesh("polyline")
    P = synth.points_on_sphere(1500, 0.01, seed=2)
    g = {"points": (dict(points=P), dict(points=P)),
         "edges": (dict(edges=(Vl * 1.2, El)), dict(edge_V=Vl * 1.2, edge_E=El)),
         "tris": (dict(tris=(V, F)), dict(tri_V=V, tri_F=F)),
         "mixed": (dict(points=P * 1.4, edges=(Vl * 1.2, El), tris=(V * 0.7, F)),
                   dict(points=P * 1.4, edge_V=Vl * 1.2, edge_E=El, tri_V=V * 0.7, tri_F=F))}[kind]
    return g


def _query_mesh(k, seed, n=400):
    """n small random edges or triangles around the data (some crossing it)."""
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(n, 3))
    c *= rng.uniform(0.6, 1.6, (n, 1)) / np.linalg.norm(c, axis=1, keepdims=True)
    V = (c[:, None, :] + 0.12 * rng.normal(size=(n, k, 3))).reshape(-1, 3).astype(np.float32)
    F = np.arange(n * k, dtype=np.int32).reshape(n, k)
    return V, F


def _data_prims(okw):
    """The data primitives' vertex arrays, in any order."""
    out = []
    if "points" in okw:
        out += [p[None].astype(np.float64) for p in okw["points"]]
    if "edge_V" in okw:
        out += [okw["edge_V"][e].astype(np.float64) for e in okw["edge_E"]]
    if "tri_V" in okw:
        out += [okw["tri_V"][f].astype(np.float64) for f in okw["tri_F"]]
    return out


def _fp32_slack(okw, V, F, alpha, reach=0.5):
    """Per query, the gradient error that fp32 arithmetic allows near contact.
    A pair at distance d whose closest points are computed from coordinates of
    size ~1 has its direction known to about u / d (u = 2^-24); the error
    enters the gradient with the pair's share e^{-alpha d} / sum e^{-alpha d}
    (touching pairs, d = 0, contribute no direction). Bound: 8 u sum_i
    share_i / d_i over the pairs within `reach` of the query."""
    prims = _data_prims(okw)
    cen = np.array([p.mean(0) for p in prims])
    u = 2.0 ** -24
    slack = np.zeros(F.shape[0])
    for j, f in enumerate(F):
        g = V[f].astype(np.float64)
        near = np.nonzero(np.linalg.norm(cen - g.mean(0), axis=1) < reach + np.ptp(g, 0).max())[0]
        d = np.array([oracle.simplex_closest(prims[i], g)[0] for i in near])
        if d.size == 0:
            continue
        e = np.exp(-alpha * d)
        far = d > 1e-12
        slack[j] = 8 * u * (e[far] / d[far]).sum() / e.sum()
    return slack


def _assert_prims_parity(v, g, rv, rg, alpha, dmin, slack, what):
    """values as for points; gradients within the point tolerance plus the
    fp32 near-contact allowance of each query"""
    assert_parity(v, None, rv, None, alpha, dmin, what)
    err = np.linalg.norm(np.asarray(g, np.float64) - rg, axis=1)
    plain = 1e-4 * np.maximum(np.linalg.norm(rg, axis=1), 1e-2)
    lim = plain + slack
    # the distribution against the plain point-query tolerance (printed with -s)
    over = err > plain
    print(f"{what}: grad err / plain 1e-4 limit: p50 {np.median(err / plain):.3f} p99 "
          f"{np.quantile(err / plain, 0.99):.3f} max {(err / plain).max():.3f}; {over.sum()} of {err.size} "
          f"above it, all within the fp32 slack (max slack / plain limit {(slack / plain).max():.2f})")
    bad = np.nonzero(err > lim)[0]
    assert bad.size == 0, f"{what}: grad err {err[bad[0]]:.3e} > {lim[bad[0]]:.3e} at {bad[0]}"
    return (err / lim).max()


def _gpu(kw, **extra):
    from paper_2108_10480_gb300 import SmoothDistance
    return SmoothDistance(device="cuda:0", **kw, **extra)


@pytest.mark.parametrize("kind", ["points", "edges", "tris", "mixed"])
@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("weights", ["paper", "unit"])
def test_exact_parity(kind, k, weights):
    gkw, okw = _data(kind)
    alpha = 30.0
    sd = _gpu(gkw, alpha=alpha, beta=0.0, weights=weights)
    sc = oracle.Scene(**okw)
    V, F = _query_mesh(k, 5 + k)
    v, g = sd.query_prims(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
    assert sd.status() == 0
    rv, rg, dmin = sc.brute_prims(V, F, alpha, unit=(weights == "unit"))
    _assert_prims_parity(v.cpu().numpy(), g.cpu().numpy(), rv, rg, alpha, dmin, _fp32_slack(okw, V, F, alpha),
                         f"{kind} k={k} {weights}")


@pytest.mark.parametrize("kind", ["tris", "mixed"])
@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("L", [1, 4])
def test_barnes_hut_parity(kind, k, L):
    """beta = 0.5: the node tests on the query's box are taken in the same
    fp32 operation order on both sides, so the work counts agree exactly."""
    gkw, okw = _data(kind)
    alpha = 30.0
    sd = _gpu(gkw, alpha=alpha, beta=0.5, leaf_size=L)
    sc = oracle.Scene(**okw)
    sc.build_tree(L)
    V, F = _query_mesh(k, 9 + k)
    v, g, cnt = sd.query_prims(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda(), counts=True)
    rv, rg, rc, _ = sc.bh_prims(V, F, alpha, 0.5)
    assert np.array_equal(cnt.cpu().numpy(), rc)
    assert np.any(rc[:, 1] > 0)
    _assert_prims_parity(v.cpu().numpy(), g.cpu().numpy(), rv, rg, alpha, None, _fp32_slack(okw, V, F, alpha),
                         f"BH {kind} k={k} L={L}")


def test_point_primitives_equal_point_queries():
    gkw, _ = _data("mixed")
    sd = _gpu(gkw, alpha=30.0, beta=0.5)
    q = torch.from_numpy(synth.uniform_box(3000, [-1.5] * 3, [1.5] * 3, 4)).cuda()
    v0, g0 = sd.query(q)
    v1, g1 = sd.query_prims(q, torch.arange(3000, dtype=torch.int32, device="cuda")[:, None])
    assert torch.equal(v0, v1) and torch.equal(g0, g1)


def test_mesh_objective_parity():
    """The query-mesh objective: the reduction itself against the FP64 formula
    on the same per-primitive inputs, and the whole path against the oracle."""
    from paper_2108_10480_gb300 import mesh_reduce
    gkw, okw = _data("tris")
    sd = _gpu(gkw, alpha=20.0, beta=0.0)
    sc = oracle.Scene(**okw)
    Vq, Fq = synth.torus(24, 12, 0.6, 0.2)
    Vq = (Vq.astype(np.float64) + [0.9, 0.0, 0.2]).astype(np.float32)
    Vt, Ft = torch.from_numpy(Vq).cuda(), torch.from_numpy(Fq.astype(np.int32)).cuda()
    v, g = sd.query_prims(Vt, Ft)
    D, VG = mesh_reduce(Ft, Vq.shape[0], v, g, 40.0)
    rD, rVG, _ = OMesh.mesh_objective(v.cpu().numpy(), g.cpu().numpy(), Fq, Vq.shape[0], 40.0)
    assert abs(D.item() - rD) <= 1e-6 * max(abs(rD), 1.0 / 40.0)
    assert np.abs(VG.cpu().numpy() - rVG).max() <= 1e-5 * np.abs(rVG).max()
    # end to end against the oracle's per-primitive values
    ov, og, _ = sc.brute_prims(Vq, Fq, 20.0)
    eD, eVG, gam = OMesh.mesh_objective(ov, og, Fq, Vq.shape[0], 40.0)
    assert abs(D.item() - eD) <= 1e-5 * max(abs(eD), 1.0 / 40.0)
    # per-primitive gradient errors reach the vertices with weights gamma_j / 3
    slack = (gam * _fp32_slack(okw, Vq, Fq, 20.0)).sum()
    assert np.linalg.norm(VG.cpu().numpy() - eVG) <= 1e-4 * np.linalg.norm(eVG) + slack


def test_invalid_primitives_are_reported():
    gkw, _ = _data("tris")
    sd = _gpu(gkw, alpha=20.0, beta=0.5)
    V, F = _query_mesh(3, 1, n=50)
    F = F.copy()
    F[7, 1] = V.shape[0] + 3
    v, g = sd.query_prims(torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda())
    assert sd.status() == 5
    vv = v.cpu().numpy()
    assert np.isnan(vv[7]) and np.all(np.isfinite(np.delete(vv, 7)))
