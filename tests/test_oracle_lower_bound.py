"""Pins of the oracle's certified lower bound (the routing test of the
learned surrogate): it never exceeds the exact d^ of Eq. 3, it is the exact
d^ where the cut reaches every point of a small point cloud, its gradient
matches finite differences, and kappa bounds every blending weight."""
import numpy as np
import pytest

import oracle
import synth


def _scenes():
    V3, F3 = synth.icosphere(2)
    # an open mesh: boundary vertices have smaller valences, so w~ is not 1
    keep = V3[F3].mean(1)[:, 2] > -0.2
    Vl, El = synth.tiny_mesh("polyline")
    P = synth.points_on_sphere(300, 0.01, seed=3)
    return {
        "points": dict(points=P),
        "polyline": dict(edge_V=Vl, edge_E=El),
        "closed": dict(tri_V=V3, tri_F=F3),
        "open": dict(tri_V=V3, tri_F=F3[keep]),
        "mixed": dict(points=P * 2.0, edge_V=Vl, edge_E=El, tri_V=V3 * 0.5, tri_F=F3[keep]),
    }


def _queries(n, seed, scale=3.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, (n, 3))


@pytest.mark.parametrize("name", ["points", "polyline", "closed", "open", "mixed"])
@pytest.mark.parametrize("L", [1, 4])
@pytest.mark.parametrize("alpha,alpha_u", [(8.0, 0.0), (30.0, 60.0)])
def test_lower_bound_below_exact(name, L, alpha, alpha_u):
    sc = oracle.Scene(**_scenes()[name])
    sc.build_tree(L)
    q = _queries(400, 1)
    exact, _, _ = sc.brute(q, alpha, alpha_u=alpha_u)
    lb, _, kappa, ncut = sc.lower_bound(q, alpha, alpha_u=alpha_u)
    assert 1 <= ncut <= 64 and kappa >= 1.0
    assert np.all(lb <= exact + 1e-12 * np.maximum(1.0, np.abs(exact)))
    # and not vacuous far away: within the cut's box size of the exact value
    far = np.linalg.norm(q, axis=1) > 2.5
    assert np.median((exact - lb)[far]) < 2.0


def test_points_all_leaves_is_exact():
    """At most 64 points with leaf size 1: the cut is every point and each
    box is the point itself, so LB is the plain LogSumExp (Eq. 3, w = 1)."""
    P = synth.points_on_sphere(50, 0.02, seed=4)
    sc = oracle.Scene(points=P)
    sc.build_tree(1)
    q = _queries(200, 2)
    lb, g, kappa, ncut = sc.lower_bound(q, 12.0)
    assert ncut == 50 and kappa == 1.0
    d = np.linalg.norm(q[:, None, :] - P[None].astype(np.float64), axis=2)
    t = -12.0 * d
    mx = t.max(1)
    ref = -(mx + np.log(np.exp(t - mx[:, None]).sum(1))) / 12.0
    assert np.allclose(lb, ref, rtol=1e-12, atol=1e-12)
    ex, eg, _ = sc.brute(q, 12.0)
    assert np.allclose(lb, ex, rtol=1e-12, atol=1e-12)
    assert np.allclose(g, eg, rtol=1e-9, atol=1e-12)


def test_single_point_closed_form():
    p = np.array([[0.5, -1.0, 2.0]], np.float32)
    sc = oracle.Scene(points=p)
    q = _queries(20, 3)
    lb, g, kappa, ncut = sc.lower_bound(q, 5.0)
    r = q - p.astype(np.float64)
    assert ncut == 1
    assert np.allclose(lb, np.linalg.norm(r, axis=1), rtol=1e-14)
    assert np.allclose(g, r / np.linalg.norm(r, axis=1)[:, None], rtol=1e-12)


@pytest.mark.parametrize("name", ["closed", "mixed"])
def test_gradient_fd(name):
    sc = oracle.Scene(**_scenes()[name])
    sc.build_tree(2)
    q = _queries(40, 5, 4.0)
    q = q[np.linalg.norm(q, axis=1) > 2.5]
    _, g, _, _ = sc.lower_bound(q, 10.0)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3); e[j] = h
        fd = (sc.lower_bound(q + e, 10.0)[0] - sc.lower_bound(q - e, 10.0)[0]) / (2 * h)
        assert np.allclose(g[:, j], fd, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("name", ["polyline", "open", "closed"])
def test_kappa_bounds_every_weight(name):
    """Each primitive's largest Bernstein coefficient lies above its w~
    everywhere and its corner coefficients are w~ at the corners (a Bernstein
    polynomial interpolates its end coefficients). A query placed on a
    primitive has its closest point there, so prim_eval reports w~ at that
    point; sample a barycentric grid."""
    kw = _scenes()[name]
    sc = oracle.Scene(**kw)
    _, _, kappa, _ = sc.lower_bound(np.zeros((1, 3)), 10.0)
    K = sc.prim_kappa()
    if name == "polyline":
        V, idx = kw["edge_V"].astype(np.float64), kw["edge_E"]
        bary = [np.array([1 - t, t]) for t in np.linspace(0, 1, 41)]
        corners = [np.array([1.0, 0.0]), np.array([0.0, 1.0])]
    else:
        V, idx = kw["tri_V"].astype(np.float64), kw["tri_F"]
        g = np.linspace(0, 1, 13)
        bary = [np.array([1 - a - b, a, b]) for a in g for b in g if a + b <= 1 + 1e-12]
        corners = [np.eye(3)[0], np.eye(3)[1], np.eye(3)[2]]
    for i, f in enumerate(idx):
        X = V[f]
        w = np.array([sc.prim_eval(i, b @ X)["wt"] for b in bary])
        assert K[i, 0] >= w.max() - 1e-12
        for c, b in enumerate(corners):
            assert abs(K[i, 1 + c] - sc.prim_eval(i, b @ X)["wt"]) <= 1e-9 * max(1.0, abs(K[i, 1 + c]))
    assert kappa == max(1.0, K[:, 0].max())
    assert not np.all(K[:, 0] == 1.0)
