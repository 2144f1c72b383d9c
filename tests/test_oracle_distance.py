"""Pins of the oracle's exact primitive distances, closest-point barycentrics
and their gradients (App. B, Eq. distsq, Eq. dgrad, Eq. dw_new): textbook
cases, dense sampling of the primitive, an independent QP solve and central
finite differences."""
import numpy as np
import pytest
import scipy.optimize

import oracle


def _scene_tri(V):
    return oracle.Scene(tri_V=np.asarray(V, np.float32), tri_F=np.array([[0, 1, 2]], np.int32))


TRI = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)


def test_point_distance_textbook():
    s = oracle.Scene(points=np.array([[1.0, 2.0, 3.0]], np.float32))
    r = s.prim_eval(0, [4.0, 6.0, 3.0])
    assert r["d"] == pytest.approx(5.0, abs=1e-15)
    assert np.allclose(r["grad_d"], [0.6, 0.8, 0.0], atol=1e-15)
    r = s.prim_eval(0, [1.0, 2.0, 3.0])
    assert r["d"] == 0.0 and np.all(r["grad_d"] == 0.0)     # Eq. dgrad, d = 0 case


def test_segment_distance_textbook():
    s = oracle.Scene(edge_V=np.array([[0, 0, 0], [2, 0, 0]], np.float32), edge_E=np.array([[0, 1]]))
    r = s.prim_eval(0, [0.5, 3.0, 4.0])
    assert r["d"] == pytest.approx(5.0) and r["phi"][0] == pytest.approx(0.25)
    assert np.allclose(r["grad_d"], [0, 0.6, 0.8])
    r = s.prim_eval(0, [-3.0, 4.0, 0.0])                    # beyond the a end
    assert r["d"] == pytest.approx(5.0) and r["phi"][0] == 0.0
    r = s.prim_eval(0, [5.0, 0.0, 4.0])                     # beyond the b end
    assert r["d"] == pytest.approx(5.0) and r["phi"][0] == 1.0


@pytest.mark.parametrize("q,d,phi", [
    ([0.25, 0.25, 2.0], 2.0, (0.25, 0.25)),      # face region: height
    ([0.5, -1.0, 0.0], 1.0, (0.5, 0.0)),         # edge v0v1
    ([-1.0, 0.5, 0.0], 1.0, (0.0, 0.5)),         # edge v0v2
    ([1.0, 1.0, 0.0], np.sqrt(0.5), (0.5, 0.5)), # hypotenuse v1v2
    ([-1.0, -1.0, 1.0], np.sqrt(3.0), (0.0, 0.0)),  # vertex v0
    ([3.0, 0.0, 0.0], 2.0, (1.0, 0.0)),          # vertex v1
])
def test_triangle_distance_textbook(q, d, phi):
    s = _scene_tri(TRI)
    r = s.prim_eval(0, q)
    assert r["d"] == pytest.approx(d, abs=1e-14)
    assert np.allclose(r["phi"], phi, atol=1e-14)


def _tri_qp(V, q):
    V = np.asarray(V, np.float64)
    f = lambda x: np.sum(((1 - x[0] - x[1]) * V[0] + x[0] * V[1] + x[1] * V[2] - q) ** 2)
    best = None
    for x0 in ([1 / 3, 1 / 3], [0.8, 0.1], [0.1, 0.8], [0.05, 0.05]):
        res = scipy.optimize.minimize(f, x0, method="SLSQP", bounds=[(0, 1), (0, 1)],
                                      constraints=[{"type": "ineq", "fun": lambda x: 1 - x[0] - x[1]}],
                                      options=dict(ftol=1e-15, maxiter=500))
        if best is None or res.fun < best.fun:
            best = res
    return np.sqrt(best.fun), best.x


def test_triangle_distance_vs_independent_qp_and_sampling():
    rng = np.random.default_rng(3)
    # dense barycentric sample grid of the triangle
    k = 400
    a, b = np.meshgrid(np.arange(k + 1) / k, np.arange(k + 1) / k, indexing="ij")
    m = a + b <= 1
    a, b = a[m], b[m]
    for _ in range(25):
        V = rng.standard_normal((3, 3)).astype(np.float32)
        s = _scene_tri(V)
        q = rng.standard_normal(3) * 1.5
        r = s.prim_eval(0, q)
        dq, x = _tri_qp(V, q)
        assert r["d"] == pytest.approx(dq, abs=2e-7)
        Vd = V.astype(np.float64)
        P = (1 - a - b)[:, None] * Vd[0] + a[:, None] * Vd[1] + b[:, None] * Vd[2]
        ds = np.sqrt(((P - q) ** 2).sum(1)).min()
        assert r["d"] <= ds + 1e-12                      # nothing on the triangle is closer
        assert ds - r["d"] < 0.02                        # sampling resolution


def _fd(f, q, h=1e-6):
    g = np.zeros(3)
    for j in range(3):
        e = np.zeros(3); e[j] = h
        g[j] = (f(q + e) - f(q - e)) / (2 * h)
    return g


def test_gradient_of_distance_fd():
    rng = np.random.default_rng(4)
    for trial in range(40):
        V = rng.standard_normal((3, 3)).astype(np.float32)
        s = _scene_tri(V)
        q = rng.standard_normal(3) * 1.2
        r = s.prim_eval(0, q)
        gd = _fd(lambda x: s.prim_eval(0, x)["d"], q)
        assert np.allclose(r["grad_d"], gd, atol=1e-6)


def test_triangle_weight_gradient_fd():
    # chain rule of Eq. dw_new: grad w~ = dw~/dphi . grad phi, checked in the
    # face, edge and vertex regions of a closed mesh (v_i = 3, e_i = 2)
    import synth
    V, F = synth.tiny_mesh("tet", seed=1)
    s = oracle.Scene(tri_V=V, tri_F=F)
    rng = np.random.default_rng(6)
    for i in range(4):
        for _ in range(25):
            q = rng.standard_normal(3) * 0.8 + 0.3
            r = s.prim_eval(i, q)
            gw = _fd(lambda x: s.prim_eval(i, x)["wt"], q)
            assert np.allclose(r["grad_wt"], gw, atol=2e-5 * max(1.0, np.abs(gw).max()))


def test_segment_weight_gradient_fd():
    rng = np.random.default_rng(5)
    V = rng.standard_normal((5, 3)).astype(np.float32)
    E = np.array([[0, 1], [1, 2], [2, 3], [1, 4]], np.int32)
    s = oracle.Scene(edge_V=V, edge_E=E)
    for i in range(4):
        for _ in range(10):
            q = rng.standard_normal(3)
            r = s.prim_eval(i, q)
            gw = _fd(lambda x: s.prim_eval(i, x)["wt"], q)
            assert np.allclose(r["grad_wt"], gw, atol=1e-6)


def test_degenerate_primitives():
    # zero-length edge behaves as a point; zero-area triangle takes its edges
    s = oracle.Scene(edge_V=np.array([[1, 1, 1], [1, 1, 1]], np.float32), edge_E=np.array([[0, 1]]))
    r = s.prim_eval(0, [1.0, 1.0, 3.0])
    assert r["d"] == pytest.approx(2.0) and np.all(r["grad_wt"] == 0)
    Vc = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], np.float32)   # collinear
    s = _scene_tri(Vc)
    r = s.prim_eval(0, [0.5, 1.0, 0.0])
    assert r["d"] == pytest.approx(1.0)
    assert np.all(r["grad_wt"] == 0)
