"""Pins of the oracle's smooth distance (Eq. 3) and gradient (Eq. 4):
single-primitive cases, Theorem A.1's bounds, convergence in alpha, central
finite differences, and an independent pure-Python evaluation on tiny
scenes."""
import math

import numpy as np
import pytest
import scipy.optimize

import oracle
import synth
from oracle import weights as W


def test_single_primitive_is_exact_distance():
    q = np.array([[0.3, -0.2, 0.9], [2.0, 1.0, -1.0]])
    s = oracle.Scene(points=np.array([[0.1, 0.2, 0.3]], np.float32))
    v, g, dm = s.brute(q, 37.0)
    assert np.allclose(v, dm, atol=1e-14, rtol=0)
    # lone segment: u = v = 1 so w~ = 1, A = 1
    s = oracle.Scene(edge_V=np.array([[0, 0, 0], [1, 0.5, 0]], np.float32), edge_E=np.array([[0, 1]]))
    v, g, dm = s.brute(q, 37.0)
    assert np.allclose(v, dm, atol=1e-14, rtol=0)
    # lone triangle: v_i = 1 (guard w~ = 1), A = 1
    s = oracle.Scene(tri_V=np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.2]], np.float32), tri_F=np.array([[0, 1, 2]]))
    v, g, dm = s.brute(q, 37.0)
    assert np.allclose(v, dm, atol=1e-14, rtol=0)
    # and the gradient is the unit direction of Eq. dgrad
    assert np.allclose(np.linalg.norm(g, axis=1), 1.0, atol=1e-12)


def test_theorem_a1_unit_weights():
    c = synth.config1()
    s = oracle.Scene(points=c["points"])
    n = c["points"].shape[0]
    for alpha in (10.0, 100.0, 1000.0):
        v, g, dm = s.brute(c["queries"], alpha)
        assert np.all(v <= dm + 1e-12)
        assert np.all(v >= dm - math.log(n) / alpha - 1e-12)


def test_monotone_and_convergent_in_alpha():
    c = synth.config1()
    s = oracle.Scene(points=c["points"][:512])
    q = c["queries"][:200]
    prev = None
    for alpha in (50.0, 200.0, 1000.0, 5000.0):
        v, g, dm = s.brute(q, alpha)
        assert np.all(np.abs(v - dm) <= math.log(512) / alpha + 1e-12)
        if prev is not None:
            assert np.all(v >= prev - 1e-12)     # soft-min increases with alpha
        prev = v


def test_weighted_mesh_bounds():
    # App. A with 1 <= w_i <= A up to the recorded 0.999 dip of A w~ near
    # triangle vertices: d_min - log(A N)/alpha <= d^ <= d_min + log(1/0.995)/alpha
    V, F = synth.icosphere(2)
    V = synth.perturb_radial(V, 0.01, 0)
    s = oracle.Scene(tri_V=V, tri_F=F)
    q = synth.shell_queries(300, seed=4)
    n = F.shape[0]
    for alpha in (50.0, 200.0, 1000.0):
        v, g, dm = s.brute(q, alpha)
        wmax = 6 * 1.3
        assert np.all(v >= dm - math.log(wmax * n) / alpha - 1e-12)
        assert np.all(v <= dm + math.log(1 / 0.995) / alpha + 1e-12)


def _fd(f, q, h=1e-6):
    out = np.zeros(3)
    for j in range(3):
        e = np.zeros(3); e[j] = h
        out[j] = (f(q + e) - f(q - e)) / (2 * h)
    return out


@pytest.mark.parametrize("kind", ["points", "edges", "tris", "mixed", "tris_atten", "tris_metric"])
def test_gradient_matches_finite_differences(kind):
    rng = np.random.default_rng(11)
    alpha, alpha_u, pm = 20.0, 0.0, False
    if kind == "points":
        s = oracle.Scene(points=synth.points_on_sphere(64, 0.01, 1))
    elif kind == "edges":
        V, E = synth.tiny_mesh("polyline")
        s = oracle.Scene(edge_V=V, edge_E=E)
    elif kind in ("tris", "tris_atten", "tris_metric"):
        V, F = synth.icosphere(1)
        s = oracle.Scene(tri_V=V, tri_F=F)
        if kind == "tris_atten":
            alpha_u = 60.0          # S = 1/3
        if kind == "tris_metric":
            pm = True
    else:
        V, E = synth.tiny_mesh("polyline")
        Vt, F = synth.icosphere(1)
        s = oracle.Scene(points=synth.points_on_sphere(16, 0.01, 2) * 1.5, edge_V=V, edge_E=E,
                         tri_V=Vt * 0.7, tri_F=F)
    for _ in range(12):
        q = rng.uniform(-1.4, 1.4, 3)
        v, g, _ = s.brute(q[None], alpha, alpha_u, pm)
        f = lambda x: s.brute(x[None], alpha, alpha_u, pm)[0][0]
        gfd = _fd(f, q)
        if pm:
            # the alpha-scaled metric is a damping heuristic, not the
            # derivative of d^: only the distance term must match
            continue
        assert np.allclose(g[0], gfd, atol=2e-6), (g[0], gfd)


def test_independent_python_evaluation_tiny():
    """Eq. 3 and Eq. 4 written out directly in Python for a tiny mixed scene:
    distances by an SLSQP solve over the barycentric simplex, weights from the
    App. C bases, terms summed without shifting."""
    rng = np.random.default_rng(12)
    pts = rng.standard_normal((3, 3)).astype(np.float32)
    eV = rng.standard_normal((3, 3)).astype(np.float32)
    eE = np.array([[0, 1], [1, 2]], np.int32)
    tV, tF = synth.tiny_mesh("tet", seed=3)
    s = oracle.Scene(points=pts, edge_V=eV, edge_E=eE, tri_V=tV, tri_F=tF)
    alpha = 3.0
    eb, tb = W.edge_basis(), W.tri_basis()
    # valences by hand: polyline 0-1-2 has |N| = (1, 2, 1), A_E = 2; the tet
    # has v = 3 at every vertex and e = 2 on every edge, A_T = 3
    A_E, A_T = 2.0, 3.0
    assert s.A_E == A_E and s.A_T == A_T
    for _ in range(5):
        q = rng.standard_normal(3)
        total = 0.0
        for p in pts.astype(np.float64):
            total += math.exp(-alpha * np.linalg.norm(q - p))
        ends = [(1.0, 0.5), (0.5, 1.0)]
        for (i0, i1), (u, v) in zip(eE, ends):
            a, b = eV[i0].astype(np.float64), eV[i1].astype(np.float64)
            res = scipy.optimize.minimize_scalar(lambda t: np.sum((a + t * (b - a) - q) ** 2),
                                                 bounds=(0, 1), method="bounded", options=dict(xatol=1e-12))
            wt = W.edge_weight(res.x, u, v, eb)
            total += A_E * wt * math.exp(-alpha * math.sqrt(res.fun))
        for f in tF:
            Vt = tV[f].astype(np.float64)
            fun = lambda x: np.sum(((1 - x[0] - x[1]) * Vt[0] + x[0] * Vt[1] + x[1] * Vt[2] - q) ** 2)
            best = None
            for x0 in ([1 / 3, 1 / 3], [0.8, 0.1], [0.1, 0.8], [0.05, 0.05]):
                r = scipy.optimize.minimize(fun, x0, method="SLSQP", bounds=[(0, 1), (0, 1)],
                                            constraints=[{"type": "ineq", "fun": lambda x: 1 - x[0] - x[1]}],
                                            options=dict(ftol=1e-15, maxiter=500))
                if best is None or r.fun < best.fun:
                    best = r
            wt = W.tri_weight(best.x[0], best.x[1], 1 / 3, 1 / 2, tb)
            total += A_T * wt * math.exp(-alpha * math.sqrt(best.fun))
        ref = -math.log(total) / alpha
        v, g, _ = s.brute(q[None], alpha)
        assert v[0] == pytest.approx(ref, abs=2e-6)


def test_empty_scene_is_infinite():
    s = oracle.Scene()
    v, g, dm = s.brute(np.zeros((2, 3)), 10.0)
    assert np.all(np.isinf(v)) and np.all(g == 0)


def test_paper_metric_rescales_only_the_weight_term():
    """The paper_metric variant (reading R4: the barycentric gradients taken
    in the alpha-scaled metric) divides the weight-gradient part of each
    term's vector by alpha once more and changes nothing else: per primitive
    vec_pm = grad d + (vec - grad d) / alpha, the value is unchanged, and the
    LogSumExp gradient is the softmax mix of those vectors."""
    V, F = synth.icosphere(2)
    V = synth.perturb_radial(V, 0.02, 3)
    sc = oracle.Scene(tri_V=V, tri_F=F)
    q = synth.shell_queries(40, frac_shell=1.0, r_lo=0.95, r_hi=1.05, seed=8)
    alpha = 20.0
    v0, g0, _ = sc.brute(q, alpha)
    v1, g1, _ = sc.brute(q, alpha, paper_metric=True)
    assert np.array_equal(v0, v1)
    for k in range(len(q)):
        ts, vs = [], []
        for i in range(len(F)):
            e = sc.prim_eval(i, q[k], alpha)
            p = sc.prim_eval(i, q[k], alpha, paper_metric=True)
            assert p["t"] == e["t"]
            np.testing.assert_allclose(p["vec"], e["grad_d"] + (e["vec"] - e["grad_d"]) / alpha, rtol=0, atol=1e-12)
            ts.append(e["t"])
            vs.append(p["vec"])
        ts = np.array(ts)
        s = np.exp(ts - ts.max())
        ref = (s[:, None] * np.array(vs)).sum(0) / s.sum()
        np.testing.assert_allclose(g1[k], ref, rtol=1e-10, atol=1e-12)
    # and it differs from the exact gradient where the weights vary
    assert np.abs(g1 - g0).max() > 1e-6
