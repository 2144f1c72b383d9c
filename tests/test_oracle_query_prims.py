"""Pins of the oracle's query primitives (Sec. 3.4, Sec. 3.6): simplex
distances against the point distances, closed forms and dense sampling;
primitive queries that are points reduce to point queries; Barnes-Hut with
the box test is exact at beta = 0 and an underestimate otherwise; Theorem
A.1's bounds; translation gradients and the query-mesh objective against
finite differences."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from oracle import mesh as OMesh


def _rand_simplex(rng, k, scale=1.0, c=None):
    c = rng.normal(size=3) if c is None else np.asarray(c, float)
    return c + scale * rng.normal(size=(k, 3))


def _grid(k, n):
    if k == 1:
        return [np.array([1.0])]
    if k == 2:
        return [np.array([1 - t, t]) for t in np.linspace(0, 1, n)]
    g = np.linspace(0, 1, n)
    return [np.array([1 - a - b, a, b]) for a in g for b in g if a + b <= 1 + 1e-12]


@pytest.mark.parametrize("ka,kb", [(1, 2), (1, 3), (2, 2), (2, 3), (3, 3)])
def test_simplex_distance_dense_sampling(ka, kb):
    rng = np.random.default_rng(ka * 10 + kb)
    for _ in range(30):
        A = _rand_simplex(rng, ka)
        B = _rand_simplex(rng, kb, c=rng.normal(size=3) * 1.5)
        d, pa, pb = oracle.simplex_closest(A, B)
        assert abs(np.linalg.norm(pa - pb) - d) <= 1e-12
        # the points lie on their simplices: d is attained, so d >= true min
        ga, gb = _grid(ka, 41), _grid(kb, 41)
        PA = np.array([w @ A for w in ga])
        PB = np.array([w @ B for w in gb])
        dmin = np.sqrt(((PA[:, None, :] - PB[None]) ** 2).sum(-1)).min()
        assert d <= dmin + 1e-12
        # and the grid's minimum is within its resolution of d
        h = max(np.ptp(A, 0).max(), np.ptp(B, 0).max()) / 40 * 2
        assert dmin <= d + h
        # symmetry
        d2, qb, qa = oracle.simplex_closest(B, A)
        assert abs(d2 - d) <= 1e-12


@pytest.mark.parametrize("k", [2, 3])
def test_point_against_simplex_matches_point_distances(k):
    """A point query against a data edge/triangle: the face-pair QP and the
    oracle's own point distance routines (Voronoi / 2x2 QP) agree."""
    rng = np.random.default_rng(k)
    if k == 2:
        V, E = synth.tiny_mesh("polyline")
        sc = oracle.Scene(edge_V=V, edge_E=E)
        prims = V[E].astype(np.float64)
    else:
        V, F = synth.icosphere(1)
        sc = oracle.Scene(tri_V=V, tri_F=F)
        prims = V[F].astype(np.float64)
    for i in range(min(len(prims), 20)):
        for q in rng.normal(size=(5, 3)) * 1.5:
            d, pf, pq = oracle.simplex_closest(prims[i], q[None])
            ref = sc.prim_eval(i, q)["d"]
            assert abs(d - ref) <= 1e-12 * max(1.0, ref)


def test_simplex_closed_forms():
    # skew segments crossing at right angles, offset 0.7 in z
    d, pa, pb = oracle.simplex_closest([[-1, 0, 0], [1, 0, 0]], [[0.3, -1, 0.7], [0.3, 1, 0.7]])
    assert abs(d - 0.7) < 1e-14 and np.allclose(pa, [0.3, 0, 0]) and np.allclose(pb, [0.3, 0, 0.7])
    # parallel overlapping segments 0.5 apart
    d, _, _ = oracle.simplex_closest([[0, 0, 0], [2, 0, 0]], [[1, 0.5, 0], [3, 0.5, 0]])
    assert abs(d - 0.5) < 1e-14
    # triangles in parallel planes, overlapping footprints
    T = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    d, _, _ = oracle.simplex_closest(T, T + [0.1, 0.1, 0.25])
    assert abs(d - 0.25) < 1e-14
    # an edge piercing a triangle, and two triangles crossing
    d, pa, pb = oracle.simplex_closest([[0.2, 0.2, -1], [0.2, 0.2, 1]], T)
    assert d < 1e-14 and np.allclose(pa, [0.2, 0.2, 0])
    d, _, _ = oracle.simplex_closest(T, [[0.3, -0.5, -0.5], [0.3, 0.5, 0.5], [0.3, 0.5, -0.5]])
    assert d < 1e-14
    # vertex above the interior of a triangle
    d, pa, _ = oracle.simplex_closest([[0.25, 0.25, 2]], T)
    assert abs(d - 2) < 1e-14


def _scene(kind):
    V, F = synth.icosphere(2)
    Vl, El = synth.tiny_mesh("polyline")
    P = synth.points_on_sphere(200, 0.01, seed=1)
    return {"points": dict(points=P), "edges": dict(edge_V=Vl, edge_E=El), "tris": dict(tri_V=V, tri_F=F),
            "mixed": dict(points=P * 1.5, edge_V=Vl, edge_E=El, tri_V=V * 0.6, tri_F=F)}[kind]


def _queries(k, m, seed, spread=0.15):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-2, 2, (m, 3))
    V = (c[:, None, :] + spread * rng.normal(size=(m, k, 3))).reshape(-1, 3).astype(np.float32)
    F = np.arange(m * k, dtype=np.int32).reshape(m, k)
    return V, F


@pytest.mark.parametrize("kind", ["points", "edges", "tris", "mixed"])
def test_point_primitives_reduce_to_point_queries(kind):
    sc = oracle.Scene(**_scene(kind))
    q = synth.uniform_box(50, [-2] * 3, [2] * 3, 3)
    v0, g0, d0 = sc.brute(q, 20.0)
    v1, g1, d1 = sc.brute_prims(q, np.arange(50, dtype=np.int32)[:, None], 20.0)
    assert np.allclose(v1, v0, rtol=1e-13, atol=1e-13) and np.allclose(g1, g0, rtol=1e-12, atol=1e-13)
    # a degenerate edge (both ends at q) is the point q
    F2 = np.stack([np.arange(50), np.arange(50)], 1).astype(np.int32)
    v2, g2, _ = sc.brute_prims(q, F2, 20.0)
    assert np.allclose(v2, v0, rtol=1e-12, atol=1e-12) and np.allclose(g2, g0, rtol=1e-9, atol=1e-10)
    # Barnes-Hut: the box test of a point query is the point test
    sc.build_tree(2)
    b0 = sc.bh(q, 20.0, 0.5)
    b1 = sc.bh_prims(q, np.arange(50, dtype=np.int32)[:, None], 20.0, 0.5)
    assert np.allclose(b1[0], b0[0], rtol=1e-13) and np.array_equal(b1[2], b0[2])


@pytest.mark.parametrize("kind", ["points", "edges", "tris", "mixed"])
@pytest.mark.parametrize("k", [2, 3])
def test_bh_prims_exact_at_beta0_and_conservative(kind, k):
    sc = oracle.Scene(**_scene(kind))
    sc.build_tree(1)
    V, F = _queries(k, 60, 7 * k)
    ex, eg, dmin = sc.brute_prims(V, F, 15.0)
    b0, g0, c0, _ = sc.bh_prims(V, F, 15.0, 0.0)
    assert np.allclose(b0, ex, rtol=1e-12, atol=1e-12) and np.allclose(g0, eg, rtol=1e-9, atol=1e-11)
    assert np.all(c0[:, 1] == 0)
    b1, g1, c1, _ = sc.bh_prims(V, F, 15.0, 0.5)
    assert np.all(b1 <= ex + 1e-12) and np.any(c1[:, 1] > 0)
    # Theorem A.1 with the weights bounded by A
    A = max(sc.A_E, sc.A_T, 1.0)
    assert np.all(ex <= dmin + 1e-12)
    assert np.all(ex >= dmin - np.log(A * sc.n) / 15.0 - 1e-12)


@pytest.mark.parametrize("k", [2, 3])
def test_translation_gradient_fd(k):
    """Unit weights: grad d^ of a query primitive is the derivative of d^
    under a rigid translation of all its vertices."""
    sc = oracle.Scene(**_scene("mixed"))
    V, F = _queries(k, 25, 11 + k)
    V = V.astype(np.float64)
    _, g, _ = sc.brute_prims(V, F, 10.0, unit=True)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3); e[j] = h
        fp = sc.brute_prims(V + e, F, 10.0, unit=True)[0]
        fm = sc.brute_prims(V - e, F, 10.0, unit=True)[0]
        assert np.allclose(g[:, j], (fp - fm) / (2 * h), atol=2e-6, rtol=1e-5)


def test_mesh_objective():
    """Eq. lse_full for a small query mesh: D between min d^ - log(m)/alpha_q
    and min d^, the vertex gradients summing to the derivative of D under a
    rigid translation (unit weights), and weights gamma summing to 1."""
    sc = oracle.Scene(**_scene("tris"))
    Vq, Fq = synth.icosphere(1)
    Vq = (Vq.astype(np.float64) * 0.3 + [1.6, 0.2, 0.1])
    val, grad, _ = sc.brute_prims(Vq, Fq, 10.0, unit=True)
    D, G, gam = OMesh.mesh_objective(val, grad, Fq, Vq.shape[0], 25.0)
    assert val.min() - np.log(len(val)) / 25.0 <= D <= val.min()
    assert abs(gam.sum() - 1.0) < 1e-12
    h = 1e-6
    fd = []
    for j in range(3):
        e = np.zeros(3); e[j] = h
        Dp = OMesh.mesh_objective(sc.brute_prims(Vq + e, Fq, 10.0, unit=True)[0], grad, Fq, Vq.shape[0], 25.0)[0]
        Dm = OMesh.mesh_objective(sc.brute_prims(Vq - e, Fq, 10.0, unit=True)[0], grad, Fq, Vq.shape[0], 25.0)[0]
        fd.append((Dp - Dm) / (2 * h))
    assert np.allclose(G.sum(0), fd, atol=1e-6, rtol=1e-5)
