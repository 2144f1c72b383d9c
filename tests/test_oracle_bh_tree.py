"""Pins of the oracle's Morton codes, radix tree and Barnes-Hut evaluation
(Sec. 3.5, Alg. 1, Alg. 2, App. D): an independent Morton/Karras
construction in Python, structural invariants, beta = 0 exactness, the
conservative (underestimate) property and its derived lower bound."""
import math

import numpy as np
import pytest

import oracle
import synth


# ------------------------------------------------------------------ Morton code
def _morton_py(c, lo, hi):
    """Morton code written out with numpy float32 scalar arithmetic."""
    f = np.float32
    k = []
    for j in range(3):
        ext = f(hi[j]) - f(lo[j])
        u = f(0.0)
        if ext > 0:
            u = (f(c[j]) - f(lo[j])) / ext
        u = min(max(u, f(0.0)), f(1.0))
        v = int(np.floor(u * f(2097152.0)))
        k.append(min(v, 2097151))
    code = 0
    for b in range(20, -1, -1):
        for j in range(3):
            code = (code << 1) | ((k[j] >> b) & 1)
    return code


def _centroids_f32(s, kind):
    f = np.float32
    if kind == "points":
        return [tuple(p) for p in s.points]
    if kind == "tris":
        out = []
        for tri in s.tri_F:
            a, b, c = (s.tri_V[i] for i in tri)
            out.append(tuple(((a[j] + b[j]) + c[j]) * f(1.0 / 3.0) for j in range(3)))
        return out
    out = []
    for e in s.edge_E:
        a, b = s.edge_V[e[0]], s.edge_V[e[1]]
        out.append(tuple((a[j] + b[j]) * f(0.5) for j in range(3)))
    return out


@pytest.mark.parametrize("kind", ["points", "tris", "edges"])
def test_morton_codes_independent(kind):
    if kind == "points":
        s = oracle.Scene(points=synth.points_on_sphere(300, 0.01, 3))
    elif kind == "tris":
        V, F = synth.icosphere(2)
        s = oracle.Scene(tri_V=V, tri_F=F)
    else:
        V, E = synth.tiny_mesh("polyline")
        s = oracle.Scene(edge_V=V, edge_E=E)
    t = s.build_tree(1)
    allv = np.concatenate([s.points, s.edge_V, s.tri_V])
    lo, hi = allv.min(0), allv.max(0)
    assert np.array_equal(t["scene_box"], np.concatenate([lo, hi]))
    ref = [_morton_py(c, lo, hi) for c in _centroids_f32(s, kind)]
    assert [int(x) for x in t["codes"]] == ref


def test_morton_corners():
    pts = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.25, 0.75]], np.float32)
    s = oracle.Scene(points=pts)
    t = s.build_tree(1)
    assert int(t["codes"][0]) == 0
    assert int(t["codes"][1]) == (1 << 63) - 1
    # x = 0.5 -> 2^20 (code bit 3*20+2), y = 0.25 -> 2^19 (bit 3*19+1),
    # z = 0.75 -> 2^20 + 2^19 (bits 3*20 and 3*19)
    assert int(t["codes"][2]) == (1 << 62) | (1 << 58) | (1 << 60) | (1 << 57)


# ------------------------------------------------------------------ radix tree
def _karras_py(keys):
    """Karras (2012) parallel construction, one internal node at a time."""
    n = len(keys)

    def delta(i, j):
        if j < 0 or j >= n:
            return -1
        x = keys[i] ^ keys[j]
        return 96 - x.bit_length()

    left, right = [0] * (n - 1), [0] * (n - 1)
    for i in range(n - 1):
        d = 1 if delta(i, i + 1) - delta(i, i - 1) > 0 else -1
        dmin = delta(i, i - d)
        lmax = 2
        while delta(i, i + lmax * d) > dmin:
            lmax *= 2
        l = 0
        t = lmax // 2
        while t >= 1:
            if delta(i, i + (l + t) * d) > dmin:
                l += t
            t //= 2
        j = i + l * d
        dnode = delta(i, j)
        s = 0
        t = (l + 1) // 2
        while True:
            if delta(i, i + (s + t) * d) > dnode:
                s += t
            if t == 1:
                break
            t = (t + 1) // 2
        g = i + s * d + min(d, 0)
        left[i] = -(g + 1) if min(i, j) == g else g
        right[i] = -(g + 2) if max(i, j) == g + 1 else g + 1
    return left, right


@pytest.mark.parametrize("L", [1, 3, 4])
@pytest.mark.parametrize("case", ["sphere", "dups", "tris"])
def test_topology_matches_independent_karras(case, L):
    if case == "sphere":
        s = oracle.Scene(points=synth.points_on_sphere(700, 0.005, 5))
    elif case == "dups":
        p = synth.points_on_sphere(50, 0.0, 6)
        s = oracle.Scene(points=np.concatenate([p, p, p[:20], p[:7]]))   # equal codes
    else:
        V, F = synth.icosphere(2)
        s = oracle.Scene(tri_V=V, tri_F=F)
    t = s.build_tree(L)
    codes, srt = t["codes"], t["sorted"]
    order = np.lexsort((np.arange(s.n), codes))
    assert np.array_equal(srt, order)
    nb = t["nb"]
    assert nb == (s.n + L - 1) // L
    keys = [(int(codes[srt[b * L]]) << 32) | int(srt[b * L]) for b in range(nb)]
    left, right = _karras_py(keys)
    assert list(t["left"]) == left and list(t["right"]) == right


def _invariants(s, t):
    nb, L = t["nb"], s.L
    seen = np.zeros(nb, int)
    allv = [s.points, s.edge_V, s.tri_V]

    def visit(node, leaf):
        if leaf:
            seen[node] += 1
            return node * L, min((node + 1) * L, s.n) - 1, t["leaf_lo"][node], t["leaf_hi"][node], t["leaf_count"][node]
        a = visit(*((-t["left"][node] - 1, True) if t["left"][node] < 0 else (t["left"][node], False)))
        b = visit(*((-t["right"][node] - 1, True) if t["right"][node] < 0 else (t["right"][node], False)))
        assert a[1] + 1 == b[0]                            # contiguous ranges
        lo, hi = t["node_lo"][node], t["node_hi"][node]
        assert np.all(lo <= a[2]) and np.all(lo <= b[2]) and np.all(hi >= a[3]) and np.all(hi >= b[3])
        assert np.array_equal(lo, np.minimum(a[2], b[2])) and np.array_equal(hi, np.maximum(a[3], b[3]))
        assert t["node_count"][node] == a[4] + b[4]
        return a[0], b[1], lo, hi, a[4] + b[4]

    if nb == 1:
        visit(0, True)
    else:
        r = visit(0, False)
        assert r[0] == 0 and r[1] == s.n - 1 and r[4] == s.n
    assert np.all(seen == 1)


@pytest.mark.parametrize("L", [1, 2, 5])
def test_tree_invariants_and_leaf_boxes(L):
    V, F = synth.icosphere(2)
    s = oracle.Scene(points=synth.points_on_sphere(100, 0.01, 2) * 1.3, tri_V=V, tri_F=F)
    t = s.build_tree(L)
    _invariants(s, t)
    # leaf boxes are exact min/max over the bucket's primitive vertices
    params, kind, iso = s.prim_params()
    srt = t["sorted"]
    for b in range(t["nb"]):
        vs = []
        for k in srt[b * L:(b + 1) * L]:
            if k < 100:
                vs.append(s.points[k])
            else:
                vs.extend(V[F[k - 100]])
        vs = np.array(vs)
        assert np.array_equal(t["leaf_lo"][b], vs.min(0)) and np.array_equal(t["leaf_hi"][b], vs.max(0))


def test_single_and_empty_trees():
    s = oracle.Scene(points=np.array([[1, 2, 3]], np.float32))
    t = s.build_tree(1)
    assert t["nb"] == 1 and t["left"].size == 0
    v, g, cnt, _ = s.bh(np.array([[1, 2, 5.0]]), 10.0, 0.5)
    assert v[0] == pytest.approx(2.0)


# ------------------------------------------------------------------ Barnes-Hut
def _scenes():
    V, F = synth.icosphere(3)
    V = synth.perturb_radial(V, 0.01, 1)
    Ve, E = synth.tiny_mesh("polyline")
    return {
        "points": oracle.Scene(points=synth.points_on_sphere(2000, 0.005, 0)),
        "tris": oracle.Scene(tri_V=V, tri_F=F),
        "mixed": oracle.Scene(points=synth.points_on_sphere(300, 0.01, 1) * 1.5, edge_V=Ve, edge_E=E,
                              tri_V=V, tri_F=F),
    }


@pytest.mark.parametrize("name", ["points", "tris", "mixed"])
@pytest.mark.parametrize("L", [1, 4])
def test_beta_zero_is_brute_force(name, L):
    s = _scenes()[name]
    s.build_tree(L)
    q = synth.shell_queries(200, seed=7)
    vb, gb, dm = s.brute(q, 80.0)
    v, g, cnt, _ = s.bh(q, 80.0, 0.0)
    assert np.abs(v - vb).max() < 1e-12
    assert np.abs(g - gb).max() < 1e-10
    t = s.tree()
    assert np.all(cnt[:, 0] == 2 * t["nb"] - 1) and np.all(cnt[:, 1] == 0) and np.all(cnt[:, 2] == s.n)


@pytest.mark.parametrize("beta", [0.25, 0.5, 1.0])
def test_points_underestimate_and_derived_bound(beta):
    # far field at the box's closest point never overestimates (Sec. 3.5);
    # every point of an accepted box lies within d_box + |B| and |B| < beta d_box
    s = _scenes()["points"]
    s.build_tree(1)
    q = synth.shell_queries(400, seed=8)
    alpha = 100.0
    vb, gb, dm = s.brute(q, alpha)
    v, g, cnt, _ = s.bh(q, alpha, beta)
    assert np.all(v <= vb + 1e-12)
    # lower bound: each accepted node contributes at most e^{alpha |B|} times
    # its exact part with |B| <= beta * d_box <= beta * (d_max of the scene)
    diag = np.linalg.norm(s.points.max(0) - s.points.min(0))
    dmax = np.linalg.norm(q, axis=1) + diag
    assert np.all(v >= vb - beta * dmax - 1e-12)
    assert np.all(cnt[:, 1] > 0) or beta == 0


def test_bh_error_shrinks_with_beta():
    s = _scenes()["tris"]
    s.build_tree(1)
    q = synth.shell_queries(300, seed=9)
    vb, _, _ = s.brute(q, 200.0)
    errs = []
    for beta in (1.0, 0.5, 0.25, 0.1):
        v, _, cnt, _ = s.bh(q, 200.0, beta)
        errs.append(np.abs(v - vb).mean())
    assert errs == sorted(errs, reverse=True)


def test_fp32_and_fp64_decisions_agree_away_from_the_margin():
    s = _scenes()["tris"]
    s.build_tree(1)
    q = synth.shell_queries(500, seed=10)
    v32, g32, c32, m32 = s.bh(q, 200.0, 0.5, decision="fp32", want_margin=True)
    v64, g64, c64, m64 = s.bh(q, 200.0, 0.5, decision="fp64", want_margin=True)
    safe = m64 > 1e-5
    assert safe.mean() > 0.95
    assert np.array_equal(c32[safe], c64[safe])
    assert np.abs(v32[safe] - v64[safe]).max() < 1e-12
