"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only makes geometry and query points (fp32 numpy arrays). It holds
none of the smooth-distance arithmetic: no distances, weights, trees or sums.
Every generator takes an explicit ``seed`` and draws from
``numpy.random.default_rng(seed)``, so the same call gives the same bytes on
every machine.

Workload recipes (the paper's scenes are not available, these stand in):

* ``points_on_sphere``  — point cloud on the unit sphere with isotropic noise
  (stands in for the point-cloud examples of Sec. 3.1).
* ``icosphere``          — recursively subdivided icosahedron, the triangle
  mesh workload (stands in for the Thingi10K meshes of Sec. 4.4).
* ``shell_queries``      — 70 % of queries near the surface, 30 % in a box.
* ``street_scene``       — synthetic lidar street with ground, box buildings,
  poles and catenary wires (stands in for the Toronto-3D scan, Sec. 4.5).
* ``geodesic_icosphere`` / ``torus`` — rigid query bodies (Sec. 4.5).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "points_on_sphere", "uniform_box", "icosphere", "perturb_radial",
    "shell_queries", "geodesic_icosphere", "torus", "random_rotation",
    "street_scene", "config1", "config2", "config3_scene", "config3_body",
    "config4_bodies", "surrogate_samples", "tiny_mesh", "mesh_edges", "blob", "trace_camera",
]


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def points_on_sphere(n: int = 4096, sigma: float = 0.005, seed: int = 0):
    """n standard-normal vectors normalised onto the unit sphere plus N(0, sigma^2) noise."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x += sigma * rng.standard_normal((n, 3))
    return _f32(x)


def uniform_box(m: int, lo, hi, seed: int = 0):
    rng = np.random.default_rng(seed)
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (3,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (3,))
    return _f32(lo + (hi - lo) * rng.random((m, 3)))


def icosphere(level: int = 6):
    """Icosahedron refined ``level`` times by 4-way midpoint subdivision; every
    new vertex is projected to the unit sphere. Level 6 gives 81,920 triangles
    and 40,962 vertices. Returns (V float32 [nv,3], F int32 [nf,3])."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = np.array(V, dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
                  (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
                  (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
                  (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)],
                 dtype=np.int64)
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
        e.sort(axis=1)
        key = e[:, 0] * nv + e[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        a, b = uniq // nv, uniq % nv
        mid = V[a] + V[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        V = np.concatenate([V, mid])
        nf = F.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        F = np.concatenate([
            np.stack([F[:, 0], m01, m20], 1),
            np.stack([F[:, 1], m12, m01], 1),
            np.stack([F[:, 2], m20, m12], 1),
            np.stack([m01, m12, m20], 1)])
    return _f32(V), np.ascontiguousarray(F.astype(np.int32))


def perturb_radial(V, sigma: float = 0.01, seed: int = 0):
    """r <- r * (1 + N(0, sigma^2)) per vertex."""
    rng = np.random.default_rng(seed)
    V = np.asarray(V, dtype=np.float64)
    return _f32(V * (1.0 + sigma * rng.standard_normal((V.shape[0], 1))))


def shell_queries(m: int = 262144, frac_shell: float = 0.7, r_lo: float = 0.9,
                  r_hi: float = 1.1, box: float = 2.0, seed: int = 0):
    """frac_shell of the queries at a uniform direction and radius uniform in
    [r_lo, r_hi]; the rest uniform in [-box, box]^3; the two groups are
    interleaved in random order."""
    rng = np.random.default_rng(seed)
    ns = int(round(frac_shell * m))
    d = rng.standard_normal((ns, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(r_lo, r_hi, size=(ns, 1))
    shell = d * r
    uni = rng.uniform(-box, box, size=(m - ns, 3))
    q = np.concatenate([shell, uni])
    q = q[rng.permutation(m)]
    return _f32(q)


def geodesic_icosphere(freq: int):
    """Class-I geodesic sphere: every icosahedron face split into freq^2
    triangles on a barycentric grid, vertices projected to the unit sphere.
    V = 10 freq^2 + 2, F = 20 freq^2."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    B = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
                  (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
                  (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], dtype=np.float64)
    Fi = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
          (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
          (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
          (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    n = int(freq)
    # grid points (i, j) with i + j <= n on each face; shared points are merged
    # through an integer key built from the (sorted) global description.
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    mask = ii + jj <= n
    ii, jj = ii[mask], jj[mask]
    kk = n - ii - jj
    loc = -np.ones((n + 1, n + 1), dtype=np.int64)
    loc[ii, jj] = np.arange(ii.size)
    # local triangles of the grid
    tris = []
    for i in range(n):
        for j in range(n - i):
            tris.append((loc[i, j], loc[i + 1, j], loc[i, j + 1]))
            if i + j < n - 1:
                tris.append((loc[i + 1, j], loc[i + 1, j + 1], loc[i, j + 1]))
    tris = np.array(tris, dtype=np.int64)
    allkeys, allpos, allF = [], [], []
    M = 13 * (n + 1) + 1
    for f, (a, b, c) in enumerate(Fi):
        # A grid point is identified by the multiset of (corner, weight) pairs
        # with non-zero weight; zero weights code as 0 and sort first, so the
        # same point seen from two faces gets the same key.
        wts = np.stack([kk, ii, jj], 1)
        cid = np.array([a, b, c])
        codes = np.where(wts > 0, (cid[None, :] + 1) * (n + 1) + wts, 0)
        codes.sort(axis=1)
        key = (codes[:, 0] * M + codes[:, 1]) * M + codes[:, 2]
        pos = (np.outer(kk, B[a]) + np.outer(ii, B[b]) + np.outer(jj, B[c])) / n
        allkeys.append(key)
        allpos.append(pos)
        allF.append(tris + f * ii.size)
    keys = np.concatenate(allkeys)
    pos = np.concatenate(allpos)
    uniq, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    V = pos[first]
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = inv[np.concatenate(allF)]
    return _f32(V), np.ascontiguousarray(F.astype(np.int32))


def torus(n: int, m: int, R: float = 1.0, r: float = 0.35):
    """n x m quad grid on a torus (major radius R, minor radius r), split into
    2 n m triangles; V = n m."""
    u = 2 * np.pi * np.arange(n) / n
    v = 2 * np.pi * np.arange(m) / m
    uu, vv = np.meshgrid(u, v, indexing="ij")
    x = (R + r * np.cos(vv)) * np.cos(uu)
    y = (R + r * np.cos(vv)) * np.sin(uu)
    z = r * np.sin(vv)
    V = np.stack([x, y, z], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    a = i * m + j
    b = ((i + 1) % n) * m + j
    c = ((i + 1) % n) * m + (j + 1) % m
    d = i * m + (j + 1) % m
    F = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3),
                        np.stack([a, c, d], -1).reshape(-1, 3)])
    return _f32(V), np.ascontiguousarray(F.astype(np.int32))


def random_rotation(rng):
    """Uniform random rotation (Shoemake's uniform unit quaternion)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


# ----------------------------------------------------------------------------
# synthetic lidar street (stand-in for the city scan of Sec. 4.5)
# ----------------------------------------------------------------------------

def _street_objects(rng):
    boxes = []
    for _ in range(40):
        sx, sy, sz = rng.uniform(5.0, 30.0, 3)
        side = rng.choice([-1.0, 1.0])
        yc = side * rng.uniform(12.0 + sy / 2, max(12.0 + sy / 2, 40.0 - sy / 2) + 1e-6)
        xc = rng.uniform(-200.0 + sx / 2, 200.0 - sx / 2)
        boxes.append((xc - sx / 2, yc - sy / 2, 0.0, xc + sx / 2, yc + sy / 2, sz))
    poles = []
    xs = -195.0 + 13.0 * np.arange(30)
    for side in (-6.0, 6.0):
        for x in xs:
            poles.append((x, side))
    return np.array(boxes), np.array(poles)


def _cast(o, d, boxes, poles, rmax=60.0, pole_r=0.15, pole_h=8.0):
    """Analytic ray cast of rays (origins o [n,3], unit directions d [n,3])
    against the ground z=0, boxes and vertical cylinders; returns the hit
    range (inf where nothing is hit within rmax)."""
    t = np.full(d.shape[0], np.inf)
    dz = d[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = -o[:, 2] / dz
        inv = 1.0 / d
    t = np.where((dz < 0) & (tg > 0), tg, t)
    for b in boxes:
        lo, hi = b[:3], b[3:]
        with np.errstate(invalid="ignore"):
            t1 = (lo - o) * inv
            t2 = (hi - o) * inv
        mn = np.fmin(t1, t2)
        mx = np.fmax(t1, t2)
        tn = np.fmax(np.fmax(mn[:, 0], mn[:, 1]), mn[:, 2])
        tf = np.fmin(np.fmin(mx[:, 0], mx[:, 1]), mx[:, 2])
        hit = (tn <= tf) & (tn > 0)
        t = np.where(hit & (tn < t), tn, t)
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    for (px, py) in poles:
        ox, oy = o[:, 0] - px, o[:, 1] - py
        bq = 2 * (ox * d[:, 0] + oy * d[:, 1])
        cq = ox * ox + oy * oy - pole_r ** 2
        disc = bq * bq - 4 * a * cq
        ok = disc > 0
        with np.errstate(invalid="ignore", divide="ignore"):
            tc = (-bq - np.sqrt(np.where(ok, disc, 0))) / (2 * a)
        z = o[:, 2] + tc * d[:, 2]
        hit = ok & (tc > 0) & (z >= 0) & (z <= pole_h)
        t = np.where(hit & (tc < t), tc, t)
    return np.where(t <= rmax, t, np.inf)


def street_scene(n_points: int = 2_000_000, n_wire_segments: int = 50_000, seed: int = 2):
    """Synthetic lidar street: 400 m x 80 m along x, sensor at y=0, z=1.8 m
    moving in 0.5 m steps, 64 scanlines at elevations in [-25, +15] degrees
    with randomly phased azimuths. Ground z=0 with N(0, 0.02^2) height noise,
    40 axis-aligned box buildings (sides 5-30 m) at |y| in [12, 40], 60 poles
    (r=0.15 m, h=8 m) at |y|=6 every 13 m, range noise N(0, 0.03^2); returns
    truncated (or repeated) to exactly n_points, inside the street rectangle.
    Catenary wires (sag 0.5 m) join consecutive pole tops on each side with
    n_wire_segments segments in total and shared vertices.
    Returns dict(points, wire_V, wire_E, boxes, poles)."""
    rng = np.random.default_rng(seed)
    boxes, poles = _street_objects(rng)
    elev = np.deg2rad(np.linspace(-25.0, 15.0, 64))
    sweeps = np.arange(-200.0, 200.0 + 1e-9, 0.5)
    naz = 96
    pts = []
    chunk = 20
    for s0 in range(0, sweeps.size, chunk):
        xs = sweeps[s0:s0 + chunk]
        az = rng.uniform(0, 2 * np.pi, size=(xs.size, 64, naz))
        el = np.broadcast_to(elev[None, :, None], az.shape)
        d = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1).reshape(-1, 3)
        o = np.zeros_like(d)
        o[:, 0] = np.repeat(xs, 64 * naz)
        o[:, 2] = 1.8
        # only objects within the sensor range of this chunk can be hit
        near_b = (boxes[:, 3] >= xs[0] - 60.0) & (boxes[:, 0] <= xs[-1] + 60.0)
        near_p = np.abs(poles[:, 0] - 0.5 * (xs[0] + xs[-1])) <= 60.0 + 0.5 * (xs[-1] - xs[0])
        t = _cast(o, d, boxes[near_b], poles[near_p])
        ok = np.isfinite(t)
        tt = t[ok] + 0.03 * rng.standard_normal(int(ok.sum()))
        p = o[ok] + d[ok] * tt[:, None]
        ground = np.abs(p[:, 2]) < 0.2
        p[:, 2] += np.where(ground, 0.02 * rng.standard_normal(p.shape[0]), 0.0)
        inside = (np.abs(p[:, 0]) <= 200.0) & (np.abs(p[:, 1]) <= 40.0)
        pts.append(p[inside])
    P = np.concatenate(pts)
    if P.shape[0] >= n_points:
        P = P[rng.permutation(P.shape[0])[:n_points]]
    else:
        extra = P[rng.integers(0, P.shape[0], n_points - P.shape[0])]
        P = np.concatenate([P, extra])
    # wires
    Vw, Ew = [], []
    nspans = 2 * (poles.shape[0] // 2 - 1)
    base, rem = divmod(n_wire_segments, nspans)
    span_id = 0
    vcount = 0
    for side in (-6.0, 6.0):
        tops = poles[poles[:, 1] == side]
        tops = tops[np.argsort(tops[:, 0])]
        prev_last = None
        for k in range(tops.shape[0] - 1):
            nseg = base + (1 if span_id < rem else 0)
            span_id += 1
            s = np.linspace(0.0, 1.0, nseg + 1)
            x = tops[k, 0] + s * (tops[k + 1, 0] - tops[k, 0])
            y = np.full_like(s, side)
            z = 8.0 - 4 * 0.5 * s * (1 - s)
            pv = np.stack([x, y, z], 1)
            if prev_last is None:
                Vw.append(pv)
                idx = vcount + np.arange(nseg + 1)
                vcount += nseg + 1
            else:
                Vw.append(pv[1:])
                idx = np.concatenate([[prev_last], vcount + np.arange(nseg)])
                vcount += nseg
            Ew.append(np.stack([idx[:-1], idx[1:]], 1))
            prev_last = idx[-1]
    Vw = np.concatenate(Vw)
    Ew = np.concatenate(Ew)
    return dict(points=_f32(P), wire_V=_f32(Vw), wire_E=np.ascontiguousarray(Ew.astype(np.int32)),
                boxes=boxes, poles=poles)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def config1(seed: int = 0):
    """4,096 noisy sphere points (sigma 0.005), 1,024 queries uniform in
    [-1.5, 1.5]^3; alpha = 100, unit weights, beta in {0, 0.5}."""
    pts = points_on_sphere(4096, 0.005, seed)
    q = uniform_box(1024, -1.5, 1.5, seed + 100)
    return dict(points=pts, queries=q, alpha=100.0, beta=0.5)


def config2(seed: int = 1, m: int = 262144, level: int = 6):
    """Level-6 icosphere (81,920 triangles) with radial noise 0.01; 262,144
    queries, 70 % in the shell |r-1| < 0.1 and 30 % uniform in [-2, 2]^3."""
    V, F = icosphere(level)
    V = perturb_radial(V, 0.01, seed)
    q = shell_queries(m, 0.7, 0.9, 1.1, 2.0, seed + 100)
    return dict(V=V, F=F, queries=q)


def config3_scene(seed: int = 2, n_points: int = 2_000_000, n_wire_segments: int = 50_000):
    return street_scene(n_points, n_wire_segments, seed)


def config3_body(seed: int = 3, freq: int = 100, scale=(2.0, 1.0, 0.7)):
    """Geodesic icosphere of frequency ``freq`` (10 freq^2 + 2 vertices)
    stretched by ``scale``; returns the rest-pose vertices and faces plus a
    random pose (rotation vector theta, translation p) placing the body
    0.5-3 m above the ground near the sensor path."""
    rng = np.random.default_rng(seed)
    V, F = geodesic_icosphere(freq)
    V = _f32(V.astype(np.float64) * np.asarray(scale))
    R = random_rotation(rng)
    theta = _rotvec(R)
    Vr = V.astype(np.float64) @ R.T
    zmin = Vr[:, 2].min()
    p = np.array([rng.uniform(-150, 150), rng.uniform(-4, 4), rng.uniform(0.5, 3.0) - zmin])
    return dict(V0=V, F=F, theta=theta.astype(np.float64), p=p.astype(np.float64))


def _rotvec(R):
    c = (np.trace(R) - 1) / 2
    c = min(1.0, max(-1.0, c))
    ang = math.acos(c)
    if ang < 1e-12:
        return np.zeros(3)
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    s = math.sin(ang)
    if s < 1e-6:
        # near pi: axis from the diagonal
        ax = np.sqrt(np.maximum((np.diag(R) + 1) / 2, 0))
        ax = ax * np.sign(np.where(w == 0, 1, w))
        return ax / np.linalg.norm(ax) * ang
    return w / (2 * s) * ang


def config4_bodies(seed: int = 4, n_bodies: int = 64, vmin: float = 1e3, vmax: float = 2e5,
                   scene_lo=(-200.0, -40.0, 0.0), scene_hi=(200.0, 40.0, 30.0)):
    """64 rigid bodies, each an icosphere (frequency chosen so V ~ target) or
    a torus (n x m grid, R/r in [2, 4]); target V log-uniform in [1e3, 2e5];
    scale 0.3-3 m; random rotation and position inside the scene bounds.
    Returns a list of dict(V0, F, theta, p)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_bodies):
        target = math.exp(rng.uniform(math.log(vmin), math.log(vmax)))
        if rng.random() < 0.5:
            freq = max(2, int(round(math.sqrt((target - 2) / 10))))
            V, F = geodesic_icosphere(freq)
        else:
            ratio = rng.uniform(2.0, 4.0)
            nm = max(16, int(round(target)))
            m = max(4, int(round(math.sqrt(nm / ratio))))
            n = max(4, int(round(nm / m)))
            V, F = torus(n, m, 1.0, 1.0 / ratio)
        scale = rng.uniform(0.3, 3.0)
        R = random_rotation(rng)
        lo, hi = np.asarray(scene_lo), np.asarray(scene_hi)
        p = lo + (hi - lo) * rng.random(3)
        out.append(dict(V0=_f32(V.astype(np.float64) * scale), F=F,
                        theta=_rotvec(R), p=p))
    return out


def surrogate_samples(lo, hi, n: int, seed: int = 5, near_points=None, near_frac: float = 0.0,
                      near_radius: float = 2.0):
    """n points: (1 - near_frac) uniform in the box [lo, hi]; near_frac within
    ``near_radius`` of randomly chosen ``near_points`` (uniform in a ball)."""
    rng = np.random.default_rng(seed)
    nn = int(round(near_frac * n)) if near_points is not None else 0
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    u = lo + (hi - lo) * rng.random((n - nn, 3))
    if nn:
        c = near_points[rng.integers(0, near_points.shape[0], nn)].astype(np.float64)
        d = rng.standard_normal((nn, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = near_radius * rng.random((nn, 1)) ** (1 / 3)
        u = np.concatenate([u, c + d * r])
        u = u[rng.permutation(n)]
    return _f32(u)


def tiny_mesh(kind: str, seed: int = 0):
    """Small fixtures for unit tests."""
    rng = np.random.default_rng(seed)
    if kind == "tet":
        V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
        F = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
        return _f32(V + 0.01 * rng.standard_normal(V.shape)), F.astype(np.int32)
    if kind == "polyline":
        t = np.linspace(0, 2 * np.pi, 25)
        V = np.stack([np.cos(t), np.sin(t), 0.3 * np.sin(3 * t)], 1)
        E = np.stack([np.arange(24), np.arange(1, 25)], 1)
        return _f32(V), E.astype(np.int32)
    raise ValueError(kind)


def mesh_edges(F):
    """Unique undirected edges of a triangle mesh, [ne, 2] int32 (lower
    index first, sorted)."""
    F = np.asarray(F, np.int64)
    E = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    E.sort(axis=1)
    return np.unique(E, axis=0).astype(np.int32)


def blob(level: int = 6, diag: float = 0.25, n_bumps: int = 12, seed: int = 6):
    """A closed, bumpy, rabbit-sized stand-in for a scanned object: an
    icosphere of the given level whose radius is modulated by a sum of
    Gaussian bumps on the sphere (random centres, widths 0.25-0.6 rad,
    heights -0.15..0.35), then scaled so that its bounding-box diagonal is
    ``diag`` (0.25 m, the size of a desktop scan). Returns (V float32, F
    int32)."""
    rng = np.random.default_rng(seed)
    V, F = icosphere(level)
    u = V.astype(np.float64)
    c = rng.normal(size=(n_bumps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    w = rng.uniform(0.25, 0.6, n_bumps)
    h = rng.uniform(-0.15, 0.35, n_bumps)
    ang = np.arccos(np.clip(u @ c.T, -1.0, 1.0))
    r = 1.0 + (h * np.exp(-(ang / w) ** 2)).sum(1)
    X = u * r[:, None] * np.array([1.0, 0.8, 0.9])
    X *= diag / np.linalg.norm(X.max(0) - X.min(0))
    return _f32(X), F


def trace_camera(V, width: int = 512, height: int = 512, dist: float = 2.2, fov_deg: float = 30.0):
    """A pinhole camera looking at the centre of V's bounding box from
    ``dist`` bounding-box diagonals away (slightly above and to the side).
    Returns dict(eye, target, up, fov_y, width, height, diag)."""
    V = np.asarray(V, np.float64)
    lo, hi = V.min(0), V.max(0)
    c = 0.5 * (lo + hi)
    diag = float(np.linalg.norm(hi - lo))
    d = np.array([0.6, -1.0, 0.45])
    d /= np.linalg.norm(d)
    return dict(eye=c + dist * diag * d, target=c, up=np.array([0.0, 0.0, 1.0]), fov_y=math.radians(fov_deg),
                width=int(width), height=int(height), diag=diag)
