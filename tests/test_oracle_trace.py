"""Pins of the oracle's sphere tracer (Sec. 4.2): closed-form hits on one
point and on a plane, the march's bound on an oblique plane, misses, and
Barnes-Hut at beta = 0 equal to the exact tracer."""
import math

import numpy as np

import oracle
import synth
from oracle import trace as OT


def _cam(eye, target, w=1, h=1, fov=0.4, up=(0.0, 0.0, 1.0)):
    return dict(eye=np.asarray(eye, float), target=np.asarray(target, float), up=np.asarray(up, float),
                fov_y=fov, width=w, height=h)


def test_camera_rays_are_unit_and_centred():
    eye, d = OT.camera_rays([0, -2, 0], [0, 0, 0], [0, 0, 1], math.radians(40), 64, 48)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    # the four centre pixels straddle the forward axis symmetrically
    c = d.reshape(48, 64, 3)[23:25, 31:33].reshape(-1, 3).mean(0)
    assert np.allclose(c / np.linalg.norm(c), [0, 1, 0], atol=1e-12)
    # the vertical field of view
    top = d.reshape(48, 64, 3)[0, 31:33].mean(0)
    ang = math.atan2(top[2], top[1])
    assert abs(ang - math.radians(20) * (1 - 1 / 48)) < 2e-3


def test_point_hit_and_miss():
    p = np.array([[0.1, 0.2, 0.3]], np.float32)
    sc = oracle.Scene(points=p)
    eye = np.array([0.1, -1.7, 0.3])
    depth, steps = OT.sphere_trace(sc, _cam(eye, p[0].astype(float)), alpha=50.0, beta=0.0, t_max=5.0)
    # one step of |eye - p| lands on the point
    assert abs(depth[0] - np.linalg.norm(eye - p[0])) < 1e-12 and steps[0] == 2
    # a ray passing 0.01 from the point never gets within eps
    depth, _ = OT.sphere_trace(sc, _cam(eye, p[0] + [0.0, 0.0, 0.01]), alpha=50.0, beta=0.0, t_max=5.0)
    assert np.isinf(depth[0])


def _plane(z=0.0, size=10.0):
    V = np.array([[-size, -size, z], [size, -size, z], [size, size, z], [-size, size, z]], np.float32)
    F = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return V, F


def test_plane_perpendicular_and_oblique():
    V, F = _plane()
    sc = oracle.Scene(tri_V=V, tri_F=F[:1])       # one large triangle: d^ is its distance
    # straight down from height 0.7 over the interior, unit weights: one step
    # of 0.7 lands on the plane, where d^ <= 0 < eps
    depth, steps = OT.sphere_trace(sc, _cam([0.3, -0.2, 0.7], [0.3, -0.2, 0.0], up=(0.0, 1.0, 0.0)), alpha=200.0,
                                   beta=0.0, t_max=5.0, unit=True)
    assert abs(depth[0] - 0.7) < 1e-7 and steps[0] == 2
    # oblique ray at points on a grid of the plane (spacing 0.025, alpha 50:
    # the zero set is a closed sheet above the grid): the
    # march stops within eps / cos(theta) before the zero set along the ray
    g = np.stack(np.meshgrid(np.linspace(-1, 1, 81), np.linspace(-1, 1, 81)), -1).reshape(-1, 2)
    P = np.concatenate([g, np.zeros((len(g), 1))], 1).astype(np.float32)
    sp = oracle.Scene(points=P)
    eye = np.array([0.0, -0.6, 0.5])
    tgt = np.array([0.02, 0.1, 0.0])
    depth, steps = OT.sphere_trace(sp, _cam(eye, tgt), alpha=50.0, beta=0.0, eps=1e-5, t_max=5.0)
    dirn = (tgt - eye) / np.linalg.norm(tgt - eye)
    # the zero set of the smooth distance along the ray, by bisection
    f = lambda s: sp.brute((eye + s * dirn)[None], 50.0)[0][0]
    lo, hi = 0.0, np.linalg.norm(tgt - eye) * 1.2
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) > 0 else (lo, mid)
    cos = abs(dirn[2])
    assert lo - 1e-5 / cos * 1.5 <= depth[0] <= lo + 1e-12 and steps[0] > 3


def test_bh_beta0_equals_exact_tracer():
    V, F = synth.blob(level=2)
    sc = oracle.Scene(tri_V=V, tri_F=F)
    cam = synth.trace_camera(V, 16, 12)
    d0, s0 = OT.sphere_trace(sc, cam, 200.0, 0.0, alpha_u=1200.0, t_max=2.0)
    sc2 = oracle.Scene(tri_V=V, tri_F=F)
    sc2.build_tree(1)
    eye, dirs = OT.camera_rays(cam["eye"], cam["target"], cam["up"], cam["fov_y"], 16, 12)
    # BH at beta = 0 through the same loop
    d1, s1 = OT.sphere_trace(sc2, cam, 200.0, 1e-30, alpha_u=1200.0, t_max=2.0)
    hit = np.isfinite(d0)
    assert np.array_equal(hit, np.isfinite(d1)) and hit.sum() > 20
    assert np.allclose(d1[hit], d0[hit], rtol=0, atol=1e-10)
    # and beta = 0.5 stays close to the exact isosurface (relative to the diagonal)
    d2, _ = OT.sphere_trace(sc2, cam, 200.0, 0.5, alpha_u=1200.0, t_max=2.0)
    both = hit & np.isfinite(d2)
    assert np.abs(d2[both] - d0[both]).max() < 0.05 * cam["diag"]
