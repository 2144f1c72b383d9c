"""Sphere tracing of the smooth distance's zero isosurface (Sec. 4.2, Hart
1996), in FP64 on the CPU.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Camera: pinhole at `eye` looking at `target`; forward f = (target - eye)/|.|,
right r = (f x up)/|.|, up u = r x f; pixel (row i from the top, column j)
has the direction normalize(f + x r + y u) with
    x = ((j + 0.5) / W * 2 - 1) tan(fov_y / 2) W / H,
    y = (1 - (i + 0.5) / H * 2) tan(fov_y / 2).
March from t = 0: at step k evaluate d = d^(eye + t dir); if d < eps the ray
hits at depth t (k steps); otherwise t += d, and the ray misses once
t > t_max or after max_steps evaluations (depth +inf).
The smooth distance at the march points is the oracle's Barnes-Hut (beta > 0,
FP32 node decisions) or exact evaluation (beta = 0), for all active rays at
once.
"""
from __future__ import annotations

import math

import numpy as np


def camera_rays(eye, target, up, fov_y, width, height):
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(fov_y / 2)
    j = (np.arange(width) + 0.5) / width * 2 - 1
    i = 1 - (np.arange(height) + 0.5) / height * 2
    x = (j * th * width / height)[None, :]
    y = (i * th)[:, None]
    d = f[None, None, :] + x[..., None] * r[None, None, :] + y[..., None] * u[None, None, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return eye, d.reshape(-1, 3)


def sphere_trace(scene, cam, alpha, beta, alpha_u=0.0, eps=1e-5, t_max=1.0, max_steps=256, leaf_size=1,
                 unit=False):
    """Returns depth [H*W] (inf for misses) and the evaluations per ray."""
    eye, dirs = camera_rays(cam["eye"], cam["target"], cam["up"], cam["fov_y"], cam["width"], cam["height"])
    n = dirs.shape[0]
    t = np.zeros(n)
    depth = np.full(n, np.inf)
    steps = np.zeros(n, np.int64)
    active = np.arange(n)
    if beta > 0:
        scene.build_tree(leaf_size)
    for k in range(max_steps):
        if active.size == 0:
            break
        x = eye[None, :] + t[active, None] * dirs[active]
        if beta > 0:
            d = scene.bh(x, alpha, beta, alpha_u=alpha_u, unit=unit)[0]
        else:
            d = scene.brute(x, alpha, alpha_u=alpha_u, unit=unit)[0]
        steps[active] = k + 1
        hit = d < eps
        depth[active[hit]] = t[active[hit]]
        go = active[~hit]
        t[go] += d[~hit]
        active = go[t[go] <= t_max]
    return depth, steps
