"""Rigid-body pose, outer LogSumExp over query vertices and the pose
gradient, in FP64 (Sec. 4.5 Eq. opt; Sec. 3.6 Eq. lse_full2, Eq. dlse_full
with point queries, n(g) = 0 so every vertex has weight 1).

TEST INFRASTRUCTURE (see oracle/__init__.py).

The pose is (theta, p): theta a rotation vector (exponential map), p a
translation; x_k = R(theta) x0_k + p.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _load, _ptr


def skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def rotation(theta):
    """Exponential map of a rotation vector: the Rodrigues formula
    R = I + sin(t)/t K + (1 - cos(t))/t^2 K^2, K = [theta]_x."""
    theta = np.asarray(theta, np.float64)
    t = float(np.linalg.norm(theta))
    K = skew(theta)
    if t < 1e-8:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + math.sin(t) / t * K + (1.0 - math.cos(t)) / (t * t) * K @ K


def left_jacobian(theta):
    """J_l with R(theta + e) = exp([J_l e]_x) R(theta) to first order:
    J_l = I + (1 - cos t)/t^2 K + (t - sin t)/t^3 K^2."""
    theta = np.asarray(theta, np.float64)
    t = float(np.linalg.norm(theta))
    K = skew(theta)
    if t < 1e-6:
        return np.eye(3) + 0.5 * K + K @ K / 6.0
    return np.eye(3) + (1.0 - math.cos(t)) / (t * t) * K + (t - math.sin(t)) / (t ** 3) * K @ K


def place(X0, pose, precision="f64"):
    """Vertices at a pose. f64: exact FP64 R x0 + p. f32: the fp32 rounding
    rule of the GPU path (R, p rounded to fp32; fma order fixed)."""
    pose = np.asarray(pose, np.float64)
    R = rotation(pose[:3])
    X0 = np.ascontiguousarray(X0, np.float32)
    if precision == "f64":
        return X0.astype(np.float64) @ R.T + pose[3:]
    out = np.zeros_like(X0)
    Rc = np.ascontiguousarray(R)
    pc = np.ascontiguousarray(pose[3:])
    _load().orc_pose_f32(_ptr(Rc), _ptr(pc), _ptr(X0), X0.shape[0], _ptr(out))
    return out


def outer_lse(d, alpha_q):
    """D = -(1/alpha_q) log sum_k exp(-alpha_q d_k) and the softmin weights."""
    t = -alpha_q * np.asarray(d, np.float64)
    m = t.max()
    e = np.exp(t - m)
    s = e.sum()
    return -(m + math.log(s)) / alpha_q, e / s


def pose_objective(scene, X0, pose, alpha, alpha_q, beta=0.0, precision="f64", threads=None):
    """D(pose) and its gradient (dD/dtheta, dD/dp) by the chain rule:
    dD/dx_k = gamma_k g_k, dD/dp = sum gamma_k g_k,
    dD/dtheta = J_l^T sum_k gamma_k (R x0_k) x g_k.
    beta = 0 uses brute force, beta > 0 the oracle's Barnes-Hut."""
    X = place(X0, pose, precision)
    if beta == 0.0:
        v, g, _ = scene.brute(X, alpha, threads=threads)
    else:
        v, g, _, _ = scene.bh(X, alpha, beta, threads=threads)
    D, gam = outer_lse(v, alpha_q)
    pose = np.asarray(pose, np.float64)
    R = rotation(pose[:3])
    Y = np.asarray(X0, np.float64) @ R.T
    dp = (gam[:, None] * g).sum(0)
    tq = (gam[:, None] * np.cross(Y, g)).sum(0)
    dth = left_jacobian(pose[:3]).T @ tq
    return D, np.concatenate([dth, dp]), v, g, gam
