"""Rigid-body time steps against a static data mesh (Sec. 4.5, Eq. opt):
minimise the incremental potential of an implicit Euler step subject to the
smooth distance constraint D(theta, p) >= 0, where D is the query mesh's
outer LogSumExp of the per-vertex smooth distances (sd_pose_query +
sd_pose_reduce, on the GPU).

The solver is a primal-dual interior-point method with the Hessian block
replaced by the identity (taken in mass-normalised coordinates, where it is
the potential's exact Hessian). The slack is reset to the exactly evaluated
constraint at every iterate, the multiplier kept positive by the
fraction-to-boundary rule, and the primal step halved until D > 0 and the
barrier function f - mu log D decreases by the Armijo fraction (the
primal-dual step with W = I is a descent direction of it). The 6-dof linear
algebra runs on the host; every constraint evaluation is one placement +
Barnes-Hut query + reduction on the device.

    body = RigidBody(sd, X0, mass, I_body, theta, p)
    for _ in range(steps):
        info = body.step(h=1e-3, gravity=(0, 0, -9.81), alpha_q=100.0)
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import pose as _pose


def _rotation(theta):
    th = np.asarray(theta, np.float64)
    t = float(np.linalg.norm(th))
    K = np.array([[0.0, -th[2], th[1]], [th[2], 0.0, -th[0]], [-th[1], th[0], 0.0]])
    if t < 1e-8:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + math.sin(t) / t * K + (1.0 - math.cos(t)) / (t * t) * K @ K


def primal_dual_direction(g, a, lam, s, c, mu):
    """Step of the perturbed KKT system with W = I for min f s.t. c - s = 0,
    s >= 0 (g = grad f, a = grad c): dy from (I + (lam/s) a a^T) dy = b by
    Sherman-Morrison, then ds and dlam."""
    k = lam / s
    b = a * ((mu - lam * c) / s) - (g - lam * a)
    dy = b - a * (k * float(a @ b) / (1.0 + k * float(a @ a)))
    ds = float(a @ dy) + (c - s)
    dl = (mu - lam * s - lam * ds) / s
    return dy, ds, dl


class RigidBody:
    """A rigid body (rest vertices X0 on the device, about its centre of
    mass) moving against the data mesh of `sd`."""

    def __init__(self, sd, X0, mass, I_body, theta, p, omega=(0.0, 0.0, 0.0), v=(0.0, 0.0, 0.0)):
        self.sd = sd
        self.X0 = X0 if torch.is_tensor(X0) else torch.from_numpy(np.asarray(X0, np.float32)).to(sd.device)
        self.mass = float(mass)
        self.I_body = np.asarray(I_body, np.float64)
        self.theta = np.asarray(theta, np.float64).copy()
        self.p = np.asarray(p, np.float64).copy()
        self.omega = np.asarray(omega, np.float64).copy()
        self.v = np.asarray(v, np.float64).copy()
        self.r_max = float(self.X0.norm(dim=1).max().item())

    def constraint(self, x, alpha_q):
        """D and dD/d(theta, p) at pose x = (theta, p)."""
        X, val, grad = _pose.pose_query(self.sd, self.X0, x)
        out, _ = _pose.pose_reduce(self.X0, val, grad, x, alpha_q=alpha_q)
        o = out.cpu().numpy().astype(np.float64)
        return float(o[0]), o[1:]          # (D, dD/dtheta (3), dD/dp (3))

    def step(self, h, gravity, alpha_q, mu0=1e-4, mu_min=1e-9, tol=1e-7, max_iter=200, conservative=False):
        """One time step; returns a dict of solver statistics."""
        R = _rotation(self.theta)
        I_w = R @ self.I_body @ R.T
        x_t = np.concatenate([self.theta, self.p])
        x_pred = np.concatenate([self.theta + h * self.omega, self.p + h * self.v + h * h * np.asarray(gravity)])
        sq = np.sqrt(np.concatenate([np.diag(I_w), np.full(3, self.mass)]))
        y, y_pred = sq * x_t, sq * x_pred
        c, dc = self.constraint(x_t, alpha_q)
        evals = 1
        if not c > 0:
            raise ValueError("the body must start clear of the data mesh (D > 0)")
        mu = mu0
        lam = mu0 / c
        it = 0
        for it in range(1, max_iter + 1):
            a = dc / sq
            g = y - y_pred
            kkt = max(float(np.linalg.norm(g - lam * a)), abs(lam * c - mu))
            if kkt < max(mu, tol):
                if mu <= mu_min and kkt < tol:
                    break
                mu = max(mu * 0.1, mu_min)
            dy, ds, dl = primal_dual_direction(g, a, lam, c, c, mu)
            al = 1.0 if ds >= 0 else min(1.0, -0.995 * c / ds)
            al_l = 1.0 if dl >= 0 else min(1.0, -0.995 * lam / dl)
            if conservative:
                dx = dy / sq
                reach = float(np.linalg.norm(dx[3:])) + self.r_max * float(np.linalg.norm(dx[:3]))
                if reach > 0:
                    al = min(al, 0.9 * c / reach)
            B0 = 0.5 * float(g @ g) - mu * math.log(c)
            dB = float(g @ dy) - mu / c * float(a @ dy)
            ok = False
            while al >= 1e-12:
                yn = y + al * dy
                cn, dcn = self.constraint(yn / sq, alpha_q)
                evals += 1
                if cn > 0:
                    gn = yn - y_pred
                    if 0.5 * float(gn @ gn) - mu * math.log(cn) <= B0 + 1e-4 * al * min(dB, 0.0):
                        ok = True
                        break
                al *= 0.5
            if not ok:
                break
            y, c, dc = yn, cn, dcn
            lam = max(lam + al_l * dl, 1e-16)
        x = y / sq
        th, p = x[:3], x[3:]
        self.omega = (th - self.theta) / h
        self.v = (p - self.p) / h
        self.theta, self.p = th, p
        return {"iterations": it, "evaluations": evals, "lambda": lam, "D": c}
