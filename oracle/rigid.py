"""One rigid-body time step as a constrained minimisation (Sec. 4.5,
Eq. opt), solved by a primal-dual interior-point method with the Hessian
block replaced by the identity, in FP64.

TEST INFRASTRUCTURE (see oracle/__init__.py).

Readings of the paper's description:
  * x = (theta, p) (rotation vector, position). The incremental potential is
    E(x) = 1/2 (x - x~)^T M (x - x~) with M = diag(I_w, m I), the predicted
    x~ = (theta_t + h omega_t, p_t + h v_t + h^2 g): an implicit Euler step in
    position and, to first order in the rotation vector, an exponential Euler
    step in orientation; I_w = R I_body R^T at the step's start.
  * The identity Hessian is taken in mass-normalised coordinates y = M^(1/2) x,
    where it is E's exact Hessian; only the constraint's curvature is left out.
  * One constraint c(x) = D(x) >= 0 (the query mesh's smooth distance, Eq.
    lse_full2), a slack s with multiplier lambda; the slack is reset to c at
    every iterate (the constraint is evaluated exactly, so s = c is feasible
    and the linearisation error of a curved c never enters the merit);
    barrier mu, shrunk by 10 once the KKT residual at mu falls below mu; the
    multiplier step cut to 0.995 of the way to its boundary; the primal step
    (also cut so the linearised c stays above 0.005 c) halved until c(x) > 0
    and the barrier function f - mu log c decreases by the Armijo fraction
    1e-4 of its directional derivative. With s = c and W = I the primal-dual
    step is dy = -(I + (lambda / c) a a^T)^-1 grad(f - mu log c), a descent
    direction of that barrier function.
  * Every iterate has c(x) > 0. The distance is unsigned and there is no
    continuous collision detection (as in the paper), so a step that jumps
    through the data mesh by more than the smooth offset (about log n / alpha
    for n nearby vertices) is not caught; time steps are kept small.
    conservative=True adds a guarantee: D is below every vertex's distance
    (Theorem A.1) and a pose step (dtheta, dp) moves no vertex farther than
    |dp| + r_max |dtheta| (r_max the largest vertex radius about the body's
    origin), so steps of at most 0.9 D in that measure cannot cross (at the
    price of short steps while sliding in contact).
  * Velocities after the step: v = (p - p_t) / h, omega = (theta - theta_t) / h.
"""
from __future__ import annotations

import numpy as np


def newton_direction(g, a, lam, s, c, mu):
    """The primal-dual step for min f s.t. c(y) - s = 0, s >= 0 with W = I:
    (I + (lam / s) a a^T) dy = -(g - lam a) + a (mu - lam c) / s, then
    ds = a . dy + (c - s), dlam = (mu - lam s - lam ds) / s."""
    r = g - lam * a
    b = -r + a * (mu - lam * c) / s
    k = lam / s
    dy = b - k * a * (a @ b) / (1.0 + k * (a @ a))
    ds = a @ dy + (c - s)
    dl = (mu - lam * s - lam * ds) / s
    return dy, ds, dl


def ipm_step(constraint, x_t, x_pred, Mdiag, r_max, mu0=1e-4, mu_min=1e-9, tol=1e-7, max_iter=200,
             conservative=False):
    """Minimise 1/2 (x - x_pred)^T diag(Mdiag) (x - x_pred) subject to
    constraint(x)[0] >= 0 from the feasible x_t; x = (theta, p), r_max bounds
    the body's vertex radii. constraint(x) returns (c, dc/dx). Returns (x,
    lam, iterations, constraint evaluations)."""
    sq = np.sqrt(np.asarray(Mdiag, np.float64))
    y = sq * np.asarray(x_t, np.float64)
    y_pred = sq * np.asarray(x_pred, np.float64)
    c, dc = constraint(y / sq)
    evals = 1
    if not c > 0:
        raise ValueError("the step must start from a feasible pose")
    lam, mu = mu0 / c, mu0
    it = 0
    for it in range(1, max_iter + 1):
        a = dc / sq
        g = y - y_pred
        kkt = max(np.linalg.norm(g - lam * a), abs(lam * c - mu))
        if kkt < max(mu, tol):
            if mu <= mu_min and kkt < tol:
                break
            mu = max(mu / 10.0, mu_min)
        dy, ds, dl = newton_direction(g, a, lam, c, c, mu)
        al = 1.0 if ds >= 0 else min(1.0, -0.995 * c / ds)
        al_l = 1.0 if dl >= 0 else min(1.0, -0.995 * lam / dl)
        if conservative:
            # no vertex may move farther than 0.9 c in the step
            dx = dy / sq
            reach = np.linalg.norm(dx[3:]) + r_max * np.linalg.norm(dx[:3])
            if reach > 0:
                al = min(al, 0.9 * c / reach)
        # Armijo on the barrier function over feasible iterates
        B0 = 0.5 * (g @ g) - mu * np.log(c)
        dB = g @ dy - mu / c * (a @ dy)
        accepted = False
        while al >= 1e-12:
            y_new = y + al * dy
            c_new, dc_new = constraint(y_new / sq)
            evals += 1
            if c_new > 0:
                gn = y_new - y_pred
                if 0.5 * (gn @ gn) - mu * np.log(c_new) <= B0 + 1e-4 * al * min(dB, 0.0):
                    accepted = True
                    break
            al *= 0.5
        if not accepted:
            break
        y, c, dc = y_new, c_new, dc_new
        lam = max(lam + al_l * dl, 1e-16)
    return y / sq, lam, it, evals


def rigid_step(constraint, theta, p, omega, v, h, mass, I_world, gravity, r_max, **kw):
    """One time step; returns (theta, p, omega, v, lam, iterations, evals)."""
    x_t = np.concatenate([theta, p])
    x_pred = np.concatenate([np.asarray(theta) + h * np.asarray(omega),
                             np.asarray(p) + h * np.asarray(v) + h * h * np.asarray(gravity)])
    Mdiag = np.concatenate([np.diag(I_world), np.full(3, mass)])
    x, lam, it, ev = ipm_step(constraint, x_t, x_pred, Mdiag, r_max, **kw)
    th, pp = x[:3], x[3:]
    return th, pp, (th - theta) / h, (pp - p) / h, lam, it, ev
