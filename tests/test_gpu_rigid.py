"""Rigid-body time steps (Sec. 4.5) driven by the GPU constraint against the
oracle's interior-point step driven by the FP64 constraint: a small body
dropped onto a small street comes to the same pose, in free flight and in
contact, without any vertex crossing the ground."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import pose as PO
from oracle import rigid as RI

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    """a 4 m x 4 m patch of lidar-like ground (5 cm grid, 1 cm jitter) and an
    ellipsoidal body"""
    rng = np.random.default_rng(3)
    g = np.stack(np.meshgrid(np.arange(-2, 2, 0.05), np.arange(-2, 2, 0.05)), -1).reshape(-1, 2)
    P = np.concatenate([g + rng.normal(0, 0.01, g.shape), rng.normal(0, 0.005, (len(g), 1))], 1).astype(np.float32)
    V, F = synth.geodesic_icosphere(3)
    X0 = (V.astype(np.float64) * np.array([0.4, 0.3, 0.2])).astype(np.float32)
    return P, X0


@pytest.mark.parametrize("clearance", [1.0, 0.01])
def test_step_matches_oracle(scene, clearance):
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.rigid import RigidBody
    P, X0 = scene
    alpha, alpha_q, beta, h = 100.0, 100.0, 0.5, 0.01
    theta = np.array([0.1, -0.05, 0.3])
    v = np.array([0.3, 0.0, -2.0])
    mass, I = 1.0, np.diag([0.02, 0.03, 0.04])
    sc = oracle.Scene(points=P)
    sc.build_tree(1)

    def cons(x):
        D, G, _, _, _ = PO.pose_objective(sc, X0, x, alpha, alpha_q, beta=beta, precision="f32")
        return D, G
    # start at the height where D = clearance (bisection)
    lo, hi = 0.15, 2.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if cons(np.concatenate([theta, [0.1, 0.2, mid]]))[0] > clearance else (mid, hi)
    p = np.array([0.1, 0.2, hi])
    sd = SmoothDistance(points=P, alpha=alpha, beta=beta, device="cuda:0")
    body = RigidBody(sd, X0, mass, I, theta, p, v=v)
    info = body.step(h, (0.0, 0.0, -9.81), alpha_q, max_iter=400)
    R = PO.rotation(theta)
    th, pp, om, vv, lam, it, ev = RI.rigid_step(cons, theta, p, np.zeros(3), v, h, mass, R @ I @ R.T,
                                                np.array([0.0, 0.0, -9.81]), r_max=0.4, max_iter=400)
    assert np.abs(body.theta - th).max() <= 2e-5 and np.abs(body.p - pp).max() <= 2e-5, (body.theta - th, body.p - pp)
    assert abs(info["lambda"] - lam) <= 1e-3 * max(lam, 1e-3)
    D, _ = cons(np.concatenate([body.theta, body.p]))
    assert D > 0
    if clearance > 0.5:
        assert lam < 1e-6                     # free flight: the unconstrained step
    else:
        assert lam > 1e-4                     # in contact
