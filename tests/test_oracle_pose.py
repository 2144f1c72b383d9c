"""Pins of the oracle's rigid-pose map and pose gradient (Sec. 4.5, Eq. opt;
Sec. 3.6, Eq. lse_full2 / Eq. dlse_full): textbook rotations, the left
Jacobian against finite differences of the exponential map, and the pose
gradient of the outer LogSumExp against central finite differences
(h = 1e-4, FP64 placement, exact evaluation beta = 0)."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import pose as PO


def test_rotation_textbook_and_orthonormal():
    t = 0.7
    Rz = PO.rotation([0.0, 0.0, t])
    assert np.allclose(Rz, [[math.cos(t), -math.sin(t), 0], [math.sin(t), math.cos(t), 0], [0, 0, 1]], atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(20):
        th = rng.standard_normal(3) * 2
        R = PO.rotation(th)
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-14
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.allclose(R @ th, th, atol=1e-14)          # the axis is fixed
    assert np.allclose(PO.rotation([0, 0, 0]), np.eye(3))


def test_left_jacobian_fd():
    rng = np.random.default_rng(1)
    eps = 1e-6
    for _ in range(10):
        th = rng.standard_normal(3)
        R = PO.rotation(th)
        J = PO.left_jacobian(th)
        for i in range(3):
            e = np.zeros(3); e[i] = eps
            A = (PO.rotation(th + e) @ R.T - PO.rotation(th - e) @ R.T) / (2 * eps)
            w = np.array([A[2, 1], A[0, 2], A[1, 0]])        # A = [J e_i]_x
            assert np.allclose(w, J[:, i], atol=1e-8)


@pytest.fixture(scope="module")
def small_street():
    s = synth.street_scene(n_points=3000, n_wire_segments=116, seed=7)
    # keep a 40 m stretch so that a small body sees both points and wires
    P = s["points"]
    keep = np.abs(P[:, 0] - 20.0) < 20.0
    V, F = synth.geodesic_icosphere(4)
    X0 = (V.astype(np.float64) * np.array([0.8, 0.5, 0.35])).astype(np.float32)
    return oracle.Scene(points=P[keep], edge_V=s["wire_V"], edge_E=s["wire_E"]), X0


def test_pose_gradient_matches_central_differences(small_street):
    sc, X0 = small_street
    alpha, alpha_q = 5.0, 10.0
    pose = np.array([0.4, -0.3, 1.1, 20.0, 5.5, 6.0])   # near the wires at y = 6, z = 8
    D, G, _, _, _ = PO.pose_objective(sc, X0, pose, alpha, alpha_q)
    h = 1e-4
    fd = np.zeros(6)
    for i in range(6):
        e = np.zeros(6); e[i] = h
        fd[i] = (PO.pose_objective(sc, X0, pose + e, alpha, alpha_q)[0]
                 - PO.pose_objective(sc, X0, pose - e, alpha, alpha_q)[0]) / (2 * h)
    assert np.abs(G - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_outer_lse_bounds():
    d = np.array([0.3, 0.5, 1.0, 0.31])
    for aq in (1.0, 10.0, 100.0):
        D, g = PO.outer_lse(d, aq)
        assert d.min() - math.log(len(d)) / aq <= D <= d.min()
        assert abs(g.sum() - 1) < 1e-15
