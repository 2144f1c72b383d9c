"""Pins of the oracle's interior-point rigid-body step (Sec. 4.5): the
constrained minimiser of a quadratic above a plane is the projection of the
unconstrained one (closed form), an inactive constraint gives the free step,
the KKT conditions hold at an active contact, and the Newton direction solves
its linear system."""
import numpy as np

import oracle
from oracle import pose as PO
from oracle import rigid as RI


def test_newton_direction_solves_the_system():
    rng = np.random.default_rng(0)
    for _ in range(20):
        g, a = rng.normal(size=6), rng.normal(size=6)
        lam, s, c, mu = rng.uniform(0.1, 2, 4)
        dy, ds, dl = RI.newton_direction(g, a, lam, s, c, mu)
        # rows of the full system
        assert np.allclose(dy - a * dl, -(g - lam * a))
        assert np.isclose(a @ dy - ds, -(c - s))
        assert np.isclose(lam * ds + s * dl, -(lam * s - mu))


def _plane_constraint():
    """c(x) = height of the single vertex at the origin of the body above
    the plane z = 0 (one large triangle, unit weight: d^ is the exact
    distance; one vertex: D = d^)."""
    V = np.array([[-50, -50, 0], [50, -50, 0], [0, 50, 0]], np.float32)
    sc = oracle.Scene(tri_V=V, tri_F=np.array([[0, 1, 2]], np.int32))
    X0 = np.zeros((1, 3), np.float32)

    def c(x):
        D, G, _, _, _ = PO.pose_objective(sc, X0, x, 100.0, 100.0)
        return D, G
    return c


def test_projection_onto_the_plane():
    """min 1/2 m |p - p~|^2 s.t. p_z >= 0 with p~ below the plane: p = (p~_x,
    p~_y, 0) up to the barrier's offset."""
    c = _plane_constraint()
    x_t = np.array([0.0, 0.0, 0.0, 0.3, -0.2, 0.05])
    x_pred = np.array([0.0, 0.0, 0.0, 0.5, 0.1, -0.4])
    x, lam, it, ev = RI.ipm_step(c, x_t, x_pred, np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0]), 0.0)
    assert np.allclose(x[3:5], x_pred[3:5], atol=1e-6)
    assert 0 < x[5] < 1e-4
    # KKT: m (p - p~) = lam grad c, grad c = (0, 0, 1) for the height
    assert np.isclose(2.0 * (x[5] - x_pred[5]), lam, rtol=1e-3)


def test_inactive_constraint_gives_the_free_step():
    c = _plane_constraint()
    x_t = np.array([0.1, -0.2, 0.3, 0.0, 0.0, 2.0])
    x_pred = np.array([0.12, -0.18, 0.31, 0.05, 0.0, 1.9])
    x, lam, it, ev = RI.ipm_step(c, x_t, x_pred, np.array([0.5, 0.7, 0.9, 3.0, 3.0, 3.0]), 0.0, max_iter=400)
    assert np.allclose(x, x_pred, atol=1e-6) and lam < 1e-6


def test_rigid_step_of_a_box_onto_a_plane():
    """A tilted box 4 mm above the plane moving down at 1 m/s: after a 5 ms
    step no vertex is below it, the constraint is active (lam > 0) and the
    Lagrangian is stationary; with the conservative step bound as well."""
    V = np.array([[-50, -50, 0], [50, -50, 0], [0, 50, 0]], np.float32)
    sc = oracle.Scene(tri_V=V, tri_F=np.array([[0, 1, 2]], np.int32))
    X0 = np.array([[x, y, z] for x in (-0.1, 0.1) for y in (-0.1, 0.1) for z in (-0.1, 0.1)], np.float32)

    def cons(x):
        D, G, _, _, _ = PO.pose_objective(sc, X0, x, 1000.0, 1000.0)
        return D, G
    theta = np.array([0.05, 0.02, 0.0])
    R = PO.rotation(theta)
    p = np.array([0.0, 0.0, 0.004 - (X0.astype(np.float64) @ R.T)[:, 2].min()])
    h = 0.005
    Md = np.array([0.01, 0.01, 0.01, 1.0, 1.0, 1.0])
    x_pred = np.concatenate([theta, p + h * np.array([0, 0, -1.0]) + h * h * np.array([0, 0, -9.81])])
    for conservative in (False, True):
        out = RI.rigid_step(cons, theta, p, np.zeros(3), np.array([0.0, 0.0, -1.0]), h, 1.0, np.eye(3) * 0.01,
                            np.array([0.0, 0.0, -9.81]), r_max=np.sqrt(3) * 0.1, max_iter=2000,
                            conservative=conservative)
        th, pp, om, vv, lam, it, ev = out
        Xn = PO.place(X0, np.concatenate([th, pp]))
        assert lam > 0 and Xn[:, 2].min() > 0
        D, G = cons(np.concatenate([th, pp]))
        grad_E = Md * (np.concatenate([th, pp]) - x_pred)
        assert np.linalg.norm(grad_E - lam * G) <= 1e-4 * np.linalg.norm(grad_E), conservative
