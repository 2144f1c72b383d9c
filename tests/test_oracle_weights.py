"""Pins of the oracle's weight polynomials (App. C) against what the paper
fixes: the constraint values, the zero normal derivatives, symmetry, the
13-coefficient structure, the scale A, an independent QR-based
minimum-norm solve, and the exact minimum-norm solution of the triangle
system rebuilt in rational arithmetic."""
import numpy as np
import pytest
import scipy.linalg

from oracle import weights as W


# ---------------------------------------------------------------- edge (App. C.2)
@pytest.mark.parametrize("u,v", [(0.5, 0.5), (1.0, 0.5), (1 / 3, 1 / 7), (0.25, 1.0), (1.0, 1.0)])
def test_edge_constraints(u, v):
    c = W.edge_basis() @ np.array([u, v, 1.0])
    w = np.polynomial.Polynomial(c)
    dw = w.deriv()
    assert abs(w(0.0) - u) < 1e-14
    assert abs(w(1.0) - v) < 1e-14
    assert abs(w(0.5) - 1.0) < 1e-14
    assert abs(dw(0.0)) < 1e-13 and abs(dw(1.0)) < 1e-13


@pytest.mark.parametrize("u", [0.5, 1 / 3, 0.2, 1.0])
def test_edge_symmetric_closed_form(u):
    # with equal end weights the five constraints are met by
    # u + (1 - u) 16 phi^2 (1 - phi)^2 (a quartic, so it is the solution)
    phi = np.linspace(0, 1, 101)
    ref = u + (1 - u) * 16 * phi ** 2 * (1 - phi) ** 2
    got = np.array([W.edge_weight(x, u, u) for x in phi])
    assert np.abs(got - ref).max() < 1e-13


def test_edge_minimum_at_endpoints_so_A_makes_it_conservative():
    # the paper sets the three extrema by construction, so A = max valence
    # gives A w~ >= 1 on the whole edge
    for nu in range(1, 9):
        for nv in range(1, 9):
            phi = np.linspace(0, 1, 2001)
            c = W.edge_basis() @ np.array([1 / nu, 1 / nv, 1.0])
            w = np.polyval(c[::-1], phi)
            A = max(nu, nv)
            assert (A * w).min() >= 1.0 - 1e-12


def test_isolated_edge_weight_is_one():
    c = W.edge_basis() @ np.array([1.0, 1.0, 1.0])
    assert np.allclose(c, [1, 0, 0, 0, 0], atol=1e-14)


# ----------------------------------------------------------- triangle (App. C.3)
def _poly(inv_v, inv_e):
    return W.tri_basis() @ np.array([inv_v, inv_e, 1 - inv_v])


def _eval(c, x, y):
    return sum(c[j] * x ** a * y ** b for j, (a, b) in enumerate(W.TRI_EXPONENTS))


def _grad(c, x, y):
    gx = sum(c[j] * a * x ** (a - 1) * y ** b for j, (a, b) in enumerate(W.TRI_EXPONENTS) if a > 0)
    gy = sum(c[j] * b * x ** a * y ** (b - 1) for j, (a, b) in enumerate(W.TRI_EXPONENTS) if b > 0)
    return gx, gy


def test_tri_system_size_rank_consistency():
    A, B = W.tri_system()
    assert A.shape == (36, 36)       # 10 point + 26 derivative equations
    assert np.linalg.matrix_rank(A) == 30
    X = W.tri_basis()
    assert np.abs(A @ X - B).max() < 1e-9   # consistent: residual ~ roundoff


@pytest.mark.parametrize("v,e", [(6, 2), (5, 2), (3, 2), (4, 1), (8, 3), (2, 2)])
def test_tri_point_constraints(v, e):
    c = _poly(1 / v, 1 / e)
    for p in [(0, 0), (1, 0), (0, 1)]:
        assert abs(_eval(c, *p) - 1 / v) < 1e-9
    t = 1 / 3
    for p in [(t, 0), (2 * t, 0), (t, 2 * t), (2 * t, t), (0, t), (0, 2 * t)]:
        assert abs(_eval(c, *p) - 1 / e) < 1e-9
    assert abs(_eval(c, t, t) - (v - 1) / v) < 1e-9


@pytest.mark.parametrize("v,e", [(6, 2), (5, 2), (7, 3)])
def test_tri_zero_normal_derivative_on_boundary(v, e):
    c = _poly(1 / v, 1 / e)
    for t in np.linspace(0, 1, 23):
        gx, gy = _grad(c, 0.0, t)          # leg phi1 = 0: d/dphi1 = 0
        assert abs(gx) < 1e-8
        gx, gy = _grad(c, t, 0.0)          # leg phi2 = 0: d/dphi2 = 0
        assert abs(gy) < 1e-8
        gx, gy = _grad(c, t, 1 - t)        # hypotenuse: (d1 + d2) = 0
        assert abs(gx + gy) < 1e-8


def test_tri_symmetry_and_13_stored_coefficients():
    X = W.tri_basis()
    idx = {m: i for i, m in enumerate(W.TRI_EXPONENTS)}
    for (a, b) in W.TRI_EXPONENTS:
        assert np.abs(X[idx[(a, b)]] - X[idx[(b, a)]]).max() < 1e-7
    zero = [m for m in W.TRI_EXPONENTS if m[0] == 1 or m[1] == 1]
    assert len(zero) == 13
    for m in zero:
        assert np.abs(X[idx[m]]).max() < 1e-9
    unique = {tuple(sorted(m)) for m in W.TRI_EXPONENTS if m not in zero}
    assert len(unique) == 13


def test_tri_min_norm_matches_independent_qr_solve():
    # complete orthogonal factorisation (LAPACK gelsy) gives the same
    # minimum-norm solution as the SVD pseudoinverse
    A, B = W.tri_system()
    Xq = scipy.linalg.lstsq(A, B, lapack_driver="gelsy", cond=1e-10)[0]
    assert np.abs(Xq - W.tri_basis()).max() < 1e-7


def test_tri_weight_scale_A():
    # icosphere-type valences: A = max v_i makes A w~ >= 1 up to the small
    # dip the minimum-norm solution leaves near the vertices (recorded, 0.999)
    phi = np.random.default_rng(0).dirichlet([1, 1, 1], 20000)[:, 1:]
    for v in (5, 6):
        c = _poly(1 / v, 1 / 2)
        w = _eval(c, phi[:, 0], phi[:, 1])
        assert (6 * w).min() > 0.995
        assert w.max() < 1.3


def test_isolated_triangle_polynomial_goes_negative():
    # (v, e) = (1, 1): the solved w~ dips below 0; the oracle's guard uses
    # w~ = 1 for such triangles
    phi = np.random.default_rng(1).dirichlet([1, 1, 1], 20000)[:, 1:]
    c = _poly(1.0, 1.0)
    assert _eval(c, phi[:, 0], phi[:, 1]).min() < 0


def test_tri_min_norm_exact_rational():
    """The triangle weight everywhere (not only at its constraint points):
    App. C.3's constraints rebuilt from the text in exact rational arithmetic
    (sympy, independent of the oracle's matrix), their minimum-norm solution
    x = A^T y with A A^T y = b solved exactly, and the oracle's coefficients
    compared with it."""
    sp = pytest.importorskip("sympy")
    p1, p2, t = sp.symbols("p1 p2 t")
    keys = [(a, b) for a in range(8) for b in range(8) if a + b <= 7]
    cs = sp.symbols("c0:%d" % len(keys))
    w = sum(c * p1 ** a * p2 ** b for c, (a, b) in zip(cs, keys))
    third = sp.Rational(1, 3)
    eqs = []     # (linear form in cs, right-hand side column: 0 vertex, 1 edge, 2 centre, None zero)
    for pt in [(0, 0), (1, 0), (0, 1)]:
        eqs.append((w.subs({p1: pt[0], p2: pt[1]}), 0))
    for pt in [(third, 0), (2 * third, 0), (0, third), (0, 2 * third), (third, 2 * third), (2 * third, third)]:
        eqs.append((w.subs({p1: pt[0], p2: pt[1]}), 1))
    eqs.append((w.subs({p1: third, p2: third}), 2))
    # zero derivative across each side: d/dphi1 on phi1 = 0, d/dphi2 on
    # phi2 = 0, (d/dphi1 + d/dphi2) on phi1 + phi2 = 1 (both directions)
    lines = [(sp.diff(w, p1), {p1: 0, p2: t}), (sp.diff(w, p2), {p1: t, p2: 0}),
             (sp.diff(w, p1) + sp.diff(w, p2), {p1: t, p2: 1 - t}),
             (sp.diff(w, p1) + sp.diff(w, p2), {p1: 1 - t, p2: t})]
    for expr, sub in lines:
        poly = sp.Poly(sp.expand(expr.subs(sub)), t)
        for coeff in poly.all_coeffs():
            eqs.append((coeff, None))
    A = sp.Matrix([[sp.diff(e, c) for c in cs] for e, _ in eqs])
    M = A * A.T
    X = W.tri_basis()
    idx = {m: i for i, m in enumerate(W.TRI_EXPONENTS)}
    scale = np.abs(X).max()
    for col in range(3):
        b = sp.Matrix([1 if r == col else 0 for _, r in eqs])
        sol, params = M.gauss_jordan_solve(b)
        y = sol.subs({p: 0 for p in params})
        x = A.T * y                                  # unique: the minimum-norm solution
        assert (A * x - b).is_zero_matrix            # the constraints hold exactly
        ref = np.array([float(x[i]) for i in range(len(keys))])
        got = np.array([X[idx[k], col] for k in keys])
        assert np.abs(got - ref).max() <= 1e-10 * scale, (col, np.abs(got - ref).max())
