"""The library's nested-Horner tables of the triangle weight (App. C.3),
the form the traversal kernels evaluate, against the oracle's own weight
polynomials (numpy pseudoinverse solve of the App. C.3 constraints, in the
monomial basis): for every class (v, e) of the tables and each orientation,
the tables evaluated in FP64 reproduce the oracle's w~ and its two partial
derivatives (phi0 = 1 - phi1 - phi2) at random barycentric points, to the
fp32 rounding of the stored coefficients. Host only: no GPU."""
import ctypes

import numpy as np
import pytest

from oracle import weights as OW

VMAX, EMAX, FLOATS = 16, 4, 92


@pytest.fixture(scope="module")
def tables():
    from paper_2108_10480_gb300 import lib
    out = np.zeros(VMAX * EMAX * 3 * FLOATS, np.float32)
    assert lib().sd_weight_horner_tables(ctypes.c_void_p(out.ctypes.data)) == 0
    return out.astype(np.float64).reshape(VMAX, EMAX, 3, FLOATS)


def _horner(c, deg, r, s):
    acc, n = 0.0, 0
    for bp in range(deg, -1, -1):
        inner = c[n]
        n += 1
        for _ in range(deg - bp):
            inner = inner * r + c[n]
            n += 1
        acc = acc * s + inner
    return acc


def _eval(t, p1, p2):
    """w~, dw~/dphi1, dw~/dphi2 from one class's three orientation tables."""
    p0 = 1.0 - p1 - p2
    ps = [p0, p1, p2]
    o = int(np.argmax(ps))
    others = [ps[k] for k in range(3) if k != o]
    base = ps[o]
    r, s = others[0] / base, others[1] / base
    c = t[o]
    return (_horner(c[:36], 7, r, s) * base ** 7, _horner(c[36:64], 6, r, s) * base ** 6,
            _horner(c[64:], 6, r, s) * base ** 6)


def _oracle(coef, p1, p2):
    w = sum(cf * p1 ** a * p2 ** b for cf, (a, b) in zip(coef, OW.TRI_EXPONENTS))
    d1 = sum(cf * a * p1 ** (a - 1) * p2 ** b for cf, (a, b) in zip(coef, OW.TRI_EXPONENTS) if a)
    d2 = sum(cf * b * p1 ** a * p2 ** (b - 1) for cf, (a, b) in zip(coef, OW.TRI_EXPONENTS) if b)
    return w, d1, d2


@pytest.mark.parametrize("v", [2, 3, 4, 5, 6, 7, 9, 12, 16])
@pytest.mark.parametrize("e", [1, 2, 3, 4])
def test_tables_reproduce_the_oracle_weight(tables, v, e):
    basis = OW.tri_basis()
    coef = basis @ np.array([1.0 / v, 1.0 / e, 1.0 - 1.0 / v])
    rng = np.random.default_rng(100 * v + e)
    pts = rng.random((400, 2))
    pts = pts[pts.sum(1) <= 1.0]
    # vertices, edge midpoints, the barycentre and points where two
    # barycentrics tie (the orientation switches)
    pts = np.concatenate([pts, [[0, 0], [1, 0], [0, 1], [0.5, 0], [0, 0.5], [0.5, 0.5], [1 / 3, 1 / 3],
                                [0.4, 0.4], [0.2, 0.4], [0.4, 0.2], [0.25, 0.5]]])
    t = tables[v - 1, e - 1]
    for p1, p2 in pts:
        w, d1, d2 = _eval(t, p1, p2)
        rw, r1, r2 = _oracle(coef, p1, p2)
        assert abs(w - rw) <= 1e-6 * max(abs(rw), 1.0), (v, e, p1, p2, w, rw)
        g = max(abs(r1), abs(r2), 1.0)
        assert abs(d1 - r1) <= 1e-5 * g and abs(d2 - r2) <= 1e-5 * g, (v, e, p1, p2, d1, r1, d2, r2)
