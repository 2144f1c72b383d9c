"""Weight-polynomial bases of the oracle (FP64, numpy).

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline use the oracle; the CUDA library never imports it.

Both bases are solved here from the constraint systems that App. C states,
with plain library linear algebra; nothing is hand-derived.

* Edge weight (App. C.2): a quartic w~(phi) with w~(0) = 1/|N_i0|,
  w~(1) = 1/|N_i1|, w~(1/2) = 1 and zero derivative at both ends (the paper
  prints the derivative constraints as "w~(0) = w~(1) = 0"; they are read as
  w~'(0) = w~'(1) = 0, the only reading that gives a C^1 weight and five
  independent equations). The solution is linear in (u, v, 1), so the basis
  is three quartics solved with numpy.linalg.solve.

* Triangle weight (App. C.3): a degree-7 polynomial in (phi1, phi2) with 36
  monomial coefficients; 10 point constraints (vertices 1/v_i, two points per
  edge 1/e_i, barycentre (v_i - 1)/v_i) and 26 normal-derivative equations
  (7 + 7 - 1 on the legs phi1 = 0 and phi2 = 0, 7 + 7 - 1 on the hypotenuse),
  36 equations in all, solved with the pseudoinverse (numpy.linalg.pinv,
  minimum-norm). The right-hand side is linear in (1/v, 1/e, (v-1)/v), so the
  basis is three 36-vectors.
"""
from __future__ import annotations

import math

import numpy as np

# monomial order: phi1^a phi2^b, a + b <= 7, a-major
TRI_EXPONENTS = [(a, b) for a in range(8) for b in range(8) if a + b <= 7]
_TIDX = {m: i for i, m in enumerate(TRI_EXPONENTS)}


def edge_system():
    """5x5 matrix of the edge constraints (rows: w(0), w(1), w(1/2), w'(0),
    w'(1)) acting on the coefficients (c0..c4) of sum_k c_k phi^k, and the
    3 right-hand sides for (u, v, 1)."""
    A = np.array([
        [1.0, 0.0, 0.0, 0.0, 0.0],
        [1.0, 1.0, 1.0, 1.0, 1.0],
        [1.0, 0.5, 0.25, 0.125, 0.0625],
        [0.0, 1.0, 0.0, 0.0, 0.0],
        [0.0, 1.0, 2.0, 3.0, 4.0],
    ])
    B = np.zeros((5, 3))
    B[0, 0] = 1.0   # w(0) = u
    B[1, 1] = 1.0   # w(1) = v
    B[2, 2] = 1.0   # w(1/2) = 1
    return A, B


def edge_basis():
    """[5, 3] array: column j holds the quartic coefficients for the unit
    right-hand side j of (u, v, 1)."""
    A, B = edge_system()
    return np.linalg.solve(A, B)


def _mono_row(x, y):
    return np.array([x ** a * y ** b for (a, b) in TRI_EXPONENTS])


def _hyp_rows(swap: bool):
    """Coefficients (in t) of (d/dphi1 + d/dphi2) w~ restricted to the
    hypotenuse, parametrised as (t, 1-t) or, if swap, (1-t, t); returns a
    [7, 36] matrix, row k = coefficient of t^k."""
    R = np.zeros((7, 36))
    for j, (a, b) in enumerate(TRI_EXPONENTS):
        # d/dphi1 + d/dphi2 of phi1^a phi2^b
        for (coef, p, r) in ((a, a - 1, b), (b, a, b - 1)):
            if coef == 0 or p < 0 or r < 0:
                continue
            # phi1 = t, phi2 = 1 - t  (or swapped)
            tp, om = (p, r) if not swap else (r, p)
            # t^tp (1 - t)^om = sum_k C(om, k) (-1)^k t^(tp + k)
            for k in range(om + 1):
                R[tp + k, j] += coef * math.comb(om, k) * (-1) ** k
    return R


def tri_system():
    """The 36 constraint equations of App. C.3 as ([36, 36] matrix, [36, 3]
    right-hand sides for the unit vectors of (1/v, 1/e, (v-1)/v))."""
    rows, rhs = [], []
    third = 1.0 / 3.0
    for (x, y) in [(0, 0), (1, 0), (0, 1)]:
        rows.append(_mono_row(x, y)); rhs.append([1, 0, 0])
    for (x, y) in [(third, 0), (2 * third, 0), (third, 2 * third), (2 * third, third),
                   (0, third), (0, 2 * third)]:
        rows.append(_mono_row(x, y)); rhs.append([0, 1, 0])
    rows.append(_mono_row(third, third)); rhs.append([0, 0, 1])
    # d/dphi1 w~(0, t) = sum_b c_{1,b} t^b == 0  -> c_{1,b} = 0, b = 0..6
    for b in range(7):
        r = np.zeros(36); r[_TIDX[(1, b)]] = 1.0
        rows.append(r); rhs.append([0, 0, 0])
    # d/dphi2 w~(t, 0) = sum_a c_{a,1} t^a == 0 -> c_{a,1} = 0; the t^1
    # coefficient c_{1,1} is already present above
    for a in range(7):
        if a == 1:
            continue
        r = np.zeros(36); r[_TIDX[(a, 1)]] = 1.0
        rows.append(r); rhs.append([0, 0, 0])
    # hypotenuse, both parametrisations; their t^6 coefficients coincide, so
    # the second family drops it
    H1 = _hyp_rows(False)
    H2 = _hyp_rows(True)
    for k in range(7):
        rows.append(H1[k]); rhs.append([0, 0, 0])
    for k in range(6):
        rows.append(H2[k]); rhs.append([0, 0, 0])
    return np.array(rows, dtype=np.float64), np.array(rhs, dtype=np.float64)


def tri_basis():
    """[36, 3] minimum-norm (pseudoinverse) solution, monomials in
    TRI_EXPONENTS order, columns for (1/v, 1/e, (v-1)/v)."""
    A, B = tri_system()
    return np.linalg.pinv(A) @ B


def tri_weight(phi1, phi2, inv_v, inv_e, basis=None):
    """FP64 w~(phi1, phi2) for one triangle (used by tests)."""
    if basis is None:
        basis = tri_basis()
    c = basis @ np.array([inv_v, inv_e, 1.0 - inv_v])
    return float(sum(c[j] * phi1 ** a * phi2 ** b for j, (a, b) in enumerate(TRI_EXPONENTS)))


def edge_weight(phi, u, v, basis=None):
    if basis is None:
        basis = edge_basis()
    c = basis @ np.array([u, v, 1.0])
    return float(sum(c[k] * phi ** k for k in range(5)))
