"""Error measures for GPU-vs-oracle parity of d^ and grad d^.

value:    |d^_gpu - d^_ref| / max(|d^_ref|, d_min, 1/alpha)         <= 1e-5
gradient: ||g_gpu - g_ref|| / max(||g_ref||, 1e-2)                   <= 1e-4
d_min is the exact distance to the data mesh where the test has it; without
it the denominator drops that term (a stricter test). The floors 1/alpha and
1e-2 keep the measure defined where d^ or its gradient crosses zero.
"""
import numpy as np

VALUE_TOL = 1e-5
GRAD_TOL = 1e-4


def value_err(v, ref, alpha, dmin=None):
    v = np.asarray(v, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1.0 / alpha)
    if dmin is not None:
        den = np.maximum(den, np.asarray(dmin, np.float64))
    return np.abs(v - ref) / den


def grad_err(g, ref):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.linalg.norm(g - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-2)


def assert_parity(v, g, rv, rg, alpha, dmin=None, what=""):
    ev = value_err(v, rv, alpha, dmin)
    assert np.all(np.isfinite(v)), what + ": non-finite value"
    assert ev.max() <= VALUE_TOL, f"{what}: value rel err {ev.max():.3e} at {int(ev.argmax())}"
    if g is not None:
        eg = grad_err(g, rg)
        assert eg.max() <= GRAD_TOL, f"{what}: grad rel err {eg.max():.3e} at {int(eg.argmax())}"
    return ev.max(), (grad_err(g, rg).max() if g is not None else 0.0)
