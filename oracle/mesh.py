"""Smooth distance between a data mesh and a query mesh, in FP64 (Sec. 3.6,
Eq. lse_full, Eq. lse_full2, Eq. dlse_full).

TEST INFRASTRUCTURE (see oracle/__init__.py).

Given per-primitive values d^_j and translation gradients grad d^_j of the
query mesh's primitives g_j (each with n(g_j) + 1 vertices),
  D = -(1/alpha_q) log sum_j exp(-alpha_q d^_j)                     (Eq. lse_full)
and the gradient with respect to query vertex k splits every primitive's
share equally between its vertices:
  grad_k D = sum_{j incident to k} exp(-alpha_q d^_j) / (n(g_j) + 1) grad d^_j
             / sum_j exp(-alpha_q d^_j)                             (Eq. dlse_full)
"""
from __future__ import annotations

import numpy as np


def mesh_objective(val, grad, QF, nverts, alpha_q):
    val = np.asarray(val, np.float64)
    grad = np.asarray(grad, np.float64).reshape(-1, 3)
    F = np.asarray(QF).reshape(val.shape[0], -1)
    t = -alpha_q * val
    m = t.max()
    e = np.exp(t - m)
    Z = e.sum()
    D = -(m + np.log(Z)) / alpha_q
    share = (e / Z / F.shape[1])[:, None] * grad
    G = np.zeros((nverts, 3))
    for c in range(F.shape[1]):
        np.add.at(G, F[:, c], share)
    return D, G, e / Z
