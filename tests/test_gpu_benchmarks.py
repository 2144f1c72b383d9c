"""The evaluation protocols of Sec. 4.3 / 4.4 at the GPU-oracle parity bar:
voxel-grid queries on a mesh normalised into the unit cube as V, E and F
with the paper's alpha heuristic, and beta = 0.5001 next to 0.5 (node
decisions identical to the oracle's FP32 test for both)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _metrics import assert_parity

pytestmark = pytest.mark.gpu


def _unit_box(X):
    X = np.asarray(X, np.float64)
    lo, hi = X.min(0), X.max(0)
    return ((X - 0.5 * (lo + hi)) * (0.5 / np.linalg.norm(hi - lo)) + 0.5).astype(np.float32)


@pytest.mark.parametrize("kind", ["V", "E", "F"])
def test_voxel_grid_parity(kind):
    from paper_2108_10480_gb300 import SmoothDistance
    V, F = synth.blob(level=3, diag=1.0, seed=13)
    V = _unit_box(V)
    E = synth.mesh_edges(F)
    emin = float(np.linalg.norm(V[E[:, 0]] - V[E[:, 1]], axis=1).min())
    kw, okw, alpha = {"V": (dict(points=V), dict(points=V), 50.0),
                      "E": (dict(edges=(V, E)), dict(edge_V=V, edge_E=E), 1.0 / emin),
                      "F": (dict(tris=(V, F)), dict(tri_V=V, tri_F=F), 1.0 / emin)}[kind]
    g = (np.arange(24) + 0.5) / 24
    q = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    sc = oracle.Scene(**okw)
    sc.build_tree(1)
    for beta in (0.5, 0.5001):
        sd = SmoothDistance(alpha=alpha, beta=beta, device="cuda:0", **kw)
        v, gr, cnt = sd.query(torch.from_numpy(q).cuda(), counts=True)
        rv, rg, rc, _ = sc.bh(q, alpha, beta)
        assert np.array_equal(cnt.cpu().numpy(), rc), (kind, beta)
        assert_parity(v.cpu().numpy(), gr.cpu().numpy(), rv, rg, alpha, None, f"voxel {kind} beta={beta}")
