"""GPU sphere tracing (sd_sphere_trace) against the oracle's tracer on a
small bumpy mesh as points, edges and triangles, exact and Barnes-Hut:
the same rays hit (every ray whose marches both end within the step
budget), at the same depth up to the march's resolution."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import trace as OT

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _kinds():
    V, F = synth.blob(level=3)
    E = synth.mesh_edges(F)
    return {"points": (dict(points=V), dict(points=V)),
            "edges": (dict(edges=(V, E)), dict(edge_V=V, edge_E=E)),
            "tris": (dict(tris=(V, F)), dict(tri_V=V, tri_F=F))}, V


@pytest.mark.parametrize("kind", ["points", "edges", "tris"])
@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_trace_matches_oracle(kind, beta):
    from paper_2108_10480_gb300 import SmoothDistance
    kinds, V = _kinds()
    gkw, okw = kinds[kind]
    cam = synth.trace_camera(V, 48, 40)
    t_max = 4.0 * cam["diag"]
    sd = SmoothDistance(alpha=200.0, alpha_u=1200.0, beta=beta, device="cuda:0", **gkw)
    depth, steps, ev = sd.sphere_trace(cam, eps=EPS, t_max=t_max, max_steps=256)
    assert sd.status() == 0
    depth = depth.cpu().numpy().ravel().astype(np.float64)
    sc = oracle.Scene(**okw)
    rd, rs = OT.sphere_trace(sc, cam, 200.0, beta, alpha_u=1200.0, eps=EPS, t_max=t_max, max_steps=256)
    hg, hr = np.isfinite(depth), np.isfinite(rd)
    assert hr.sum() > 200 and (~hr).sum() > 200            # the object and the background both in view
    # A ray's hit decision may differ only where one of the two marches ran
    # out of steps (a grazing ray still closing in on the surface, where
    # fp32 and fp64 steps part ways); everywhere else both must agree.
    gs = steps.cpu().numpy().ravel()
    differ = (hg != hr) & (gs < 256) & (rs < 256)
    assert not differ.any(), f"{kind} beta={beta}: hit masks differ on {differ.sum()} rays"
    both = hg & hr
    err = np.abs(depth[both] - rd[both])
    assert np.all(err <= 4 * EPS + 1e-5 * rd[both]), f"{kind} beta={beta}: depth err {err.max():.3e}"
    assert ev == int(steps.sum().item()) and ev >= rs.sum() * 0.98
