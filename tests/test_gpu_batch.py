"""Batched multi-body evaluation (sd_batch_*): per-body outer LogSumExp and
pose gradients against the FP64 oracle at the same fp32 vertices, graph
capture and replay, and the autotuner's admissibility rule."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import pose as PO

pytestmark = pytest.mark.gpu


def _vec_err(a, b, floor=1e-2):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def _bodies(n, seed, lo, hi, vmax=3000):
    rng = np.random.default_rng(seed)
    out, poses = [], []
    for b in range(n):
        if b % 2 == 0:
            V, _ = synth.geodesic_icosphere(int(rng.integers(3, 12)))
        else:
            V, _ = synth.torus(int(rng.integers(12, 40)), int(rng.integers(6, 16)), 1.0, 0.3)
        V = (V.astype(np.float64) * rng.uniform(0.3, 2.0)).astype(np.float32)[:vmax]
        out.append(V)
        poses.append(np.concatenate([rng.standard_normal(3), lo + (hi - lo) * rng.random(3)]))
    return out, np.array(poses)


@pytest.fixture(scope="module")
def small_scene():
    s = synth.street_scene(n_points=6000, n_wire_segments=116, seed=9)
    P = s["points"]
    P = P[np.abs(P[:, 0] - 20.0) < 25.0]
    return P, s["wire_V"], s["wire_E"]


def _check_bodies(out, sc, bodies, poses, alpha, alpha_q, beta, which):
    o = out.cpu().numpy().astype(np.float64)
    for b in which:
        D, G, _, _, _ = PO.pose_objective(sc, bodies[b], poses[b], alpha, alpha_q, beta=beta, precision="f32")
        assert abs(o[b, 0] - D) / max(abs(D), 1.0 / alpha_q) <= 1e-5, (b, o[b, 0], D)
        # library order (D, dD/dp, dD/dtheta) vs oracle (dtheta, dp)
        assert _vec_err(np.concatenate([o[b, 4:7], o[b, 1:4]]), G) <= 1e-4, (b, o[b], G)


@pytest.mark.parametrize("L", [1, 4])
def test_batch_small_vs_oracle_and_graph(small_scene, L):
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.batch import BatchedBodies
    P, Vw, Ew = small_scene
    alpha, beta, alpha_q = 8.0, 0.5, 20.0
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=alpha, beta=beta, leaf_size=L, device="cuda:0")
    sc = oracle.Scene(points=P, edge_V=Vw, edge_E=Ew)
    sc.build_tree(L)
    bodies, poses = _bodies(7, 3, np.array([0.0, -8.0, 0.5]), np.array([40.0, 8.0, 9.0]))
    bb = BatchedBodies(sd, bodies)
    bb.set_poses(poses)
    out = bb.run(alpha_q).clone()
    torch.cuda.synchronize()
    _check_bodies(out, sc, bodies, poses, alpha, alpha_q, beta, range(len(bodies)))
    # a captured graph replays the same computation bit for bit
    g = bb.capture(alpha_q)
    bb.out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(bb.out, out)
    # new poses, same graph
    poses2 = poses.copy()
    poses2[:, 3] += 1.5
    poses2[:, :3] *= -0.5
    bb.set_poses(poses2)
    g.replay()
    torch.cuda.synchronize()
    _check_bodies(bb.out, sc, bodies, poses2, alpha, alpha_q, beta, range(len(bodies)))


def test_batch_matches_single_body_path(small_scene):
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    from paper_2108_10480_gb300.batch import BatchedBodies
    P, Vw, Ew = small_scene
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=8.0, beta=0.5, device="cuda:0")
    bodies, poses = _bodies(5, 4, np.array([0.0, -8.0, 0.5]), np.array([40.0, 8.0, 9.0]))
    bb = BatchedBodies(sd, bodies)
    bb.set_poses(poses)
    out = bb.run(20.0).cpu().numpy()
    for b in range(len(bodies)):
        X0 = torch.from_numpy(bodies[b]).cuda()
        X, v, g = gp.pose_query(sd, X0, poses[b])
        res, _ = gp.pose_reduce(X0, v, g, poses[b], alpha_q=20.0)
        r = res.cpu().numpy()
        assert abs(out[b, 0] - r[0]) <= 1e-5 * max(abs(r[0]), 0.05)
        assert _vec_err(np.concatenate([out[b, 4:7], out[b, 1:4]]), r[1:]) <= 1e-4


def test_autotuner_admissibility(small_scene):
    from paper_2108_10480_gb300.batch import autotune
    P, Vw, Ew = small_scene
    bodies, poses = _bodies(4, 5, np.array([0.0, -8.0, 0.5]), np.array([40.0, 8.0, 9.0]))
    q = synth.uniform_box(512, [0.0, -10.0, 0.0], [40.0, 10.0, 10.0], 6)
    kw = dict(points=P, edges=(Vw, Ew), alpha=8.0, beta=0.5, device="cuda:0")
    best, recs = autotune(kw, bodies, poses, 20.0, q, leaf_sizes=(1, 2, 8), blocks=(64, 128), reps=2)
    assert len(recs) == 6
    assert best is not None and best["admissible"]
    err1 = [r["bh_err"] for r in recs if r["leaf_size"] == 1][0]
    for r in recs:
        assert r["admissible"] == (r["bh_err"] <= 2.0 * max(err1, 1e-7))
    assert best["ms"] == min(r["ms"] for r in recs if r["admissible"])


def test_batch_full_street_64_bodies():
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.batch import BatchedBodies
    s = synth.config3_scene()
    bl = synth.config4_bodies()
    bodies = [b["V0"] for b in bl]
    poses = np.array([np.concatenate([b["theta"], b["p"]]) for b in bl])
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5,
                        device="cuda:0")
    bb = BatchedBodies(sd, bodies)
    bb.set_poses(poses)
    g = bb.capture(100.0)
    g.replay()
    torch.cuda.synchronize()
    out = bb.out.clone()
    assert torch.isfinite(out).all()
    sc = oracle.Scene(points=s["points"], edge_V=s["wire_V"], edge_E=s["wire_E"])
    sc.build_tree(1)
    sizes = np.array([b.shape[0] for b in bodies])
    which = list(np.argsort(sizes)[:3]) + [int(np.argmax(sizes))]
    _check_bodies(out, sc, bodies, poses, 50.0, 100.0, 0.5, which)
