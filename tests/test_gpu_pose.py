"""GPU pose adjoint (sd_pose_query / sd_pose_reduce and the autograd
Function) against the FP64 oracle evaluated at the same fp32 query points,
on a small street at beta = 0 and on the full street workload (2,000,000
lidar points + 50,000 wire segments, a 100,002-vertex body) at beta = 0.5."""
import numpy as np
import pytest
import torch

import oracle
import synth
from _metrics import assert_parity
from oracle import pose as PO

pytestmark = pytest.mark.gpu


def _vec_err(a, b, floor=1e-2):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def _check(sd, sc, X0, pose, alpha, alpha_q, beta):
    from paper_2108_10480_gb300 import pose as gp
    X0t = torch.from_numpy(X0).cuda()
    X, v, g = gp.pose_query(sd, X0t, pose)
    res, dX0 = gp.pose_reduce(X0t, v, g, pose, alpha_q=alpha_q, want_dx0=True)
    D, G, rv, rg, gam = PO.pose_objective(sc, X0, pose, alpha, alpha_q, beta=beta, precision="f32")
    # identical query points
    assert np.array_equal(X.cpu().numpy(), PO.place(X0, pose, "f32"))
    assert_parity(v.cpu().numpy(), g.cpu().numpy(), rv, rg, alpha, None, "per-vertex")
    r = res.cpu().numpy().astype(np.float64)
    assert abs(r[0] - D) / max(abs(D), 1.0 / alpha_q) <= 1e-5, (r[0], D)
    assert _vec_err(r[1:], G) <= 1e-4, (r[1:], G)
    R = PO.rotation(pose[:3])
    ref_dx0 = gam[:, None] * (rg @ R)
    assert np.abs(dX0.cpu().numpy() - ref_dx0).max() <= 1e-4 * max(np.abs(ref_dx0).max(), 1e-6)
    return r


@pytest.fixture(scope="module")
def small_street():
    s = synth.street_scene(n_points=3000, n_wire_segments=116, seed=7)
    P = s["points"]
    P = P[np.abs(P[:, 0] - 20.0) < 20.0]
    V, F = synth.geodesic_icosphere(4)
    X0 = (V.astype(np.float64) * np.array([0.8, 0.5, 0.35])).astype(np.float32)
    return P, s["wire_V"], s["wire_E"], X0


def test_pose_small_exact(small_street):
    from paper_2108_10480_gb300 import SmoothDistance
    P, Vw, Ew, X0 = small_street
    sc = oracle.Scene(points=P, edge_V=Vw, edge_E=Ew)
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=5.0, beta=0.0, device="cuda:0")
    for pose in ([0.4, -0.3, 1.1, 20.0, 5.5, 6.0], [0.0, 0.0, 0.0, 18.0, -2.0, 1.5], [2.5, 1.0, -0.7, 30.0, 6.0, 7.5]):
        _check(sd, sc, X0, np.array(pose), 5.0, 10.0, 0.0)


def test_autograd_function(small_street):
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.pose import SmoothDistancePose
    P, Vw, Ew, X0 = small_street
    sc = oracle.Scene(points=P, edge_V=Vw, edge_E=Ew)
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=5.0, beta=0.0, device="cuda:0")
    pose0 = np.array([0.4, -0.3, 1.1, 20.0, 5.5, 6.0])
    D_ref, G_ref, rv, rg, gam = PO.pose_objective(sc, X0, pose0, 5.0, 10.0, precision="f32")
    # scalar constraint
    pose = torch.tensor(pose0, dtype=torch.float64, requires_grad=True)
    X0t = torch.from_numpy(X0).cuda().requires_grad_(True)
    D = SmoothDistancePose.apply(pose, X0t, sd, 10.0)
    D.backward()
    assert abs(D.item() - D_ref) <= 1e-5 * max(abs(D_ref), 0.1)
    assert _vec_err(pose.grad.numpy(), G_ref) <= 1e-4
    R = PO.rotation(pose0[:3])
    assert np.abs(X0t.grad.cpu().numpy() - gam[:, None] * (rg @ R)).max() <= 1e-4 * np.abs(gam[:, None] * rg).max()
    # per-vertex values with an arbitrary upstream gradient
    pose = torch.tensor(pose0, dtype=torch.float64, requires_grad=True)
    X0t = torch.from_numpy(X0).cuda().requires_grad_(True)
    v = SmoothDistancePose.apply(pose, X0t, sd, None)
    w = torch.linspace(-1.0, 2.0, v.shape[0], device="cuda")
    (v * w).sum().backward()
    wn = w.cpu().numpy().astype(np.float64)
    Y = X0.astype(np.float64) @ R.T
    ref = np.concatenate([PO.left_jacobian(pose0[:3]).T @ (wn[:, None] * np.cross(Y, rg)).sum(0),
                          (wn[:, None] * rg).sum(0)])
    assert _vec_err(pose.grad.numpy(), ref) <= 1e-4
    assert np.abs(X0t.grad.cpu().numpy() - wn[:, None] * (rg @ R)).max() <= 1e-4 * np.abs(wn[:, None] * rg).max()


def test_pose_gradient_fd_on_gpu(small_street):
    """Central differences of the GPU's own fp32 constraint (h = 1e-3; fp32
    rounding of D limits the accuracy of the difference quotient)."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    P, Vw, Ew, X0 = small_street
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=5.0, beta=0.0, device="cuda:0")
    X0t = torch.from_numpy(X0).cuda()
    pose0 = np.array([0.4, -0.3, 1.1, 20.0, 5.5, 6.0])

    def Dof(ps):
        X, v, g = gp.pose_query(sd, X0t, ps)
        return gp.pose_reduce(X0t, v, g, ps, alpha_q=10.0)[0].cpu().numpy().astype(np.float64)

    G = Dof(pose0)[1:]
    h = 1e-3
    fd = np.array([(Dof(pose0 + h * e)[0] - Dof(pose0 - h * e)[0]) / (2 * h) for e in np.eye(6)])
    assert _vec_err(G, fd, floor=1e-1) <= 2e-2


def test_pose_full_street():
    from paper_2108_10480_gb300 import SmoothDistance
    s = synth.config3_scene()
    b = synth.config3_body()
    pose = np.concatenate([b["theta"], b["p"]])
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5,
                        device="cuda:0")
    sc = oracle.Scene(points=s["points"], edge_V=s["wire_V"], edge_E=s["wire_E"])
    sc.build_tree(1)
    _check(sd, sc, b["V0"], pose, 50.0, 100.0, 0.5)


def test_sharded_reduction_matches_the_whole_body(small_street):
    """Sec. 3.6's outer sum split into shards: sd_pose_partial on uneven
    slices of the body's vertices (one of them empty), merged on the host by
    sd_pose_merge, equals sd_pose_reduce over the whole body and the FP64
    oracle, in the LSE mode and in the upstream-gradient (linear) mode."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300 import pose as gp
    P, Vw, Ew, X0 = small_street
    sc = oracle.Scene(points=P, edge_V=Vw, edge_E=Ew)
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=5.0, beta=0.0, device="cuda:0")
    pose = np.array([0.4, -0.3, 1.1, 20.0, 5.5, 6.0])
    X0t = torch.from_numpy(X0).cuda()
    X, v, g = gp.pose_query(sd, X0t, pose)
    M = X0.shape[0]
    cuts = [0, 7, 7, M // 3, M - 1, M]
    whole, _ = gp.pose_reduce(X0t, v, g, pose, alpha_q=10.0)
    whole = whole.cpu().numpy().astype(np.float64)
    parts = np.stack([gp.pose_partial(X0t[a:b], v[a:b], g[a:b], pose, alpha_q=10.0).cpu().numpy()
                      for a, b in zip(cuts[:-1], cuts[1:])])
    assert parts[1, 0] == -np.inf and not parts[1, 1:].any()        # the empty shard
    for order in (slice(None), slice(None, None, -1)):
        r = gp.merge_partials(parts[order], pose, alpha_q=10.0)
        assert abs(r[0] - whole[0]) <= 1e-6 * max(abs(whole[0]), 0.1), (r[0], whole[0])
        assert _vec_err(r[1:], whole[1:]) <= 1e-5
    D, G, _, _, _ = PO.pose_objective(sc, X0, pose, 5.0, 10.0, precision="f32")
    assert abs(r[0] - D) / max(abs(D), 0.1) <= 1e-5 and _vec_err(r[1:], G) <= 1e-4
    # linear mode: an upstream gradient gamma per vertex
    w = torch.linspace(-1.0, 2.0, M, device="cuda")
    lin, _ = gp.pose_reduce(X0t, v, g, pose, gamma=w)
    parts = np.stack([gp.pose_partial(X0t[a:b], v[a:b], g[a:b], pose, gamma=w[a:b]).cpu().numpy()
                      for a, b in zip(cuts[:-1], cuts[1:])])
    r = gp.merge_partials(parts, pose)
    lin = lin.cpu().numpy().astype(np.float64)
    assert _vec_err(r[1:], lin[1:]) <= 1e-5 and abs(r[0] - lin[0]) <= 1e-5 * max(abs(lin[0]), 1.0)
