"""Learned far-field surrogate: the MLP kernels against the FP64 oracle
network (oracle/mlp.py), the certified lower bound against exact and
Barnes-Hut values, and what a trained surrogate gains over the method alone."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import mlp as OM

pytestmark = pytest.mark.gpu


def _net(seed=0, sigma=4.0):
    from paper_2108_10480_gb300.surrogate import Surrogate
    lo, hi = np.array([-8.0, -3.0, -1.0]), np.array([12.0, 5.0, 4.0])
    sur = Surrogate(lo, hi, sigma=sigma, seed=seed, scale=2.0)
    # perturb the zero biases so that every parameter is exercised
    g = torch.Generator(device="cuda").manual_seed(seed + 7)
    sur.params.add_(0.05 * torch.randn(sur.params.shape, device="cuda", generator=g) *
                    (torch.arange(sur.params.numel(), device="cuda") >= 96))
    return sur, lo, hi


def _frame(sur):
    f = sur.frame.astype(np.float64)
    return f[:3], f[3:6], f[6]


def test_train_step_gradient_and_adam_vs_oracle():
    sur, lo, hi = _net(1)
    rng = np.random.default_rng(2)
    n = 1000
    x = lo + (hi - lo) * rng.random((n, 3))
    t = rng.uniform(0, 4, n)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    th = sur.params.cpu().numpy().astype(np.float64)
    c, h, s = _frame(sur)
    L, G = OM.loss_and_grad(th, x.astype(np.float32), t.astype(np.float32), c, h, s, bf16=True)
    loss, g = sur.train_step(xt, tt, 0.0)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - L) <= 1e-4 * L
    assert np.abs(g - G).max() <= 1e-4 * np.abs(G).max()
    # per parameter block
    o = 0
    for name, shp in OM.SHAPES:
        k = int(np.prod(shp))
        if name != "B":
            assert np.linalg.norm(g[o:o + k] - G[o:o + k]) <= 1e-4 * max(np.linalg.norm(G[o:o + k]), 1e-12), name
        o += k
    # one Adam step
    t2, _, _ = OM.adam(th, G, np.zeros_like(G), np.zeros_like(G), 1, 1e-3)
    sur.train_step(xt, tt, 1e-3)
    p2 = sur.params.cpu().numpy().astype(np.float64)
    assert np.abs(p2 - t2).max() <= 1e-6 + 1e-5 * np.abs(t2).max()


def test_forward_and_input_gradient_vs_oracle():
    sur, lo, hi = _net(3)
    rng = np.random.default_rng(4)
    x = (lo + (hi - lo) * rng.random((5003, 3))).astype(np.float32)      # ragged last tile
    y, dy = sur.forward(torch.from_numpy(x).cuda())
    th = sur.params.cpu().numpy().astype(np.float64)
    c, h, s = _frame(sur)
    y = y.cpu().numpy().astype(np.float64)
    dy = dy.cpu().numpy().astype(np.float64)

    def errs(ry, rdy):
        ey = np.abs(y - ry) / (np.abs(ry) + s * 0.05)
        eg = np.linalg.norm(dy - rdy, axis=1) / (np.linalg.norm(rdy, axis=1) + 0.05 * np.linalg.norm(s / h))
        return ey, eg

    # against the network evaluated at the kernel's storage precisions: what
    # remains is fp32 accumulation order and sincospi, plus rare one-unit
    # bfloat16 rounding flips of an operand near a tie
    ey, eg = errs(*OM.forward(th, x, c, h, s, mixed=True)[:2])
    print(f"surrogate forward vs stored-precision oracle: value rel err max {ey.max():.2e} "
          f"mean {ey.mean():.2e}; grad rel err max {eg.max():.2e} mean {eg.mean():.2e}")
    # a flip moves one operand by one bfloat16 unit and is rare, so the mean
    # and the 99th percentile are tight and the maximum is one flip's reach
    # (measured: value 1.5e-5 / 9.9e-5 / 8.1e-3, gradient 5.3e-5 / 1.8e-3 / 1.5e-2)
    assert ey.mean() <= 1e-4 and np.quantile(ey, 0.99) <= 5e-4 and ey.max() <= 2e-2
    assert eg.mean() <= 2e-4 and np.quantile(eg, 0.99) <= 5e-3 and eg.max() <= 4e-2
    # against the bf16-weight network with exact activations: the cost of
    # bfloat16 activations (measured 2.7e-2 max / 2.7e-3 mean on this net)
    ey, eg = errs(*OM.forward(th, x, c, h, s, bf16=True)[:2])
    print(f"surrogate forward vs exact-activation oracle: value rel err max {ey.max():.2e} "
          f"mean {ey.mean():.2e}; grad rel err max {eg.max():.2e} mean {eg.mean():.2e}")
    assert ey.max() <= 6e-2 and ey.mean() <= 6e-3
    assert eg.max() <= 1e-1 and eg.mean() <= 1e-2


@pytest.fixture(scope="module")
def street_small():
    s = synth.street_scene(n_points=6000, n_wire_segments=116, seed=9)
    P = s["points"]
    P = P[np.abs(P[:, 0] - 20.0) < 25.0]
    return P, s["wire_V"], s["wire_E"]


def _lb_scenes(street):
    P, Vw, Ew = street
    V, F = synth.icosphere(3)
    V = (V * 3.0 + np.array([20.0, 0.0, 5.0])).astype(np.float32)
    keep = V[F].mean(1)[:, 2] > 4.0                       # open mesh: w~ up to its Bernstein bound
    return [(dict(points=P, edges=(Vw, Ew)), dict(points=P, edge_V=Vw, edge_E=Ew)),
            (dict(tris=(V, F)), dict(tri_V=V, tri_F=F)),
            (dict(tris=(V, F[keep])), dict(tri_V=V, tri_F=F[keep]))]


@pytest.mark.parametrize("n", [1, 127, 129, 77777])
def test_forward_tile_edges_vs_oracle(n):
    """Sizes around the 128-query tile of the tensor-core kernel: a single
    query, one row short of and one past a tile, and enough tiles that every
    warp group walks several (the next tile's queries are fetched early).
    Value only gives the same values bit for bit."""
    sur, lo, hi = _net(5)
    rng = np.random.default_rng(n)
    x = (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    y, dy = sur.forward(xt)
    y2, none = sur.forward(xt, grad=False)
    assert none is None and torch.equal(y, y2)
    th = sur.params.cpu().numpy().astype(np.float64)
    c, h, s = _frame(sur)
    ry, rdy = OM.forward(th, x, c, h, s, mixed=True)[:2]
    y = y.cpu().numpy().astype(np.float64)
    dy = dy.cpu().numpy().astype(np.float64)
    assert np.isfinite(y).all() and np.isfinite(dy).all()
    ey = np.abs(y - ry) / (np.abs(ry) + s * 0.05)
    eg = np.linalg.norm(dy - rdy, axis=1) / (np.linalg.norm(rdy, axis=1) + 0.05 * np.linalg.norm(s / h))
    print(f"n={n}: value rel err mean {ey.mean():.2e} max {ey.max():.2e}; grad rel err mean {eg.mean():.2e} "
          f"max {eg.max():.2e}")
    # the statistics of test_forward_and_input_gradient_vs_oracle where there
    # are enough queries for them; the maximum is one bfloat16 rounding flip's
    # reach, whose tail grows with the sample (77,777 queries: 2.4e-2)
    assert ey.max() <= 5e-2 and eg.max() <= 1e-1
    if n >= 1000:
        assert ey.mean() <= 1e-4 and np.quantile(ey, 0.99) <= 5e-4
        assert eg.mean() <= 2e-4 and np.quantile(eg, 0.99) <= 5e-3


@pytest.mark.parametrize("L", [1, 4])
def test_lower_bound_vs_oracle(street_small, L):
    """GPU bound and gradient against the FP64 oracle's on the same cut:
    the GPU value is the oracle's lowered by its fp32 allowances (kappa x
    1.0001, then 1e-3 + 1e-5 |LB|); both lie below the exact d^."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.surrogate import lower_bound
    q = synth.uniform_box(4000, [-10.0, -30.0, -5.0], [50.0, 30.0, 25.0], 12)
    for kw, okw in _lb_scenes(street_small):
        for alpha, alpha_u in ((8.0, 0.0), (50.0, 100.0)):
            sd = SmoothDistance(alpha=alpha, alpha_u=alpha_u, beta=0.5, leaf_size=L, device="cuda:0", **kw)
            lb, g, flag = lower_bound(sd, torch.from_numpy(q).cuda(), margin=1.0)
            lb = lb.cpu().numpy().astype(np.float64)
            g = g.cpu().numpy().astype(np.float64)
            sc = oracle.Scene(**okw)
            sc.build_tree(L)
            olb, og, kappa, ncut = sc.lower_bound(q, alpha, alpha_u=alpha_u)
            S = alpha / max(alpha, alpha_u)
            raw = olb - S * np.log(1.0001) / alpha
            expect = raw - (1e-3 + 1e-5 * np.abs(raw))
            assert np.all(np.abs(lb - expect) <= 2e-5 * np.maximum(np.abs(expect), 1.0)), \
                np.abs(lb - expect).max()
            gn = np.linalg.norm(og, axis=1)
            assert np.all(np.linalg.norm(g - og, axis=1) <= 1e-4 * np.maximum(gn, 1e-2))
            exact, _, _ = sc.brute(q, alpha, alpha_u=alpha_u)
            assert np.all(lb <= exact)
            assert np.array_equal(flag.cpu().numpy(), (lb > 1.0).astype(np.int32))


def test_lower_bound_and_barnes_hut(street_small):
    """The Barnes-Hut value also lies below the exact d^ (far fields at the
    nearest box point) and may fall below LB where it takes a far field above
    the cut; LB stays within a few metres of the exact value far away."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.surrogate import lower_bound
    q = synth.uniform_box(4000, [-10.0, -30.0, -5.0], [50.0, 30.0, 25.0], 12)
    for kw, okw in _lb_scenes(street_small)[:2]:
        sd = SmoothDistance(alpha=8.0, beta=0.5, device="cuda:0", **kw)
        lb, _, _ = lower_bound(sd, torch.from_numpy(q).cuda())
        v, _ = sd.query(torch.from_numpy(q).cuda())
        exact, _, _ = oracle.Scene(**okw).brute(q, 8.0)
        assert np.all(v.cpu().numpy() <= exact + 1e-5 * np.maximum(np.abs(exact), 1.0 / 8.0))
        assert np.median(exact - lb.cpu().numpy()) < 3.0


def test_trained_surrogate_routing_and_error(street_small):
    """Train the residual over LB on Barnes-Hut samples of a small street
    where LB > 0.5 m, then answer 1M queries: those with LB > 1 m by LB + the
    network, the rest by the traversal (the same values up to summation
    order); the routed answers must beat LB alone as an estimate."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.surrogate import Surrogate, lower_bound
    P, Vw, Ew = street_small
    sd = SmoothDistance(points=P, edges=(Vw, Ew), alpha=8.0, beta=0.5, device="cuda:0")
    lo = np.minimum(P.min(0), Vw.min(0)) - 5.0
    hi = np.maximum(P.max(0), Vw.max(0)) + 5.0
    xs = torch.from_numpy(synth.uniform_box(2000000, lo, hi, 13)).cuda()
    lbs, _, far = lower_bound(sd, xs, margin=0.5, grad=False)
    xs = xs[far.bool()].contiguous()
    ts, _ = sd.query(xs, grad=False)
    res = ts - lbs[far.bool()]
    sur = Surrogate(lo, hi, sigma=12.0, seed=1, scale=float(res.abs().max()))
    loss0, _ = sur.train_step(xs[:65536], res[:65536].contiguous(), 0.0)
    hist = sur.fit_residual(sd, xs, ts, epochs=3, batch=4096, lr=1e-3)
    assert hist[-1] < 0.1 * loss0.item()
    q = torch.from_numpy(synth.uniform_box(1 << 20, lo, hi, 14)).cuda()
    v_bh, g_bh = sd.query(q)
    v, g, routed, nr = sur.query(sd, q, margin=1.0)
    r = routed.cpu().numpy().astype(bool)
    assert nr == int(r.sum()) and nr > 0.3 * q.shape[0]
    lb, glb, _ = lower_bound(sd, q, margin=1.0)
    assert np.array_equal(r, lb.cpu().numpy() > 1.0)
    vb, vv = v_bh.cpu().numpy(), v.cpu().numpy()
    # queries not routed are the method's answers (the same traversal, run
    # on the gathered subset, so only the summation order differs)
    den = np.maximum(np.abs(vb[~r]), 1.0 / 8.0)
    assert np.all(np.abs(vv[~r] - vb[~r]) <= 1e-5 * den)
    gb_, gg_ = g_bh.cpu().numpy()[~r], g.cpu().numpy()[~r]
    assert np.all(np.linalg.norm(gg_ - gb_, axis=1) <= 1e-4 * np.maximum(np.linalg.norm(gb_, axis=1), 1e-2))
    # routed answers are LB + the network, summed in fp32
    rt = torch.from_numpy(r).cuda()
    ys, dys = sur.forward(q[rt])
    assert torch.equal((ys + lb[rt]).cpu(), v[rt].cpu())
    assert torch.equal((dys + glb[rt]).cpu(), g[rt].cpu())
    err = np.abs(vv[r] - vb[r])
    lbr = lb.cpu().numpy()[r]
    gerr = np.linalg.norm(g.cpu().numpy()[r] - g_bh.cpu().numpy()[r], axis=1)
    print(f"surrogate: routed {nr}/{q.shape[0]}, abs err p50 {np.median(err):.3f} p99 {np.quantile(err, 0.99):.3f} "
          f"max {err.max():.3f} m (LB alone p50 {np.median(vb[r] - lbr):.3f}); grad err p50 {np.median(gerr):.3f}")
    assert np.median(err) < 0.5 * np.median(np.abs(vb[r] - lbr))


def test_surrogate_gain_over_the_method_at_stated_error():
    """What the trained network gains over the method alone, at a stated
    accuracy, on the street workload (2,000,000 lidar points + 50,000 wire
    segments, alpha 50, beta 0.5): trained for 3 epochs on Barnes-Hut values
    of 2M uniform samples of the box padded by 5 m (those with LB > 0.5 m),
    it answers 4M uniform queries of the same box with LB > 1 m routed to
    LB + the network. The routed evaluation must be at least 1.15x faster
    than the traversal alone on the same queries (measured 1.38x with 56 %
    routed) while the routed answers stay within the stated error: 99th
    percentile of |d^ - d^_BH| below 2.5 m and maximum below 8 m (measured
    1.6 m and 4.7 m at this training budget; the benchmark's surrogate leg
    reports longer training and other routing margins)."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.surrogate import Surrogate, lower_bound
    s = synth.config3_scene()
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=50.0, beta=0.5, device="cuda:0")
    lo = np.minimum(s["points"].min(0), s["wire_V"].min(0)) - 5.0
    hi = np.maximum(s["points"].max(0), s["wire_V"].max(0)) + 5.0
    xs = torch.from_numpy(synth.uniform_box(2_000_000, lo, hi, 31)).cuda()
    lbs, _, far = lower_bound(sd, xs, margin=0.5, grad=False)
    xs = xs[far.bool()].contiguous()
    ts, _ = sd.query(xs, grad=False)
    sur = Surrogate(lo, hi, sigma=12.0, seed=1, scale=float((ts - lbs[far.bool()]).abs().max()))
    sur.fit_residual(sd, xs, ts, epochs=3, batch=4096, lr=1e-3)
    q = torch.from_numpy(synth.uniform_box(4 * 1024 * 1024, lo, hi, 32)).cuda()
    vb, gb = torch.empty(q.shape[0], device="cuda"), torch.empty(q.shape[0], 3, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out
    ms_bh, _ = timed(lambda: sd.query(q, out=(vb, gb)))
    ms_sur, (v, g, routed, nr) = timed(lambda: sur.query(sd, q, margin=1.0))
    r = routed.bool()
    err = (v[r] - vb[r]).abs().cpu().numpy()
    p99 = float(np.quantile(err, 0.99))
    print(f"surrogate gain: routed {nr / q.shape[0]:.3f}, traversal {ms_bh:.3f} ms, routed {ms_sur:.3f} ms "
          f"(x{ms_bh / ms_sur:.2f}); routed abs err p50 {np.median(err):.3f} p99 {p99:.3f} max {err.max():.3f} m")
    assert nr > 0.3 * q.shape[0]
    assert p99 < 2.5 and err.max() < 8.0
    assert ms_bh / ms_sur > 1.15


def test_lower_bound_is_certified_at_alpha_1000_on_the_street():
    """The certified bound at the sharpest alpha of the workloads, on the
    street (2,000,000 points + 50,000 wire segments, coordinates up to
    420 m): at 512 queries spread over the box padded by 5 m, the GPU's LB
    (fp32, lowered by its 1e-3 + 1e-5 |LB| allowance) stays at or below the
    FP64 oracle's exact d^ (brute force over every primitive). The
    allowance covers the fp32 rounding bound
    6 u (|q|_inf + d_max) + 70 u / alpha + u |LB| (u = 2^-24), about 2e-4 m
    here."""
    from paper_2108_10480_gb300 import SmoothDistance
    from paper_2108_10480_gb300.surrogate import lower_bound
    s = synth.config3_scene()
    sd = SmoothDistance(points=s["points"], edges=(s["wire_V"], s["wire_E"]), alpha=1000.0, beta=0.5,
                        device="cuda:0")
    lo = np.minimum(s["points"].min(0), s["wire_V"].min(0)) - 5.0
    hi = np.maximum(s["points"].max(0), s["wire_V"].max(0)) + 5.0
    q = synth.uniform_box(512, lo, hi, 41)
    lb, _, _ = lower_bound(sd, torch.from_numpy(q).cuda(), margin=0.0, grad=False)
    lb = lb.cpu().numpy().astype(np.float64)
    exact, _, _ = oracle.Scene(points=s["points"], edge_V=s["wire_V"], edge_E=s["wire_E"]).brute(q, 1000.0)
    assert np.all(lb <= exact), (lb - exact).max()
    assert np.median(exact - lb) < 20.0     # a bound, not a vacuous one
