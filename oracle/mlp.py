"""Fourier-feature MLP of the learned far-field surrogate, in FP64 numpy.

TEST INFRASTRUCTURE (see oracle/__init__.py): the reference for the GPU
surrogate's forward pass, its input gradient and its parameter gradients.

Network (the surrogate's definition):
  xh   = (x - c) / h                     box centre c, half extents h (per axis)
  f    = [xh, sin(pi B xh), cos(pi B xh)]  B: [32, 3] frequencies -> 67 features
  z1 = W1 f + b1,  a1 = silu(z1)          W1: [128, 67]
  z2 = W2 a1 + b2, a2 = silu(z2)          W2: [128, 128]
  z3 = W3 a2 + b3, a3 = silu(z3)          W3: [128, 128]
  y  = s * (w4 . a3 + b4)                 w4: [128], output scale s
silu(z) = z / (1 + exp(-z)). Loss for a batch: mean (y - t)^2.
Parameters flattened in this order: B, W1, b1, W2, b2, W3, b3, w4, b4.
"""
from __future__ import annotations

import numpy as np

NF, H, NIN = 32, 128, 67
SHAPES = [("B", (NF, 3)), ("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
          ("W3", (H, H)), ("b3", (H,)), ("w4", (H,)), ("b4", (1,))]
NPARAMS = int(sum(np.prod(s) for _, s in SHAPES))


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def init(seed=0, sigma=8.0):
    """Gaussian Fourier frequencies N(0, sigma^2); layers with variance
    1/fan_in; zero biases."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((NF, 3)) * sigma,
             rng.standard_normal((H, NIN)) / np.sqrt(NIN), np.zeros(H),
             rng.standard_normal((H, H)) / np.sqrt(H), np.zeros(H),
             rng.standard_normal((H, H)) / np.sqrt(H), np.zeros(H),
             rng.standard_normal(H) / np.sqrt(H), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, c, h, s, bf16=False, mixed=False):
    """Returns y [n], dy/dx [n, 3] and the cache for backward. bf16=True
    rounds the four weight matrices to bfloat16 first (the GPU's weights).
    mixed=True (implies bf16) also stores every GEMM operand the way the
    tensor-core inference does: the features, a1, a2 and the three
    back-propagated factors rounded to bfloat16, dsilu(z1), dsilu(z2) to
    binary16; sums, biases, a3 and the output stay exact."""
    bf16 = bf16 or mixed
    p = unpack(theta)
    if bf16:
        for k in ("W1", "W2", "W3", "w4"):
            p[k] = round_bf16(p[k])
    rb = round_bf16 if mixed else (lambda a: a)
    rh = (lambda a: np.asarray(a, np.float16).astype(np.float64)) if mixed else (lambda a: a)
    x = np.asarray(x, np.float64)
    xh = (x - c) / h
    ph = np.pi * xh @ p["B"].T
    f = np.concatenate([xh, np.sin(ph), np.cos(ph)], axis=1)
    z1 = rb(f) @ p["W1"].T + p["b1"]; a1 = silu(z1)
    z2 = rb(a1) @ p["W2"].T + p["b2"]; a2 = silu(z2)
    z3 = rb(a2) @ p["W3"].T + p["b3"]; a3 = silu(z3)
    y = s * (a3 @ p["w4"] + p["b4"][0])
    # input gradient: back through the layers to the features, then xh, x
    g3 = rb(s * p["w4"] * dsilu(z3))
    g2 = rb((g3 @ p["W3"]) * rh(dsilu(z2)))
    g1 = rb((g2 @ p["W2"]) * rh(dsilu(z1)))
    gf = g1 @ p["W1"]
    gxh = gf[:, :3] + (np.cos(ph) * gf[:, 3:3 + NF]) @ (np.pi * p["B"]) \
        - (np.sin(ph) * gf[:, 3 + NF:]) @ (np.pi * p["B"])
    dx = gxh / h
    cache = dict(p=p, xh=xh, ph=ph, f=f, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, s=s)
    return y, dx, cache


def loss_and_grad(theta, x, t, c, h, s, bf16=False):
    """Mean squared error and its gradient with respect to every parameter
    except the (fixed) Fourier frequencies, whose gradient entries are 0."""
    y, _, C = forward(theta, x, c, h, s, bf16)
    n = y.shape[0]
    r = y - np.asarray(t, np.float64)
    L = float((r * r).mean())
    dy = 2.0 * r / n
    p = C["p"]
    g = {"B": np.zeros_like(p["B"])}
    g["b4"] = np.array([s * dy.sum()])
    g["w4"] = s * C["a3"].T @ dy
    d3 = (s * dy[:, None] * p["w4"][None, :]) * dsilu(C["z3"])
    g["W3"] = d3.T @ C["a2"]; g["b3"] = d3.sum(0)
    d2 = (d3 @ p["W3"]) * dsilu(C["z2"])
    g["W2"] = d2.T @ C["a1"]; g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"]) * dsilu(C["z1"])
    g["W1"] = d1.T @ C["f"]; g["b1"] = d1.sum(0)
    return L, np.concatenate([g[name].ravel() for name, _ in SHAPES])


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, skip=NF * 3):
    """One Adam step (Kingma & Ba) on every parameter but the frequencies."""
    theta = np.asarray(theta, np.float64).copy()
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    upd = lr * mh / (np.sqrt(vh) + eps)
    upd[:skip] = 0.0
    return theta - upd, m, v


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32).view(np.float32)).astype(np.float64).reshape(np.shape(a))
