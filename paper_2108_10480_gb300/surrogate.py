"""Learned far-field surrogate behind a certified lower bound.

    sur = Surrogate(lo, hi)                       # scene box (already padded)
    sur.fit_residual(sd, x, target, epochs=3)     # libsd training kernels + Adam
    value, grad, routed, n = sur.query(sd, q, margin=1.0)

A query whose certified lower bound LB (sd_lower_bound) exceeds `margin` is
answered by LB plus the network, every other by the Barnes-Hut evaluation,
so the constraint is never approximated near contact. The network models
the residual d^ - LB, which is small and smooth where LB > margin (outside
every cut box LB is a LogSumExp of distances to convex sets, continuously
differentiable). The forward pass, gradients, optimiser step, bound and
routing all run in libsd's kernels; this module initialises parameters,
shuffles batches and marshals calls.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _native, lib
from . import _ptr, _stream_handle

NF, HID, NIN = 32, 128, 67


def num_params() -> int:
    return int(lib().sd_mlp_num_params())


def init_params(seed=0, sigma=16.0):
    """Gaussian Fourier frequencies N(0, sigma^2); layer weights with
    variance 1/fan_in; zero biases (host RNG, uploaded once)."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((NF, 3)) * sigma,
             rng.standard_normal((HID, NIN)) / math.sqrt(NIN), np.zeros(HID),
             rng.standard_normal((HID, HID)) / math.sqrt(HID), np.zeros(HID),
             rng.standard_normal((HID, HID)) / math.sqrt(HID), np.zeros(HID),
             rng.standard_normal(HID) / math.sqrt(HID), np.zeros(1)]
    p = np.concatenate([a.ravel() for a in parts]).astype(np.float32)
    assert p.size == num_params()
    return p


class Surrogate:
    def __init__(self, lo, hi, sigma=16.0, seed=0, scale=10.0, isotropic=True, device="cuda"):
        """Box [lo, hi] mapped to xh in [-1, 1] per axis, or (isotropic) by
        the largest half extent on every axis so that the Fourier
        frequencies keep one physical scale."""
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        c = 0.5 * (lo + hi)
        h = 0.5 * (hi - lo)
        if isotropic:
            h = np.full(3, h.max())
        self.frame = np.array([c[0], c[1], c[2], h[0], h[1], h[2], scale], np.float32)
        self.device = torch.device(device)
        self.params = torch.from_numpy(init_params(seed, sigma)).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._ws = None

    def _frame_ptr(self):
        return ctypes.c_void_p(self.frame.ctypes.data)

    def train_step(self, x, t, lr, grad_out=None, loss_out=None, stream=None):
        n = x.shape[0]
        need = int(lib().sd_mlp_workspace_bytes(n))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        g = grad_out if grad_out is not None else torch.empty_like(self.params)
        loss = loss_out if loss_out is not None else torch.empty(1, device=self.device)
        if lr > 0:
            self.step += 1
        rc = lib().sd_mlp_train_step(_ptr(self.params), _ptr(self.m), _ptr(self.v), max(self.step, 1), float(lr),
                                     self._frame_ptr(), _ptr(x), _ptr(t), n, _ptr(loss), _ptr(g),
                                     _ptr(self._ws), self._ws.numel(), _stream_handle(stream))
        _native.check(rc, "sd_mlp_train_step")
        return loss, g

    def fit(self, x, t, epochs=4, batch=16384, lr=2e-3, lr_end=1e-4, seed=0):
        """Adam on mean squared error, cosine-decayed learning rate; returns
        the loss of the last batch of every epoch."""
        x = x.to(self.device, torch.float32).contiguous()
        t = t.to(self.device, torch.float32).contiguous()
        n = x.shape[0]
        steps_per_epoch = max(1, n // batch)
        total = epochs * steps_per_epoch
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        xb = torch.empty(batch, 3, device=self.device)
        tb = torch.empty(batch, device=self.device)
        g = torch.empty_like(self.params)
        loss = torch.empty(1, device=self.device)
        hist = []
        k = 0
        for ep in range(epochs):
            perm = torch.randperm(n, device=self.device, generator=gen)
            for s in range(steps_per_epoch):
                idx = perm[s * batch:(s + 1) * batch]
                torch.index_select(x, 0, idx, out=xb)
                torch.index_select(t, 0, idx, out=tb)
                a = k / max(1, total - 1)
                lr_k = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * a))
                self.train_step(xb, tb, lr_k, grad_out=g, loss_out=loss)
                k += 1
            hist.append(float(loss.item()))
        return hist

    def fit_residual(self, sd, x, t, **kw):
        """fit() on the residual t - LB(x) (the network's target in routed
        queries)."""
        lb, _, _ = lower_bound(sd, x, grad=False)
        return self.fit(x, t - lb, **kw)

    def forward(self, x, grad=True, stream=None):
        x = x.to(self.device, torch.float32).contiguous()
        n = x.shape[0]
        y = torch.empty(n, device=self.device)
        dy = torch.empty(n, 3, device=self.device) if grad else None
        rc = lib().sd_mlp_forward(_ptr(self.params), self._frame_ptr(), _ptr(x), n, _ptr(y),
                                  _ptr(dy) if dy is not None else None, _stream_handle(stream))
        _native.check(rc, "sd_mlp_forward")
        return y, dy

    def query(self, sd, q, margin=1.0, grad=True, stream=None):
        q = q.to(self.device, torch.float32).contiguous()
        M = q.shape[0]
        value = torch.empty(M, device=self.device)
        g = torch.empty(M, 3, device=self.device) if grad else None
        routed = torch.empty(M, device=self.device, dtype=torch.int32)
        nr = ctypes.c_int64(0)
        rc = lib().sd_surrogate_query(sd.handle, _ptr(self.params), self._frame_ptr(), float(margin), _ptr(q), M,
                                      _ptr(value), _ptr(g) if g is not None else None, _ptr(routed),
                                      ctypes.byref(nr), _stream_handle(stream))
        _native.check(rc, "sd_surrogate_query")
        return value, g, routed, int(nr.value)


def lower_bound(sd, q, margin=1.0, grad=True, stream=None):
    """Certified lower bound of d^ per query, its gradient and the routing
    flags (LB > margin)."""
    q = q.contiguous()
    M = q.shape[0]
    lb = torch.empty(M, device=q.device)
    g = torch.empty(M, 3, device=q.device) if grad else None
    flag = torch.empty(M, device=q.device, dtype=torch.int32)
    rc = lib().sd_lower_bound(sd.handle, _ptr(q), M, float(margin), _ptr(lb), _ptr(g) if g is not None else None,
                              _ptr(flag), _stream_handle(stream))
    _native.check(rc, "sd_lower_bound")
    return lb, g, flag
