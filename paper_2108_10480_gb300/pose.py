"""Rigid-body smooth-distance constraint and its pose adjoint (Sec. 4.5,
Eq. opt; Sec. 3.6, Eq. lse_full2 / Eq. dlse_full for point queries).

    D = SmoothDistancePose.apply(pose, X0, sd, alpha_q)   # scalar constraint
    D.backward()                                           # pose.grad, X0.grad

`pose` is a 6-vector (rotation vector theta, translation p); X0 the body's
rest vertices [M,3] on the device. Forward runs sd_pose_query (placement +
Barnes-Hut query) and sd_pose_reduce (outer LogSumExp, pose gradient);
backward scales the saved gradients. With alpha_q = None the function
returns the per-vertex d^ [M] and backward reduces the upstream gradient
with sd_pose_reduce. All arithmetic runs in libsd's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native, lib
from . import _dev_f32, _ptr, _stream_handle


def _pose_array(pose):
    p = np.ascontiguousarray(torch.as_tensor(pose).detach().cpu().to(torch.float64).numpy().reshape(6))
    return p


def pose_query(sd, X0, pose, stream=None):
    """Place X0 at `pose` and query: returns (X, value, grad)."""
    X0 = _dev_f32(X0, sd.device)
    M = X0.shape[0]
    X = torch.empty_like(X0)
    value = torch.empty(M, device=sd.device, dtype=torch.float32)
    grad = torch.empty(M, 3, device=sd.device, dtype=torch.float32)
    pa = _pose_array(pose)
    rc = lib().sd_pose_query(sd.handle, _ptr(X0), M, ctypes.c_void_p(pa.ctypes.data), _ptr(X), _ptr(value),
                             _ptr(grad), None, _stream_handle(stream))
    _native.check(rc, "sd_pose_query")
    return X, value, grad


def pose_reduce(X0, value, grad, pose, alpha_q=None, gamma=None, want_dx0=False, stream=None):
    """Outer LogSumExp (alpha_q > 0) or gamma-weighted sum over vertices and
    the pose adjoint: returns (out[7] = D, dD/dtheta, dD/dp reordered as
    (D, dtheta(3), dp(3)), dX0 or None)."""
    M = value.shape[0]
    out = torch.empty(7, device=value.device, dtype=torch.float32)
    dX0 = torch.empty(M, 3, device=value.device, dtype=torch.float32) if want_dx0 else None
    pa = _pose_array(pose)
    aq = float(alpha_q) if alpha_q else 0.0
    g = gamma.contiguous().to(torch.float32) if gamma is not None else None
    rc = lib().sd_pose_reduce(_ptr(X0), _ptr(value), _ptr(grad), _ptr(g) if g is not None else None, M,
                              ctypes.c_void_p(pa.ctypes.data), aq, _ptr(out), _ptr(dX0) if dX0 is not None else None,
                              _stream_handle(stream))
    _native.check(rc, "sd_pose_reduce")
    # library order: (D, dD/dp, dD/dtheta) -> (D, dD/dtheta, dD/dp) to match pose = (theta, p)
    res = torch.cat([out[:1], out[4:7], out[1:4]])
    return res, dX0


def pose_partial(X0, value, grad, pose, alpha_q=None, gamma=None, stream=None):
    """This shard's partial of the outer reduction (sd_pose_partial): device
    float32 [9] = (m, s, v, gp (3), gt (3)) over the given vertices."""
    M = value.shape[0]
    part = torch.empty(9, device=value.device, dtype=torch.float32)
    pa = _pose_array(pose)
    aq = float(alpha_q) if alpha_q else 0.0
    g = gamma.contiguous().to(torch.float32) if gamma is not None else None
    rc = lib().sd_pose_partial(_ptr(X0), _ptr(value), _ptr(grad), _ptr(g) if g is not None else None, M,
                               ctypes.c_void_p(pa.ctypes.data), aq, _ptr(part), _stream_handle(stream))
    _native.check(rc, "sd_pose_partial")
    return part


def merge_partials(parts, pose, alpha_q=None):
    """Merge shard partials (host [n, 9], any order) with the library's
    host-only sd_pose_merge: float64 (D, dD/dtheta (3), dD/dp (3)), the pose
    order of pose_reduce."""
    P = np.ascontiguousarray(np.asarray(parts, np.float64).reshape(-1, 9))
    pa = _pose_array(pose)
    out = np.zeros(7, np.float64)
    aq = float(alpha_q) if alpha_q else 0.0
    rc = lib().sd_pose_merge(ctypes.c_void_p(P.ctypes.data), int(P.shape[0]), ctypes.c_void_p(pa.ctypes.data), aq,
                             ctypes.c_void_p(out.ctypes.data))
    _native.check(rc, "sd_pose_merge")
    return np.concatenate([out[:1], out[4:7], out[1:4]])


def reduce_shards(part, pose, alpha_q=None, group=None):
    """The body's reduction when its vertices are split over the ranks of a
    torch.distributed group: every rank's 9-float partial is all-gathered
    (the one exchange of the split) and merged on the host by
    sd_pose_merge. Without an initialised process group the partial is
    merged alone."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        parts = [torch.empty_like(part) for _ in range(dist.get_world_size(group))]
        dist.all_gather(parts, part, group=group)
        host = torch.stack(parts).double().cpu().numpy()
    else:
        host = part.double().cpu().numpy()[None]
    return merge_partials(host, pose, alpha_q)


class SmoothDistancePose(torch.autograd.Function):
    """d^ of a rigid body against a built data mesh, differentiable in the
    6-DoF pose and the rest vertices."""

    @staticmethod
    def forward(ctx, pose, X0, sd, alpha_q=None):
        X0c = _dev_f32(X0, sd.device)
        X, value, grad = pose_query(sd, X0c, pose)
        ctx.sd, ctx.alpha_q = sd, alpha_q
        ctx.pose_dtype, ctx.pose_device = pose.dtype, pose.device
        if alpha_q:
            res, dX0 = pose_reduce(X0c, value, grad, pose, alpha_q=alpha_q, want_dx0=X0.requires_grad)
            ctx.save_for_backward(res, dX0 if dX0 is not None else torch.empty(0))
            ctx.scalar = True
            return res[0].clone()
        ctx.save_for_backward(X0c, value, grad, _pose_tensor(pose))
        ctx.scalar = False
        return value

    @staticmethod
    def backward(ctx, gout):
        if ctx.scalar:
            res, dX0 = ctx.saved_tensors
            gp = (res[1:7] * gout).to(device=ctx.pose_device, dtype=ctx.pose_dtype)
            gx = dX0 * gout if dX0.numel() else None
            return gp, gx, None, None
        X0c, value, grad, pose = ctx.saved_tensors
        res, dX0 = pose_reduce(X0c, value, grad, pose, gamma=gout.contiguous(), want_dx0=ctx.needs_input_grad[1])
        gp = res[1:7].to(device=ctx.pose_device, dtype=ctx.pose_dtype)
        return gp, dX0, None, None


def _pose_tensor(pose):
    return torch.as_tensor(pose).detach().to(torch.float64).reshape(6).cpu()
