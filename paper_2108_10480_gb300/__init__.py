"""Smooth distance constraints on co-dimensional geometry, on one GB300.

Python binding of libsd (include/sd.h): torch tensors supply device memory
and streams; the work runs in the library's CUDA kernels.

    sd = SmoothDistance(points=P, edges=(V, E), tris=(V, F), alpha=100, beta=0.5)
    value, grad = sd.query(q)          # Eq. 3 / Eq. 4 with Barnes-Hut (Alg. 1-2)
    value, grad = sd.query_brute(q)    # the plain all-pairs method
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import SdError

__all__ = ["SmoothDistance", "SdError", "lib", "weight_basis", "kernel_launches"]


def lib():
    return _native.lib()


def mesh_reduce(F, nverts, value, grad, alpha_q, stream=None):
    """Smooth distance to a query mesh and its per-vertex gradient
    (sd_mesh_reduce) from query_prims' outputs: (D [1], vgrad [nverts, 3])."""
    F = F.to(torch.int32).contiguous()
    m, k = F.shape
    out = torch.empty(1, device=F.device)
    vg = torch.empty(int(nverts), 3, device=F.device)
    rc = lib().sd_mesh_reduce(_ptr(F), int(k), m, int(nverts), _ptr(value), _ptr(grad), float(alpha_q), _ptr(out),
                              _ptr(vg), None, _stream_handle(stream))
    _native.check(rc, "sd_mesh_reduce")
    return out, vg


def kernel_launches() -> int:
    """CUDA kernels libsd has launched in this process."""
    return int(lib().sd_kernel_launches())


def weight_basis() -> np.ndarray:
    """The library's App. C.3 triangle weight basis in Bernstein form
    ([3, 36] float64; host-only, no GPU needed)."""
    out = np.zeros(108, np.float64)
    _native.check(lib().sd_weight_basis(ctypes.c_void_p(out.ctypes.data)), "sd_weight_basis")
    return out.reshape(3, 36)


def _dev_f32(x, device, k=3):
    if x is None:
        return None
    t = torch.as_tensor(x)
    t = t.to(device=device, dtype=torch.float32).reshape(-1, k).contiguous()
    return t


def _dev_i32(x, device, k):
    if x is None:
        return None
    t = torch.as_tensor(x)
    return t.to(device=device, dtype=torch.int32).reshape(-1, k).contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class SmoothDistance:
    """A built acceleration structure over a data mesh (points, an edge mesh
    and/or a triangle mesh) for fixed alpha and beta (sd_build)."""

    def __init__(self, points=None, edges=None, tris=None, alpha=100.0, beta=0.5, alpha_u=0.0,
                 leaf_size=1, weights="paper", paper_metric=False, device=None, stream=None, check=True):
        """check=True: the build waits for the device and raises on invalid
        input; check=False: it only enqueues the work (same kernels) and
        invalid input is reported by status()."""
        L = lib()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            pts = _dev_f32(points, self.device)
            eV = eE = tV = tF = None
            if edges is not None:
                eV, eE = _dev_f32(edges[0], self.device), _dev_i32(edges[1], self.device, 2)
            if tris is not None:
                tV, tF = _dev_f32(tris[0], self.device), _dev_i32(tris[1], self.device, 3)
            g = _native.SdGeometry()
            g.pts = _native.SdPoints(_ptr(pts), 0 if pts is None else pts.shape[0])
            g.edges = _native.SdEdges(_ptr(eV), 0 if eV is None else eV.shape[0], _ptr(eE), 0 if eE is None else eE.shape[0])
            g.tris = _native.SdTris(_ptr(tV), 0 if tV is None else tV.shape[0], _ptr(tF), 0 if tF is None else tF.shape[0])
            o = _native.SdBuildOpts()
            L.sd_default_build_opts(ctypes.byref(o))
            o.alpha_u = float(alpha_u)
            o.leaf_size = int(leaf_size)
            o.weights = 1 if weights == "unit" else 0
            o.paper_metric = 1 if paper_metric else 0
            o.defer_checks = 0 if check else 1
            h = ctypes.c_void_p()
            rc = L.sd_build(ctypes.byref(g), float(alpha), float(beta), ctypes.byref(o), _stream_handle(stream),
                            ctypes.byref(h))
            _native.check(rc, "sd_build")
            self._h = h
            self.alpha, self.beta = float(alpha), float(beta)
            self.leaf_size = int(leaf_size)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _native._lib is not None:
            _native._lib.sd_free(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = _native.SdTreeInfo()
        _native.check(lib().sd_tree_get_info(self._h, ctypes.byref(i)), "sd_tree_get_info")
        d = {k: getattr(i, k) for k, _ in _native.SdTreeInfo._fields_}
        d["scene_lo"] = list(i.scene_lo)
        d["scene_hi"] = list(i.scene_hi)
        return d

    def _run(self, fn, q, grad, sort, counts, block, stream, out, order=None):
        q = _dev_f32(q, self.device)
        M = q.shape[0]
        if out is None:
            value = torch.empty(M, device=self.device, dtype=torch.float32)
            g = torch.empty(M, 3, device=self.device, dtype=torch.float32) if grad else None
        else:
            value, g = out
        cnt = torch.zeros(M, 3, device=self.device, dtype=torch.int32) if counts else None
        o = _native.SdQueryOpts()
        lib().sd_default_query_opts(ctypes.byref(o))
        o.sort_queries = 1 if sort else 0
        o.block = int(block)
        o.counts = _ptr(cnt) if cnt is not None else None
        o.order = _ptr(order) if order is not None else None
        rc = fn(self._h, _ptr(q), M, _ptr(value), _ptr(g) if g is not None else None, ctypes.byref(o),
                _stream_handle(stream))
        _native.check(rc, fn.__name__)
        res = (value, g)
        if counts:
            res = res + (cnt,)
        return res

    def query(self, q, grad=True, sort=True, counts=False, block=0, stream=None, out=None, order=None):
        """Barnes-Hut d^ and grad d^ at queries q [M,3] (sd_query). Returns
        (value [M], grad [M,3] or None[, counts [M,3] int32]). `order` is an
        optional int32 device permutation from query_order()."""
        return self._run(lib().sd_query, q, grad, sort, counts, block, stream, out, order)

    def query_order(self, q, stream=None, out=None):
        """Hilbert traversal order of the queries (sd_query_order)."""
        q = _dev_f32(q, self.device)
        order = out if out is not None else torch.empty(q.shape[0], device=self.device, dtype=torch.int32)
        _native.check(lib().sd_query_order(self._h, _ptr(q), q.shape[0], _ptr(order), _stream_handle(stream)),
                      "sd_query_order")
        return order

    def query_brute(self, q, grad=True, stream=None, out=None):
        """Plain all-pairs d^ and grad d^ (sd_query_brute)."""
        return self._run(lib().sd_query_brute, q, grad, False, False, 0, stream, out)

    def query_prims(self, V, F, sort=True, counts=False, block=0, stream=None, out=None, order=None):
        """Smooth distance of edge (F [m,2]) or triangle (F [m,3]) queries over
        vertices V [n,3] (sd_query_prims): value [m] and the gradient [m,3]
        for a rigid translation of each primitive (plus work counts)."""
        V = _dev_f32(V, self.device)
        F = torch.as_tensor(F).to(device=self.device, dtype=torch.int32)
        F = F.reshape(F.shape[0], -1).contiguous()
        m, k = F.shape
        val, grad = out if out is not None else (torch.empty(m, device=self.device),
                                                 torch.empty(m, 3, device=self.device))
        cnt = torch.empty(m, 3, dtype=torch.int32, device=self.device) if counts else None
        o = _native.SdQueryOpts()
        lib().sd_default_query_opts(ctypes.byref(o))
        o.sort_queries = 1 if sort else 0
        o.block = int(block)
        o.counts = _ptr(cnt)
        o.order = _ptr(order)
        rc = lib().sd_query_prims(self._h, _ptr(V), V.shape[0], _ptr(F), int(k), m, _ptr(val), _ptr(grad),
                                  ctypes.byref(o), _stream_handle(stream))
        _native.check(rc, "sd_query_prims")
        return (val, grad, cnt) if counts else (val, grad)

    def sphere_trace(self, cam, eps=1e-5, t_max=1.0, max_steps=256, block=0, stream=None):
        """Sphere-traced depth image of the zero isosurface (sd_sphere_trace).
        cam: dict(eye, target, up, fov_y, width, height). Returns depth [H, W]
        (+inf for misses), evaluations per ray [H, W] and their total."""
        o = _native.SdTraceOpts()
        for name in ("eye", "target", "up"):
            getattr(o, name)[:] = [float(x) for x in cam[name]]
        o.fov_y = float(cam["fov_y"])
        o.width, o.height = int(cam["width"]), int(cam["height"])
        o.eps, o.t_max, o.max_steps, o.block = float(eps), float(t_max), int(max_steps), int(block)
        H, W = o.height, o.width
        depth = torch.empty(H, W, device=self.device)
        steps = torch.empty(H, W, dtype=torch.int32, device=self.device)
        ev = ctypes.c_int64(0)
        rc = lib().sd_sphere_trace(self._h, ctypes.byref(o), _ptr(depth), _ptr(steps), ctypes.byref(ev),
                                   _stream_handle(stream))
        _native.check(rc, "sd_sphere_trace")
        return depth, steps, int(ev.value)

    def status(self, stream=None) -> int:
        """Synchronise and return (then clear) the device status word."""
        return lib().sd_query_status(self._h, _stream_handle(stream))

    def export(self) -> dict:
        """Host copies of the build results (sd_tree_export)."""
        i = self.info()
        n, nb = i["n_prims"], i["n_buckets"]
        ni = max(nb - 1, 0)
        t = dict(codes=np.zeros(n, np.uint64), sorted=np.zeros(n, np.int32), left=np.zeros(ni, np.int32),
                 right=np.zeros(ni, np.int32), node_lo=np.zeros((ni, 3), np.float32),
                 node_hi=np.zeros((ni, 3), np.float32), node_count=np.zeros(ni, np.int32),
                 leaf_lo=np.zeros((nb, 3), np.float32), leaf_hi=np.zeros((nb, 3), np.float32),
                 leaf_count=np.zeros(nb, np.int32), params=np.zeros((n, 2), np.float32))
        v = _native.SdTreeView(*[ctypes.c_void_p(t[k].ctypes.data) if t[k].size else None
                                 for k, _ in _native.SdTreeView._fields_])
        _native.check(lib().sd_tree_export(self._h, ctypes.byref(v)), "sd_tree_export")
        t["nb"] = nb
        return t


from . import pose  # noqa: E402,F401  (rigid-body constraint and its adjoint)
