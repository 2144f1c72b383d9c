"""FP64 CPU oracle for the smooth distance of Madan & Levin (Eq. 3, Eq. 4,
Alg. 1, Alg. 2, App. B-D).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package. The CUDA library in
``paper_2108_10480_gb300`` shares no code with it: no kernels, headers,
tables or constant generators. The two meet only in the seeded input
generators of ``synth``.

Layout:
  weights.py     weight-polynomial bases solved from App. C (numpy)
  sd_oracle.c    distances, weights, LSE, Morton/radix tree, Barnes-Hut (C, FP64)
  pose.py        rigid pose map, outer LSE and pose gradient (numpy, FP64)
  mlp.py         Fourier-feature MLP forward/backward (numpy, FP64)

Every function is pinned by tests/test_oracle_*.py: the triangle weight
everywhere by an exact rational minimum-norm solve of App. C.3, the
``paper_metric`` (alpha-scaled barycentric gradient) variant by its defining
relation to the exact gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import weights

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_SRC = os.path.join(_HERE, "sd_oracle.c")
_lock = threading.Lock()
_lib = None

K_POINT, K_SEG, K_TRI = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile sd_oracle.c into _build/liboracle.so with gcc (no FMA
    contraction, so the FP32 Morton codes and Barnes-Hut decisions follow the
    written operation order exactly)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        i = ctypes.c_int
        lib.orc_scene_new.restype = P
        lib.orc_scene_new.argtypes = [P, i64, P, i64, P, i64, P, i64, P, i64, P, P]
        lib.orc_scene_free.argtypes = [P]
        lib.orc_scene_info.argtypes = [P, P]
        lib.orc_prim_params.argtypes = [P, P, P, P]
        lib.orc_prim_eval.argtypes = [P, i64, d, d, i, P, P]
        lib.orc_brute.argtypes = [P, d, d, i, i, P, i64, P, P, P, i]
        lib.orc_tree_build.argtypes = [P, i]
        lib.orc_tree_build.restype = i
        lib.orc_tree_nb.argtypes = [P]
        lib.orc_tree_nb.restype = i64
        lib.orc_tree_export.argtypes = [P] * 12
        lib.orc_bh.argtypes = [P, d, d, d, i, i, i, P, i64, P, P, P, P, i]
        lib.orc_bh.restype = i
        lib.orc_pose_f32.argtypes = [P, P, P, i64, P]
        lib.orc_lower_bound.argtypes = [P, d, d, i, P, i64, P, P, P]
        lib.orc_lower_bound.restype = i
        lib.orc_prim_kappa.argtypes = [P, P]
        lib.orc_simplex_closest.argtypes = [P, i, P, i, P, P]
        lib.orc_simplex_closest.restype = d
        lib.orc_brute_prims.argtypes = [P, d, d, i, i, P, P, i, i64, P, P, P, i]
        lib.orc_bh_prims.argtypes = [P, d, d, d, i, i, i, P, P, i, i64, P, P, P, P, i]
        lib.orc_bh_prims.restype = i
        _lib = lib
        return lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def simplex_closest(A, B):
    """Distance and closest points of two simplices (1-3 vertices each)."""
    A = np.ascontiguousarray(np.asarray(A, np.float64).reshape(-1, 3))
    B = np.ascontiguousarray(np.asarray(B, np.float64).reshape(-1, 3))
    pa = np.zeros(3); pb = np.zeros(3)
    d = _load().orc_simplex_closest(_ptr(A), A.shape[0], _ptr(B), B.shape[0], _ptr(pa), _ptr(pb))
    return d, pa, pb


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


class Scene:
    """A data mesh M_d = (V, F) holding points, an edge mesh and a triangle
    mesh (any of them may be empty). Primitive order: points, edges,
    triangles. Vertices are fp32 (as the GPU receives them) promoted exactly
    to FP64."""

    def __init__(self, points=None, edge_V=None, edge_E=None, tri_V=None, tri_F=None):
        lib = _load()
        f32 = lambda a: np.ascontiguousarray(np.zeros((0, 3), np.float32) if a is None else np.asarray(a, np.float32).reshape(-1, 3))
        i32 = lambda a, k: np.ascontiguousarray(np.zeros((0, k), np.int32) if a is None else np.asarray(a, np.int32).reshape(-1, k))
        self.points = f32(points)
        self.edge_V, self.edge_E = f32(edge_V), i32(edge_E, 2)
        self.tri_V, self.tri_F = f32(tri_V), i32(tri_F, 3)
        # a vertex array without primitives does not belong to the data mesh
        if self.edge_E.shape[0] == 0:
            self.edge_V = f32(None)
        if self.tri_F.shape[0] == 0:
            self.tri_V = f32(None)
        self.ebasis = np.ascontiguousarray(weights.edge_basis(), dtype=np.float64)
        self.tbasis = np.ascontiguousarray(weights.tri_basis(), dtype=np.float64)
        self._h = lib.orc_scene_new(
            _ptr(self.points), self.points.shape[0],
            _ptr(self.edge_V), self.edge_V.shape[0], _ptr(self.edge_E), self.edge_E.shape[0],
            _ptr(self.tri_V), self.tri_V.shape[0], _ptr(self.tri_F), self.tri_F.shape[0],
            _ptr(self.ebasis), _ptr(self.tbasis))
        info = np.zeros(6)
        lib.orc_scene_info(self._h, _ptr(info))
        self.A_E, self.A_T = float(info[0]), float(info[1])
        self.n = int(info[2])
        self.L = None

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_scene_free(self._h)
            self._h = None

    # -- per-primitive data ------------------------------------------------
    def prim_params(self):
        """(params [n,2], kind [n], isolated [n]): segment (u, v), triangle
        (1/v_i, 1/e_i)."""
        out = np.zeros((self.n, 2))
        kind = np.zeros(self.n, np.int32)
        iso = np.zeros(self.n, np.int32)
        _load().orc_prim_params(self._h, _ptr(out), _ptr(kind), _ptr(iso))
        return out, kind, iso

    def prim_kappa(self):
        """[n, 4]: largest Bernstein coefficient of each primitive's w~ and
        its corner coefficients (x = 0, x = 1, y = 1; NaN where absent)."""
        out = np.zeros((self.n, 4))
        _load().orc_prim_kappa(self._h, _ptr(out))
        return out

    def prim_eval(self, i, q, alpha=100.0, alpha_u=0.0, paper_metric=False):
        """One primitive at one FP64 query: dict(d, grad_d, phi, wt, grad_wt,
        t, vec) where t = ln w - alpha d and vec = grad d - grad(w)/(alpha w)."""
        q = np.ascontiguousarray(q, np.float64)
        out = np.zeros(14)
        _load().orc_prim_eval(self._h, int(i), float(alpha), float(alpha_u), int(bool(paper_metric)), _ptr(q), _ptr(out))
        return dict(d=out[0], grad_d=out[1:4].copy(), phi=out[4:6].copy(), wt=out[6],
                    grad_wt=out[7:10].copy(), t=out[10], vec=out[11:14].copy())

    # -- brute force ---------------------------------------------------------
    def brute(self, q, alpha, alpha_u=0.0, paper_metric=False, threads=None, unit=False):
        """Exact d^ and grad d^ over every primitive (Eq. 3, Eq. 4) plus the
        exact minimum distance d_min (Eq. 2). q: [m,3] (promoted to FP64).
        unit=True sets every weight to 1 (the plain LogSumExp)."""
        q = np.ascontiguousarray(np.asarray(q, np.float64).reshape(-1, 3))
        m = q.shape[0]
        val = np.zeros(m); grad = np.zeros((m, 3)); dmin = np.zeros(m)
        _load().orc_brute(self._h, float(alpha), float(alpha_u), int(bool(paper_metric)), int(bool(unit)), _ptr(q), m,
                          _ptr(val), _ptr(grad), _ptr(dmin), int(threads or default_threads()))
        return val, grad, dmin

    # -- tree and Barnes-Hut --------------------------------------------------
    def build_tree(self, leaf_size=1):
        rc = _load().orc_tree_build(self._h, int(leaf_size))
        if rc != 0:
            raise ValueError("leaf_size must be >= 1")
        self.L = int(leaf_size)
        return self.tree()

    def tree(self):
        """Morton codes (original order), sorted primitive order, Karras-
        numbered children (leaf child = -(bucket + 1)), internal and leaf
        AABBs and primitive counts, scene AABB."""
        lib = _load()
        nb = int(lib.orc_tree_nb(self._h))
        ni = max(nb - 1, 0)
        t = dict(codes=np.zeros(self.n, np.uint64), sorted=np.zeros(self.n, np.int64),
                 left=np.zeros(ni, np.int32), right=np.zeros(ni, np.int32),
                 node_lo=np.zeros((ni, 3), np.float32), node_hi=np.zeros((ni, 3), np.float32),
                 node_count=np.zeros(ni, np.int64),
                 leaf_lo=np.zeros((nb, 3), np.float32), leaf_hi=np.zeros((nb, 3), np.float32),
                 leaf_count=np.zeros(nb, np.int64), scene_box=np.zeros(6, np.float32))
        lib.orc_tree_export(self._h, _ptr(t["codes"]), _ptr(t["sorted"]), _ptr(t["left"]), _ptr(t["right"]),
                            _ptr(t["node_lo"]), _ptr(t["node_hi"]), _ptr(t["node_count"]),
                            _ptr(t["leaf_lo"]), _ptr(t["leaf_hi"]), _ptr(t["leaf_count"]),
                            _ptr(t["scene_box"]))
        t["nb"] = nb
        return t

    def bh(self, q, alpha, beta, alpha_u=0.0, paper_metric=False, decision="fp32",
           threads=None, want_margin=False, unit=False):
        """Barnes-Hut d^ and grad d^ (Alg. 1, Alg. 2) on this scene's tree.
        decision: "fp32" takes the test |B|^2 < beta^2 d^2 in FP32 in a fixed
        operation order (the precision of the GPU kernels); "fp64" takes
        |B| / d < beta in FP64. Returns (val, grad, counts[m,3] = nodes
        tested, far-field accepts, leaf primitives evaluated, margin or None)."""
        if self.L is None:
            self.build_tree(1)
        q = np.ascontiguousarray(np.asarray(q, np.float64).reshape(-1, 3))
        m = q.shape[0]
        val = np.zeros(m); grad = np.zeros((m, 3)); counts = np.zeros((m, 3), np.int64)
        margin = np.zeros(m) if want_margin else None
        rc = _load().orc_bh(self._h, float(alpha), float(alpha_u), float(beta), int(bool(paper_metric)),
                            int(bool(unit)), 0 if decision == "fp32" else 1, _ptr(q), m, _ptr(val), _ptr(grad), _ptr(counts),
                            _ptr(margin) if margin is not None else ctypes.c_void_p(0),
                            int(threads or default_threads()))
        if rc != 0:
            raise RuntimeError("orc_bh failed")
        return val, grad, counts, margin

    # -- query primitives (Sec. 3.4) -------------------------------------
    def brute_prims(self, QV, QF, alpha, alpha_u=0.0, paper_metric=False, unit=False, threads=None):
        """Exact d^ and its translation gradient for query primitives QF [m, k]
        (k = 1, 2, 3) over vertices QV [*, 3], and the exact minimum distance."""
        V = np.ascontiguousarray(np.asarray(QV, np.float64).reshape(-1, 3))
        F = np.ascontiguousarray(np.asarray(QF, np.int32))
        F = F.reshape(F.shape[0], -1)
        m, k = F.shape
        val = np.zeros(m); grad = np.zeros((m, 3)); dmin = np.zeros(m)
        _load().orc_brute_prims(self._h, float(alpha), float(alpha_u), int(bool(paper_metric)), int(bool(unit)),
                                _ptr(V), _ptr(F), int(k), m, _ptr(val), _ptr(grad), _ptr(dmin),
                                int(threads or default_threads()))
        return val, grad, dmin

    def bh_prims(self, QV, QF, alpha, beta, alpha_u=0.0, paper_metric=False, decision="fp32", threads=None,
                 want_margin=False, unit=False):
        """Barnes-Hut d^ for query primitives, the node test taken on the
        query's box (see orc_bh_prims); returns (val, grad, counts, margin)."""
        if self.L is None:
            self.build_tree(1)
        V = np.ascontiguousarray(np.asarray(QV, np.float64).reshape(-1, 3))
        F = np.ascontiguousarray(np.asarray(QF, np.int32))
        F = F.reshape(F.shape[0], -1)
        m, k = F.shape
        val = np.zeros(m); grad = np.zeros((m, 3)); counts = np.zeros((m, 3), np.int64)
        margin = np.zeros(m) if want_margin else None
        rc = _load().orc_bh_prims(self._h, float(alpha), float(alpha_u), float(beta), int(bool(paper_metric)),
                                  int(bool(unit)), 0 if decision == "fp32" else 1, _ptr(V), _ptr(F), int(k), m,
                                  _ptr(val), _ptr(grad), _ptr(counts),
                                  _ptr(margin) if margin is not None else ctypes.c_void_p(0),
                                  int(threads or default_threads()))
        if rc != 0:
            raise RuntimeError("orc_bh_prims failed")
        return val, grad, counts, margin

    def lower_bound(self, q, alpha, alpha_u=0.0, unit=False):
        """Certified lower bound of the exact d^ over the top cut (at most 64
        nodes) of this scene's tree, its gradient, kappa and the cut size."""
        if self.L is None:
            self.build_tree(1)
        q = np.ascontiguousarray(np.asarray(q, np.float64).reshape(-1, 3))
        m = q.shape[0]
        lb = np.zeros(m); grad = np.zeros((m, 3)); info = np.zeros(2)
        rc = _load().orc_lower_bound(self._h, float(alpha), float(alpha_u), int(bool(unit)), _ptr(q), m, _ptr(lb),
                                     _ptr(grad), _ptr(info))
        if rc != 0:
            raise RuntimeError("orc_lower_bound failed")
        return lb, grad, float(info[0]), int(info[1])
