"""Many rigid bodies against one data mesh in one persistent launch, with
CUDA-graph replay and an autotuner for the traversal block size and the
tree's leaf size.

    bb = BatchedBodies(sd, [X0_body0, X0_body1, ...])
    bb.set_poses(poses)                  # [B, 6]: (theta, p) per body
    out = bb.run(alpha_q)                # [B, 7]: D_b, dD/dp, dD/dtheta
    g = bb.capture(alpha_q)              # torch.cuda.CUDAGraph of run()
    bb.set_poses(new_poses); g.replay()  # same buffers, new poses

All arithmetic runs in libsd (sd_batch_*); this module only marshals.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import SmoothDistance, _native, lib
from . import _ptr, _stream_handle


class BatchedBodies:
    def __init__(self, sd, bodies_X0, device=None):
        self.sd = sd
        self.device = sd.device
        sizes = [int(np.asarray(b).shape[0]) if not torch.is_tensor(b) else int(b.shape[0]) for b in bodies_X0]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        X0 = torch.cat([torch.as_tensor(b, dtype=torch.float32).reshape(-1, 3).to(self.device) for b in bodies_X0])
        self.X0 = X0.contiguous()
        self.B = len(sizes)
        self.M = int(self.offsets[-1])
        h = ctypes.c_void_p()
        _native.check(lib().sd_batch_create(sd.handle, _ptr(self.X0), ctypes.c_void_p(self.offsets.ctypes.data),
                                            self.B, ctypes.byref(h)), "sd_batch_create")
        self._h = h
        self.out = torch.zeros(self.B, 7, device=self.device, dtype=torch.float32)
        self.block = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _native._lib is not None:
            _native._lib.sd_batch_free(h)
            self._h = None

    def set_poses(self, poses, stream=None):
        p = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(self.B, 6))
        _native.check(lib().sd_batch_set_poses(self._h, ctypes.c_void_p(p.ctypes.data), _stream_handle(stream)),
                      "sd_batch_set_poses")

    def run(self, alpha_q, stream=None):
        _native.check(lib().sd_batch_run(self._h, float(alpha_q), int(self.block), _ptr(self.out),
                                          _stream_handle(stream)), "sd_batch_run")
        return self.out

    def vertex_outputs(self):
        X, v, g = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _native.check(lib().sd_batch_vertex_outputs(self._h, ctypes.byref(X), ctypes.byref(v), ctypes.byref(g)),
                      "sd_batch_vertex_outputs")
        return X.value, v.value, g.value

    def capture(self, alpha_q):
        """Capture run(alpha_q) into a CUDA graph (poses must be set)."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.run(alpha_q, stream=s)          # warm-up outside the capture
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(alpha_q, stream=s)
        return g


def autotune(build_kwargs, bodies_X0, poses, alpha_q, sample_queries, leaf_sizes=(1, 2, 4, 8),
             blocks=(64, 128, 256), err_factor=2.0, reps=5):
    """Pick the traversal block size and the leaf size L.

    Every candidate L builds its own tree. A candidate is admissible only if
    its Barnes-Hut error against the exact (plain, all-pairs) evaluation on
    `sample_queries` is at most `err_factor` times the error of L = 1 (L is
    part of the tree's definition, so it changes results). Among admissible
    candidates the fastest graph-replayed batch evaluation wins.
    Returns (best dict, list of all candidate records)."""
    q = torch.as_tensor(sample_queries, dtype=torch.float32).cuda()
    kw = dict(build_kwargs)
    ref_err = None
    records = []
    best = None
    for L in leaf_sizes:
        kw["leaf_size"] = L
        sd = SmoothDistance(**kw)
        vb, _ = sd.query_brute(q, grad=False)
        v, _ = sd.query(q, grad=False)
        err = float((v - vb).abs().max().item())
        if ref_err is None:
            ref_err = err
        ok = err <= err_factor * max(ref_err, 1e-7)
        bb = BatchedBodies(sd, bodies_X0)
        bb.set_poses(poses)
        for blk in blocks:
            bb.block = blk
            g = bb.capture(alpha_q)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            rec = dict(leaf_size=L, block=blk, ms=ms, bh_err=err, admissible=ok)
            records.append(rec)
            if ok and (best is None or ms < best["ms"]):
                best = rec
            del g
        del bb, sd
    return best, records
