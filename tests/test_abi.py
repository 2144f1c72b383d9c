"""The C-ABI library loads and exports every symbol include/sd.h declares;
host-only entry points run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sd_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2108_10480_gb300 import _native
    lib = _native.lib()
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
        assert n in _native.SIGNATURES, n


def test_status_strings_and_defaults():
    from paper_2108_10480_gb300 import _native
    lib = _native.lib()
    assert lib.sd_status_str(0) == b"ok"
    assert lib.sd_status_str(4) == b"non-finite coordinate"
    o = _native.SdBuildOpts()
    lib.sd_default_build_opts(ctypes.byref(o))
    assert o.leaf_size == 1 and o.weights == 0 and o.alpha_u == 0.0
    q = _native.SdQueryOpts()
    lib.sd_default_query_opts(ctypes.byref(q))
    assert q.sort_queries == 1 and q.block == 0


def test_build_rejects_bad_arguments_without_a_gpu():
    # argument checks happen before any CUDA call
    from paper_2108_10480_gb300 import _native
    lib = _native.lib()
    g = _native.SdGeometry()
    h = ctypes.c_void_p()
    assert lib.sd_build(ctypes.byref(g), -1.0, 0.5, None, None, ctypes.byref(h)) == 1
    assert lib.sd_build(ctypes.byref(g), 10.0, -0.5, None, None, ctypes.byref(h)) == 1
    g.pts.n = 5     # count without a pointer
    assert lib.sd_build(ctypes.byref(g), 10.0, 0.5, None, None, ctypes.byref(h)) == 1
    assert lib.sd_query(None, None, 0, None, None, None, None) == 1


def test_library_weight_basis_matches_oracle():
    """The library solves App. C.3 with its own Gram-Schmidt minimum-norm
    solver and Bernstein conversion; the oracle uses numpy's pseudoinverse in
    the monomial basis. Both define the same polynomial."""
    from math import factorial as F

    from oracle import weights as W
    import paper_2108_10480_gb300 as P
    B = P.weight_basis()
    X = W.tri_basis()
    idx = [(7 - r, r - k, k) for r in range(8) for k in range(r + 1)]
    phi = np.random.default_rng(0).dirichlet([1, 1, 1], 300)
    bern = np.array([[F(7) / (F(i) * F(j) * F(k)) * p[0] ** i * p[1] ** j * p[2] ** k for (i, j, k) in idx]
                     for p in phi])
    mono = np.array([[p[1] ** a * p[2] ** b for (a, b) in W.TRI_EXPONENTS] for p in phi])
    assert np.abs(bern @ B.T - mono @ X).max() < 1e-9
    # Bernstein coefficients stay of the size of the weight (well conditioned)
    assert np.abs(B).max() < 10


def test_package_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2108_10480_gb300 import _native, build_ext
    monkeypatch.setattr(build_ext, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setenv("SD_AUTOBUILD", "0")
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(OSError):
        _native.lib()
