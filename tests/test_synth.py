"""The seeded synthetic inputs (the stand-ins for the paper's data): sizes,
structure and distributions of the named workloads, and determinism. These
generators hold none of the method's arithmetic; the tests pin the recipe the
benchmarks and parity tests are stated on."""
import numpy as np

import synth


def _edges(F):
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    u, c = np.unique(e, axis=0, return_counts=True)
    return u, c


def test_icosphere_level6():
    V, F = synth.icosphere(6)
    assert V.shape == (40962, 3) and F.shape == (81920, 3)
    assert V.dtype == np.float32 and F.dtype == np.int32
    assert np.allclose(np.linalg.norm(V.astype(np.float64), axis=1), 1.0, atol=1e-6)
    # closed 2-manifold: every edge in two triangles; valences 5 and 6
    _, c = _edges(F)
    assert np.all(c == 2)
    val = np.bincount(F.ravel(), minlength=len(V))
    assert set(np.unique(val)) == {5, 6} and (val == 5).sum() == 12


def test_config2_mesh_and_query_mix():
    c = synth.config2()
    V, F, q = c["V"], c["F"], c["queries"]
    assert F.shape == (81920, 3) and q.shape == (262144, 3) and q.dtype == np.float32
    r = np.linalg.norm(V.astype(np.float64), axis=1)
    assert 0.003 < np.std(r) < 0.02 and abs(r.mean() - 1.0) < 0.002          # radial noise 0.01
    rq = np.linalg.norm(q.astype(np.float64), axis=1)
    shell = np.abs(rq - 1.0) < 0.1
    assert 0.70 <= shell.mean() < 0.72          # 70 % in the shell (plus box queries that fall in it)
    assert np.abs(q).max() <= 2.0
    # the shell part is uniform in radius over [0.9, 1.1]
    h, _ = np.histogram(rq[shell], bins=4, range=(0.9, 1.1))
    assert h.min() > 0.8 * h.max()


def test_config1_points_and_queries():
    c = synth.config1()
    P, q = c["points"], c["queries"]
    assert P.shape == (4096, 3) and q.shape == (1024, 3)
    r = np.linalg.norm(P.astype(np.float64), axis=1)
    assert abs(r.mean() - 1.0) < 1e-3 and 0.003 < np.std(r) < 0.008
    assert np.abs(q).max() <= 1.5


def test_geodesic_body_size():
    V, F = synth.geodesic_icosphere(100)
    assert V.shape == (100002, 3) and F.shape == (200000, 3)
    _, c = _edges(F)
    assert np.all(c == 2)


def test_street_scene_structure():
    s = synth.street_scene(n_points=50000, n_wire_segments=2000, seed=2)
    P = s["points"].astype(np.float64)
    assert P.shape == (50000, 3)
    assert np.abs(P[:, 0]).max() <= 200.0 + 1e-3 and np.abs(P[:, 1]).max() <= 40.0 + 1e-3
    # most returns are on the ground, within its height noise
    ground = np.abs(P[:, 2]) < 0.1
    assert ground.mean() > 0.3
    E = s["wire_E"]
    assert E.shape == (2000, 2) and s["wire_V"].shape[1] == 3
    # wires: chains with shared vertices (interior valence 2)
    val = np.bincount(E.ravel())
    assert val.max() <= 2 and (val == 2).sum() > 0.9 * (val > 0).sum()


def test_generators_are_deterministic():
    a = synth.config2(m=1000)
    b = synth.config2(m=1000)
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["queries"], b["queries"])
    assert not np.array_equal(synth.shell_queries(1000, seed=1), synth.shell_queries(1000, seed=2))
