"""Seeded input generators: sizes, determinism, closedness. CPU only."""
import numpy as np

import sbr_inputs as S


def _edge_counts(tri):
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e.sort(axis=1)
    _, c = np.unique(e, axis=0, return_counts=True)
    return c


def test_icosphere_sizes_closed():
    xyz, tri = S.icosphere(5)
    assert xyz.dtype == np.float32 and tri.dtype == np.int32
    assert tri.shape == (20480, 3) and xyz.shape == (10242, 3)
    assert np.allclose(np.linalg.norm(xyz.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.all(_edge_counts(tri) == 2)  # closed 2-manifold


def test_trihedral_sizes():
    xyz, tri = S.trihedral(1.0, 32)
    assert tri.shape == (3072, 3)
    assert np.array_equal(S.mesh_bbox(xyz), np.array([0, 0, 0, 1, 1, 1], np.float32))


def test_generators_deterministic():
    a = S.aircraft(seed=1, target_tris=20_000)
    b = S.aircraft(seed=1, target_tris=20_000)
    c = S.aircraft(seed=2, target_tris=20_000)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])


def test_aircraft_size_and_extent():
    xyz, tri = S.aircraft(seed=1)
    assert 900_000 < len(tri) < 1_100_000
    bb = S.mesh_bbox(xyz)
    assert 15.0 < bb[3] - bb[0] < 16.0          # fuselage 15 m (+ tail overhang)
    assert 16.0 < bb[4] - bb[1] < 17.0          # wing span
    assert tri.min() >= 0 and tri.max() < len(xyz)


def test_batched_requests_mix():
    r = S.batched_requests(256, seed=2)
    assert len(r) == 256
    nf = np.array([len(x["freqs"]) for x in r])
    assert nf.min() >= 1 and nf.max() <= 64
    assert set(x["mesh"] for x in r) == {0, 1, 2}
    for x in r:
        assert 1e9 <= x["freqs"].min() and x["freqs"].max() <= 12e9
        assert -30 <= x["el"] <= 30 and 0 <= x["az"] < 360
