"""C-ABI library: builds, loads, exports every declared symbol, host-only logic
(ray grid, spacing, error paths) works without a GPU. CPU only."""
import os
import re

import numpy as np
import pytest

import sbr_inputs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    from paper_2604_09243_gb300 import build

    build.build()
    import paper_2604_09243_gb300 as G

    return G


def _declared():
    txt = open(os.path.join(ROOT, "include", "sbr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sbr_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(G):
    names = _declared()
    assert len(names) >= 14
    L = G.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(G.EXPORTS) == names


def test_version_and_spacing(G):
    assert G.version() == 1
    assert G.spacing_for(10e9, 10.0) == pytest.approx(0.0299792458 / 10, rel=1e-15)
    with pytest.raises(ValueError):
        G.spacing_for(-1.0, 10.0)


def test_ray_grid_bit_identical_to_oracle(G, orc):
    # both sides implement the written grid convention independently
    rng = np.random.default_rng(0)
    for xyz, tri in (S.trihedral(), S.icosphere(3), S.aircraft(target_tris=20_000)):
        bb = S.mesh_bbox(xyz)
        for k in range(600):
            az, el = rng.uniform(0, 360), rng.uniform(-90, 90)
            ds, eta = rng.uniform(0.001, 0.05), rng.uniform(0, 0.2)
            win = rng.uniform(0.5, 3) if k % 3 == 0 else 0.0
            off = (rng.uniform(0, 1), rng.uniform(0, 1)) if k % 2 else (0.0, 0.0)
            g = G.ray_grid(bb, az, el, ds, eta, win, off)
            f = orc.make_frame(bb, az, el, ds, eta, win, off)
            assert (g["nu"], g["nv"]) == (f.nu, f.nv)
            for a, b in (("p0", "P0"), ("du", "U"), ("dv", "V"), ("dir", "d")):
                assert np.array_equal(g[a], np.array(getattr(f, b), np.float32)), (a, az, el)
            assert g["eps"] == f.eps


def test_ray_grid_rejects_bad_arguments(G):
    with pytest.raises(G.SbrError):
        G.ray_grid(np.zeros(6, np.float32), 0.0, 0.0, -1.0)


def test_no_device_reports_nodev(G):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.SbrError) as e:
        G.Context(0)
    assert e.value.code == -7


def test_gemm_entry_points_refuse_bad_arguments(G):
    """Both GEMM entry points check pointers and shapes on the host, before any device work."""
    for fn in (lambda *a: G.gemm_bf16_tn(*a), lambda *a: G.gemm_bf16_tn_async(*a, 8)):
        for args in ((0, 512, 8, 512, 128, 128, 512, 8, 128),      # null A
                     (8, 512, 8, 512, 100, 128, 512, 8, 128),      # M not a multiple of 128
                     (8, 512, 8, 512, 128, 128, 96, 8, 128),       # K not a multiple of 64
                     (8, 500, 8, 512, 128, 128, 512, 8, 128)):     # lda not a multiple of 8
            with pytest.raises(G.SbrError) as e:
                fn(*args)
            assert e.value.code == -1
    with pytest.raises(G.SbrError):  # no error flag for the enqueue-only call
        G.gemm_bf16_tn_async(8, 512, 8, 512, 128, 128, 512, 8, 128, 0)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2604_09243_gb300.sbr as mod

    monkeypatch.setattr(mod, "_lib", None)
    monkeypatch.setattr(mod, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mod.lib()
