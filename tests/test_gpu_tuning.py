"""Tuning parameters (ray tile, stack depth, blocks per SM, PO item, chunk size)
and the autotuner: hits are the same under every setting, fields agree to
rounding, and the autotuner keeps only settings whose results agree."""
import numpy as np
import pytest

import sbr_inputs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2604_09243_gb300 import build

    build.build()
    import paper_2604_09243_gb300 as G

    return G


@pytest.fixture(scope="module")
def tri_case():
    return S.trihedral_case()


def _trace(c, case, angles, **kw):
    c.trace(angles, case["spacing"], eta=case["eta"], max_bounces=case["max_bounces"], offset=case["offset"],
            flags=kw.pop("flags", 0), **kw)


@pytest.mark.parametrize("setting", [dict(tile_w=1), dict(tile_w=4), dict(tile_w=32), dict(stack_depth=32),
                                     dict(stack_depth=128), dict(blocks_per_sm=1), dict(po_item=512),
                                     dict(po_item=2048), dict(chunk_rays_log2=20), dict(bvh_width=4),
                                     dict(bvh_width=4, stack_depth=32, tile_w=4), dict(packet=1),
                                     dict(packet=1, stack_depth=32, tile_w=32), dict(raster=0),
                                     dict(raster=0, silhouette=1), dict(octant=1),
                                     dict(octant=1, stack_depth=32, tile_w=16, raster=0),
                                     dict(raster=0, silhouette=1, bvh_width=4, tile_w=16)])
def test_setting_keeps_hits_and_fields(G, tri_case, setting):
    case = tri_case
    angles = case["angles"][[0, 45, 90, 135, 180]]
    out = []
    for s in ({}, setting):
        with G.Context(0) as c:
            c.load_mesh(case["xyz"], case["tri"])
            if s:
                c.set_tuning(**s)
                assert all(c.tuning()[k] == v for k, v in s.items())
            _trace(c, case, angles, flags=G.TRACE_RECORD_HITS)
            hits = [c.get_hits(a) for a in range(len(angles))]
            E, R = c.po_integrate([10e9, 7e9], "HH,VV")
            out.append((hits, E, R))
    (h0, E0, R0), (h1, E1, R1) = out
    for a, b in zip(h0, h1):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.max(np.abs(E1 - E0)) <= 1e-5 * np.max(np.abs(E0))
    big = R0 > -40
    assert np.max(np.abs(R1[big] - R0[big])) < 1e-3


def test_bad_settings_refused(G):
    with G.Context(0) as c:
        before = c.tuning()
        for bad in (dict(tile_w=3), dict(tile_w=64), dict(blocks_per_sm=0), dict(blocks_per_sm=5),
                    dict(stack_depth=48), dict(po_item=300), dict(chunk_rays_log2=19), dict(chunk_rays_log2=30),
                    dict(bvh_width=3), dict(packet=2), dict(packet=1, bvh_width=4), dict(packet=1, stack_depth=128),
                    dict(silhouette=2), dict(octant=1, bvh_width=4), dict(octant=1, packet=1), dict(octant=2),
                    dict(raster=2), dict(raster=-1)):
            with pytest.raises(G.SbrError):
                c.set_tuning(**bad)
        assert c.tuning() == before


def test_submitted_batch_follows_tuning(G, tri_case):
    torch = pytest.importorskip("torch")
    case = tri_case
    rng = np.random.default_rng(3)
    reqs = [dict(az=float(rng.uniform(0, 90)), el=35.26, freqs=np.array([6e9, 10e9]),
                 spacing=S.spacing_for(10e9, 6.0)) for _ in range(6)]
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        c.set_tuning(tile_w=16, po_item=512, stack_depth=32)
        _, Rb, _ = c.run_batch(reqs, max_bounces=3, offset=case["offset"])
        R = torch.zeros((12, 2), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        c.submit_batch(reqs, None, R, max_bounces=3, offset=case["offset"])
        c.sync()
        assert np.array_equal(R.cpu().numpy(), np.concatenate(Rb))


def test_autotune_keeps_an_accepted_setting(G, tri_case):
    case = tri_case
    rng = np.random.default_rng(4)
    reqs = [dict(az=float(rng.uniform(0, 90)), el=35.26, freqs=np.array([10e9]), spacing=case["spacing"])
            for _ in range(8)]
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        best, ms, trials = c.autotune(reqs, max_bounces=3, offset=case["offset"], reps=2)
        assert c.tuning() == best
        assert len(trials) >= 10 and ms > 0
        ok = [t for t in trials if t["status"] == 0]
        # every kept change beat the setting before it, timed beside it, by 1 %; separate timings of the
        # starting setting and the kept one can still differ by noise
        assert ms <= 1.05 * ok[0]["ms"]
        assert any(all(t[k] == best[k] for k in best) for t in ok)
        # best_ms is the fastest of all the kept setting's timings, its own trial's among them
        assert ms <= min(t["ms"] for t in ok if all(t[k] == best[k] for k in best))


def test_wide_tree_same_hits_aircraft(G):
    """The 4-wide tree and the warp-cooperative traversal of the ~1M-triangle
    aircraft give every ray the same hits (bit for bit) as the per-ray binary
    traversal, over 10 bounces."""
    case = S.aircraft_case(1e9, n_az=360)
    angles = case["angles"][[0, 90, 180, 270]]
    out = []
    for w, pk, oc in ((2, 0, 0), (4, 0, 0), (2, 1, 0), (2, 0, 1)):
        with G.Context(0) as c:
            c.load_mesh(case["xyz"], case["tri"])
            c.set_tuning(bvh_width=w, packet=pk, octant=oc)
            st = c.trace(angles, case["spacing"], eta=case["eta"], max_bounces=case["max_bounces"],
                         offset=case["offset"], flags=G.TRACE_RECORD_HITS | G.TRACE_COUNT_VISITS)
            out.append((st, [c.get_hits(a) for a in range(len(angles))], c.po_integrate([1e9])[1]))
    (s2, h2, R2) = out[0]
    for k, (s4, h4, R4) in enumerate(out[1:]):
        assert s2["ray_bounces"] == s4["ray_bounces"] and s2["valid_rays"] == s4["valid_rays"]
        assert s4["stack_overflows"] == 0
        if k == 0:
            assert s4["node_visits"] < s2["node_visits"]
        for a, b in zip(h2, h4):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
        assert np.array_equal(R2, R4)


def test_depth_first_layout_keeps_the_reachable_nodes(G):
    """After the build the node array holds only the nodes reachable from the
    root, in depth-first order: the aircraft's tree shrinks below its n - 1
    node slots while its rays keep the oracle's hits (the parity tests), a
    single triangle keeps one node, and the Karras tree of a plate hits as the
    clustered one does."""
    case = S.aircraft_case(1e9, n_az=360)
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        info = c.bvh_info()
        assert info["n_tri"] == len(case["tri"])
        assert 0 < info["n_nodes"] < len(case["tri"]) - 1
        assert 0 < info["n_nodes4"] <= info["n_nodes"]
        c.build_bvh(builder="lbvh")
        assert 0 < c.bvh_info()["n_nodes"] < len(case["tri"]) - 1
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    with G.Context(0) as c:
        c.load_mesh(xyz, np.array([[0, 1, 2]], np.int32))
        assert c.bvh_info()["n_nodes"] == 1
        st = c.trace([[0.0, 90.0]], 0.05, eta=0.0, max_bounces=1)
        assert st["valid_rays"] > 0
        for builder in ("ploc", "lbvh"):
            c.build_bvh(builder=builder)
            assert c.trace([[0.0, 90.0]], 0.05, eta=0.0, max_bounces=1)["valid_rays"] == st["valid_rays"]


def test_silhouette_mask_skips_only_misses(G):
    """With the silhouette mask (primary rays traversing the tree) the
    aircraft's rays keep their hits (bit for bit) and valid count while fewer
    queries run; with the rasterised primary hits they keep them too and every
    grid ray is answered. A two-triangle plate much larger than the grid cells
    takes the all-rays path of the mask and the traversal fallback of the
    rasterisation, and keeps its RCS."""
    case = S.aircraft_case(1e9, n_az=360)
    angles = case["angles"][[0, 45, 180, 300]]
    out = []
    for sil, ras in ((0, 0), (1, 0), (0, 1)):
        with G.Context(0) as c:
            c.load_mesh(case["xyz"], case["tri"])
            c.set_tuning(silhouette=sil, raster=ras)
            st = c.trace(angles, case["spacing"], eta=case["eta"], max_bounces=case["max_bounces"],
                         offset=case["offset"], flags=G.TRACE_RECORD_HITS)
            out.append((st, [c.get_hits(a) for a in range(len(angles))], c.po_integrate([1e9])[1]))
    (s0, h0, R0), (s1, h1, R1), (s2, h2, R2) = out
    assert s1["valid_rays"] == s0["valid_rays"] and s1["rays_launched"] == s0["rays_launched"]
    assert s1["ray_bounces"] < s0["ray_bounces"]
    assert s2["ray_bounces"] == s0["ray_bounces"] and s2["valid_rays"] == s0["valid_rays"]
    for hh in (h1, h2):
        for a, b in zip(h0, hh):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    assert np.array_equal(R0, R1) and np.array_equal(R0, R2)
    xyz, tri = S.square_plate(1.0, m=1)  # two 1 m triangles: 500 x 500 cells each at 2 mm
    res = []
    for sil, ras in ((0, 0), (1, 0), (0, 1)):
        with G.Context(0) as c:
            c.load_mesh(xyz, tri)
            c.set_tuning(silhouette=sil, raster=ras)
            c.trace([[0.0, 90.0], [10.0, 80.0]], 0.002, max_bounces=1)
            res.append(c.po_integrate([10e9])[1])
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


def test_raster_primary_hits_equal_traversal(G, tri_case):
    """Primary hits found by rasterisation (one FP32 test per triangle and
    covered grid ray, 64-bit atomic minimum of (t, index)) equal those of the
    tree traversal bit for bit: sphere with its window, aircraft at 3 GHz over
    10 bounces, a bistatic trihedral, and the submitted batch path; the
    rasterisation counts its triangle tests and the primary pass visits no
    nodes."""
    torch = pytest.importorskip("torch")
    sph = S.sphere_case(n_random=3)
    air = S.aircraft_case(3e9, n_az=360)
    cases = [(sph["xyz"], sph["tri"], sph["angles"], sph["spacing"], 1, dict(window=sph["window"])),
             (air["xyz"], air["tri"], air["angles"][[10, 100, 250]], air["spacing"], air["max_bounces"],
              dict(eta=air["eta"], offset=air["offset"])),
             (tri_case["xyz"], tri_case["tri"], tri_case["angles"][[20, 90, 150]], tri_case["spacing"], 3,
              dict(eta=tri_case["eta"], offset=tri_case["offset"], rx=tri_case["angles"][[30, 60, 100]] + [0, 5]))]
    for xyz, tri, ang, sp, B, kw in cases:
        out = []
        for ras in (0, 1):
            with G.Context(0) as c:
                c.load_mesh(xyz, tri)
                c.set_tuning(raster=ras)
                st = c.trace(ang, sp, max_bounces=B, flags=G.TRACE_RECORD_HITS | G.TRACE_COUNT_VISITS, **kw)
                p1 = c.trace(ang, sp, max_bounces=1, flags=G.TRACE_COUNT_VISITS,
                             **{k: v for k, v in kw.items() if k != "rx"})
                out.append((st, p1, c.po_integrate([3e9, 10e9])[1]))
        (s0, p0, R0), (s1, q1, R1) = out
        assert s0["ray_bounces"] == s1["ray_bounces"] and s0["valid_rays"] == s1["valid_rays"]
        assert s1["stack_overflows"] == 0
        assert q1["node_visits"] == 0 and q1["tri_tests"] > 0 and p0["node_visits"] > 0
        assert np.array_equal(R0, R1)
    # hits ray by ray (aircraft) and the submitted batch path (trihedral)
    hits = []
    for ras in (0, 1):
        with G.Context(0) as c:
            c.load_mesh(air["xyz"], air["tri"])
            c.set_tuning(raster=ras)
            c.trace(air["angles"][[10, 100]], air["spacing"], eta=air["eta"], max_bounces=air["max_bounces"],
                    offset=air["offset"], flags=G.TRACE_RECORD_HITS)
            hits.append([c.get_hits(a) for a in range(2)])
    for a, b in zip(*hits):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    rng = np.random.default_rng(5)
    reqs = [dict(az=float(rng.uniform(0, 90)), el=35.26, freqs=np.array([6e9, 10e9]),
                 spacing=S.spacing_for(10e9, 6.0)) for _ in range(5)]
    res = []
    for ras in (0, 1):
        with G.Context(0) as c:
            c.load_mesh(tri_case["xyz"], tri_case["tri"])
            c.set_tuning(raster=ras)
            R = torch.zeros((10, 2), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            c.submit_batch(reqs, None, R, max_bounces=3, offset=tri_case["offset"])
            c.sync()
            res.append(R.cpu().numpy())
    assert np.array_equal(res[0], res[1])


def test_raster_with_flagged_and_rasterised_aspects_in_one_chunk(G, orc):
    """A chunk whose aspects split between rasterised primary hits and the
    traversal fallback: a 1 m plate triangle spans ~20,000 grid cells seen
    face-on (flagged: its aspect traverses) and ~1,700 at grazing incidence
    (rasterised), beside a small-triangle sphere. The traversing rays are
    appended after the rasterised ones; every hit equals the traversal's and
    the oracle's, in the plain and the submitted batch paths."""
    torch = pytest.importorskip("torch")
    from parity import assert_hit_parity, compare_hits

    xs, ts = S.icosphere(3, radius=0.3)
    xs = xs + np.array([0.0, 0.0, 0.8], np.float32)
    xp = np.array([[-0.5, -0.5, 0.0], [0.5, -0.5, 0.0], [-0.5, 0.5, 0.0]], np.float32)
    xyz = np.concatenate([xs, xp])
    tri = np.concatenate([ts, np.array([[0, 1, 2]], np.int32) + len(xs)])
    ang = np.array([[0.0, 90.0], [30.0, 5.0], [200.0, 60.0], [45.0, 5.0]])
    sp = 0.005
    om = orc.Mesh(xyz, tri)
    out = []
    for ras in (0, 1):
        with G.Context(0) as c:
            c.load_mesh(xyz, tri)
            c.set_tuning(raster=ras)
            st = c.trace(ang, sp, max_bounces=3, flags=G.TRACE_RECORD_HITS | G.TRACE_COUNT_VISITS)
            hits = [c.get_hits(a) for a in range(len(ang))]
            out.append((st, hits, c.po_integrate([10e9])[1]))
            if ras:
                for a, (az, el) in enumerate(ang):
                    fr = orc.make_frame(om.bbox, az, el, sp)
                    assert_hit_parity(compare_hits(*hits[a], orc.trace(om, fr, 3)))
                # the same aspects again in reverse order, in the same context: the raster keys left by
                # the first trace (a flagged aspect's included) must all read "no hit" again
                c.trace(ang[::-1], sp, max_bounces=3, flags=G.TRACE_RECORD_HITS)
                again = [c.get_hits(a) for a in range(len(ang))][::-1]
                for x0, y0 in zip(hits, again):
                    for x, y in zip(x0, y0):
                        assert np.array_equal(x, y)
    (s0, h0, R0), (s1, h1, R1) = out
    assert s1["raster_tests"] > 0 and 0 < s1["node_visits"]
    assert s0["ray_bounces"] == s1["ray_bounces"] and s0["valid_rays"] == s1["valid_rays"]
    for a, b in zip(h0, h1):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.array_equal(R0, R1)
    reqs = [dict(az=float(az), el=float(el), freqs=np.array([10e9]), spacing=sp) for az, el in ang]
    res = []
    for ras in (0, 1):
        with G.Context(0) as c:
            c.load_mesh(xyz, tri)
            c.set_tuning(raster=ras)
            R = torch.zeros((len(reqs), 2), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            c.submit_batch(reqs, None, R, max_bounces=3)
            c.sync()
            res.append(R.cpu().numpy())
    assert np.array_equal(res[0], res[1])
    assert np.array_equal(res[1], R1[:, 0, :])



def test_roofline_probes(G):
    """The L2 read probe sees more than the HBM copy bandwidth and the FP32 probe
    at most the nominal rate (SMs x 128 lanes x 2 FLOP x the top SM clock)."""
    torch = pytest.importorskip("torch")
    props = torch.cuda.get_device_properties(0)
    l2 = G.probe_l2_bandwidth(0, nbytes=64 << 20, passes=20)
    fp32 = G.probe_fp32_fma(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert l2 > 5000.0, l2
    assert 0.3 * nominal < fp32 <= 1.02 * nominal, (fp32, nominal)
    with pytest.raises(G.SbrError):
        G.probe_l2_bandwidth(0, nbytes=1024, passes=1)
