"""CUDA path vs the oracle on the same seeded inputs, through the C ABI.

Parity rule (tests/parity.py): the oracle decides every hit exactly; every
ray outside the edge band (exact hit within 1e-6 barycentric of an edge, or a
runner-up within 1e-6 relative in t) must have the oracle's triangle sequence
and bounce count, band rays that differ must stay below 1e-5 of all rays, and
hit distances agree within 1e-5 relative. RCS (FP64 oracle sums vs FP32/FP64
kernel sums) within 0.1 dB wherever the oracle is above -40 dBsm.
"""
import math

import numpy as np
import pytest

import sbr_inputs as S
from parity import HitTally, assert_hit_parity, assert_rcs_close, compare_hits

pytestmark = pytest.mark.gpu
C0 = 299_792_458.0
HITS = 4  # SBR_TRACE_RECORD_HITS


@pytest.fixture(scope="module")
def G():
    from paper_2604_09243_gb300 import build

    build.build()
    import paper_2604_09243_gb300 as G

    return G


@pytest.fixture()
def ctx(G):
    c = G.Context(0)
    yield c
    c.close()


def _trace_both(G, ctx, orc, om, angles, spacing, B, eta=0.05, window=0.0, offset=(0.0, 0.0), flags=0, **kw):
    st = ctx.trace(angles, spacing, eta=eta, max_bounces=B, window=window, offset=offset, flags=flags | HITS, **kw)
    out = []
    for a, (az, el) in enumerate(angles):
        fr = orc.make_frame(om.bbox, az, el, spacing, eta=eta, window=window, offset=offset)
        o = orc.trace(om, fr, B, require_escape=bool(flags & 2))
        g = ctx.get_hits(a)
        out.append((g, o, fr))
    return st, out


# ----------------------------------------------------------------------------- C1 sphere
def test_sphere_hits_rcs_and_mie(G, ctx, orc):
    case = S.sphere_case(n_random=4)
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    assert np.array_equal(ctx.get_bbox(), om.bbox)
    f = case["freqs"]
    st, res = _trace_both(G, ctx, orc, om, case["angles"], case["spacing"], 1, window=case["window"])
    assert st["rays_launched"] == 220 * 220 * len(case["angles"])
    Ev, Rv = ctx.po_integrate(f, "HH,VV", mode="vector")
    Es, Rs = ctx.po_integrate(f, "HH,VV", mode="scalar")
    mie = 10 * math.log10(math.pi * orc.mie_pec_backscatter(2 * math.pi * f[0] / C0))
    n_valid = 0
    for a, (g, o, fr) in enumerate(res):
        s = compare_hits(*g, o)
        assert_hit_parity(s)
        n_valid += int(o["valid"].sum())
        Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], f)
        assert_rcs_close(Rv[a, 0], Ro[0, :2])
        o2 = orc.trace(om, fr, 1, po_mode="scalar")
        Eo2, Ro2 = orc.po(o2["coef"], o2["L"], o2["valid"], f)
        assert_rcs_close(Rs[a, 0], Ro2[0, :2])
        assert np.all(np.abs(Rs[a, 0] - mie) < 0.5)  # paper's Eq. po_sum vs Mie at ka = 62.9
    assert st["valid_rays"] == n_valid


# ----------------------------------------------------------------------------- C2 trihedral
def test_trihedral_hits_and_rcs_subset(G, ctx, orc):
    case = S.trihedral_case()
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ang = case["angles"][[0, 1, 37, 60, 90, 91, 133, 179, 180]]
    st, res = _trace_both(G, ctx, orc, om, ang, case["spacing"], 3, eta=case["eta"], offset=case["offset"])
    E, R = ctx.po_integrate(case["freqs"], "HH,VV,HV,VH")
    T = HitTally()
    for a, (g, o, fr) in enumerate(res):
        T.add(compare_hits(*g, o))
        Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], case["freqs"])
        assert_rcs_close(R[a, 0], Ro[0])
    tot = T.check()
    print("edge band and mismatches:", tot)
    # the edge band itself (with the seeded sub-cell grid offset) stays below 1e-5 of the rays
    assert tot["band"] / tot["n"] < 1e-5, tot


def test_trihedral_full_sweep_rcs(G, ctx, orc):
    # the benchmark workload: 181 aspects in one call, vector PO, HH/VV
    case = S.trihedral_case()
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    st = ctx.trace(case["angles"], case["spacing"], eta=case["eta"], max_bounces=3, offset=case["offset"])
    E, R = ctx.po_integrate(case["freqs"], "HH,VV")
    worst = 0.0
    for a, (az, el) in enumerate(case["angles"]):
        _, Ro, _, _ = orc.rcs_angle(om, om.bbox, az, el, case["spacing"], case["freqs"], 3, eta=case["eta"],
                                    offset=case["offset"])
        worst = max(worst, assert_rcs_close(R[a, 0], Ro[0, :2]))
    assert st["ray_bounces"] > st["rays_launched"]
    print("worst dB error over the sweep:", worst)


def test_full_size_sampled_rays(G, ctx, orc):
    # full sweep in the benchmark's launch configuration; sampled rays checked one by one
    case = S.trihedral_case()
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ctx.trace(case["angles"], case["spacing"], eta=case["eta"], max_bounces=3, flags=HITS, offset=case["offset"])
    rng = np.random.default_rng(9)
    for a in (0, 45, 90, 120, 180):
        az, el = case["angles"][a]
        fr = orc.make_frame(om.bbox, az, el, case["spacing"], eta=case["eta"], offset=case["offset"])
        ids = rng.choice(fr.n_rays, 4000, replace=False)
        o = orc.trace(om, fr, 3, ids=ids)
        s = compare_hits(*ctx.get_hits(a), o, ids=ids)
        assert_hit_parity(s)


def test_aircraft_10ghz_full_grid_sampled_rays(G, ctx, orc):
    """The aircraft at 10 GHz: full lambda/10 ray grids (about 12 M primary rays per aspect, up to 10 bounces) traced in the
    configuration the autotuner picks for the aircraft (4-wide tree, 32 x 1 ray tiles); sampled rays checked one
    by one against the oracle."""
    case = S.aircraft_case(10e9, n_az=360)
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ctx.set_tuning(bvh_width=4, tile_w=32)
    ang = case["angles"][[0, 200]]
    st = ctx.trace(ang, case["spacing"], eta=case["eta"], max_bounces=case["max_bounces"], flags=HITS,
                   offset=case["offset"])
    assert st["stack_overflows"] == 0 and st["rays_launched"] > 20_000_000
    rng = np.random.default_rng(10)
    for a, (az, el) in enumerate(ang):
        fr = orc.make_frame(om.bbox, az, el, case["spacing"], eta=case["eta"], offset=case["offset"])
        ids = rng.choice(fr.n_rays, 3000, replace=False)
        o = orc.trace(om, fr, case["max_bounces"], ids=ids)
        assert_hit_parity(compare_hits(*ctx.get_hits(a), o, ids=ids))
    ctx.set_tuning(bvh_width=2, tile_w=8)


# ----------------------------------------------------------------------------- closed forms
def test_flat_plate_and_dihedral_closed_forms(G, ctx, orc):
    xyz, tri = S.square_plate(1.0, 4)
    ctx.load_mesh(xyz, tri)
    f = 3e9
    lam = C0 / f
    ctx.trace([[0.0, 90.0]], 0.01, max_bounces=1, window=1.2)
    for mode in ("vector", "scalar"):
        _, R = ctx.po_integrate([f], "HH,VV", mode=mode)
        assert np.allclose(R[0, 0], 10 * math.log10(4 * math.pi / lam**2), atol=1e-4)
    xyz, tri = S.dihedral(1.0, 8)
    ctx.load_mesh(xyz, tri)
    f = 10e9
    lam = C0 / f
    st = ctx.trace([[45.0, 0.0]], lam / 10, max_bounces=2, offset=(0.25, 0.25))
    E, R = ctx.po_integrate([f], "HH,VV,HV")
    n = st["valid_rays"]
    assert R[0, 0, 0] == pytest.approx(10 * math.log10(4 * math.pi * (n * (lam / 10) ** 2) ** 2 / lam**2), abs=2e-3)
    assert abs(E[0, 0, 0] + E[0, 0, 1]) < 1e-4 * abs(E[0, 0, 0])  # HH = -VV after two reflections


def test_trihedral_peak(G, ctx):
    xyz, tri = S.trihedral(1.0, 32)
    ctx.load_mesh(xyz, tri)
    f = 10e9
    lam = C0 / f
    el = math.degrees(math.atan(1 / math.sqrt(2)))
    ctx.trace([[45.0, el]], lam / 10, max_bounces=3)
    _, R = ctx.po_integrate([f], "HH,VV,HV,VH")
    assert abs(R[0, 0, 0] - 10 * math.log10(4 * math.pi / (3 * lam**2))) < 0.1
    assert R[0, 0, 2] < R[0, 0, 0] - 40


# ----------------------------------------------------------------------------- edge cases
def test_single_and_two_triangles(G, ctx, orc):
    xyz = np.array([[-1, -1, 0.3], [1, -1, 0.3], [0, 1, 0.3], [0, 1, 0.9]], np.float32)
    for tri in (np.array([[0, 1, 2]], np.int32), np.array([[0, 1, 2], [0, 2, 3]], np.int32)):
        ctx.load_mesh(xyz, tri)
        om = orc.Mesh(xyz, tri)
        ang = np.array([[0.0, 90.0], [30.0, 60.0], [200.0, -45.0]])
        st, res = _trace_both(G, ctx, orc, om, ang, 0.013, 2)
        for g, o, fr in res:
            assert_hit_parity(compare_hits(*g, o))


def test_degenerate_duplicate_and_non_finite_meshes(G, ctx, orc):
    """Degenerate triangles (parallel edges within a sine of 2^-20: repeated
    vertices, a collinear midpoint, a 5e-7 sliver), exact copies and
    reversed-winding copies of every triangle on the trihedral (3 bounces): the
    GPU takes every hit decision of the oracle; the degenerate ones are never
    hit. Non-finite vertices are refused from host and device memory, and the
    context stays usable."""
    torch = pytest.importorskip("torch")
    xyz0, tri0 = S.trihedral(1.0, 16)
    a0, b0 = np.array([0.21, 0.33, 0.27], np.float32), np.array([0.62, 0.18, 0.44], np.float32)
    mid = ((a0.astype(np.float64) + b0) / 2).astype(np.float32)
    v = np.stack([a0, b0, mid, np.array([0.1, 0.1, 0.6], np.float32), np.array([0.9, 0.1, 0.6], np.float32),
                  np.array([0.9, 0.1 + 4e-7, 0.6], np.float32)])
    n = len(xyz0)
    deg = np.array([[n, n + 1, n + 1], [n, n, n + 1], [n, n + 1, n + 2], [n + 3, n + 4, n + 5]], np.int32)
    xyz = np.concatenate([xyz0, v])
    nt = len(tri0)
    tri = np.concatenate([tri0, deg, tri0, tri0[:, [0, 2, 1]]])
    ctx.load_mesh(xyz, tri)
    om = orc.Mesh(xyz, tri)
    assert om.n_degenerate == len(deg)
    ang = np.array([[45.0, 35.26], [20.0, 50.0], [71.0, 30.0]])
    st, res = _trace_both(G, ctx, orc, om, ang, 0.006, 3)
    E, R = ctx.po_integrate([10e9], "HH,VV")
    for a, (g, o, fr) in enumerate(res):
        assert_hit_parity(compare_hits(*g, o))
        ht = g[0]
        assert not np.any((ht >= nt) & (ht < nt + len(deg)))
        assert np.any(ht >= 0)
        Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], [10e9])
        assert_rcs_close(R[a, 0], Ro[0][:2])  # oracle order HH, VV, HV, VH
    # refused meshes: host arrays, then device tensors; a valid mesh loads and traces afterwards
    for bad in (np.nan, np.inf):
        x = xyz0.copy()
        x[5, 2] = bad
        with pytest.raises(G.SbrError):
            ctx.load_mesh(x, tri0)
        with pytest.raises(G.SbrError):
            ctx.load_mesh(torch.from_numpy(x).cuda(), torch.from_numpy(tri0).cuda())
    ctx.load_mesh(xyz0, tri0)
    om0 = orc.Mesh(xyz0, tri0)
    st, res = _trace_both(G, ctx, orc, om0, ang[:1], 0.006, 3)
    assert_hit_parity(compare_hits(*res[0][0], res[0][1]))


@pytest.mark.parametrize("n_tri", [16383, 16384, 16385])
def test_tree_build_size_limits(G, ctx, orc, n_tri):
    """Meshes at the size where the tree build changes from one block (sort,
    clustering and collapse in one launch, up to 16384 triangles) to a launch
    per clustering round: both trees give every ray the oracle's hits."""
    xyz, tri = S.icosphere(5)
    tri = tri[:n_tri]
    ctx.load_mesh(xyz, tri)
    om = orc.Mesh(xyz, tri)
    st, res = _trace_both(G, ctx, orc, om, np.array([[10.0, 20.0], [200.0, -35.0]]), 0.01, 2, window=2.2)
    assert st["stack_overflows"] == 0
    for g, o, fr in res:
        assert_hit_parity(compare_hits(*g, o))


def test_bounce_hit_count(G, ctx, orc):
    """The counting run's bounce_hits is the number of hits the bounce passes processed: every hit after a
    ray's first, i.e. the sum of (bounces - 1) over the rays, on the GPU's own records and on the oracle's."""
    case = S.trihedral_case()
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ang = case["angles"][[10, 77, 150]]
    for raster in (1, 0):
        ctx.set_tuning(raster=raster)
        st, res = _trace_both(G, ctx, orc, om, ang, case["spacing"], 3, eta=case["eta"], offset=case["offset"],
                              flags=G.TRACE_COUNT_VISITS)
        own = sum(int(np.maximum(g[2] - 1, 0).sum()) for g, o, fr in res)
        ref = sum(int(np.maximum(o["nb"].astype(np.int64) - 1, 0).sum()) for g, o, fr in res)
        assert st["bounce_hits"] == own
        assert abs(own - ref) <= 1e-5 * max(ref, 1) + 2  # hit decisions equal outside the edge band
        assert st["bounce_hits"] > 0
        # rasterised primary hits are rebuilt by bounce pass 1 from the hit list (no aspect falls back here)
        assert st["listed_hits"] == (st["valid_rays"] if raster else 0)
    ctx.set_tuning(raster=1)


def test_all_rays_miss_gives_empty_sum(G, ctx):
    xyz, tri = S.square_plate(1.0, 2)
    ctx.load_mesh(xyz, tri)
    st = ctx.trace([[0.0, 0.0]], 0.01, max_bounces=2)  # grazing along the plate plane
    assert st["valid_rays"] == 0 and st["ray_bounces"] == st["rays_launched"]
    E, R = ctx.po_integrate([1e9, 2e9], "HH,VV")
    assert np.all(E == 0) and np.all(np.isneginf(R))


@pytest.mark.parametrize("leaf", [1, 2, 8, 16])
def test_leaf_sizes_same_hits(G, ctx, orc, leaf):
    xyz, tri = S.icosphere(4)
    ctx.load_mesh(xyz, tri)
    ctx.build_bvh(leaf_max=leaf, builder="lbvh")
    om = orc.Mesh(xyz, tri)
    st, res = _trace_both(G, ctx, orc, om, np.array([[12.0, 34.0]]), 0.01, 1, window=2.2)
    assert_hit_parity(compare_hits(*res[0][0], res[0][1]))


@pytest.mark.parametrize("leaf,radius", [(1, 0), (4, 0), (4, 1), (16, 64)])
def test_ploc_tree_same_hits(G, ctx, orc, leaf, radius):
    """The clustering-built tree gives every ray the oracle's hits (sphere and
    trihedral, 3 bounces) and, on the trihedral, fewer node visits than the
    Karras LBVH."""
    for xyz, tri, ang, sp, B, win in ((*S.icosphere(4), [[12.0, 34.0]], 0.01, 1, 2.2),
                                      (*S.trihedral(1.0, 32), [[30.0, 35.26], [72.5, 35.26]], 0.006, 3, 0.0)):
        ctx.load_mesh(xyz, tri)
        om = orc.Mesh(xyz, tri)
        ctx.build_bvh(leaf_max=leaf, builder="lbvh")
        lb = ctx.trace(ang, sp, max_bounces=B, window=win, flags=G.TRACE_COUNT_VISITS)
        ctx.build_bvh(leaf_max=leaf, builder="ploc", ploc_radius=radius)
        st, res = _trace_both(G, ctx, orc, om, np.array(ang), sp, B, window=win)
        for g, o, _ in res:
            assert_hit_parity(compare_hits(*g, o))
        pl = ctx.trace(ang, sp, max_bounces=B, window=win, flags=G.TRACE_COUNT_VISITS)
        assert pl["ray_bounces"] == lb["ray_bounces"] and pl["stack_overflows"] == 0
        if B == 3 and radius != 1 and leaf == 4:
            assert pl["node_visits"] < lb["node_visits"], (pl["node_visits"], lb["node_visits"])


def test_ploc_tree_aircraft(G, ctx, orc):
    """~1M triangles: the clustering tree traces the same hits as the Karras
    tree on both tree widths."""
    case = S.aircraft_case(1e9, n_az=360)
    ctx.load_mesh(case["xyz"], case["tri"])
    ang = case["angles"][[0, 120]]
    kw = dict(eta=case["eta"], max_bounces=case["max_bounces"], offset=case["offset"])
    ctx.build_bvh(builder="lbvh")
    ctx.trace(ang, case["spacing"], flags=G.TRACE_RECORD_HITS, **kw)
    ref = [ctx.get_hits(a) for a in range(len(ang))]
    ctx.build_bvh(builder="ploc")
    for w in (2, 4):
        ctx.set_tuning(bvh_width=w)
        st = ctx.trace(ang, case["spacing"], flags=G.TRACE_RECORD_HITS, **kw)
        assert st["stack_overflows"] == 0
        for a in range(len(ang)):
            for x, y in zip(ref[a], ctx.get_hits(a)):
                assert np.array_equal(x, y)
    ctx.set_tuning(bvh_width=2)


def test_chunked_trace_matches_single_chunk(G, ctx):
    case = S.trihedral_case(az_step=10.0)
    ctx.load_mesh(case["xyz"], case["tri"])
    sp = 3 * case["spacing"]
    a = ctx.trace(case["angles"], sp, max_bounces=3)
    E1, R1 = ctx.po_integrate([10e9, 11e9], "HH,VV,HV,VH")
    b = ctx.trace(case["angles"], sp, max_bounces=3, chunk_rays=70_000)
    E2, R2 = ctx.po_integrate([10e9, 11e9], "HH,VV,HV,VH")
    for k in ("rays_launched", "ray_bounces", "valid_rays", "stack_overflows"):
        assert a[k] == b[k], k
    assert b["kernel_launches"] > a["kernel_launches"]  # several chunks
    assert np.array_equal(E1, E2)


def _hits_fields(G, case, angles, B, chunk_rays, flags=0, sp=1.0):
    """Trace in a fresh context (its ray queues sized by this trace's chunks)."""
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        st = c.trace(angles, sp * case["spacing"], eta=case["eta"], max_bounces=B, offset=case["offset"],
                     flags=HITS | flags, chunk_rays=chunk_rays)
        hits = [c.get_hits(a) for a in range(len(angles))]
        E, R = c.po_integrate([float(case["freqs"][0]), 0.9 * float(case["freqs"][0])], "HH,VV,HV,VH")
        recs = [c.get_records(a) for a in range(len(angles))]
    return st, hits, E, R, recs


def _assert_same(a, b):
    sa, ha, Ea, Ra, ra = a
    sb, hb, Eb, Rb, rb = b
    for k in ("rays_launched", "ray_bounces", "valid_rays", "stack_overflows", "bounce_hits"):
        assert sa[k] == sb[k], k
    for x, y in zip(ha, hb):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)
    for x, y in zip(ra, rb):
        for k in x:
            assert np.array_equal(x[k], y[k]), k
    assert np.array_equal(Ea, Eb) and np.array_equal(Ra, Rb)


def test_pooled_late_passes_match_per_chunk_passes(G):
    """A trace of several chunks runs the bounce passes after the first once
    over the rays of all chunks (the ray pool). On the aircraft at 1 GHz (ten
    bounces, 12 aspects in chunks of 2^18 rays) every ray's hits, every record
    and the fields equal, bit for bit, those of the same aspects traced as one
    chunk, whose passes all run per chunk."""
    case = S.aircraft_case(1e9, n_az=360)
    ang = case["angles"][::30]
    B = case["max_bounces"]
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        n_chunks = c.trace(ang, case["spacing"], eta=case["eta"], max_bounces=2, offset=case["offset"],
                           chunk_rays=1 << 18)["pass_launches"] // 2
    assert n_chunks >= 6
    one = _hits_fields(G, case, ang, B, 0)
    pooled = _hits_fields(G, case, ang, B, 1 << 18)
    # per chunk the primary pass and bounce pass 1; passes 2 .. B - 1 once over the pool
    assert pooled[0]["pass_launches"] == 2 * n_chunks + (B - 2)
    _assert_same(one, pooled)


def test_ray_pool_overflow_flushes_and_keeps_results(G):
    """When the rays a chunk leaves for the late passes do not fit the pool
    (which holds as many rays as a chunk), the pool is traced first and the
    chunk's rays appended again: the trihedral's multi-bounce rays in chunks of
    2^16 rays overflow it several times, and the hits, records and fields still
    equal those of one chunk. The escape-required variant (one extra query per
    ray still hitting) goes through the same pooled passes."""
    case = S.trihedral_case()
    ang = case["angles"][::20]
    # chunks: with B = 2 no pass is pooled, one primary and one bounce pass per chunk
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        n_chunks = c.trace(ang, 3 * case["spacing"], eta=case["eta"], max_bounces=2, offset=case["offset"],
                           chunk_rays=1 << 16)["pass_launches"] // 2
    assert n_chunks >= 4
    one = _hits_fields(G, case, ang, 3, 0, sp=3.0)
    pooled = _hits_fields(G, case, ang, 3, 1 << 16, sp=3.0)
    # one pooled pass per flush: more than one flush means the pool overflowed
    assert pooled[0]["pass_launches"] - 2 * n_chunks >= 2
    _assert_same(one, pooled)
    esc = G.TRACE_REQUIRE_ESCAPE
    _assert_same(_hits_fields(G, case, ang, 3, 0, esc, sp=3.0), _hits_fields(G, case, ang, 3, 1 << 16, esc, sp=3.0))


def test_many_aspects_match_split_calls(G, ctx):
    """20,000 aspects in one call (a staging upload above the first pinned
    buffer, a PO work list of 20,000 aspect rows expanded on the device) give
    the same fields, bit for bit, as the same aspects in four calls."""
    xyz, tri = S.dihedral(1.0, 4)
    ctx.load_mesh(xyz, tri)
    rng = np.random.default_rng(21)
    ang = np.stack([rng.uniform(0.0, 360.0, 20_000), rng.uniform(-30.0, 60.0, 20_000)], 1)
    st = ctx.trace(ang, 0.1, max_bounces=2)
    E1, R1 = ctx.po_integrate([3e9, 5e9], "HH,VV")
    assert st["n_angles"] == 20_000 and st["valid_rays"] > 0
    valid = 0
    for k in range(4):
        part = ctx.trace(ang[k * 5000:(k + 1) * 5000], 0.1, max_bounces=2)
        valid += part["valid_rays"]
        E2, R2 = ctx.po_integrate([3e9, 5e9], "HH,VV")
        assert np.array_equal(E1[k * 5000:(k + 1) * 5000], E2)
        assert np.array_equal(R1[k * 5000:(k + 1) * 5000], R2)
    assert valid == st["valid_rays"]


def test_deterministic_results(G, ctx):
    case = S.trihedral_case(az_step=15.0)
    ctx.load_mesh(case["xyz"], case["tri"])
    outs = []
    for _ in range(2):
        ctx.trace(case["angles"], case["spacing"], max_bounces=3)
        outs.append(ctx.po_integrate([9e9, 10e9, 11e9], "HH,VV,HV,VH")[0])
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("B", [1, 2, 3, 5])
def test_bounce_limits_and_escape(G, ctx, orc, B):
    xyz, tri = S.trihedral(1.0, 8)
    ctx.load_mesh(xyz, tri)
    om = orc.Mesh(xyz, tri)
    ang = np.array([[45.0, 35.26], [20.0, 20.0]])
    for flags in (0, 2):
        st, res = _trace_both(G, ctx, orc, om, ang, 0.01, B, flags=flags)
        E, R = ctx.po_integrate([10e9], "HH,VV")
        for a, (g, o, fr) in enumerate(res):
            assert_hit_parity(compare_hits(*g, o))
            Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], [10e9])
            assert_rcs_close(R[a, 0], Ro[0, :2])


def test_multifrequency_and_phase_precision(G, ctx, orc):
    case = S.trihedral_case()
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ang = case["angles"][[30, 90]]
    freqs = np.linspace(8e9, 12e9, 17)
    ctx.trace(ang, case["spacing"], max_bounces=3, offset=case["offset"])
    errs = {}
    for ph in ("compensated", "fp64", "fp32"):
        E, R = ctx.po_integrate(freqs, "HH,VV", phase=ph)
        e = 0.0
        for a, (az, el) in enumerate(ang):
            _, Ro, _, _ = orc.rcs_angle(om, om.bbox, az, el, case["spacing"], freqs, 3, eta=case["eta"],
                                        offset=case["offset"])
            e = max(e, assert_rcs_close(R[a], Ro[:, :2], tol=0.5))
        errs[ph] = e
    assert errs["compensated"] <= 0.1 and errs["fp64"] <= 0.1
    print("max dB error by phase precision:", errs)


def test_device_outputs_and_torch_stream(G, orc):
    torch = pytest.importorskip("torch")
    st = torch.cuda.Stream()
    c = G.Context(0, stream=st)
    case = S.trihedral_case(az_step=30.0)
    xyz = torch.from_numpy(case["xyz"]).cuda()
    tri = torch.from_numpy(case["tri"]).cuda()
    torch.cuda.synchronize()
    c.load_mesh(xyz, tri)
    c.trace(case["angles"], case["spacing"], max_bounces=3)
    Eh, Rh = c.po_integrate([10e9], "HH,VV")
    Ed = torch.empty((len(case["angles"]), 1, 2, 2), dtype=torch.float64, device="cuda")
    Rd = torch.empty((len(case["angles"]), 1, 2), dtype=torch.float64, device="cuda")
    c.po_integrate([10e9], "HH,VV", E_out=Ed, rcs_out=Rd)
    st.synchronize()
    assert np.array_equal(Rd.cpu().numpy(), Rh)
    assert np.array_equal(Ed.cpu().numpy()[..., 0], Eh.real)
    c.close()


def test_records_match_oracle_coefficients(G, ctx, orc):
    case = S.trihedral_case()
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    az, el = case["angles"][70]
    ctx.trace([[az, el]], case["spacing"], max_bounces=3, offset=case["offset"])
    r = ctx.get_records(0)
    fr = orc.make_frame(om.bbox, az, el, case["spacing"], eta=case["eta"], offset=case["offset"])
    o = orc.trace(om, fr, 3, ids=r["ray"])
    o_s = orc.trace(om, fr, 3, ids=r["ray"], po_mode="scalar")
    assert np.all(o["valid"] == 1)
    scale = 2 * case["spacing"] ** 2
    assert np.max(np.abs(r["coef"][:, :4] - o["coef"])) < 1e-4 * scale
    assert np.max(np.abs(r["coef"][:, 4] - o_s["coef"][:, 0])) < 1e-4 * scale
    assert np.max(np.abs(r["L"] - o["L"])) < 2e-6


def test_aircraft_sampled_parity(G, ctx, orc):
    # 1M-triangle aircraft at 1 GHz (lambda/10 grid), two aspects, up to 10 bounces
    case = S.aircraft_case(1e9, n_az=360)
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ang = case["angles"][[0, 30]]
    st, res = _trace_both(G, ctx, orc, om, ang, case["spacing"], 10, eta=case["eta"], offset=case["offset"])
    E, R = ctx.po_integrate(case["freqs"], "HH,VV")
    for a, (g, o, fr) in enumerate(res):
        s = compare_hits(*g, o)
        assert_hit_parity(s)
        Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], case["freqs"])
        assert_rcs_close(R[a, 0], Ro[0, :2])


def test_deep_cavity_escape_parity(G, ctx, orc):
    """Nose-on view into the two 3 m engine inlets of the aircraft at 1 GHz: up
    to 100 bounces, a ray still hitting after them is invalid. Every ray's hits,
    bounce count and the RCS match the oracle."""
    case = S.aircraft_case(1e9, n_az=360)
    ctx.load_mesh(case["xyz"], case["tri"])
    om = orc.Mesh(case["xyz"], case["tri"])
    ang = case["angles"][[180]]
    st, res = _trace_both(G, ctx, orc, om, ang, case["spacing"], 100, eta=case["eta"], offset=case["offset"],
                          flags=G.TRACE_REQUIRE_ESCAPE)
    E, R = ctx.po_integrate(case["freqs"], "HH,VV")
    g, o, fr = res[0]
    assert_hit_parity(compare_hits(*g, o))
    assert int(o["nb"].max()) > 10  # rays do bounce deep inside the inlets
    Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], case["freqs"])
    assert_rcs_close(R[0, 0], Ro[0, :2])


# ----------------------------------------------------------------------------- bistatic variant
def _blocked_plate():
    plate_xyz, plate_tri = S.square_plate(1.0, 8)
    xb, z0, z1 = 0.30131, 0.05, 0.35
    bl = np.array([[xb, -0.6, z0], [xb, 0.6, z0], [xb, 0.6, z1], [xb, -0.6, z1]], np.float32)
    nv = len(plate_xyz)
    xyz = np.concatenate([plate_xyz, bl]).astype(np.float32)
    tri = np.concatenate([plate_tri, np.array([[nv, nv + 1, nv + 2], [nv, nv + 2, nv + 3]])]).astype(np.int32)
    return xyz, tri


def _bistatic_compare(G, ctx, orc, xyz, tri, tx, rx, sp, B, freqs, window=0.0, offset=(0.0, 0.0)):
    ctx.load_mesh(xyz, tri)
    om = orc.Mesh(xyz, tri)
    ctx.trace(tx, sp, max_bounces=B, window=window, offset=offset, rx=rx, flags=HITS)
    E, R = ctx.po_integrate(freqs, "HH,VV,HV,VH")
    for a in range(len(tx)):
        fr = orc.make_frame(om.bbox, tx[a][0], tx[a][1], sp, window=window, offset=offset, rx=rx[a])
        o = orc.trace(om, fr, B)
        assert_hit_parity(compare_hits(*ctx.get_hits(a), o))
        rec = ctx.get_records(a)
        vis = np.zeros(fr.n_rays, bool)
        vis[rec["ray"]] = np.any(rec["coef"][:, :4] != 0, axis=1)
        assert np.array_equal(vis, o["valid"].astype(bool))  # every visibility decision
        Eo, Ro = orc.po(o["coef"], o["L"], o["valid"], freqs)
        assert_rcs_close(R[a, :, :2], Ro[:, :2])
    return R


def test_bistatic_blocker_and_plate(G, ctx, orc):
    # a sub-cell grid offset keeps the regular ray grid off the plate's regular mesh edges (an aligned grid
    # puts whole rows of rays exactly on edges, all in the edge band)
    xyz, tri = _blocked_plate()
    _bistatic_compare(G, ctx, orc, xyz, tri, [[0.0, 90.0], [0.0, 90.0], [0.0, 60.0]],
                      [[0.0, 30.0], [180.0, 40.0], [180.0, 60.0]], 0.004, 1, [10e9, 9e9], window=1.3,
                      offset=(0.37, 0.21))
    # without the blocker, the specular receiver of a 30 deg incidence sees the whole plate:
    # sigma = 4 pi (A cos 30)^2 / lambda^2 (PO closed form)
    pxyz, ptri = S.square_plate(1.0, 8)
    R = _bistatic_compare(G, ctx, orc, pxyz, ptri, [[0.0, 60.0]], [[180.0, 60.0]], 0.003, 1, [10e9], window=1.3,
                          offset=(0.37, 0.21))
    lam = C0 / 10e9
    want = 10 * math.log10(4 * math.pi * math.cos(math.radians(30.0)) ** 2 / lam**2)
    assert abs(R[0, 0, 0] - want) < 0.15 and abs(R[0, 0, 1] - want) < 0.15


def test_bistatic_trihedral_multibounce(G, ctx, orc):
    case = S.trihedral_case()
    tx = case["angles"][[60, 90]]
    rx = np.array([[40.0, 30.0], [60.0, 40.0]])
    _bistatic_compare(G, ctx, orc, case["xyz"], case["tri"], tx, rx, 2 * case["spacing"], 3, [10e9],
                      offset=case["offset"])


def test_bistatic_pooled_passes_match_one_chunk(G):
    """Bistatic aspects in chunks: the pooled late passes keep each aspect's
    receiver (its visibility queries and radiation toward it), so the trihedral
    traced in chunks of 2^16 rays gives the hits, records and fields of one
    chunk, bit for bit."""
    case = S.trihedral_case()
    tx = case["angles"][::30]
    rx = np.stack([np.linspace(20.0, 70.0, len(tx)), np.linspace(25.0, 45.0, len(tx))], 1)
    out = []
    for chunk in (0, 1 << 16):
        with G.Context(0) as c:
            c.load_mesh(case["xyz"], case["tri"])
            st = c.trace(tx, 3 * case["spacing"], eta=case["eta"], max_bounces=3, offset=case["offset"], flags=HITS,
                         chunk_rays=chunk, rx=rx)
            out.append((st, [c.get_hits(a) for a in range(len(tx))], *c.po_integrate([10e9], "HH,VV,HV,VH"),
                        [c.get_records(a) for a in range(len(tx))]))
    assert out[1][0]["pass_launches"] > out[0][0]["pass_launches"]  # several chunks
    _assert_same(out[0], out[1])


def test_bistatic_at_transmitter_matches_monostatic_single_bounce(G, ctx):
    xyz, tri = S.square_plate(1.0, 8)
    ctx.load_mesh(xyz, tri)
    ang = np.array([[0.0, 90.0], [20.0, 75.0]])
    ctx.trace(ang, 0.004, max_bounces=1, window=1.3)
    E0, R0 = ctx.po_integrate([10e9], "HH,VV")
    ctx.trace(ang, 0.004, max_bounces=1, window=1.3, rx=ang)
    E1, R1 = ctx.po_integrate([10e9], "HH,VV")
    assert np.array_equal(E0, E1)
