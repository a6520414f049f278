"""Pins of the FP64 CPU oracle against results fixed by the paper and by
mathematics (closed forms, limits, invariants, brute force), independent of the
oracle's own code. CPU only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import sbr_inputs as S

C0 = 299_792_458.0
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def db(x):
    return 10.0 * math.log10(x)


# ----------------------------------------------------------------------------- Mie series
def test_mie_rayleigh_limit(orc):
    # PEC sphere, ka << 1: sigma = 9 pi a^2 (ka)^4 (Rayleigh)
    for x in (1e-3, 1e-2):
        q = orc.mie_pec_backscatter(x)
        assert abs(q / (9 * x**4) - 1) < 5 * x**2


def test_mie_optical_limit(orc):
    # ka >> 1: sigma -> pi a^2 (geometric optics)
    for x in (500.0, 2000.0, 8000.0):
        assert abs(db(orc.mie_pec_backscatter(x))) < 0.01


def test_mie_matches_library_bessel(orc):
    # same series evaluated with scipy's spherical Bessel routines (independent recurrences)
    sp = pytest.importorskip("scipy.special")
    for x in (0.7, 3.0, 12.5, 62.9):
        n = np.arange(1, int(x + 4 * x ** (1 / 3) + 10) + 1)
        jn, yn = sp.spherical_jn(n, x), sp.spherical_yn(n, x)
        jd, yd = sp.spherical_jn(n, x, True), sp.spherical_yn(n, x, True)
        psi, dpsi = x * jn, jn + x * jd
        chi, dchi = -x * yn, -(yn + x * yd)
        a = dpsi / (dpsi - 1j * dchi)
        b = psi / (psi - 1j * chi)
        s = np.sum((2 * n + 1) * (-1.0) ** n * (a - b))
        q = abs(s) ** 2 / x**2
        assert orc.mie_pec_backscatter(x) == pytest.approx(q, rel=1e-9)


def test_mie_near_pi_a2_at_ka63(orc):
    ka = 2 * math.pi * 3.0e9 / C0
    assert abs(db(orc.mie_pec_backscatter(ka))) < 0.1


# ----------------------------------------------------------------------------- frame (Eq. L1-L3)
def test_frame_extents_and_grid(orc):
    bbox = np.array([-0.5, -0.5, -0.5, 0.5, 0.5, 0.5], np.float32)
    ds = 0.01
    f = orc.make_frame(bbox, 0.0, 0.0, ds, eta=0.05)
    assert f.Lu == pytest.approx(1.0) and f.Lv == pytest.approx(1.0)
    assert f.nu == math.ceil(1.05 / ds - 1e-9) and f.nv == f.nu
    f = orc.make_frame(bbox, 45.0, 0.0, ds, eta=0.05)
    assert f.Lu == pytest.approx(math.sqrt(2.0)) and f.Lv == pytest.approx(1.0)
    # the eight corners of a unit cube seen along the body diagonal span 2*sqrt(2/3) in v
    f = orc.make_frame(bbox, 45.0, math.degrees(math.atan(1 / math.sqrt(2))), ds, eta=0.0)
    assert f.Lv == pytest.approx(2 * math.sqrt(2.0 / 3.0))
    # ray grid: centred on the box, spacing ds, direction -r, basis orthonormal
    f = orc.make_frame(bbox, 30.0, 20.0, ds, eta=0.05)
    d = np.array(f.d, np.float64)
    r = np.array([math.cos(math.radians(20)) * math.cos(math.radians(30)),
                  math.cos(math.radians(20)) * math.sin(math.radians(30)), math.sin(math.radians(20))])
    assert np.allclose(d, -r, atol=1e-7)
    o00 = np.array(orc.ray(f, 0, 0)[0], np.float64)
    o11 = np.array(orc.ray(f, f.nu - 1, f.nv - 1)[0], np.float64)
    mid = 0.5 * (o00 + o11)
    assert np.linalg.norm(mid - np.dot(mid, d) * d) < 1e-5  # centre ray passes through the box centre
    o10 = np.array(orc.ray(f, 1, 0)[0], np.float64)
    o01 = np.array(orc.ray(f, 0, 1)[0], np.float64)
    assert np.linalg.norm(o10 - o00) == pytest.approx(ds, rel=1e-4)
    assert abs(np.dot(o10 - o00, o01 - o00)) < 1e-8 and abs(np.dot(o10 - o00, d)) < 1e-8
    # origins lie on the upstream side of the box
    assert np.dot(o00, d) < -0.87


def test_window_mode_counts(orc):
    bbox = np.array([-1, -1, -1, 1, 1, 1], np.float32)
    f = orc.make_frame(bbox, 0.0, 0.0, 0.01, window=2.2)
    assert (f.nu, f.nv) == (220, 220)


# ----------------------------------------------------------------------------- reflection
def test_reflection_invariants(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        e1 = np.cross(d, rng.normal(size=3)); e1 /= np.linalg.norm(e1)
        e2 = np.cross(d, e1)
        d2, f1, f2 = orc.reflect(n, d, e1, e2)
        assert abs(np.linalg.norm(d2) - 1) < 1e-14
        assert np.dot(d2, n) == pytest.approx(-np.dot(d, n), abs=1e-14)
        for e, f in ((e1, f1), (e2, f2)):
            assert abs(np.linalg.norm(f) - 1) < 1e-14
            assert abs(np.dot(f, d2)) < 1e-14              # stays transverse
            assert np.dot(f, n) == pytest.approx(np.dot(e, n), abs=1e-14)  # normal part kept
            t_in, t_out = e - np.dot(e, n) * n, f - np.dot(f, n) * n
            assert np.allclose(t_out, -t_in, atol=1e-14)   # tangential part reversed (PEC)


# ----------------------------------------------------------------------------- intersection
def _random_soup(n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, size=(n, 1, 3))
    v = (c + 0.15 * rng.normal(size=(n, 3, 3))).reshape(-1, 3).astype(np.float32)
    return v, np.arange(3 * n, dtype=np.int32).reshape(n, 3)


@pytest.mark.parametrize("which", ["ico3", "trihedral", "soup"])
def test_bvh_equals_brute_force(orc, which):
    if which == "ico3":
        xyz, tri = S.icosphere(3)
    elif which == "trihedral":
        xyz, tri = S.trihedral(1.0, 8)
    else:
        xyz, tri = _random_soup(300, 7)
    m = orc.Mesh(xyz, tri, bvh_leaf=2)
    rng = np.random.default_rng(3)
    for leaf in (1, 2, 4):
        m.build_bvh(leaf)
        for az, el in ((10.0, 20.0), (45.0, 35.26), (200.0, -40.0)):
            f = orc.make_frame(m.bbox, az, el, 0.05, eta=0.05)
            ids = rng.choice(f.n_rays, size=min(400, f.n_rays), replace=False)
            a = orc.trace(m, f, 3, ids=ids, use_bvh=True)
            b = orc.trace(m, f, 3, ids=ids, use_bvh=False)
            for key in ("hit_tri", "hit_t", "coef", "band", "bmin", "nb", "valid"):
                assert np.array_equal(a[key], b[key]), key
            assert a["counters"][0] < b["counters"][0]


def test_single_triangle_hit_distance(orc):
    # one triangle in the plane z = 0.3; a ray straight down from z = 2 hits at t = 1.7
    xyz = np.array([[-1, -1, 0.3], [1, -1, 0.3], [0, 1, 0.3]], np.float32)
    m = orc.Mesh(xyz, np.array([[0, 1, 2]], np.int32), bvh_leaf=None)
    k, t, bmin, t2 = m.closest_hit([0.1, 0.0, 2.0], [0, 0, -1.0])
    assert k == 0 and t == pytest.approx(2.0 - np.float64(np.float32(0.3)), rel=1e-15)
    assert math.isinf(t2)
    # outside the triangle: miss; exactly on the edge y = -1: inclusive hit, in the edge band
    assert m.closest_hit([1.5, 0.0, 2.0], [0, 0, -1.0])[0] == -1
    k, t, bmin, _ = m.closest_hit([0.0, -1.0, 2.0], [0, 0, -1.0])
    assert k == 0 and bmin < 1e-6
    # the skipped triangle is never reported
    assert m.closest_hit([0.1, 0.0, 2.0], [0, 0, -1.0], skip=0)[0] == -1


def _degenerate_extras(n_vert):
    """Vertices inside the unit trihedral's box and triangles on them whose
    edges are parallel or nearly so: repeated vertices, an exactly collinear
    midpoint, a sliver with edge-angle sine ~5e-7 (all degenerate), plus one
    thin but valid sliver (sine ~1e-3)."""
    a = np.array([0.21, 0.33, 0.27], np.float32)
    b = np.array([0.62, 0.18, 0.44], np.float32)
    mid = ((a.astype(np.float64) + b) / 2).astype(np.float32)
    v = np.stack([a, b, mid,
                  np.array([0.1, 0.1, 0.6], np.float32), np.array([0.9, 0.1, 0.6], np.float32),
                  np.array([0.9, 0.1 + 4e-7, 0.6], np.float32), np.array([0.9, 0.1008, 0.6], np.float32)])
    n = n_vert
    deg = np.array([[n, n + 1, n + 1], [n, n, n + 1], [n + 1, n + 1, n + 1], [n, n + 1, n + 2],
                    [n + 3, n + 4, n + 5]], np.int32)
    thin = np.array([[n + 3, n + 4, n + 6]], np.int32)
    return v, deg, thin


def test_degenerate_triangles_take_no_hits(orc):
    """A triangle whose edges are parallel to within a sine of 2^-20 has no
    usable normal and is never hit: a ray aimed through the inside of such
    a sliver misses it while the same ray hits a thin but valid sliver (sine
    ~1e-3); the ordinary meshes have no such triangle; adding degenerate
    triangles to a mesh leaves every ray's hits, fields and path bit for bit."""
    xyz0, tri0 = S.trihedral(1.0, 8)
    v, deg, thin = _degenerate_extras(len(xyz0))
    xyz = np.concatenate([xyz0, v])
    # the sliver spans x in [0.1, 0.9] at y = 0.1 .. 0.1 + 4e-7 x' / 0.8 in the plane z = 0.6
    for use_bvh in (True, False):
        m = orc.Mesh(xyz, deg[4:5], bvh_leaf=4 if use_bvh else None)
        assert m.n_degenerate == 1
        assert m.closest_hit([0.8, 0.1 + 1e-7, 1.5], [0, 0, -1.0], use_bvh=use_bvh)[0] == -1
        m = orc.Mesh(xyz, thin, bvh_leaf=4 if use_bvh else None)
        assert m.n_degenerate == 0
        k, t, _, _ = m.closest_hit([0.8, 0.1 + 1e-4, 1.5], [0, 0, -1.0], use_bvh=use_bvh)
        assert k == 0 and t == pytest.approx(1.5 - 0.6, rel=1e-6)
    for xyz_m, tri_m in (S.trihedral(1.0, 32), S.icosphere(4), S.square_plate(1.0, 8, tilt_deg=30.0)):
        assert orc.Mesh(xyz_m, tri_m, bvh_leaf=None).n_degenerate == 0
    base = orc.Mesh(xyz0, tri0)
    more = orc.Mesh(xyz, np.concatenate([tri0, deg, thin]))
    assert more.n_degenerate == len(deg)
    assert np.array_equal(base.bbox, more.bbox)
    for az, el in ((45.0, 35.26), (20.0, 50.0)):
        fa = orc.make_frame(base.bbox, az, el, 0.01)
        ta, tb = orc.trace(base, fa, 3), orc.trace(more, fa, 3)
        hit_thin = np.any(tb["hit_tri"] == len(tri0) + len(deg), axis=1)
        assert not np.any((tb["hit_tri"] >= len(tri0)) & (tb["hit_tri"] < len(tri0) + len(deg)))
        keep = ~hit_thin
        assert keep.sum() > 0.99 * len(keep)
        for key in ("hit_tri", "hit_t", "nb", "valid", "coef", "L"):
            assert np.array_equal(ta[key][keep], tb[key][keep]), key


def test_duplicate_triangles_resolve_to_the_lower_index(orc):
    """A copy of every triangle appended to the mesh ties with its original at
    every hit (same vertices, same t); the lower index wins, so every ray's
    hits, fields and path equal those of the mesh without copies."""
    xyz, tri = S.trihedral(1.0, 8)
    base = orc.Mesh(xyz, tri)
    dup = orc.Mesh(xyz, np.concatenate([tri, tri]))
    for az, el in ((45.0, 35.26), (10.0, 20.0)):
        f = orc.make_frame(base.bbox, az, el, 0.01)
        ta, tb = orc.trace(base, f, 3), orc.trace(dup, f, 3)
        assert ta["valid"].sum() > 1000
        for key in ("hit_tri", "hit_t", "nb", "valid", "coef", "L"):
            assert np.array_equal(ta[key], tb[key]), key


def test_non_finite_vertices_refused(orc):
    xyz, tri = S.square_plate(1.0, 2)
    for bad in (np.nan, np.inf, -np.inf):
        x = xyz.copy()
        x[3, 1] = bad
        with pytest.raises(ValueError):
            orc.Mesh(x, tri)
    # an unreferenced vertex counts too: it would set the scene box
    x = np.concatenate([xyz, np.array([[0.0, np.nan, 0.0]], np.float32)])
    with pytest.raises(ValueError):
        orc.Mesh(x, tri)


def test_watertight_closed_icosphere(orc):
    # every ray aimed inside the silhouette of a closed mesh must hit it
    xyz, tri = S.icosphere(4)
    m = orc.Mesh(xyz, tri)
    for az, el in ((0.0, 0.0), (17.0, 33.0), (123.4, -61.0)):
        f = orc.make_frame(m.bbox, az, el, 0.004, window=2.2)
        tr = orc.trace(m, f, 1)
        i = np.arange(f.n_rays) % f.nu
        j = np.arange(f.n_rays) // f.nu
        u = (i + 0.5 - f.nu / 2) * f.spacing
        v = (j + 0.5 - f.nv / 2) * f.spacing
        inside = np.hypot(u, v) < 0.97  # inscribed polyhedron covers radius > 0.98
        assert inside.sum() > 150_000
        assert np.all(tr["nb"][inside] == 1)


# ----------------------------------------------------------------------------- PO closed forms
@pytest.mark.parametrize("mode", ["vector", "scalar"])
def test_flat_plate_normal_incidence_exact(orc, mode):
    # sigma = 4 pi A^2 / lambda^2: every ray hitting the plate adds the same phase
    xyz, tri = S.square_plate(1.0, 4)
    m = orc.Mesh(xyz, tri)
    for f in (1e9, 3e9, 10e9):
        lam = C0 / f
        E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, 0.0, 90.0, 0.01, [f], 1, window=1.2, po_mode=mode)
        assert tr["valid"].sum() == 100 * 100
        assert rcs[0, 0] == pytest.approx(db(4 * math.pi * 1.0 / lam**2), abs=1e-8)
        assert rcs[0, 1] == pytest.approx(rcs[0, 0], abs=1e-8)


@pytest.mark.parametrize("mode", ["vector", "scalar"])
def test_tilted_plate_discrete_sum_closed_form(orc, mode):
    # Plate tilted by alpha about x, radar overhead. Hit rows are spaced ds along y;
    # the round trip differs by 2 ds tan(alpha) between rows, so the discrete sum is a
    # Dirichlet kernel: |S| = 2 dA Nx |sin(M b/2) / sin(b/2)|, b = 2 k ds tan(alpha),
    # and the scalar form carries one more cos(alpha).
    a, ds, W = 1.0, 0.01, 1.2
    off = 0.3
    for alpha in (3.0, 10.0, 25.0):
        xyz, tri = S.square_plate(a, 4, tilt_deg=alpha)
        m = orc.Mesh(xyz, tri)
        g = (np.arange(120) + 0.5 - 60 + off) * ds
        nx = int(np.sum(np.abs(g) <= a / 2))
        my = int(np.sum(np.abs(g) <= (a / 2) * math.cos(math.radians(alpha))))
        for f in (3e9, 5e9):
            k = 2 * math.pi * f / C0
            E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, 0.0, 90.0, ds, [f], 1, window=W, offset=(off, off),
                                           po_mode=mode)
            assert tr["valid"].sum() == nx * my
            b = 2 * k * ds * math.tan(math.radians(alpha))
            S_ = 2 * ds * ds * nx * abs(math.sin(my * b / 2) / math.sin(b / 2))
            if mode == "scalar":
                S_ *= math.cos(math.radians(alpha))
            Emag = k / (4 * math.pi) * S_
            peak = k / (4 * math.pi) * 2 * ds * ds * nx * my
            assert abs(abs(E[0, 0]) - Emag) < 2e-4 * peak
            assert abs(abs(E[0, 1]) - Emag) < 2e-4 * peak


def test_two_plate_round_trip_phase(orc):
    # Two plates side by side at heights 0 and dz, normal incidence: the round trip
    # differs by 2 dz, so sigma follows |N1 + N2 exp(j 2 k dz)|^2.
    v1, t1 = S.square_plate(0.4, 2, z0=0.0)
    v2, t2 = S.square_plate(0.4, 2, z0=0.0137)
    v1 = v1 + np.array([-0.3, 0, 0], np.float32)
    v2 = v2 + np.array([0.3, 0, 0], np.float32)
    xyz = np.concatenate([v1, v2])
    tri = np.concatenate([t1, t2 + len(v1)]).astype(np.int32)
    m = orc.Mesh(xyz, tri)
    dz = float(np.float32(0.0137))
    for f in (2e9, 4.4e9, 7.1e9):
        k = 2 * math.pi * f / C0
        E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, 0.0, 90.0, 0.01, [f], 1, window=1.2, offset=(0.25, 0.25))
        n = tr["valid"].sum() // 2
        S_ = 2 * 1e-4 * abs(n + n * np.exp(2j * k * dz))
        # the stored hit distances are FP32 (one rounding of a ~2 m path)
        assert abs(E[0, 0]) == pytest.approx(k / (4 * math.pi) * S_, rel=1e-4)


def test_dihedral_double_bounce_peak(orc):
    # 90-degree dihedral seen along its bisector: every ray bounces twice and returns
    # with the same path, sigma = 4 pi (N dA)^2 / lambda^2 -> 8 pi a^2 b^2 / lambda^2,
    # with HH and VV in antiphase (two reflections).
    f = 10e9
    lam = C0 / f
    ds = lam / 10
    xyz, tri = S.dihedral(1.0, 8)
    m = orc.Mesh(xyz, tri)
    E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, 45.0, 0.0, ds, [f], 2, eta=0.05, offset=(0.25, 0.25))
    nb = tr["nb"][tr["valid"] == 1]
    assert np.all(nb == 2)
    n = int(tr["valid"].sum())
    assert rcs[0, 0] == pytest.approx(db(4 * math.pi * (n * ds * ds) ** 2 / lam**2), abs=1e-3)
    assert abs(db(8 * math.pi / lam**2) - rcs[0, 0]) < 0.05
    assert E[0, 0] == pytest.approx(-E[0, 1], rel=1e-9)
    assert abs(E[0, 2]) < 1e-9 * abs(E[0, 0])


def test_trihedral_peak_and_polarisation(orc):
    # triangular trihedral on its symmetry axis: sigma = 4 pi L^4 / (3 lambda^2),
    # co-polar HH = VV, no cross-polar return; triple-bounce paths all equal.
    f = 10e9
    lam = C0 / f
    xyz, tri = S.trihedral(1.0, 32)
    m = orc.Mesh(xyz, tri)
    el = math.degrees(math.atan(1 / math.sqrt(2)))
    E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, 45.0, el, lam / 10, [f], 3, eta=0.05)
    assert abs(rcs[0, 0] - db(4 * math.pi / (3 * lam**2))) < 0.1
    assert abs(rcs[0, 1] - rcs[0, 0]) < 0.01
    assert rcs[0, 2] < rcs[0, 0] - 60 and rcs[0, 3] < rcs[0, 0] - 60
    L3 = tr["L"][tr["nb"] == 3]
    assert len(L3) > 50_000 and np.ptp(L3) < 1e-4  # retro-reflection: common round trip


def test_trihedral_mirror_symmetry(orc):
    f = 10e9
    lam = C0 / f
    xyz, tri = S.trihedral(1.0, 32)
    m = orc.Mesh(xyz, tri)
    for dlt in (7.0, 21.5):
        r = [orc.rcs_angle(m, m.bbox, 45.0 + s * dlt, 35.26, lam / 10, [f], 3)[1][0] for s in (1, -1)]
        assert abs(r[0][0] - r[1][0]) < 0.25 and abs(r[0][1] - r[1][1]) < 0.25


def test_phase_literal_equals_default_single_bounce(orc):
    xyz, tri = S.icosphere(3)
    m = orc.Mesh(xyz, tri)
    f = orc.make_frame(m.bbox, 20.0, 10.0, 0.02, window=2.2)
    a = orc.trace(m, f, 1, po_mode="scalar")
    b = orc.trace(m, f, 1, po_mode="scalar", phase_literal=True)
    # equal up to the FP32 rounding of the ray direction (|d - k| ~ 1e-7)
    assert np.allclose(a["L"], b["L"], atol=2e-6)


def test_require_escape_drops_trapped(orc):
    # dihedral along the bisector with one allowed bounce: every ray would hit again
    xyz, tri = S.dihedral(1.0, 4)
    m = orc.Mesh(xyz, tri)
    f = orc.make_frame(m.bbox, 45.0, 0.0, 0.05, offset=(0.25, 0.25))
    a = orc.trace(m, f, 1)
    b = orc.trace(m, f, 1, require_escape=True)
    assert a["valid"].sum() > 100 and b["valid"].sum() == 0
    c = orc.trace(m, f, 2, require_escape=True)
    assert c["valid"].sum() == a["valid"].sum()


# ----------------------------------------------------------------------------- sphere vs Mie
def test_sphere_against_mie(orc):
    # C1 geometry: icosphere subdivision 5, r = 1 m, 3 GHz (ka = 62.9), 220 x 220
    # rays over 2.2 m (10 rays per wavelength). The paper's Eq. po_sum (scalar form)
    # is held to the Mie series: 0.5 dB per aspect, and the aspect average within
    # twice the paper's 2.5 % optical-region spread (Fig. 4).
    case = S.sphere_case(n_random=6)
    m = orc.Mesh(case["xyz"], case["tri"])
    f = case["freqs"][0]
    ka = 2 * math.pi * f / C0
    mie = db(math.pi * orc.mie_pec_backscatter(ka))
    vals = []
    for az, el in case["angles"]:
        E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, az, el, case["spacing"], [f], 1, window=case["window"],
                                       po_mode="scalar")
        vals.append(rcs[0, :2])
        assert abs(rcs[0, 0] - mie) < 0.5 and abs(rcs[0, 1] - mie) < 0.5
    mean_lin = np.mean(10 ** (np.array(vals) / 10))
    tol = GOLD["mie_optical_std_fraction"]["value"] * 2
    assert abs(mean_lin / 10 ** (mie / 10) - 1) < tol


def test_sphere_vector_mode_converges_to_mie(orc):
    # The vector form weights every ray alike (no obliquity taper), so the silhouette
    # band, where the round-trip phase changes fastest, is undersampled at 10 rays per
    # wavelength; the error must shrink as the grid is refined (Sec. 4 sampling rule).
    case = S.sphere_case(n_random=0)
    m = orc.Mesh(case["xyz"], case["tri"])
    f = case["freqs"][0]
    mie = db(math.pi * orc.mie_pec_backscatter(2 * math.pi * f / C0))
    err = {}
    for ds in (0.01, 0.00125):
        E, rcs, tr, fr = orc.rcs_angle(m, m.bbox, 0.0, 0.0, ds, [f], 1, window=2.2)
        err[ds] = abs(rcs[0, 0] - mie)
    assert err[0.01] < 1.0
    assert err[0.00125] < 0.1


# ----------------------------------------------------------------------------- edge band and FP32 ray state
def _fl32(x: Fraction) -> float:
    """x rounded to the nearest FP32 value (ties to even), exactly."""
    if x == 0:
        return 0.0
    sgn = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)  # subnormals share the smallest exponent
    q = a / Fraction(2) ** (e - 23)  # 24-bit significand scale
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sgn * float(Fraction(n) * Fraction(2) ** (e - 23))


def _square(z, i0=0):
    """unit square [0, 1]^2 at height z, split along its diagonal (0,0)-(1,1) into two triangles"""
    v = np.array([[0, 0, z], [1, 0, z], [1, 1, z], [0, 1, z]], np.float32)
    return v, np.array([[i0, i0 + 1, i0 + 2], [i0, i0 + 2, i0 + 3]], np.int32)


def test_runner_up_band_on_a_shared_edge(orc):
    """A ray through the shared diagonal of two coplanar triangles hits both at
    the same t: the lower index wins, the hit is on an edge (bit 0) and the
    runner-up ties (bit 1), by brute force and through the BVH alike."""
    xyz, tri = _square(0.5)
    for use_bvh, leaf in ((False, None), (True, 1)):
        m = orc.Mesh(xyz, tri, bvh_leaf=leaf)
        k, t, bmin, t2 = m.closest_hit([0.25, 0.25, 2.0], [0, 0, -1.0], use_bvh=use_bvh)
        assert k == 0 and t == 1.5 and t2 == 1.5 and bmin == 0.0
        # off the diagonal: one triangle, no runner-up
        k, t, bmin, t2 = m.closest_hit([0.75, 0.25, 2.0], [0, 0, -1.0], use_bvh=use_bvh)
        assert k == 0 and math.isinf(t2) and bmin == pytest.approx(0.25)
        k, t, bmin, t2 = m.closest_hit([0.25, 0.75, 2.0], [0, 0, -1.0], use_bvh=use_bvh)
        assert k == 1 and math.isinf(t2)
    # traced from an aperture (el = 90 deg: the FP32 direction keeps a 6e-17 tilt from cos 90 deg, so a
    # diagonal ray meets one triangle at barycentric ~1e-16 from the edge): the rays with i = j, and only
    # they, are in the barycentric band
    m = orc.Mesh(xyz, tri, bvh_leaf=1)
    f = orc.make_frame(m.bbox, 0.0, 90.0, 0.125, window=1.0)
    tr = orc.trace(m, f, 1)
    i, j = np.arange(f.n_rays) % f.nu, np.arange(f.n_rays) // f.nu
    assert tr["valid"].sum() == f.n_rays == 64
    assert np.array_equal((tr["band"] & 1) != 0, i == j)
    assert np.all(tr["bmin"][i == j] < 1e-15) and np.all(tr["bmin"][i != j] > 0.06)


@pytest.mark.parametrize("gap_rel, in_band", [(5e-7, True), (5e-6, False)])
def test_runner_up_band_on_parallel_facets(orc, gap_rel, in_band):
    """Two parallel squares a relative distance gap_rel apart along the ray: the
    nearer one is hit, and the ray is in the edge band (bit 1) exactly when the
    other lies within 1e-6 relative in t; the BVH sees the same runner-up as
    brute force (it keeps boxes up to 1e-5 beyond the closest hit)."""
    t_near = 1.5
    z_far = np.float32(0.5 - gap_rel * t_near)
    va, ta = _square(0.5)
    vb, tb = _square(z_far, i0=4)
    xyz, tri = np.concatenate([va, vb]), np.concatenate([ta, tb])
    got = []
    for use_bvh, leaf in ((False, None), (True, 1), (True, 4)):
        m = orc.Mesh(xyz, tri, bvh_leaf=leaf)
        k, t, bmin, t2 = m.closest_hit([0.7, 0.2, 2.0], [0, 0, -1.0], use_bvh=use_bvh)
        assert k == 0 and t == t_near
        assert t2 == 2.0 - float(z_far)
        assert ((t2 - t) <= 1e-6 * t) == in_band
        got.append((k, t, bmin, t2))
    assert got[0] == got[1] == got[2]
    m = orc.Mesh(xyz, tri, bvh_leaf=2)
    f = orc.make_frame(m.bbox, 0.0, 90.0, 0.1, window=0.8, offset=(0.3, 0.3))
    a, b = orc.trace(m, f, 1, use_bvh=True), orc.trace(m, f, 1, use_bvh=False)
    hit = a["nb"] == 1
    assert hit.sum() > 30
    assert np.all(((a["band"][hit] & 2) != 0) == in_band)
    assert np.array_equal(a["band"], b["band"]) and np.array_equal(a["hit_tri"], b["hit_tri"])


def test_fp32_state_is_the_rounded_formula(orc):
    """After a hit, the stored distance is t32 = fl32(((v0 - o).n32) / (d.n32))
    and n32 = fl32(unit normal): both checked against exact rational (and
    60-digit decimal) arithmetic on random triangles and rays, so a dropped
    term, a wrong sign or a transposed operand in either shows up."""
    from decimal import Decimal, getcontext

    getcontext().prec = 60
    rng = np.random.default_rng(17)
    xyz, tri = _random_soup(60, 23)
    m = orc.Mesh(xyz, tri, bvh_leaf=None)
    n32 = m.normals
    for k in range(len(tri)):
        P = [[Fraction(float(c)) for c in xyz[i]] for i in tri[k]]
        e1 = [P[1][c] - P[0][c] for c in range(3)]
        e2 = [P[2][c] - P[0][c] for c in range(3)]
        N = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]]
        ln = sum(Decimal(x.numerator) / Decimal(x.denominator) * Decimal(x.numerator) / Decimal(x.denominator)
                 for x in N).sqrt()
        for c in range(3):
            want = _fl32(Fraction(Decimal(N[c].numerator) / Decimal(N[c].denominator) / ln))
            assert n32[k, c] == np.float32(want), (k, c)
    hits = 0
    for _ in range(300):
        k = int(rng.integers(len(tri)))
        w = rng.dirichlet([1, 1, 1])
        p = (w[:, None] * xyz[tri[k]].astype(np.float64)).sum(0)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = (p - 3.0 * d).astype(np.float32)
        d32 = d.astype(np.float32)
        kk, t, _, _ = m.closest_hit(o.astype(np.float64), d32.astype(np.float64))
        if kk < 0:
            continue
        # the oracle's trace of this one ray: a frame whose grid has the ray at (0, 0) is not available, so
        # the single-ray entry closest_hit gives the triangle and the stored t32 is recomputed here
        v0 = [Fraction(float(c)) for c in xyz[tri[kk]][0]]
        nn = [Fraction(float(c)) for c in n32[kk]]
        of = [Fraction(float(c)) for c in o]
        df = [Fraction(float(c)) for c in d32]
        num = sum((v0[c] - of[c]) * nn[c] for c in range(3))
        den = sum(df[c] * nn[c] for c in range(3))
        t32 = _fl32(num / den)
        # t32 is the distance along the ray to the plane of n32 through v0: within
        # FP32 rounding of the exact hit distance of the triangle itself
        assert abs(t32 - t) <= 4e-7 * t
        hits += 1
    assert hits > 200


def test_trace_stores_the_rounded_distance(orc):
    """Along a traced path the stored hit distances are FP32 values, and on an
    axis-aligned plate seen head-on they equal the plate's distance from the
    aperture (a difference of FP32 values, exact in FP64) rounded once."""
    xyz, tri = S.square_plate(1.0, 4, z0=0.3)
    m = orc.Mesh(xyz, tri)
    f = orc.make_frame(m.bbox, 0.0, 90.0, 0.02, window=1.2)
    tr = orc.trace(m, f, 2)
    hit = tr["nb"] >= 1
    o0 = np.array([orc.ray(f, int(r % f.nu), int(r // f.nu))[0] for r in np.nonzero(hit)[0][:50]])
    # exact in FP64 (a difference of FP32 values), then rounded once to FP32
    want = (o0[:, 2].astype(np.float64) - np.float64(np.float32(0.3))).astype(np.float32).astype(np.float64)
    assert np.array_equal(tr["hit_t"][np.nonzero(hit)[0][:50], 0], want)
    assert np.all(tr["hit_t"].astype(np.float32).astype(np.float64) == tr["hit_t"])


# ----------------------------------------------------------------------------- bistatic variant
def test_bistatic_monostatic_limit(orc):
    # a receiver at the transmitter reproduces the monostatic fields bit for bit (plate, one bounce)
    xyz, tri = S.square_plate(1.0, 4)
    m = orc.Mesh(xyz, tri)
    for az, el in ((0.0, 90.0), (30.0, 70.0)):
        E0, _, _, _ = orc.rcs_angle(m, m.bbox, az, el, 0.01, [10e9, 3e9], 1, window=1.5)
        E1, _, t1, _ = orc.rcs_angle(m, m.bbox, az, el, 0.01, [10e9, 3e9], 1, window=1.5, rx=(az, el))
        assert np.array_equal(E0, E1)


def _plate_bistatic(orc, th_deg, phi_deg, f=10e9, ds=0.003):
    # 1 m x 1 m plate in z = 0; transmitter theta from the normal on the +x side, receiver phi on the -x side
    xyz, tri = S.square_plate(1.0, 8)
    m = orc.Mesh(xyz, tri)
    E, R, tr, fr = orc.rcs_angle(m, m.bbox, 0.0, 90.0 - th_deg, ds, [f], 1, window=1.3,
                                 rx=(180.0, 90.0 - phi_deg))
    return R[0], tr


@pytest.mark.parametrize("th", [0.0, 30.0, 50.0])
def test_bistatic_plate_specular_closed_form(orc, th):
    # PO in the specular direction of a flat PEC plate: sigma = 4 pi (A cos theta)^2 / lambda^2, both polarisations
    lam = C0 / 10e9
    want = db(4 * math.pi * (1.0 * math.cos(math.radians(th))) ** 2 / lam**2)
    R, _ = _plate_bistatic(orc, th, th)
    assert abs(R[0] - want) < 0.15 and abs(R[1] - want) < 0.15, (R[:2], want)


def test_bistatic_plate_null_and_sidelobe(orc):
    # along x the plate is a uniform aperture of length a: |sum| ~ sinc(k a q / 2), q = sin(th) - sin(phi);
    # first null at q = lambda / a, first sidelobe (-13.26 dB) near q = 1.4303 lambda / a. A wrong sign of the
    # receiver path term would move the peak away from the specular direction.
    lam, a, th = C0 / 10e9, 1.0, 30.0
    spec, _ = _plate_bistatic(orc, th, th)
    s_th = math.sin(math.radians(th))
    null, _ = _plate_bistatic(orc, th, math.degrees(math.asin(s_th - lam / a)))
    side, _ = _plate_bistatic(orc, th, math.degrees(math.asin(s_th - 1.4303 * lam / a)))
    # the obliquity factor changes by < 0.1 dB over these few degrees
    assert null[0] < spec[0] - 25.0 and null[1] < spec[1] - 25.0
    assert abs((side[0] - spec[0]) + 13.26) < 0.6 and abs((side[1] - spec[1]) + 13.26) < 0.6
    mono, _ = _plate_bistatic(orc, th, -th)  # receiver back at the transmitter: far off specular
    assert mono[0] < spec[0] - 25.0


def test_bistatic_visibility_by_brute_force(orc):
    # plate in z = 0 lit from the normal; a vertical blocker (normal along x, parallel to the incident rays,
    # so no incident ray hits it) hides part of the plate from a receiver 60 deg toward +x. A hit point at x
    # is hidden exactly when x lies in [xb - z1 tan60, xb - z0 tan60].
    plate_xyz, plate_tri = S.square_plate(1.0, 8)
    xb, z0, z1 = 0.30131, 0.05, 0.35
    bl = np.array([[xb, -0.6, z0], [xb, 0.6, z0], [xb, 0.6, z1], [xb, -0.6, z1]], np.float32)
    xyz = np.concatenate([plate_xyz, bl]).astype(np.float32)
    nv = len(plate_xyz)
    tri = np.concatenate([plate_tri, np.array([[nv, nv + 1, nv + 2], [nv, nv + 2, nv + 3]])]).astype(np.int32)
    m = orc.Mesh(xyz, tri)
    fr = orc.make_frame(m.bbox, 0.0, 90.0, 0.004, window=1.3, rx=(0.0, 30.0))
    tr = orc.trace(m, fr, 1)
    n_blk = len(plate_tri)
    hit_plate = (tr["hit_tri"][:, 0] >= 0) & (tr["hit_tri"][:, 0] < n_blk)
    assert not np.any(tr["hit_tri"][:, 0] >= n_blk)  # the blocker is edge-on to the incident rays
    ids = np.arange(fr.n_rays)
    xs = np.array([orc.ray(fr, int(i % fr.nu), int(i // fr.nu))[0][0] for i in ids[hit_plate]])
    t60 = math.tan(math.radians(60.0))
    lo, hi = xb - z1 * t60, xb - z0 * t60
    hidden = (xs > lo) & (xs < hi)
    near = (np.abs(xs - lo) < 1e-4) | (np.abs(xs - hi) < 1e-4)
    vis = tr["valid"][hit_plate].astype(bool)
    assert np.array_equal(vis[~near], ~hidden[~near])
    assert hidden.sum() > 1000 and (~hidden).sum() > 1000
