"""Procedural PEC meshes: icosphere, trihedral corner reflector, square plate,
dihedral and a seeded aircraft-like body.

Every generator returns ``(xyz, tri)`` with ``xyz`` a C-contiguous
``float32[nv, 3]`` array (metres) and ``tri`` an ``int32[nt, 3]`` array of
vertex indices. Geometry is computed in float64 and rounded once to float32, so
the same call gives bit-identical arrays on every machine.
"""
from __future__ import annotations

import math

import numpy as np


def mesh_bbox(xyz: np.ndarray) -> np.ndarray:
    """Axis-aligned bounding box ``[xmin, ymin, zmin, xmax, ymax, zmax]`` (float32)."""
    xyz = np.asarray(xyz, dtype=np.float32)
    return np.concatenate([xyz.min(axis=0), xyz.max(axis=0)]).astype(np.float32)


def _finish(v: np.ndarray, f: np.ndarray):
    return (np.ascontiguousarray(v, dtype=np.float64).astype(np.float32),
            np.ascontiguousarray(f, dtype=np.int32))


# --------------------------------------------------------------------------- sphere
def icosphere(subdiv: int = 5, radius: float = 1.0):
    """Icosahedron refined ``subdiv`` times by edge midpoints pushed to the sphere.

    ``subdiv = 5`` gives 20 * 4**5 = 20480 triangles and 10242 vertices, all on
    the sphere of the given radius (the mesh is closed and inscribed).
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return _finish(np.array(v) * radius, np.array(faces))


# --------------------------------------------------------------------------- plates
def _tri_grid(p0, p1, p2, n):
    """Split triangle (p0, p1, p2) into n*n congruent triangles.

    Vertex (a, b) sits at p0 + a/n (p1 - p0) + b/n (p2 - p0), a + b <= n.
    """
    p0, p1, p2 = (np.asarray(p, dtype=np.float64) for p in (p0, p1, p2))
    idx = {}
    verts = []
    for a in range(n + 1):
        for b in range(n + 1 - a):
            idx[(a, b)] = len(verts)
            verts.append(p0 + (a / n) * (p1 - p0) + (b / n) * (p2 - p0))
    faces = []
    for a in range(n):
        for b in range(n - a):
            faces.append((idx[(a, b)], idx[(a + 1, b)], idx[(a, b + 1)]))
            if a + b + 1 < n:
                faces.append((idx[(a + 1, b)], idx[(a + 1, b + 1)], idx[(a, b + 1)]))
    return np.array(verts), np.array(faces)


def _merge(parts):
    vs, fs, off = [], [], 0
    for v, f in parts:
        vs.append(v)
        fs.append(f + off)
        off += len(v)
    return np.concatenate(vs), np.concatenate(fs)


def trihedral(leg: float = 1.0, n_seg: int = 32):
    """Triangular trihedral corner reflector with its corner at the origin.

    Three mutually orthogonal isosceles right-triangle plates with legs of
    length ``leg`` along the positive axes; the opening faces (1, 1, 1).
    Each plate is split into ``n_seg**2`` triangles (1024 for n_seg = 32), so
    the whole reflector has ``3 * n_seg**2`` triangles.
    """
    o = (0.0, 0.0, 0.0)
    ex, ey, ez = (leg, 0.0, 0.0), (0.0, leg, 0.0), (0.0, 0.0, leg)
    return _finish(*_merge([_tri_grid(o, ex, ey, n_seg),
                            _tri_grid(o, ey, ez, n_seg),
                            _tri_grid(o, ez, ex, n_seg)]))


def square_plate(side: float = 1.0, m: int = 8, tilt_deg: float = 0.0, z0: float = 0.0):
    """Square plate of the given side, centred on the z axis at height ``z0``.

    The plate starts in the z = z0 plane (normal +z) and is then rotated by
    ``tilt_deg`` about the x axis. It is split into ``2 m**2`` triangles.
    """
    s = np.linspace(-side / 2, side / 2, m + 1)
    gx, gy = np.meshgrid(s, s, indexing="ij")
    v = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, 0.0)], axis=1)
    a = math.radians(tilt_deg)
    rot = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    v = v @ rot.T
    v[:, 2] += z0
    f = []
    for i in range(m):
        for j in range(m):
            p = i * (m + 1) + j
            q = (i + 1) * (m + 1) + j
            f.append((p, q, p + 1))
            f.append((q, q + 1, p + 1))
    return _finish(v, np.array(f))


def dihedral(side: float = 1.0, m: int = 8):
    """Right-angle dihedral: two square plates of the given side meeting along
    the z axis, one in the x-z plane (x >= 0) and one in the y-z plane (y >= 0)."""
    s = np.linspace(0.0, side, m + 1)
    t = np.linspace(-side / 2, side / 2, m + 1)
    parts = []
    for plane in ("xz", "yz"):
        v = []
        for a in s:
            for b in t:
                v.append((a, 0.0, b) if plane == "xz" else (0.0, a, b))
        f = []
        for i in range(m):
            for j in range(m):
                p = i * (m + 1) + j
                q = (i + 1) * (m + 1) + j
                f.append((p, q, p + 1))
                f.append((q, q + 1, p + 1))
        parts.append((np.array(v, dtype=np.float64), np.array(f)))
    return _finish(*_merge(parts))


# --------------------------------------------------------------------------- aircraft
def _naca_half_thickness(x, t=0.12):
    """Symmetric NACA 4-digit half thickness at chord fraction x (closed trailing edge)."""
    return 5 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2 + 0.2843 * x**3 - 0.1036 * x**4)


def _grid_mesh(P, close_u=False):
    """Quad grid of points P[nu, nv, 3] -> triangles; ``close_u`` wraps the u index."""
    nu, nv = P.shape[:2]
    idx = np.arange(nu * nv).reshape(nu, nv)
    f = []
    ur = nu if close_u else nu - 1
    for i in range(ur):
        i2 = (i + 1) % nu
        a = idx[i, :-1]
        b = idx[i2, :-1]
        c = idx[i2, 1:]
        d = idx[i, 1:]
        f.append(np.stack([a, b, c], 1))
        f.append(np.stack([a, c, d], 1))
    return P.reshape(-1, 3), np.concatenate(f)


def _fan_cap(ring_pts, centre):
    """Disk closing a ring of points (n, 3) with a centre vertex."""
    n = len(ring_pts)
    v = np.concatenate([ring_pts, centre[None]])
    f = np.array([(i, (i + 1) % n, n) for i in range(n)])
    return v, f


def _fuselage(L, R, nu, nv):
    # ellipsoid of revolution along x, length L (x in [-L/2, L/2]), max radius R;
    # nv interior rings plus one vertex at each pole, so every vertex is shared
    th = np.linspace(0.0, math.pi, nv + 2)[1:-1]
    ph = np.linspace(0.0, 2 * math.pi, nu, endpoint=False)
    x = -(L / 2) * np.cos(th)
    r = R * np.sin(th)
    P = np.empty((nu, nv, 3))
    P[:, :, 0] = x[None, :]
    P[:, :, 1] = np.cos(ph)[:, None] * r[None, :]
    P[:, :, 2] = np.sin(ph)[:, None] * r[None, :]
    v, f = _grid_mesh(P, close_u=True)
    nose = _fan_cap(P[:, 0, :], np.array([-L / 2, 0.0, 0.0]))
    tail = _fan_cap(P[:, -1, :], np.array([L / 2, 0.0, 0.0]))
    return _merge([(v, f), (nose[0], nose[1][:, ::-1]), tail])


def _wing(root_x, root_chord, tip_chord, semi_span, sweep_deg, y0, z0, n_chord, n_span, side,
          vertical=False, t=0.12):
    """One lifting surface with a symmetric NACA section; ``side`` = +1/-1 mirrors it."""
    # cosine-spaced chord stations, upper then lower surface -> closed loop around the section
    s = 0.5 * (1 - np.cos(np.linspace(0, math.pi, n_chord)))
    xs = np.concatenate([s, s[::-1][1:-1]])
    sign = np.concatenate([np.ones(n_chord), -np.ones(n_chord - 2)])
    ht = _naca_half_thickness(xs, t) * sign
    etas = np.linspace(0.0, 1.0, n_span)
    tan_sw = math.tan(math.radians(sweep_deg))
    P = np.empty((len(xs), n_span, 3))
    for k, eta in enumerate(etas):
        chord = root_chord + (tip_chord - root_chord) * eta
        span = eta * semi_span
        xle = root_x + span * tan_sw
        px = xle + xs * chord
        pt = ht * chord
        if vertical:
            P[:, k, 0], P[:, k, 1], P[:, k, 2] = px, y0 + pt, z0 + span
        else:
            P[:, k, 0], P[:, k, 1], P[:, k, 2] = px, y0 + side * span, z0 + pt
    v, f = _grid_mesh(P, close_u=True)
    # close the tip with a fan
    tip = P[:, -1, :]
    vc, fc = _fan_cap(tip, tip.mean(axis=0))
    if (side < 0) and not vertical:
        f = f[:, ::-1]
        fc = fc[:, ::-1]
    return _merge([(v, f), (vc, fc)])


def _inlet(cx, cy, cz, radius, depth, n_ang, n_depth, wall=0.04):
    """Open cylindrical duct along +x starting at x = cx (mouth) and ending in a
    closed back disk at x = cx + depth; inner wall plus outer skin and a lip."""
    ph = np.linspace(0.0, 2 * math.pi, n_ang, endpoint=False)
    xs = np.linspace(cx, cx + depth, n_depth)
    parts = []
    for r in (radius, radius + wall):
        P = np.empty((n_ang, n_depth, 3))
        P[:, :, 0] = xs[None, :]
        P[:, :, 1] = cy + r * np.cos(ph)[:, None]
        P[:, :, 2] = cz + r * np.sin(ph)[:, None]
        parts.append(_grid_mesh(P, close_u=True))
    # lip: annulus at the mouth
    P = np.empty((n_ang, 2, 3))
    for j, r in enumerate((radius, radius + wall)):
        P[:, j, 0] = cx
        P[:, j, 1] = cy + r * np.cos(ph)
        P[:, j, 2] = cz + r * np.sin(ph)
    parts.append(_grid_mesh(P, close_u=True))
    # back disk closing the duct
    ring = np.stack([np.full(n_ang, cx + depth), cy + radius * np.cos(ph), cz + radius * np.sin(ph)], 1)
    parts.append(_fan_cap(ring, np.array([cx + depth, cy, cz])))
    return _merge(parts)


def aircraft(seed: int = 1, target_tris: int = 1_000_000, jitter_sigma: float = 1e-3):
    """Seeded aircraft-like PEC body of roughly ``target_tris`` triangles.

    Fuselage: 15 m ellipsoid of revolution, radius 1.5 m, along x (nose at -x).
    Wings: root chord 4 m, tip chord 1.2 m, semi-span 7 m, 30 deg sweep, NACA
    0012-like section. Horizontal tail: semi-span 3 m; vertical tail 3 m high.
    Two open cylindrical engine inlets (radius 0.5 m, 3 m deep, closed back
    disk) under the wings, mouths facing -x. Every vertex is jittered once by
    N(0, jitter_sigma^2) per coordinate with ``numpy.random.default_rng(seed)``
    (shared vertices move together, so each component stays watertight).
    """
    # resolution scale: triangles grow ~ s^2
    s = math.sqrt(target_tris / 1_000_000)

    def n(x):
        return max(4, int(round(x * s)))

    parts = [_fuselage(15.0, 1.5, n(600), n(340))]
    for side in (+1, -1):
        parts.append(_wing(-2.0, 4.0, 1.2, 7.0, 30.0, side * 1.2, -0.4, n(150), n(300), side))
        parts.append(_wing(4.6, 1.8, 0.8, 3.0, 35.0, side * 0.4, 0.3, n(70), n(110), side))
        parts.append(_inlet(-2.5, side * 3.2, -1.3, 0.5, 3.0, n(200), n(80)))
    parts.append(_wing(4.2, 2.2, 1.0, 3.0, 40.0, 0.0, 0.5, n(70), n(110), +1, vertical=True))
    v, f = _merge(parts)
    # weld coincident vertices (seams, caps, lips) so the jitter keeps them together
    v, inv = np.unique(v, axis=0, return_inverse=True)
    f = inv.reshape(-1)[f]
    f = f[(f[:, 0] != f[:, 1]) & (f[:, 1] != f[:, 2]) & (f[:, 0] != f[:, 2])]
    rng = np.random.default_rng(seed)
    v = v + rng.normal(0.0, jitter_sigma, size=v.shape)
    return _finish(v, f)
