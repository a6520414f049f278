"""Seeded workload descriptions (meshes, aspect angles, frequencies, ray density).

Each ``*_case`` function returns a plain dict; nothing here evaluates any part
of the scattering method. Angles are in degrees: azimuth ``az`` measured in the
x-y plane from +x, elevation ``el`` from the x-y plane toward +z.
"""
from __future__ import annotations

import math

import numpy as np

from . import meshes

C0 = 299_792_458.0  # speed of light in vacuum, m/s


def spacing_for(freq_hz: float, rays_per_lambda: float) -> float:
    """Ray-grid spacing (m) giving ``rays_per_lambda`` rays per wavelength."""
    return C0 / (freq_hz * rays_per_lambda)


def grid_offset(seed: int) -> tuple:
    """Seeded sub-cell shift (du, dv) of the aperture grid, in units of the ray
    spacing, drawn U[0, 1)^2. It keeps a regular grid from lining up with the
    edges of a regular mesh (whole rows of rays on edges otherwise)."""
    rng = np.random.default_rng(seed)
    return tuple(float(x) for x in rng.uniform(0.0, 1.0, 2))


def _random_aspects(n: int, seed: int) -> np.ndarray:
    """``n`` aspects uniform over the unit sphere, as (az, el) degrees."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 360.0, n)
    el = np.degrees(np.arcsin(rng.uniform(-1.0, 1.0, n)))
    return np.stack([az, el], axis=1)


def sphere_case(n_random: int = 64, seed: int = 11) -> dict:
    """PEC sphere r = 1 m, icosphere subdivision 5 (20480 triangles), 3 GHz
    (ka = 62.9), 220 x 220 rays over a fixed 2.2 m square window (spacing 1 cm,
    about 10 rays per wavelength), one bounce, HH and VV. Aspects: (0, 0) plus
    ``n_random`` seeded aspects uniform over the sphere."""
    xyz, tri = meshes.icosphere(5, 1.0)
    ang = np.concatenate([[[0.0, 0.0]], _random_aspects(n_random, seed)])
    return dict(name="sphere_r1m_ico5_3GHz", xyz=xyz, tri=tri, freqs=np.array([3.0e9]),
                angles=ang, spacing=0.01, eta=0.0, window=2.2, max_bounces=1, radius=1.0, offset=(0.0, 0.0))


def trihedral_case(az_step: float = 0.5, el: float = 35.26) -> dict:
    """Triangular trihedral (1 m legs, 3 x 1024 triangles), 10 GHz, spacing
    lambda/10, aperture margin 0.05, up to 3 bounces, azimuth 0..90 deg in
    ``az_step`` steps at elevation ``el`` (181 angles for 0.5 deg); grid offset
    from seed 5 (the axis-aligned plates would otherwise put whole rows of rays
    on edges at 0 and 90 deg)."""
    xyz, tri = meshes.trihedral(1.0, 32)
    az = np.arange(0.0, 90.0 + 1e-9, az_step)
    ang = np.stack([az, np.full_like(az, el)], axis=1)
    return dict(name="trihedral_1m_10GHz_sweep", xyz=xyz, tri=tri, freqs=np.array([10.0e9]),
                angles=ang, spacing=spacing_for(10.0e9, 10.0), eta=0.05, window=0.0, max_bounces=3,
                offset=grid_offset(5))


def aircraft_case(freq_hz: float = 1.0e9, n_az: int = 360, target_tris: int = 1_000_000,
                  seed: int = 1) -> dict:
    """Seeded aircraft-like body, ``n_az`` azimuths at elevation 0, spacing
    lambda/10 at ``freq_hz``, up to 10 bounces."""
    xyz, tri = meshes.aircraft(seed=seed, target_tris=target_tris)
    az = np.arange(n_az) * (360.0 / n_az)
    ang = np.stack([az, np.zeros_like(az)], axis=1)
    return dict(name=f"aircraft_{freq_hz / 1e9:g}GHz", xyz=xyz, tri=tri, freqs=np.array([freq_hz]),
                angles=ang, spacing=spacing_for(freq_hz, 10.0), eta=0.05, window=0.0, max_bounces=10,
                offset=grid_offset(6))


def batched_requests(n: int = 4096, seed: int = 2, n_meshes: int = 3) -> list:
    """Mixed request list: mesh index ~ U{0..n_meshes-1}, az ~ U[0, 360),
    el ~ U[-30, 30], density ~ U[5, 10] rays per wavelength at the request's
    highest frequency, n_f ~ U{1..64} frequencies drawn U[1, 12] GHz (sorted)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        m = int(rng.integers(0, n_meshes))
        az = float(rng.uniform(0.0, 360.0))
        el = float(rng.uniform(-30.0, 30.0))
        dens = float(rng.uniform(5.0, 10.0))
        nf = int(rng.integers(1, 65))
        f = np.sort(rng.uniform(1.0e9, 12.0e9, nf))
        out.append(dict(mesh=m, az=az, el=el, rays_per_lambda=dens, freqs=f,
                        spacing=spacing_for(float(f[-1]), dens)))
    return out


def surrogate_samples(n: int = 200_000, seed: int = 3) -> np.ndarray:
    """Training inputs (az deg, el deg, f Hz): az ~ U[0, 360), el ~ U[-30, 30],
    log f ~ U[log 1 GHz, log 12 GHz]."""
    rng = np.random.default_rng(seed)
    az = rng.uniform(0.0, 360.0, n)
    el = rng.uniform(-30.0, 30.0, n)
    f = np.exp(rng.uniform(math.log(1.0e9), math.log(12.0e9), n))
    return np.stack([az, el, f], axis=1)
