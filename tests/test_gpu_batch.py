"""Batched form (sbr_run_batch) against the plain per-request path, and against
the oracle on a sample. Requests mix ray spacings and frequency lists, so ray
counts are uneven and several chunks are needed."""
import numpy as np
import pytest

import sbr_inputs as S
from parity import assert_rcs_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_2604_09243_gb300 import build

    build.build()
    import paper_2604_09243_gb300 as G

    return G


def _requests(n, seed, fmax=12e9):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nf = int(rng.integers(1, 9))
        f = np.sort(rng.uniform(1e9, fmax, nf))
        dens = rng.uniform(5, 10)
        out.append(dict(az=float(rng.uniform(0, 360)), el=float(rng.uniform(-30, 30)), freqs=f,
                        spacing=S.spacing_for(float(f[-1]), dens)))
    return out


@pytest.mark.parametrize("chunk", [0, 200_000])
def test_batch_equals_plain_trihedral(G, chunk):
    case = S.trihedral_case()
    reqs = _requests(24, 5, fmax=6e9)
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        Eb, Rb, st = c.run_batch(reqs, eta=0.05, max_bounces=3, pols="HH,VV,HV,VH", chunk_rays=chunk,
                                 offset=case["offset"])
        tot_b = 0
        for k, r in enumerate(reqs):
            s = c.trace([[r["az"], r["el"]]], r["spacing"], eta=0.05, max_bounces=3, offset=case["offset"])
            E, R = c.po_integrate(r["freqs"], "HH,VV,HV,VH")
            tot_b += s["ray_bounces"]
            assert np.array_equal(Eb[k], E[0]), k
            assert np.array_equal(Rb[k], R[0])
        assert st["ray_bounces"] == tot_b
        if chunk:
            assert st["kernel_launches"] > 8 * 2


def test_batch_against_oracle_sphere(G, orc):
    case = S.sphere_case(n_random=0)
    reqs = _requests(6, 8, fmax=4e9)
    om = orc.Mesh(case["xyz"], case["tri"])
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        Eb, Rb, st = c.run_batch(reqs, eta=0.05, max_bounces=1, pols="HH,VV")
    for k, r in enumerate(reqs):
        _, Ro, _, _ = orc.rcs_angle(om, om.bbox, r["az"], r["el"], r["spacing"], r["freqs"], 1, eta=0.05)
        assert_rcs_close(Rb[k], Ro[:, :2])
