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


@pytest.mark.parametrize("chunk,no_graph", [(0, False), (200_000, False), (200_000, True)])
def test_submitted_batch_equals_run_batch(G, chunk, no_graph):
    """sbr_submit_batch (device-built PO work lists, CUDA graph replay) gives the
    run_batch results bit for bit, on the first launch and on replays."""
    torch = pytest.importorskip("torch")
    case = S.trihedral_case()
    reqs = _requests(24, 7, fmax=6e9)
    rows = sum(len(r["freqs"]) for r in reqs)
    flags = G.TRACE_NO_GRAPH if no_graph else 0
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        Eb, Rb, st = c.run_batch(reqs, eta=0.05, max_bounces=3, pols="HH,VV,HV,VH", chunk_rays=chunk,
                                 offset=case["offset"])
        Eb, Rb = np.concatenate(Eb), np.concatenate(Rb)
        E = torch.full((rows, 4, 2), float("nan"), dtype=torch.float64, device="cuda")
        R = torch.full((rows, 4), float("nan"), dtype=torch.float64, device="cuda")
        for rep in range(3):
            E.fill_(float("nan"))
            R.fill_(float("nan"))
            torch.cuda.synchronize()  # the context runs on its own stream
            c.submit_batch(reqs, E, R, eta=0.05, max_bounces=3, pols="HH,VV,HV,VH", chunk_rays=chunk,
                           offset=case["offset"], flags=flags)
            ss = c.sync()
            Eg = E.cpu().numpy()
            assert np.array_equal(Eg[..., 0] + 1j * Eg[..., 1], Eb), rep
            assert np.array_equal(R.cpu().numpy(), Rb), rep
            for k in ("ray_bounces", "valid_rays", "rays_launched", "n_angles"):
                assert ss[k] == st[k], (k, ss[k], st[k])
        if chunk:
            assert ss["kernel_launches"] > 8 * 2


def test_submitted_batch_replans_on_change_and_refuses_bad_flags(G):
    torch = pytest.importorskip("torch")
    case = S.trihedral_case()
    reqs = _requests(5, 9, fmax=6e9)
    rows = sum(len(r["freqs"]) for r in reqs)
    with G.Context(0) as c:
        c.load_mesh(case["xyz"], case["tri"])
        with pytest.raises(G.SbrError):
            c.sync()  # nothing submitted
        R = torch.zeros((rows, 2), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()  # the context runs on its own stream
        c.submit_batch(reqs, None, R, max_bounces=2, offset=case["offset"])
        c.sync()
        r1 = R.cpu().numpy().copy()
        # another bounce limit: a new plan, results of run_batch with that limit
        c.submit_batch(reqs, None, R, max_bounces=1, offset=case["offset"])
        c.sync()
        _, Rb, _ = c.run_batch(reqs, eta=0.05, max_bounces=1, offset=case["offset"])
        assert np.array_equal(R.cpu().numpy(), np.concatenate(Rb))
        assert not np.array_equal(R.cpu().numpy(), r1)
        for bad in (G.TRACE_RECORD_HITS, G.TRACE_TIME_PASSES):
            with pytest.raises(G.SbrError):
                c.submit_batch(reqs, None, R, flags=bad)
        # a new mesh invalidates the captured graph
        sph = S.sphere_case(n_random=0)
        c.load_mesh(sph["xyz"], sph["tri"])
        c.submit_batch(reqs, None, R, max_bounces=1, offset=case["offset"])
        c.sync()
        _, Rs, _ = c.run_batch(reqs, eta=0.05, max_bounces=1, offset=case["offset"])
        assert np.array_equal(R.cpu().numpy(), np.concatenate(Rs))
