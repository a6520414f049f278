"""Helpers that compare the CUDA path with the oracle ray by ray (tests only).

Parity rule for the hits: the oracle decides every hit exactly (FP64 on the
FP32 ray and vertices). A ray is in the edge band when, at some bounce, its
exact hit lies within 1e-6 barycentric of a triangle edge, or a runner-up
triangle lies within 1e-6 relative in t. The GPU must give every ray outside
the band the oracle's triangle sequence and bounce count, and the rays of the
band on which the two differ must stay below 1e-5 of all rays. Hit distances
of agreeing rays must agree within 1e-5 relative.
"""
import numpy as np

RCS_DB = 0.1
RCS_FLOOR = -40.0
T_REL = 1e-5
BAND_MISMATCH_FRACTION = 1e-5


def compare_hits(g_tri, g_t, g_nb, o, ids=None):
    """Compare GPU per-ray hits (tri [n,B], t [n,B] float32, nb [n]) with an oracle
    trace dict. ``ids`` selects GPU rows when the oracle traced a subset.
    Returns a summary dict: rays, mismatching rays outside / inside the edge
    band, rays in the band, largest relative t difference of agreeing rays."""
    if ids is not None:
        g_tri, g_t, g_nb = g_tri[ids], g_t[ids], g_nb[ids]
    o_tri, o_t, o_nb = o["hit_tri"], o["hit_t"], o["nb"]
    same = np.all(g_tri == o_tri, axis=1) & (g_nb == o_nb)
    band = o["band"] != 0
    hit = same[:, None] & (o_tri >= 0)
    rel = np.abs(g_t.astype(np.float64)[hit] - o_t[hit]) / np.maximum(np.abs(o_t[hit]), 1e-30)
    return dict(n=len(o_nb), mismatch=int((~same).sum()), mismatch_out=int((~same & ~band).sum()),
                mismatch_band=int((~same & band).sum()), band=int(band.sum()),
                t_exact=int((g_t.astype(np.float64)[hit] == o_t[hit]).sum()), t_hits=int(hit.sum()),
                max_rel_t=float(rel.max()) if rel.size else 0.0, bad_ids=np.nonzero(~same & ~band)[0][:10])


def assert_hit_parity(s):
    """No mismatch outside the edge band, band mismatches below 1e-5 of the
    compared rays, agreeing rays' distances within 1e-5 relative."""
    assert s["mismatch_out"] == 0, s
    assert s["mismatch_band"] <= BAND_MISMATCH_FRACTION * s["n"], s
    assert s["max_rel_t"] <= T_REL, s


class HitTally:
    """Totals over the compared rays of a test: the band-mismatch fraction is a
    property of all the rays, so it is asserted on the totals."""

    def __init__(self):
        self.n = self.mismatch_band = self.mismatch_out = self.band = 0

    def add(self, s):
        assert s["mismatch_out"] == 0 and s["max_rel_t"] <= T_REL, s
        self.n += s["n"]
        self.mismatch_band += s["mismatch_band"]
        self.mismatch_out += s["mismatch_out"]
        self.band += s["band"]
        return s

    def check(self):
        assert self.n > 0
        assert self.mismatch_out == 0
        assert self.mismatch_band <= BAND_MISMATCH_FRACTION * self.n, vars(self)
        return vars(self)


def assert_rcs_close(g_db, o_db, tol=RCS_DB, floor=RCS_FLOOR):
    g_db, o_db = np.asarray(g_db), np.asarray(o_db)
    m = o_db > floor
    d = np.abs(g_db[m] - o_db[m])
    assert d.size == 0 or d.max() <= tol, (d.max(), np.argmax(d))
    return float(d.max()) if d.size else 0.0
