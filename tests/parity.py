"""Helpers that compare the CUDA path with the oracle ray by ray (tests only).

The hit decisions (triangle, distance, bounce count) are taken by both sides in
FP32 in the same written operation order, so they must agree bit for bit for
every ray. The edge band of the parity rule (rays whose exact FP64 hit lies
within 1e-6 barycentric of a triangle edge, or whose runner-up triangle is within
1e-6 relative in t) is measured with the oracle's exact transport and reported.
"""
import numpy as np

RCS_DB = 0.1
RCS_FLOOR = -40.0
T_REL = 1e-5


def compare_hits(g_tri, g_t, g_nb, o, ids=None):
    """Compare GPU per-ray hits (tri [n,B], t [n,B] float32, nb [n]) with an oracle
    trace dict (FP32 transport). ``ids`` selects GPU rows when the oracle traced
    a subset. Returns a summary dict."""
    if ids is not None:
        g_tri, g_t, g_nb = g_tri[ids], g_t[ids], g_nb[ids]
    o_tri, o_t, o_nb = o["hit_tri"], o["hit_t"].astype(np.float32), o["nb"]
    same_tri = np.all(g_tri == o_tri, axis=1) & (g_nb == o_nb)
    same_t = np.all(g_t == o_t, axis=1)
    both = (g_tri >= 0) & (o_tri >= 0)
    rel = np.abs(g_t[both].astype(np.float64) - o_t[both]) / np.maximum(np.abs(o_t[both]), 1e-30)
    bad = ~(same_tri & same_t)
    return dict(n=len(o_nb), mismatch=int((~same_tri).sum()), t_mismatch=int((~same_t).sum()),
                max_rel_t=float(rel.max()) if rel.size else 0.0, bad_ids=np.nonzero(bad)[0][:10],
                band=int((o["band"] != 0).sum()))


def assert_hit_parity(s):
    assert s["mismatch"] == 0 and s["t_mismatch"] == 0, s
    assert s["max_rel_t"] <= T_REL, s


def assert_rcs_close(g_db, o_db, tol=RCS_DB, floor=RCS_FLOOR):
    g_db, o_db = np.asarray(g_db), np.asarray(o_db)
    m = o_db > floor
    d = np.abs(g_db[m] - o_db[m])
    assert d.size == 0 or d.max() <= tol, (d.max(), np.argmax(d))
    return float(d.max()) if d.size else 0.0
