"""FP64 CPU oracle of the SBR trace-integrate path (ctypes wrapper of sbr_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference legs of ``bench.py``. The product package
never imports it, and it never imports the product package.

Conventions (angles, aperture grid, polarisation order, phase path) are listed
at the top of ``sbr_oracle.c``. Polarisation index order everywhere is
``HH, VV, HV, VH`` where the first letter is the receive polarisation and the
second the transmit polarisation (V = theta_hat, H = phi_hat).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbr_oracle.c")
_LIB = os.path.join(_HERE, "lib", "libsbr_oracle.so")
C0 = 299_792_458.0
POLS = ("HH", "VV", "HV", "VH")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, IEEE semantics)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-pthread", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class Frame(C.Structure):
    _fields_ = [("az_deg", C.c_double), ("el_deg", C.c_double),
                ("rhat", C.c_double * 3), ("khat", C.c_double * 3),
                ("vhat", C.c_double * 3), ("hhat", C.c_double * 3),
                ("centre", C.c_double * 3), ("diag", C.c_double), ("D", C.c_double),
                ("Lu", C.c_double), ("Lv", C.c_double),
                ("spacing", C.c_double), ("dA", C.c_double), ("eps", C.c_double),
                ("nu", C.c_int64), ("nv", C.c_int64),
                ("P0", C.c_float * 3), ("U", C.c_float * 3), ("V", C.c_float * 3), ("d", C.c_float * 3),
                ("bistatic", C.c_int), ("rx_rhat", C.c_double * 3), ("rx_hhat", C.c_double * 3),
                ("rx_vhat", C.c_double * 3), ("rx_r32", C.c_float * 3)]

    @property
    def n_rays(self) -> int:
        return int(self.nu * self.nv)


class TraceOpts(C.Structure):
    _fields_ = [("max_bounces", C.c_int), ("po_mode", C.c_int), ("phase_literal", C.c_int),
                ("require_escape", C.c_int), ("use_bvh", C.c_int), ("n_threads", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orc_make_frame.argtypes = [P(C.c_float), C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double, P(Frame)]
        L.orc_make_frame.restype = C.c_int
        L.orc_ray.argtypes = [P(Frame), C.c_int64, C.c_int64, P(C.c_float), P(C.c_float)]
        L.orc_frame_set_receiver.argtypes = [P(Frame), C.c_double, C.c_double]
        L.orc_frame_set_receiver.restype = C.c_int
        L.orc_ray.restype = None
        L.orc_mesh_create.argtypes = [P(C.c_float), C.c_int64, P(C.c_int32), C.c_int64]
        L.orc_mesh_create.restype = C.c_void_p
        L.orc_mesh_free.argtypes = [C.c_void_p]
        L.orc_mesh_free.restype = None
        L.orc_mesh_bbox.argtypes = [C.c_void_p, P(C.c_float)]
        L.orc_mesh_bbox.restype = None
        L.orc_mesh_normals.argtypes = [C.c_void_p, P(C.c_float)]
        L.orc_mesh_normals.restype = None
        L.orc_mesh_n_degenerate.argtypes = [C.c_void_p]
        L.orc_mesh_n_degenerate.restype = C.c_int64
        L.orc_mesh_build_bvh.argtypes = [C.c_void_p, C.c_int]
        L.orc_mesh_build_bvh.restype = C.c_int
        L.orc_mesh_bvh_nodes.argtypes = [C.c_void_p]
        L.orc_mesh_bvh_nodes.restype = C.c_int64
        L.orc_closest_hit.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_double), C.c_int64,
                                      P(C.c_double), P(C.c_int64), P(C.c_double), P(C.c_double)]
        L.orc_closest_hit.restype = C.c_int
        L.orc_trace.argtypes = [C.c_void_p, P(Frame), P(TraceOpts), P(C.c_int64), C.c_int64,
                                P(C.c_int32), P(C.c_double), P(C.c_int32), P(C.c_uint8), P(C.c_uint8),
                                P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_int64)]
        L.orc_trace.restype = C.c_int
        L.orc_po.argtypes = [P(C.c_double), P(C.c_double), P(C.c_uint8), C.c_int64, P(C.c_double),
                             C.c_int64, P(C.c_double), P(C.c_double)]
        L.orc_po.restype = C.c_int
        L.orc_reflect.argtypes = [P(C.c_double)] * 4
        L.orc_reflect.restype = None
        L.orc_mie_pec_backscatter.argtypes = [C.c_double]
        L.orc_mie_pec_backscatter.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def make_frame(bbox, az_deg, el_deg, spacing, eta=0.05, window=0.0, offset=(0.0, 0.0), rx=None) -> Frame:
    """Aperture frame and ray grid of one aspect (Eq. L1-L3). ``rx`` = (az, el) of a
    bistatic receiver (None: monostatic)."""
    b = np.ascontiguousarray(bbox, dtype=np.float32)
    f = Frame()
    rc = lib().orc_make_frame(_ptr(b, C.c_float), float(az_deg), float(el_deg), float(spacing), float(eta),
                              float(window), float(offset[0]), float(offset[1]), C.byref(f))
    if rc != 0:
        raise ValueError("orc_make_frame failed")
    if rx is not None:
        lib().orc_frame_set_receiver(C.byref(f), float(rx[0]), float(rx[1]))
    return f


def ray(frame: Frame, i: int, j: int):
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    lib().orc_ray(C.byref(frame), int(i), int(j), _ptr(o, C.c_float), _ptr(d, C.c_float))
    return o, d


class Mesh:
    """Triangle mesh held in FP64 by the oracle, with an optional median-split BVH."""

    def __init__(self, xyz, tri, bvh_leaf: int | None = 4):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        h = lib().orc_mesh_create(_ptr(self.xyz, C.c_float), len(self.xyz), _ptr(self.tri, C.c_int32),
                                  len(self.tri))
        if not h:
            raise ValueError("orc_mesh_create failed (bad indices or non-finite coordinates)")
        self._h = h
        self.has_bvh = False
        if bvh_leaf:
            self.build_bvh(bvh_leaf)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_mesh_free(h)
            self._h = None

    @property
    def n_tri(self) -> int:
        return len(self.tri)

    def build_bvh(self, leaf: int = 4):
        if lib().orc_mesh_build_bvh(self._h, int(leaf)) != 0:
            raise ValueError("bvh build failed")
        self.has_bvh = True

    @property
    def n_degenerate(self) -> int:
        """Triangles that take no hits: sine of the edge angle at most 2^-20."""
        return int(lib().orc_mesh_n_degenerate(self._h))

    @property
    def normals(self) -> np.ndarray:
        """FP32 unit normals [n_tri, 3] (the rounded FP64 normal; 0 for a degenerate triangle)."""
        n = np.zeros((self.n_tri, 3), np.float32)
        lib().orc_mesh_normals(self._h, _ptr(n, C.c_float))
        return n

    @property
    def bvh_nodes(self) -> int:
        return int(lib().orc_mesh_bvh_nodes(self._h))

    @property
    def bbox(self) -> np.ndarray:
        b = np.zeros(6, np.float32)
        lib().orc_mesh_bbox(self._h, _ptr(b, C.c_float))
        return b

    def closest_hit(self, o, d, skip=-1, use_bvh=True):
        o = np.ascontiguousarray(o, dtype=np.float64)
        d = np.ascontiguousarray(d, dtype=np.float64)
        t, k, bm, t2 = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
        lib().orc_closest_hit(self._h, int(bool(use_bvh) and self.has_bvh), _ptr(o, C.c_double),
                              _ptr(d, C.c_double), int(skip), C.byref(t), C.byref(k), C.byref(bm), C.byref(t2))
        return (int(k.value), float(t.value), float(bm.value), float(t2.value))


def trace(mesh: Mesh, frame: Frame, max_bounces: int, po_mode: str = "vector", phase_literal: bool = False,
          require_escape: bool = False, use_bvh: bool = True, ids=None, threads: int | None = None) -> dict:
    """Trace rays of ``frame`` (all, or the ray ids ``ids`` = j*nu + i) through
    ``mesh`` (Algorithm 2) and return per-ray arrays: hit_tri/hit_t [n, B],
    nb, valid, band (bit 0: a hit within 1e-6 barycentric of an edge, bit 1: a
    runner-up within 1e-6 relative in t), bmin, coef [n, 4] (HH, VV, HV, VH)
    and L.

    Hit decisions are exact (FP64 on the FP32 ray and vertices); the ray state
    between bounces is FP32, each value the rounding of its defining formula
    (hit_t is the stored FP32 distance t32). Path length, fields and
    coefficients are FP64."""
    B = int(max_bounces)
    if ids is None:
        n = frame.n_rays
        idp = None
    else:
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        n = len(ids)
        idp = ids
    out = dict(hit_tri=np.empty((n, B), np.int32), hit_t=np.empty((n, B), np.float64),
               nb=np.empty(n, np.int32), valid=np.empty(n, np.uint8), band=np.empty(n, np.uint8),
               coef=np.empty((n, 4), np.float64), L=np.empty(n, np.float64), bmin=np.empty(n, np.float64),
               counters=np.zeros(2, np.int64))
    o = TraceOpts(B, 1 if po_mode == "scalar" else 0, int(bool(phase_literal)), int(bool(require_escape)),
                  int(bool(use_bvh) and mesh.has_bvh), int(threads or default_threads()))
    rc = lib().orc_trace(mesh._h, C.byref(frame), C.byref(o), _ptr(idp, C.c_int64), n,
                         _ptr(out["hit_tri"], C.c_int32), _ptr(out["hit_t"], C.c_double),
                         _ptr(out["nb"], C.c_int32), _ptr(out["valid"], C.c_uint8), _ptr(out["band"], C.c_uint8),
                         _ptr(out["coef"], C.c_double), _ptr(out["L"], C.c_double), _ptr(out["bmin"], C.c_double),
                         _ptr(out["counters"], C.c_int64))
    if rc != 0:
        raise ValueError("orc_trace failed")
    out["ids"] = np.arange(n, dtype=np.int64) if ids is None else ids
    return out


def po(coef, L, valid, freqs):
    """PO ray-tube sum (Eq. po_sum / em6): returns (E complex [nf, 4], rcs_dbsm [nf, 4])."""
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    valid = None if valid is None else np.ascontiguousarray(valid, dtype=np.uint8)
    freqs = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
    nf = len(freqs)
    E = np.empty((nf, 4, 2), np.float64)
    rcs = np.empty((nf, 4), np.float64)
    with np.errstate(divide="ignore"):
        rc = lib().orc_po(_ptr(coef, C.c_double), _ptr(L, C.c_double), _ptr(valid, C.c_uint8), len(L),
                          _ptr(freqs, C.c_double), nf, _ptr(E, C.c_double), _ptr(rcs, C.c_double))
    if rc != 0:
        raise ValueError("orc_po failed")
    return E[..., 0] + 1j * E[..., 1], rcs


def reflect(n, d, E1, E2):
    """Oracle's specular reflection + PEC field update for unit normal n."""
    n = np.ascontiguousarray(n, dtype=np.float64)
    d = np.array(d, dtype=np.float64)
    E1 = np.array(E1, dtype=np.float64)
    E2 = np.array(E2, dtype=np.float64)
    lib().orc_reflect(_ptr(n, C.c_double), _ptr(d, C.c_double), _ptr(E1, C.c_double), _ptr(E2, C.c_double))
    return d, E1, E2


def mie_pec_backscatter(x: float) -> float:
    """sigma / (pi a^2) of a PEC sphere with k a = x (Mie series)."""
    return float(lib().orc_mie_pec_backscatter(float(x)))


def rcs_angle(mesh: Mesh, bbox, az, el, spacing, freqs, max_bounces, eta=0.05, window=0.0, offset=(0.0, 0.0),
              po_mode="vector", phase_literal=False, require_escape=False, threads=None, ids=None, rx=None):
    """Convenience: one aspect, trace + PO. Returns (E [nf,4], rcs_dbsm [nf,4], trace dict, frame).
    ``rx`` = (az, el) of a bistatic receiver (None: monostatic)."""
    fr = make_frame(bbox, az, el, spacing, eta=eta, window=window, offset=offset, rx=rx)
    tr = trace(mesh, fr, max_bounces, po_mode=po_mode, phase_literal=phase_literal,
               require_escape=require_escape, ids=ids, threads=threads)
    E, rcs = po(tr["coef"], tr["L"], tr["valid"], freqs)
    return E, rcs, tr, fr
