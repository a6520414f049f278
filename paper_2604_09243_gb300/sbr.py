"""Thin ctypes binding of libsbr (include/sbr.h): argument marshalling only.

Every step of the trace-integrate path runs in the CUDA library. If
``lib/libsbr.so`` is missing or cannot be loaded, every entry point raises;
there is no CPU fallback. PyTorch is optional: device tensors (``torch.Tensor``
on CUDA) are accepted wherever the C ABI takes a device pointer, and a torch
stream may be passed as the context's stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsbr.so")

SBR_OK = 0
ERRORS = {-1: "SBR_ERR_ARG", -2: "SBR_ERR_CUDA", -3: "SBR_ERR_OOM", -4: "SBR_ERR_STATE",
          -5: "SBR_ERR_STACK_OVERFLOW", -6: "SBR_ERR_TIMEOUT", -7: "SBR_ERR_NODEV"}
POL_BITS = {"HH": 1, "VV": 2, "HV": 4, "VH": 8}
POL_ORDER = ("HH", "VV", "HV", "VH")
PO_VECTOR, PO_PAPER_SCALAR = 0, 1
PHASE = {"compensated": 0, "fp32": 16, "fp64": 32}
TRACE_PHASE_LITERAL_2R, TRACE_REQUIRE_ESCAPE, TRACE_RECORD_HITS, TRACE_COUNT_VISITS, TRACE_TIME_PASSES = 1, 2, 4, 8, 16
TRACE_NO_GRAPH = 32

# every symbol declared in include/sbr.h
EXPORTS = ("sbr_version", "sbr_create", "sbr_destroy", "sbr_last_error", "sbr_load_mesh", "sbr_get_bbox",
           "sbr_build_bvh", "sbr_ray_grid_for", "sbr_ray_grid_box", "sbr_trace", "sbr_po_integrate", "sbr_get_hits",
           "sbr_get_records", "sbr_spacing_for", "sbr_po_integrate_noalloc", "sbr_run_batch", "sbr_submit_batch",
           "sbr_sync", "sbr_get_tuning", "sbr_set_tuning", "sbr_autotune", "sbr_trace_bistatic",
           "sbr_surrogate_create", "sbr_surrogate_destroy", "sbr_surrogate_last_error", "sbr_surrogate_num_params",
           "sbr_surrogate_params", "sbr_surrogate_fourier", "sbr_surrogate_train", "sbr_surrogate_grads",
           "sbr_surrogate_predict", "sbr_gemm_bf16_tn", "sbr_gemm_bf16_tn_async", "sbr_probe_l2_bandwidth",
           "sbr_probe_fp32_fma", "sbr_get_bvh_info")


class SbrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class BvhOpts(C.Structure):
    _fields_ = [("leaf_max", C.c_int), ("cost_traverse", C.c_float), ("cost_intersect", C.c_float),
                ("builder", C.c_int), ("ploc_radius", C.c_int)]


class TraceOpts(C.Structure):
    _fields_ = [("window_m", C.c_double), ("offset_u", C.c_double), ("offset_v", C.c_double),
                ("flags", C.c_int), ("chunk_rays", C.c_int)]


class Tuning(C.Structure):
    _fields_ = [("tile_w", C.c_int), ("blocks_per_sm", C.c_int), ("stack_depth", C.c_int),
                ("chunk_rays_log2", C.c_int), ("po_item", C.c_int), ("bvh_width", C.c_int), ("packet", C.c_int),
                ("octant", C.c_int), ("silhouette", C.c_int), ("raster", C.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class TuneTrial(C.Structure):
    _fields_ = [("tuning", Tuning), ("ms", C.c_double), ("status", C.c_int), ("reserved", C.c_int)]


class BvhInfo(C.Structure):
    _fields_ = [("n_tri", C.c_int64), ("n_nodes", C.c_int64), ("n_nodes4", C.c_int64)]


class TraceStats(C.Structure):
    _fields_ = [("n_angles", C.c_int64), ("rays_launched", C.c_int64), ("ray_bounces", C.c_int64),
                ("valid_rays", C.c_int64), ("node_visits", C.c_int64), ("tri_tests", C.c_int64),
                ("stack_overflows", C.c_int64), ("kernel_launches", C.c_int64), ("pass_launches", C.c_int64),
                ("pass_ms", C.c_double), ("raster_tests", C.c_int64), ("primary_ms", C.c_double),
                ("bounce_hits", C.c_int64), ("listed_hits", C.c_int64), ("open_tests", C.c_int64),
                ("fp64_tests", C.c_int64), ("warp_node_visits", C.c_int64)]

    def as_dict(self):
        return {k: (float if k.endswith("_ms") else int)(getattr(self, k)) for k, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("az_deg", C.c_double), ("el_deg", C.c_double), ("ray_spacing_m", C.c_double),
                ("freq_offset", C.c_int64), ("n_freq", C.c_int32), ("reserved", C.c_int32)]


class RayGrid(C.Structure):
    _fields_ = [("nu", C.c_int64), ("nv", C.c_int64), ("lu", C.c_double), ("lv", C.c_double),
                ("spacing", C.c_double), ("eps", C.c_double),
                ("rhat", C.c_double * 3), ("khat", C.c_double * 3), ("vhat", C.c_double * 3),
                ("hhat", C.c_double * 3),
                ("p0", C.c_float * 3), ("du", C.c_float * 3), ("dv", C.c_float * 3), ("dir", C.c_float * 3)]


_lib = None


def lib() -> C.CDLL:
    """Load libsbr.so (built in-tree by ``paper_2604_09243_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsbr.so not found at {LIB_PATH}: run paper_2604_09243_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    P, vp, i64, d = C.POINTER, C.c_void_p, C.c_int64, C.c_double
    sig = {
        "sbr_version": ([], C.c_int),
        "sbr_create": ([P(vp), C.c_int, vp], C.c_int),
        "sbr_destroy": ([vp], None),
        "sbr_last_error": ([vp], C.c_char_p),
        "sbr_load_mesh": ([vp, vp, i64, vp, i64, C.c_int], C.c_int),
        "sbr_get_bbox": ([vp, P(C.c_float)], C.c_int),
        "sbr_build_bvh": ([vp, P(BvhOpts)], C.c_int),
        "sbr_get_bvh_info": ([vp, P(BvhInfo)], C.c_int),
        "sbr_ray_grid_for": ([vp, d, d, d, d, P(TraceOpts), P(RayGrid)], C.c_int),
        "sbr_ray_grid_box": ([P(C.c_float), d, d, d, d, P(TraceOpts), P(RayGrid)], C.c_int),
        "sbr_trace": ([vp, P(d), i64, d, d, C.c_int, P(TraceOpts), P(TraceStats)], C.c_int),
        "sbr_trace_bistatic": ([vp, P(d), P(d), i64, d, d, C.c_int, P(TraceOpts), P(TraceStats)], C.c_int),
        "sbr_po_integrate": ([vp, P(d), i64, C.c_int, C.c_int, vp, vp, C.c_int], C.c_int),
        "sbr_get_hits": ([vp, i64, vp, vp, vp], C.c_int),
        "sbr_get_records": ([vp, i64, i64, vp, vp, vp, P(i64)], C.c_int),
        "sbr_spacing_for": ([d, d], d),
        "sbr_probe_l2_bandwidth": ([C.c_int, i64, C.c_int, P(d)], C.c_int),
        "sbr_probe_fp32_fma": ([C.c_int, P(d)], C.c_int),
        "sbr_run_batch": ([vp, P(Request), i64, P(d), i64, d, C.c_int, C.c_int, C.c_int, P(TraceOpts), vp, vp,
                           C.c_int, P(TraceStats)], C.c_int),
        "sbr_po_integrate_noalloc": ([vp, P(i64), i64, P(d), i64, C.c_int, C.c_int, vp, vp, vp], C.c_int),
        "sbr_submit_batch": ([vp, P(Request), i64, P(d), i64, d, C.c_int, C.c_int, C.c_int, P(TraceOpts), vp, vp],
                             C.c_int),
        "sbr_sync": ([vp, P(TraceStats)], C.c_int),
        "sbr_get_tuning": ([vp, P(Tuning)], C.c_int),
        "sbr_set_tuning": ([vp, P(Tuning)], C.c_int),
        "sbr_autotune": ([vp, P(Request), i64, P(d), i64, d, C.c_int, C.c_int, C.c_int, P(TraceOpts), C.c_int,
                          P(TuneTrial), C.c_int, P(C.c_int), P(Tuning), P(d)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def version() -> int:
    return int(lib().sbr_version())


def spacing_for(f_max_hz: float, rays_per_lambda: float) -> float:
    """Ray spacing ds = c0 / (f * rays_per_lambda) (Sec. 4 sampling rule asks ds <= lambda / 5)."""
    v = lib().sbr_spacing_for(float(f_max_hz), float(rays_per_lambda))
    if v < 0:
        raise ValueError("frequency and rays per wavelength must be > 0")
    return v


def probe_l2_bandwidth(device: int = 0, nbytes: int = 64 << 20, passes: int = 50) -> float:
    """L2 read bandwidth in GB/s (sbr_probe_l2_bandwidth): a buffer below the L2
    capacity read ``passes`` times with loads that bypass L1."""
    v = C.c_double()
    rc = lib().sbr_probe_l2_bandwidth(int(device), int(nbytes), int(passes), C.byref(v))
    if rc != SBR_OK:
        raise SbrError(rc, "sbr_probe_l2_bandwidth failed")
    return float(v.value)


def probe_fp32_fma(device: int = 0) -> float:
    """FP32 fused multiply-add throughput in TFLOP/s (two operations each; sbr_probe_fp32_fma)."""
    v = C.c_double()
    rc = lib().sbr_probe_fp32_fma(int(device), C.byref(v))
    if rc != SBR_OK:
        raise SbrError(rc, "sbr_probe_fp32_fma failed")
    return float(v.value)


def po_integrate_noalloc(records_ptr: int, rec_offsets, freqs, pols="HH,VV", mode="vector", phase="compensated",
                        E_ptr: int | None = None, rcs_ptr: int | None = None, stream=None) -> None:
    """Allocation-free PO sum (sbr_po_integrate_noalloc) over caller-owned device
    records; ``records_ptr``, ``E_ptr`` and ``rcs_ptr`` are device addresses,
    ``rec_offsets`` host int64 [n_angles + 1]. Raises SbrError on a refused call."""
    off = np.ascontiguousarray(rec_offsets, dtype=np.int64)
    f = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
    m = (PO_PAPER_SCALAR if mode == "scalar" else PO_VECTOR) | PHASE[phase]
    s = int(getattr(stream, "cuda_stream", stream)) if stream is not None else None
    rc = lib().sbr_po_integrate_noalloc(C.c_void_p(int(records_ptr)), off.ctypes.data_as(C.POINTER(C.c_int64)),
                                        len(off) - 1, f.ctypes.data_as(C.POINTER(C.c_double)), len(f), _pols(pols),
                                        m, C.c_void_p(E_ptr) if E_ptr else None,
                                        C.c_void_p(rcs_ptr) if rcs_ptr else None, C.c_void_p(s) if s else None)
    if rc != SBR_OK:
        raise SbrError(rc, (lib().sbr_last_error(None) or b"").decode())


def _opts(window=0.0, offset=(0.0, 0.0), flags=0, chunk_rays=0) -> TraceOpts:
    return TraceOpts(float(window), float(offset[0]), float(offset[1]), int(flags), int(chunk_rays))


def _grid_dict(g: RayGrid) -> dict:
    out = {k: getattr(g, k) for k, _ in RayGrid._fields_}
    for k in ("rhat", "khat", "vhat", "hhat"):
        out[k] = np.array(out[k], np.float64)
    for k in ("p0", "du", "dv", "dir"):
        out[k] = np.array(out[k], np.float32)
    out["nu"], out["nv"] = int(g.nu), int(g.nv)
    return out


def ray_grid(bbox, az_deg, el_deg, spacing, eta=0.05, window=0.0, offset=(0.0, 0.0)) -> dict:
    """Aperture grid of one aspect for a scene box (Eq. L1-L3); host only, no GPU."""
    b = np.ascontiguousarray(bbox, dtype=np.float32)
    g = RayGrid()
    o = _opts(window, offset)
    rc = lib().sbr_ray_grid_box(b.ctypes.data_as(C.POINTER(C.c_float)), float(az_deg), float(el_deg), float(spacing),
                            float(eta), C.byref(o), C.byref(g))
    if rc != SBR_OK:
        raise SbrError(rc, "sbr_ray_grid_box: bad arguments")
    return _grid_dict(g)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


def _pols(pols) -> int:
    if isinstance(pols, int):
        return pols
    if isinstance(pols, str):
        pols = [p.strip() for p in pols.split(",") if p.strip()]
    m = 0
    for p in pols:
        m |= POL_BITS[p.upper()]
    return m


class Context:
    """One libsbr context on one CUDA device; methods mirror the sbr_* calls."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        h = C.c_void_p()
        s = None
        if stream is not None:
            s = int(getattr(stream, "cuda_stream", stream))
        rc = L.sbr_create(C.byref(h), int(device), C.c_void_p(s) if s else None)
        if rc != SBR_OK:
            raise SbrError(rc, (L.sbr_last_error(None) or b"").decode())
        self._h = h
        self.device = device
        self._stream_ref = stream  # keep a passed stream alive
        self.n_tri = 0
        self.max_bounces = 0
        self.grids: list[dict] = []

    # ------------------------------------------------------------------ plumbing
    def _check(self, rc: int):
        if rc != SBR_OK:
            raise SbrError(rc, (lib().sbr_last_error(self._h) or b"").decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sbr_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ calls
    def load_mesh(self, xyz, tri):
        """Copy a mesh (numpy host arrays or CUDA torch tensors: float32 [nv,3], int32 [nt,3])."""
        if _is_torch_cuda(xyz) or _is_torch_cuda(tri):
            if not (_is_torch_cuda(xyz) and _is_torch_cuda(tri)):
                raise ValueError("xyz and tri must both be host arrays or both CUDA tensors")
            xyz_c, tri_c = xyz.contiguous(), tri.contiguous()
            self._check(lib().sbr_load_mesh(self._h, xyz_c.data_ptr(), xyz_c.shape[0], tri_c.data_ptr(),
                                            tri_c.shape[0], 1))
            self.n_tri = int(tri_c.shape[0])
            return
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        if xyz.ndim != 2 or xyz.shape[1] != 3 or tri.ndim != 2 or tri.shape[1] != 3:
            raise ValueError("xyz must be [nv, 3] and tri [nt, 3]")
        self._check(lib().sbr_load_mesh(self._h, xyz.ctypes.data, len(xyz), tri.ctypes.data, len(tri), 0))
        self.n_tri = len(tri)

    def build_bvh(self, leaf_max: int = 4, cost_traverse: float = 1.0, cost_intersect: float = 1.0,
                  builder: str = "ploc", ploc_radius: int = 0):
        """sbr_build_bvh; builder "ploc" (nearest-neighbour clustering, default) or "lbvh" (Karras)."""
        o = BvhOpts(int(leaf_max), float(cost_traverse), float(cost_intersect), {"ploc": 0, "lbvh": 1}[builder],
                    int(ploc_radius))
        self._check(lib().sbr_build_bvh(self._h, C.byref(o)))

    def bvh_info(self) -> dict:
        """sbr_get_bvh_info: triangles, reachable binary nodes, 4-wide nodes."""
        o = BvhInfo()
        self._check(lib().sbr_get_bvh_info(self._h, C.byref(o)))
        return {"n_tri": int(o.n_tri), "n_nodes": int(o.n_nodes), "n_nodes4": int(o.n_nodes4)}

    def get_bbox(self) -> np.ndarray:
        b = np.zeros(6, np.float32)
        self._check(lib().sbr_get_bbox(self._h, b.ctypes.data_as(C.POINTER(C.c_float))))
        return b

    def ray_grid_for(self, az_deg, el_deg, spacing, eta=0.05, window=0.0, offset=(0.0, 0.0)) -> dict:
        g = RayGrid()
        o = _opts(window, offset)
        self._check(lib().sbr_ray_grid_for(self._h, float(az_deg), float(el_deg), float(spacing), float(eta),
                                           C.byref(o), C.byref(g)))
        return _grid_dict(g)

    def trace(self, angles, spacing, eta=0.05, max_bounces=1, window=0.0, offset=(0.0, 0.0), flags=0,
              stats=True, chunk_rays=0, rx=None) -> dict | None:
        """Trace aspects ``angles`` ([n, 2] az, el degrees); returns the trace stats. ``rx``: [n, 2]
        bistatic receiver directions (sbr_trace_bistatic), None for monostatic."""
        a = np.ascontiguousarray(np.atleast_2d(angles), dtype=np.float64)
        if a.shape[1] != 2:
            raise ValueError("angles must be [n, 2] (az, el)")
        o = _opts(window, offset, flags, chunk_rays)
        st = TraceStats()
        sp = C.byref(st) if stats else None
        dp = C.POINTER(C.c_double)
        if rx is None:
            self._check(lib().sbr_trace(self._h, a.ctypes.data_as(dp), len(a), float(spacing), float(eta),
                                        int(max_bounces), C.byref(o), sp))
        else:
            r = np.ascontiguousarray(np.atleast_2d(rx), dtype=np.float64)
            if r.shape != a.shape:
                raise ValueError("rx must be [n, 2] like angles")
            self._check(lib().sbr_trace_bistatic(self._h, a.ctypes.data_as(dp), r.ctypes.data_as(dp), len(a),
                                                 float(spacing), float(eta), int(max_bounces), C.byref(o), sp))
        self.max_bounces = int(max_bounces)
        self.n_angles = len(a)
        self._last_angles = a.copy()
        self._trace_args = (spacing, eta, window, offset)
        return st.as_dict() if stats else None

    def run_batch(self, requests, eta=0.05, max_bounces=1, pols="HH,VV", mode="vector", phase="compensated",
                  flags=0, chunk_rays=0, window=0.0, offset=(0.0, 0.0)):
        """Batched trace + PO (sbr_run_batch). ``requests``: iterable of dicts with az, el,
        spacing and freqs (array). Returns (list of E [n_freq, n_pol] complex, list of
        rcs [n_freq, n_pol], stats)."""
        reqs, arr, freqs = _requests(requests)
        pm = _pols(pols)
        npol = bin(pm).count("1")
        m = (PO_PAPER_SCALAR if mode == "scalar" else PO_VECTOR) | PHASE[phase]
        E = np.empty((len(freqs), npol, 2), np.float64)
        R = np.empty((len(freqs), npol), np.float64)
        o = _opts(window, offset, flags, chunk_rays)
        st = TraceStats()
        self._check(lib().sbr_run_batch(self._h, arr, len(reqs), freqs.ctypes.data_as(C.POINTER(C.c_double)),
                                        len(freqs), float(eta), int(max_bounces), pm, m, C.byref(o), E.ctypes.data,
                                        R.ctypes.data, 0, C.byref(st)))
        Ec = E[..., 0] + 1j * E[..., 1]
        outE, outR, off = [], [], 0
        for k in range(len(reqs)):
            nf = arr[k].n_freq
            outE.append(Ec[off:off + nf])
            outR.append(R[off:off + nf])
            off += nf
        return outE, outR, st.as_dict()

    def submit_batch(self, requests, E_out=None, rcs_out=None, eta=0.05, max_bounces=1, pols="HH,VV",
                     mode="vector", phase="compensated", flags=0, chunk_rays=0, window=0.0, offset=(0.0, 0.0)):
        """Asynchronous batch (sbr_submit_batch): enqueue the batch as a CUDA graph on the context's stream
        and return at once. ``E_out`` / ``rcs_out``: CUDA float64 tensors [rows, n_pol, 2] / [rows, n_pol]
        (rows = total frequencies), written when the stream gets there; ``sync()`` waits. Submitting the
        same requests, options and tensors again replays the captured graph."""
        reqs, arr, freqs = _requests(requests)
        self._submit_keep = (arr, freqs)
        pm = _pols(pols)
        m = (PO_PAPER_SCALAR if mode == "scalar" else PO_VECTOR) | PHASE[phase]
        o = _opts(window, offset, flags, chunk_rays)
        ep = E_out.data_ptr() if E_out is not None else None
        rp = rcs_out.data_ptr() if rcs_out is not None else None
        self._check(lib().sbr_submit_batch(self._h, arr, len(reqs), freqs.ctypes.data_as(C.POINTER(C.c_double)),
                                           len(freqs), float(eta), int(max_bounces), pm, m, C.byref(o), ep, rp))

    def tuning(self) -> dict:
        t = Tuning()
        self._check(lib().sbr_get_tuning(self._h, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        """Change some tuning fields (tile_w, blocks_per_sm, stack_depth, chunk_rays_log2, po_item, bvh_width,
        packet, octant, silhouette, raster)."""
        t = Tuning(**{**self.tuning(), **kw})
        self._check(lib().sbr_set_tuning(self._h, C.byref(t)))

    def autotune(self, requests, eta=0.05, max_bounces=1, pols="HH,VV", mode="vector", phase="compensated",
                 flags=0, chunk_rays=0, window=0.0, offset=(0.0, 0.0), reps=3):
        """sbr_autotune on a sample batch; returns (best tuning dict, best ms, list of trials)."""
        reqs, arr, freqs = _requests(requests)
        pm = _pols(pols)
        m = (PO_PAPER_SCALAR if mode == "scalar" else PO_VECTOR) | PHASE[phase]
        o = _opts(window, offset, flags, chunk_rays)
        cap = 64
        tr = (TuneTrial * cap)()
        n = C.c_int()
        best = Tuning()
        ms = C.c_double()
        self._check(lib().sbr_autotune(self._h, arr, len(reqs), freqs.ctypes.data_as(C.POINTER(C.c_double)),
                                       len(freqs), float(eta), int(max_bounces), pm, m, C.byref(o), int(reps), tr, cap,
                                       C.byref(n), C.byref(best), C.byref(ms)))
        trials = [dict(tr[k].tuning.as_dict(), ms=float(tr[k].ms), status=int(tr[k].status))
                  for k in range(min(n.value, cap))]
        return best.as_dict(), float(ms.value), trials

    def sync(self) -> dict:
        """Wait for the last submitted batch; its statistics."""
        st = TraceStats()
        self._check(lib().sbr_sync(self._h, C.byref(st)))
        return st.as_dict()

    def po_integrate(self, freqs, pols="HH,VV", mode="vector", phase="compensated", E_out=None, rcs_out=None):
        """PO sum of the last trace. Returns (E complex128 [n_angles, n_freq, n_pol], rcs_dbsm [...]) as
        numpy arrays, or fills the given CUDA float64 tensors E_out [.., 2] / rcs_out (device path)."""
        f = np.ascontiguousarray(np.atleast_1d(freqs), dtype=np.float64)
        pm = _pols(pols)
        npol = bin(pm).count("1")
        m = (PO_PAPER_SCALAR if mode == "scalar" else PO_VECTOR) | PHASE[phase]
        fp = f.ctypes.data_as(C.POINTER(C.c_double))
        if E_out is not None or rcs_out is not None:
            ep = E_out.data_ptr() if E_out is not None else None
            rp = rcs_out.data_ptr() if rcs_out is not None else None
            self._check(lib().sbr_po_integrate(self._h, fp, len(f), pm, m, ep, rp, 1))
            return E_out, rcs_out
        E = np.empty((self.n_angles, len(f), npol, 2), np.float64)
        R = np.empty((self.n_angles, len(f), npol), np.float64)
        self._check(lib().sbr_po_integrate(self._h, fp, len(f), pm, m, E.ctypes.data, R.ctypes.data, 0))
        return E[..., 0] + 1j * E[..., 1], R

    def get_hits(self, angle: int):
        """Per-ray hits of aspect ``angle`` (needs TRACE_RECORD_HITS): (tri [n, B], t [n, B], n_bounce [n])."""
        sp, eta, window, offset = self._trace_args
        g = self.ray_grid_for(*self._angle(angle), sp, eta, window, offset)
        n = g["nu"] * g["nv"]
        B = self.max_bounces
        tri = np.empty((n, B), np.int32)
        t = np.empty((n, B), np.float32)
        nb = np.empty(n, np.int32)
        self._check(lib().sbr_get_hits(self._h, int(angle), tri.ctypes.data, t.ctypes.data, nb.ctypes.data))
        return tri, t, nb

    def _angle(self, angle):
        return self._last_angles[angle]

    def get_records(self, angle: int) -> dict:
        n = C.c_int64()
        self._check(lib().sbr_get_records(self._h, int(angle), 0, None, None, None, C.byref(n)))
        cnt = int(n.value)
        ids = np.empty(cnt, np.int64)
        coef = np.empty((cnt, 5), np.float32)
        path = np.empty(cnt, np.float64)
        self._check(lib().sbr_get_records(self._h, int(angle), cnt, ids.ctypes.data, coef.ctypes.data,
                                          path.ctypes.data, C.byref(n)))
        return dict(ray=ids, coef=coef, L=path)


# ---------------------------------------------------------------------------- surrogate
def _requests(requests):
    """(list of request dicts, sbr_request array, concatenated frequency array)."""
    reqs = list(requests)
    freqs = np.ascontiguousarray(np.concatenate([np.atleast_1d(np.asarray(r["freqs"], np.float64)) for r in reqs]))
    arr = (Request * len(reqs))()
    off = 0
    for k, r in enumerate(reqs):
        nf = len(np.atleast_1d(r["freqs"]))
        arr[k] = Request(float(r["az"]), float(r["el"]), float(r["spacing"]), off, nf, 0)
        off += nf
    return reqs, arr, freqs


class SurrogateOpts(C.Structure):
    _fields_ = [("n_members", C.c_int), ("width", C.c_int), ("depth", C.c_int), ("n_fourier", C.c_int),
                ("fourier_sigma", C.c_float), ("seed", C.c_uint64)]


def _surrogate_sigs(L):
    P, vp, i64, d = C.POINTER, C.c_void_p, C.c_int64, C.c_double
    sig = {
        "sbr_surrogate_create": ([P(vp), C.c_int, vp, P(SurrogateOpts)], C.c_int),
        "sbr_surrogate_destroy": ([vp], None),
        "sbr_surrogate_last_error": ([vp], C.c_char_p),
        "sbr_surrogate_num_params": ([vp], i64),
        "sbr_surrogate_params": ([vp, C.c_int, vp, vp], C.c_int),
        "sbr_surrogate_fourier": ([vp, C.c_int, vp], C.c_int),
        "sbr_surrogate_train": ([vp, vp, vp, i64, C.c_int, C.c_int, C.c_float, vp], C.c_int),
        "sbr_surrogate_grads": ([vp, C.c_int, vp, vp, i64, P(d), vp], C.c_int),
        "sbr_surrogate_predict": ([vp, vp, i64, vp, vp], C.c_int),
        "sbr_gemm_bf16_tn": ([vp, C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp], C.c_int),
        "sbr_gemm_bf16_tn_async": ([vp, C.c_int, vp, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, vp],
                                   C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def gemm_bf16_tn(A_ptr: int, lda: int, B_ptr: int, ldb: int, M: int, N: int, K: int, C_ptr: int, ldc: int,
                 stream=None) -> None:
    """C [M x N] FP32 = A [M x K] B^T on the tensor cores (device pointers; BF16 inputs, K contiguous)."""
    L = _surrogate_sigs(lib())
    s = int(getattr(stream, "cuda_stream", stream)) if stream is not None else None
    rc = L.sbr_gemm_bf16_tn(A_ptr, lda, B_ptr, ldb, M, N, K, C_ptr, ldc, C.c_void_p(s) if s else None)
    if rc != SBR_OK:
        raise SbrError(rc, "sbr_gemm_bf16_tn failed")


def gemm_bf16_tn_async(A_ptr: int, lda: int, B_ptr: int, ldb: int, M: int, N: int, K: int, C_ptr: int, ldc: int,
                       err_ptr: int, stream=None) -> None:
    """As gemm_bf16_tn, only enqueued (sbr_gemm_bf16_tn_async); err_ptr: a zeroed device int32 set to 1 if a
    bounded wait in the kernel gave up."""
    L = _surrogate_sigs(lib())
    s = int(getattr(stream, "cuda_stream", stream)) if stream is not None else None
    rc = L.sbr_gemm_bf16_tn_async(A_ptr, lda, B_ptr, ldb, M, N, K, C_ptr, ldc, err_ptr, C.c_void_p(s) if s else None)
    if rc != SBR_OK:
        raise SbrError(rc, "sbr_gemm_bf16_tn_async failed")


class Surrogate:
    """Fourier-feature MLP ensemble trained on SBR samples (sbr_surrogate_*)."""

    def __init__(self, device=0, stream=None, n_members=4, width=512, depth=6, n_fourier=256, fourier_sigma=4.0,
                 seed=1):
        L = _surrogate_sigs(lib())
        o = SurrogateOpts(n_members, width, depth, n_fourier, fourier_sigma, seed)
        h = C.c_void_p()
        s = int(getattr(stream, "cuda_stream", stream)) if stream is not None else None
        rc = L.sbr_surrogate_create(C.byref(h), int(device), C.c_void_p(s) if s else None, C.byref(o))
        if rc != SBR_OK:
            raise SbrError(rc, "sbr_surrogate_create failed")
        self._h = h
        self._stream_ref = stream
        self.n_members, self.width, self.depth, self.n_fourier = n_members, width, depth, n_fourier
        self.n_params = int(L.sbr_surrogate_num_params(h))

    def _check(self, rc):
        if rc != SBR_OK:
            raise SbrError(rc, (lib().sbr_surrogate_last_error(self._h) or b"").decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sbr_surrogate_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, member=0, set_to=None):
        out = np.empty(self.n_params, np.float32)
        if set_to is not None:
            set_to = np.ascontiguousarray(set_to, dtype=np.float32)
            assert set_to.size == self.n_params
        self._check(lib().sbr_surrogate_params(self._h, member, out.ctypes.data,
                                               None if set_to is None else set_to.ctypes.data))
        return out

    def fourier(self, member=0):
        B = np.empty((self.n_fourier // 2, 4), np.float32)
        self._check(lib().sbr_surrogate_fourier(self._h, member, B.ctypes.data))
        return B

    def train(self, x, y, epochs=10, batch=8192, lr=1e-3):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        loss = np.zeros((self.n_members, epochs), np.float32)
        self._check(lib().sbr_surrogate_train(self._h, x.ctypes.data, y.ctypes.data, len(x), int(epochs),
                                              int(batch), float(lr), loss.ctypes.data))
        return loss

    def grads(self, x, y, member=0):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        g = np.empty(self.n_params, np.float32)
        loss = C.c_double()
        self._check(lib().sbr_surrogate_grads(self._h, member, x.ctypes.data, y.ctypes.data, len(x),
                                              C.byref(loss), g.ctypes.data))
        return float(loss.value), g

    def predict(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        ym = np.empty((len(x), 4), np.float64)
        sp = np.empty(len(x), np.float32)
        self._check(lib().sbr_surrogate_predict(self._h, x.ctypes.data, len(x), ym.ctypes.data, sp.ctypes.data))
        return ym, sp
