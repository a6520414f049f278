"""Benchmark of the SBR trace-integrate path on one GB300 (replicas on N GPUs).

Workload (default, the largest configuration): seeded procedural aircraft
(983,270 triangles), 10 GHz, ray spacing lambda/10 (margin 0.05), up to 10
bounces, 360 azimuths at elevation 0 (about 4.8 G launched rays per sweep),
vector PO, HH and VV. One step = one full sweep: sbr_trace over all 360
aspects + sbr_po_integrate. The trihedral sweep (C2) runs beside it and is
reported under "trihedral".

Metric: ray-bounces per second (closest-hit queries on live rays, hit or
miss), aggregated over all ranks; angles per second is reported beside it.

  value     device-resident: mesh and BVH already on the GPU, outputs to device
  e2e       through the public API from host buffers every step: mesh upload
            from pinned host memory, BVH build, trace, PO, results read back
  roofline  the bounce passes (the dominant kernel): R* = min(BW / B_rb,
            P / F_rb) with B_rb = 32 n_node + 48 n_tri bytes and
            F_rb = 28 n_node + 30 n_tri FP32 operations per bounce query
            (n_node, n_tri: node visits and triangle tests per query from a
            counting run), BW the probed L2 bandwidth when the tree and the
            triangles fit in L2 (else the measured HBM bandwidth), P the probed
            FP32 FMA rate; frac = measured bounce queries/s / R*
  cpu_baseline  the FP64 oracle on a seeded sample of the sweep's rays, all host cores

``--impl reference`` times the oracle (the CPU reference of this method) on
the same workload and prints its own line. N > 1 (torchrun): every rank runs
the full workload on its own GPU (replicas, no collective on the data path);
the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import sbr_inputs as S  # noqa: E402

# Roofline of the traversal (the bounce passes): per bounce query, B_rb = 32 bytes per node visit + 48 per
# triangle test (one node's box, one triangle record) and F_rb = 28 FP32 operations per node visit (slab tests
# of two children) + 30 per triangle test (Moller-Trumbore).
BYTES_NODE, BYTES_TRI = 32, 48
FLOP_NODE, FLOP_TRI = 28, 30
# one rasterised cell test: the ray's FP32 origin (12) and the triangle test with the per-(aspect, triangle)
# constants (38), FMA counted as 2; the roofline of workloads without bounce passes (B = 1)
FLOP_CELL = 50
# FP32 operations of the per-hit arithmetic (apply_hit: hit point, path, normal orientation, receiver path
# term, H field, tube area, the vector PO terms and coefficients, scalar coefficient, PEC field update,
# reflection, new origin), reported beside the roofline: 157 per hit of a bounce pass, 185 for a primary hit
# rebuilt by bounce pass 1.
OPS_HIT = 157
OPS_PRIMARY_HIT = 185
# DRAM bytes per bounce query of the bounce passes (dram__bytes_read.sum + dram__bytes_write.sum over the
# k_bounce launches of one ncu capture, divided by their queries), per workload and setting; scaled by the
# bounce queries of a step. None where no capture of the current kernels exists.
TRAFFIC_PER_QUERY = {
    # k_bounce, warm L2 (ncu --cache-control none), 36 of the 360 aspects, five identical sweeps, grouped ray pool
    "aircraft10": [(116.8, {"bvh_width": 2, "octant": 0, "packet": 0})],
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="gloo")
        pg = dist
    return ws, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload(name: str) -> dict:
    if name == "trihedral":
        return S.trihedral_case()
    if name == "sphere":
        return S.sphere_case(n_random=64)
    if name == "aircraft3deep":
        # deep cavities: up to 100 bounces, a ray still hitting after them is invalid (escape required)
        c = S.aircraft_case(3e9, n_az=360)
        c.update(name="aircraft_3GHz_B100_escape", max_bounces=100, escape=True)
        return c
    if name.startswith("aircraft"):
        f = {"aircraft1": 1e9, "aircraft3": 3e9, "aircraft10": 10e9}[name]
        return S.aircraft_case(f, n_az=360)
    raise ValueError(name)


def wl_config(case: dict, name: str) -> dict:
    return {"workload": case["name"], "mesh_triangles": int(len(case["tri"])), "aspects": int(len(case["angles"])),
            "freq_ghz": [float(f) / 1e9 for f in case["freqs"]], "ray_spacing_m": float(case["spacing"]),
            "max_bounces": int(case["max_bounces"]), "require_escape": bool(case.get("escape", False)),
            "grid_offset": list(case.get("offset", (0.0, 0.0))),
            "po": "vector", "pols": "HH,VV",
            "l2": "flushed between timed steps (512 MB write)"}


# ----------------------------------------------------------------------------- oracle timing
_ORACLE_MESH = {}


def oracle_sample(case, n_angles: int, threads: int, frac: float = 1.0, seed: int = 0):
    """The oracle on ``n_angles`` evenly spaced aspects of the workload, each with a
    seeded fraction ``frac`` of its ray grid (all rays when 1): ray-bounces,
    seconds of trace + PO (the oracle's mesh and BVH are built once, untimed)."""
    import oracle

    key = case["name"]
    if key not in _ORACLE_MESH:
        _ORACLE_MESH.clear()
        _ORACLE_MESH[key] = oracle.Mesh(case["xyz"], case["tri"])
    om = _ORACLE_MESH[key]
    idx = np.linspace(0, len(case["angles"]) - 1, n_angles).round().astype(int)
    rng = np.random.default_rng(seed)
    frames = []
    for a in idx:
        az, el = case["angles"][a]
        fr = oracle.make_frame(om.bbox, az, el, case["spacing"], eta=case["eta"], window=case.get("window", 0.0),
                               offset=case.get("offset", (0.0, 0.0)))
        ids = None if frac >= 1.0 else np.sort(rng.choice(fr.n_rays, max(1, int(fr.n_rays * frac)), replace=False))
        frames.append((fr, ids))
    t0 = time.perf_counter()
    bounces = 0
    for fr, ids in frames:
        tr = oracle.trace(om, fr, case["max_bounces"], threads=threads, require_escape=case.get("escape", False),
                          ids=ids)
        oracle.po(tr["coef"], tr["L"], tr["valid"], case["freqs"])
        nb = tr["nb"]
        bounces += int(np.sum(nb + (nb < case["max_bounces"])))
    dt = time.perf_counter() - t0
    return bounces, dt, idx


def oracle_sample_size(case):
    """Oracle sample of a step: the whole sweep's aspects for the small meshes, a seeded fraction of
    the rays of 12 evenly spaced aspects for the aircraft (about 1 M rays per aspect at 10 GHz)."""
    if "aircraft" in case["name"]:
        f = float(case["freqs"][0])
        return 12, min(1.0, 0.4 * (10e9 / f) ** 2)
    return min(24, len(case["angles"])), 1.0


def run_reference(args, case, ws, rank, pg):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    n, frac = oracle_sample_size(case)
    t1 = 0.0
    for _ in range(max(1, args.warmup)):
        t1 = oracle_sample(case, 1, threads, frac)[1]
    # aspects per step: fewer when the steps would take more than about two minutes
    n = max(1, min(n, args.ref_angles, int(120.0 / (max(1, args.steps) * max(t1, 1e-3)))))
    tot_b, tot_t = 0, 0.0
    for k in range(args.steps):
        b, t, idx = oracle_sample(case, n, threads, frac, seed=k)
        tot_b += b
        tot_t += t
    v = tot_b / tot_t
    sample = (f"{n} of {len(case['angles'])} aspects per step (evenly spaced), "
              + ("full ray grids" if frac >= 1.0 else f"a seeded {100 * frac:.3g} % of each aspect's rays"))
    line = {"impl": "reference", "metric": "ray-bounces/s", "value": v, "unit": "ray-bounces/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(wl_config(case, args.workload), bvh_builder=args.builder),
            "cpu_baseline": {"value": v, "unit": "ray-bounces/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "ray-bounces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- GPU arm
def sweep_value(G, torch, dev, case, tuning, steps, warmup, flush):
    """Ray-bounces/s of another sweep (device-resident, CUDA events, L2 flushed between steps) with a fixed
    tuning: reported beside the headline workload."""
    stream = torch.cuda.Stream(dev)
    ctx = G.Context(dev, stream=stream)
    ctx.load_mesh(case["xyz"], case["tri"])
    ctx.set_tuning(**tuning)
    ang = np.ascontiguousarray(case["angles"], np.float64)
    kw = dict(eta=case["eta"], max_bounces=case["max_bounces"], window=case.get("window", 0.0),
              offset=case.get("offset", (0.0, 0.0)))
    E = torch.empty((len(ang), len(case["freqs"]), 2, 2), dtype=torch.float64, device=f"cuda:{dev}")
    R = torch.empty((len(ang), len(case["freqs"]), 2), dtype=torch.float64, device=f"cuda:{dev}")

    def step():
        st = ctx.trace(ang, case["spacing"], **kw)
        ctx.po_integrate(case["freqs"], "HH,VV", E_out=E, rcs_out=R)
        return st

    for _ in range(warmup):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        ev[k][0].record(stream)
        st = step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ctx.close()
    return {"workload": case["name"], "value": st["ray_bounces"] / (ms * 1e-3), "unit": "ray-bounces/s",
            "ms_per_step": ms, "angles_per_s": len(ang) / (ms * 1e-3), "aspects": len(ang),
            "ray_bounces_per_step": st["ray_bounces"], "tuning": tuning}


def precision_report(G, torch, dev, n_az=4, freq=(8e9, 12e9, 17)):
    """Precision form: the same traced records of the aircraft at 10 GHz
    (lambda/10, B = 10, n_az azimuths at el 0) integrated with the three phase
    modes. Paths reach ~60 m, so k L ~ 1.3e4 rad. Errors are against the FP64
    phase (same records, same FP64 cross-item sums), in dB where that result
    is above -40 dBsm; times are the PO kernels alone (CUDA events)."""
    case = S.aircraft_case(10e9, n_az=360)
    ang = case["angles"][np.linspace(0, 359, n_az).round().astype(int)]
    freqs = np.linspace(*freq)
    stream = torch.cuda.Stream(dev)
    ctx = G.Context(dev, stream=stream)
    ctx.load_mesh(case["xyz"], case["tri"])
    st = ctx.trace(ang, case["spacing"], eta=case["eta"], max_bounces=case["max_bounces"], offset=case["offset"])
    out, ms = {}, {}
    for ph in ("fp64", "compensated", "fp32"):
        E = torch.empty((len(ang), len(freqs), 2, 2), dtype=torch.float64, device=f"cuda:{dev}")
        R = torch.empty((len(ang), len(freqs), 2), dtype=torch.float64, device=f"cuda:{dev}")
        ctx.po_integrate(freqs, "HH,VV", phase=ph, E_out=E, rcs_out=R)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            ctx.po_integrate(freqs, "HH,VV", phase=ph, E_out=E, rcs_out=R)
        e1.record(stream)
        torch.cuda.synchronize()
        ms[ph] = e0.elapsed_time(e1) / 5
        out[ph] = R.cpu().numpy()
    ctx.close()
    ref = out["fp64"]
    big = ref > -40.0
    return {"case": f"aircraft 10 GHz, lambda/10, B = 10, {n_az} azimuths at el 0, {len(freqs)} frequencies "
                    f"{freq[0] / 1e9:g}-{freq[1] / 1e9:g} GHz, HH and VV",
            "valid_rays": st["valid_rays"],
            "max_db_error_vs_fp64_phase": {k: float(np.max(np.abs(out[k][big] - ref[big])))
                                           for k in ("compensated", "fp32")},
            "median_db_error_vs_fp64_phase": {k: float(np.median(np.abs(out[k][big] - ref[big])))
                                              for k in ("compensated", "fp32")},
            "po_ms": ms}


def batched_vs_plain(G, torch, dev, n_req, passes=5):
    """Batched form against plain per-request SBR on the first ``n_req`` requests
    of the mixed-request workload (4096 requests, seed 2, over the sphere,
    trihedral and aircraft meshes): requests (= aspects) per second, same
    requests, same outputs (HH, VV for every requested frequency)."""
    import time as _t

    reqs = S.batched_requests(4096, seed=2)[:n_req]
    meshes = [S.icosphere(5), S.trihedral(1.0, 32), S.aircraft(seed=1)]
    offs = [(0.0, 0.0), S.grid_offset(5), S.grid_offset(6)]
    bounces = [1, 3, 10]
    ctxs = []
    for xyz, tri in meshes:
        c = G.Context(dev)
        c.load_mesh(xyz, tri)
        ctxs.append(c)
    groups = [[r for r in reqs if r["mesh"] == m] for m in range(3)]

    def batched():
        rb = 0
        for m in range(3):
            if groups[m]:
                rb += ctxs[m].run_batch(groups[m], eta=0.05, max_bounces=bounces[m], offset=offs[m])[2]["ray_bounces"]
        torch.cuda.synchronize()
        return rb

    def plain():
        for m in range(3):
            for r in groups[m]:
                ctxs[m].trace([[r["az"], r["el"]]], r["spacing"], eta=0.05, max_bounces=bounces[m], offset=offs[m],
                              stats=False)
                ctxs[m].po_integrate(r["freqs"], "HH,VV")
        torch.cuda.synchronize()

    rows = [sum(len(r["freqs"]) for r in groups[m]) for m in range(3)]
    outs = [torch.zeros((max(1, rows[m]), 2), dtype=torch.float64, device=f"cuda:{dev}") for m in range(3)]
    torch.cuda.synchronize()

    def graphed():
        # one asynchronous submission per mesh (each context has its own stream), then wait for all
        for m in range(3):
            if groups[m]:
                ctxs[m].submit_batch(groups[m], None, outs[m], eta=0.05, max_bounces=bounces[m], offset=offs[m])
        return sum(ctxs[m].sync()["ray_bounces"] for m in range(3) if groups[m])

    batched()
    plain()
    graphed()
    tb_l, tp_l, tg_l = [], [], []
    rb = rg = 0
    for _ in range(passes):
        t0 = _t.perf_counter()
        rb = batched()
        tb_l.append(_t.perf_counter() - t0)
        t0 = _t.perf_counter()
        plain()
        tp_l.append(_t.perf_counter() - t0)
        t0 = _t.perf_counter()
        rg = graphed()
        tg_l.append(_t.perf_counter() - t0)
    tb, tp, tg = float(np.median(tb_l)), float(np.median(tp_l)), float(np.median(tg_l))
    same = True
    for m in range(3):
        if groups[m]:
            _, Rb, _ = ctxs[m].run_batch(groups[m], eta=0.05, max_bounces=bounces[m], offset=offs[m])
            same = same and bool(np.array_equal(outs[m][:rows[m]].cpu().numpy(), np.concatenate(Rb)))
    for c in ctxs:
        c.close()
    return {"requests": n_req, "meshes": "icosphere5 / trihedral / aircraft (1M)",
            "frequencies": int(sum(len(r["freqs"]) for r in reqs)),
            "batched_requests_per_s": n_req / tb, "plain_requests_per_s": n_req / tp, "speedup": tp / tb,
            "graph_requests_per_s": n_req / tg, "graph_speedup": tp / tg, "graph_equals_batched": same,
            "batched_ray_bounces_per_s": rb / tb, "graph_ray_bounces_per_s": rg / tg,
            "seconds_per_pass": {"plain": [min(tp_l), tp, max(tp_l)], "batched": [min(tb_l), tb, max(tb_l)],
                                 "graph": [min(tg_l), tg, max(tg_l)]},
            "timing": f"host wall clock, median of {passes} passes each (min, median, max listed) after one warm-up "
                      "pass; graph = sbr_submit_batch replay (one CUDA graph per mesh, three streams) + sbr_sync"}


SURROGATE_DOMAINS = {
    # the configured case: the whole sweep space, 200k samples
    "full": dict(az=(0.0, 360.0), el=(-30.0, 30.0), f=(1e9, 12e9), n_aspects=2000, f_per=100, n_heldout=10000,
                 lattice=(500, 40, 50), sigmas=(1.0, 4.0, 16.0, 64.0)),
    # a dense sweep patch around nose-on: 4 deg x 2 deg x 1.0-1.2 GHz, 200k samples
    # held-out points traced on the training data's ray grid (10 rays per wavelength of 1.2 GHz)
    "patch": dict(az=(178.0, 182.0), el=(-1.0, 1.0), f=(1e9, 1.2e9), n_aspects=2000, f_per=100, n_heldout=10000,
                  lattice=(100, 20, 500), sigmas=(16.0, 32.0, 64.0, 128.0, 256.0), heldout_grid="domain"),
    # the same patch with SBR (training data and judge) at 50 rays per wavelength, where SBR's own
    # dependence on the ray grid (0.28 dB median) is below the 0.5 dB target
    "patch_dense": dict(az=(178.0, 182.0), el=(-1.0, 1.0), f=(1e9, 1.2e9), n_aspects=2000, f_per=100,
                        n_heldout=10000, lattice=(100, 20, 500), sigmas=(16.0, 32.0, 64.0, 128.0, 256.0),
                        heldout_grid="domain", rpl=50.0),
}


def _tensor_roofline(points, members, seconds, width=512, depth=6, n_fourier=256):
    """Ensemble prediction as a tensor-core contraction: 2 (n_fourier W + (D - 1) W^2 + 4 W) FLOP per point
    and member (BF16 GEMMs with FP32 accumulation), over the whole prediction call (host wall clock, so
    the Fourier features, head, ensemble statistics and transfers count against it)."""
    flops = 2.0 * (n_fourier * width + (depth - 1) * width * width + 4 * width) * points * members
    pk, src = peaks()
    peak = pk.get("bf16_tflops", 1900.0)
    ach = flops / seconds / 1e12
    return {"bound": "tensor", "kernel": "k_gemm_tn (tcgen05, BF16 in, FP32 accumulate) in sbr_surrogate_predict",
            "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
            "peak_source": f"bf16 dense GEMM burst, {src}", "flop": flops}


def surrogate_eval(G, torch, ctx, dom, epochs=60, batch=2048, spread_db=1.0, scale=1.0):
    """Learned surrogate on the aircraft mesh against plain SBR over one domain.

    Training data: ``n_aspects`` aspects uniform over the domain's (az, el) box
    (seed 3), each with ``f_per`` frequencies log-uniform over its band, traced
    once at 10 rays per wavelength of its highest frequency (batched form) ->
    samples (az, el, f) -> (Re, Im of HH and VV). sigma_B is picked on a 90/10
    split. Held out: ``n_heldout`` points (seed 4), each its own aspect and
    frequency, computed by plain SBR at 10 rays per wavelength of that
    frequency. The ensemble answers a point when its spread is <= ``spread_db``;
    otherwise SBR does. ``scale`` shrinks the sample counts (quick runs)."""
    import time as _t

    off = S.grid_offset(6)
    rpl = dom.get("rpl", 10.0)  # rays per wavelength of the SBR runs
    n_aspects = max(8, int(dom["n_aspects"] * scale))
    n_heldout = max(64, int(dom["n_heldout"] * scale))
    f_per = dom["f_per"]
    (a0, a1), (e0, e1), (f0, f1) = dom["az"], dom["el"], dom["f"]
    rng = np.random.default_rng(3)
    reqs = []
    for _ in range(n_aspects):
        f = np.sort(np.exp(rng.uniform(np.log(f0), np.log(f1), f_per)))
        reqs.append(dict(az=float(rng.uniform(a0, a1)), el=float(rng.uniform(e0, e1)), freqs=f,
                         spacing=S.spacing_for(float(f[-1]), rpl)))
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    E, _, st = ctx.run_batch(reqs, eta=0.05, max_bounces=10, offset=off)
    t_data = _t.perf_counter() - t0
    x = np.concatenate([np.stack([np.full(len(r["freqs"]), r["az"]), np.full(len(r["freqs"]), r["el"]), r["freqs"]], 1)
                        for r in reqs])
    Ec = np.concatenate(E)
    y = np.stack([Ec[:, 0].real, Ec[:, 0].imag, Ec[:, 1].real, Ec[:, 1].imag], 1)
    # Fourier scale sigma_B tuned on a 90/10 split of the training samples (one member, short runs)
    t0 = _t.perf_counter()
    perm = np.random.default_rng(5).permutation(len(x))
    cut = (int(0.9 * len(x)) // 128) * 128
    tr, va = perm[:cut], perm[cut:]
    tune = {}
    for sig in dom["sigmas"]:
        m = G.Surrogate(ctx.device, n_members=1, width=512, depth=6, n_fourier=256, fourier_sigma=sig, seed=11)
        m.train(x[tr], y[tr], epochs=max(1, epochs // 4), batch=batch, lr=1e-3)
        yv, _ = m.predict(x[va])
        m.close()
        tune[sig] = float(np.sqrt(np.mean((yv - y[va]) ** 2)) / np.sqrt(np.mean(y[va] ** 2)))
    sigma = min(tune, key=tune.get)
    t_tune = _t.perf_counter() - t0
    sur = G.Surrogate(ctx.device, n_members=4, width=512, depth=6, n_fourier=256, fourier_sigma=sigma, seed=1)
    t0 = _t.perf_counter()
    loss = sur.train(x, y, epochs=epochs, batch=batch, lr=1e-3)
    t_train = _t.perf_counter() - t0
    # held-out points, plain SBR (one frequency per aspect)
    rng = np.random.default_rng(4)
    hx = np.stack([rng.uniform(a0, a1, n_heldout), rng.uniform(e0, e1, n_heldout),
                   np.exp(rng.uniform(np.log(f0), np.log(f1), n_heldout))], 1)
    # plain SBR of each held-out point: 10 rays per wavelength of its own frequency, or of the domain's
    # highest frequency (the training data's grid) when the domain says so
    domain_grid = dom.get("heldout_grid") == "domain"
    hreq = [dict(az=a, el=e, freqs=np.array([f]), spacing=S.spacing_for(f1 if domain_grid else f, rpl))
            for a, e, f in hx]
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    _, Rh, _ = ctx.run_batch(hreq, eta=0.05, max_bounces=10, offset=off)
    t_sbr = _t.perf_counter() - t0
    Rh = np.concatenate(Rh)  # [n, 2] dBsm HH, VV
    grid_sens = None
    if domain_grid:
        # how much plain SBR itself moves between the two ray grids (its own discretisation)
        _, Rg, _ = ctx.run_batch([dict(r, spacing=S.spacing_for(float(r["freqs"][0]), rpl)) for r in hreq],
                                 eta=0.05, max_bounces=10, offset=off)
        dg = np.max(np.abs(np.concatenate(Rg) - Rh), axis=1)
        grid_sens = {"median_db": float(np.median(dg)), "within_0.5dB": float(np.mean(dg <= 0.5))}
    t0 = _t.perf_counter()
    ym, spread = sur.predict(hx)
    t_pred = _t.perf_counter() - t0
    with np.errstate(divide="ignore"):
        Rp = 10 * np.log10(4 * np.pi * np.stack([ym[:, 0] ** 2 + ym[:, 1] ** 2, ym[:, 2] ** 2 + ym[:, 3] ** 2], 1))
    err = np.max(np.abs(Rp - Rh), axis=1)
    above = np.min(Rh, axis=1) > -40.0
    served = spread <= spread_db
    # hybrid: surrogate for served points, SBR for the rest (timed)
    fb = [hreq[i] for i in np.nonzero(~served)[0]]
    t0 = _t.perf_counter()
    if fb:
        ctx.run_batch(fb, eta=0.05, max_bounces=10, offset=off)
    t_fb = _t.perf_counter() - t0
    # dense (az, el, log f) lattice: surrogate query, and SBR on the same lattice (each aspect traced once)
    naz, nel, nfq = dom["lattice"]
    if scale < 1.0:
        naz = max(4, int(naz * scale))
    la, le = np.linspace(a0, a1, naz), np.linspace(e0, e1, nel)
    lf = np.exp(np.linspace(np.log(f0), np.log(f1), nfq))
    A, El, F = np.meshgrid(la, le, lf, indexing="ij")
    q = np.stack([A.ravel(), El.ravel(), F.ravel()], 1)
    t0 = _t.perf_counter()
    _, qs = sur.predict(q)
    t_q = _t.perf_counter() - t0
    lat_aspects = naz * nel
    n_lat_sbr = min(lat_aspects, 256)
    pick = np.linspace(0, lat_aspects - 1, n_lat_sbr).round().astype(int)
    lreq = [dict(az=float(la[k // nel]), el=float(le[k % nel]), freqs=lf, spacing=S.spacing_for(f1, rpl))
            for k in pick]
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    ctx.run_batch(lreq, eta=0.05, max_bounces=10, offset=off)
    t_lat = (_t.perf_counter() - t0) * lat_aspects / n_lat_sbr
    bands = {}
    edges = np.exp(np.linspace(np.log(f0), np.log(f1), 4))
    edges[-1] *= 1.0001
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (hx[:, 2] >= lo) & (hx[:, 2] < hi)
        sm = m & served
        bands[f"{lo / 1e9:.3g}-{min(hi, f1) / 1e9:.3g} GHz"] = {
            "points": int(m.sum()), "served_fraction": float(sm.sum() / max(1, m.sum())),
            "served_median_db_error": float(np.median(err[sm])) if sm.any() else None,
            "served_within_0.5dB": float(np.mean(err[sm] <= 0.5)) if sm.any() else None,
            "all_median_db_error": float(np.median(err[m])) if m.any() else None}
    sur.close()
    return {"domain": {k: dom[k] for k in ("az", "el", "f")}, "training_samples": int(len(x)),
            "heldout_grid": f"{rpl:g} rays per wavelength of " + ("the domain's highest frequency" if domain_grid
                                                                   else "each point's frequency"),
            "rays_per_wavelength": rpl,
            "sbr_grid_sensitivity": grid_sens,
            "training_aspects": n_aspects, "data_gen_s": t_data, "data_ray_bounces": st["ray_bounces"],
            "sigma_validation_rel_rms": {str(k): v for k, v in tune.items()}, "fourier_sigma": sigma,
            "tune_s": t_tune, "train_s": t_train, "epochs": epochs, "batch": batch,
            "final_loss_per_member": [float(v) for v in loss[:, -1]],
            "heldout_points": n_heldout, "plain_sbr_points_per_s": n_heldout / t_sbr,
            "surrogate_points_per_s": n_heldout / t_pred,
            "served_fraction": float(served.mean()), "spread_threshold_db": spread_db,
            "served_median_db_error": float(np.median(err[served])) if served.any() else None,
            "served_within_0.5dB": float(np.mean(err[served] <= 0.5)) if served.any() else None,
            "served_above_m40dBsm_within_0.5dB": float(np.mean(err[served & above] <= 0.5))
            if (served & above).any() else None,
            "all_median_db_error": float(np.median(err)),
            "hybrid_points_per_s": n_heldout / (t_pred + t_fb), "hybrid_vs_plain": t_sbr / (t_pred + t_fb),
            "lattice_points": int(len(q)), "lattice_surrogate_s": t_q,
            "lattice_roofline": _tensor_roofline(len(q), 4, t_q),
            "lattice_served_fraction": float(np.mean(qs <= spread_db)),
            "lattice_sbr_s": t_lat, "lattice_sbr_sample": f"{n_lat_sbr} of {lat_aspects} lattice aspects, scaled",
            "bands": bands}


def surrogate_leg(G, torch, dev, ctx=None, scale=0.25, epochs=30):
    """Bounded surrogate run beside the headline: the configured sweep space (C5) and the dense nose-on patch
    at a quarter of the sample counts and half the epochs (each domain a few tens of seconds). Reports the
    served fraction, the served error against plain SBR per frequency band, and the hybrid's speed against
    plain SBR on the held-out points."""
    own = ctx is None
    if own:
        xyz, tri = S.aircraft(seed=1)
        ctx = G.Context(dev)
        ctx.load_mesh(xyz, tri)
    out = {"scale": scale, "epochs": epochs}
    for name in ("full", "patch_dense"):
        r = surrogate_eval(G, torch, ctx, dict(SURROGATE_DOMAINS[name]), epochs=epochs, scale=scale)
        out[name] = {k: r[k] for k in ("domain", "training_samples", "rays_per_wavelength", "fourier_sigma",
                                       "served_fraction", "served_median_db_error", "served_within_0.5dB",
                                       "all_median_db_error", "hybrid_vs_plain", "plain_sbr_points_per_s",
                                       "hybrid_points_per_s", "lattice_served_fraction", "lattice_points",
                                       "lattice_surrogate_s", "bands", "train_s")}
    if own:
        ctx.close()
    return out


def run_surrogate(args, ws, rank, local, pg):
    """Surrogate-with-fallback against plain SBR on the aircraft (one replica per rank)."""
    import torch
    import paper_2604_09243_gb300 as G

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the surrogate has no oracle counterpart; "
                              "its judge is the plain SBR path"}))
        return
    torch.cuda.set_device(local)
    xyz, tri = S.aircraft(seed=1)
    ctx = G.Context(local)
    ctx.load_mesh(xyz, tri)
    res = {}
    for name in args.sur_domains.split(","):
        dom = dict(SURROGATE_DOMAINS[name])
        if args.sur_rpl > 0:
            dom["rpl"] = args.sur_rpl
        res[name] = surrogate_eval(G, torch, ctx, dom, epochs=args.sur_epochs, scale=args.sur_scale)
    ctx.close()
    head = res[args.sur_domains.split(",")[0]]
    if rank == 0:
        print(json.dumps({"metric": "RCS points/s, surrogate with SBR fallback (spread > 1 dB)",
                          "value": head["hybrid_points_per_s"] * ws, "unit": "points/s", "n_gpus": ws,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                          "data": "synthetic", "config": {"workload": "aircraft_surrogate", "mesh": "aircraft seed 1",
                                                          "parallelism": f"replicas{ws}"},
                          "roofline": head["lattice_roofline"], "surrogate": res}))


def run_gemm(args, ws, rank, local, pg):
    """The surrogate's tensor-core GEMM alone (C = A B^T, BF16 in, FP32 out) on its layer shapes:
    K = 512 hidden layers and K = 256 first layer, M = batch rows. Device time per GEMM from CUDA events
    over args.steps back-to-back launches (sbr_gemm_bf16_tn_async) after args.warmup, inputs resident."""
    import torch
    import paper_2604_09243_gb300 as G

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "no CPU counterpart of the tensor-core GEMM"}))
        return
    torch.cuda.set_device(local)
    pk, src = peaks()
    peak = pk.get("bf16_tflops", 1900.0)
    res = []
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for M, N, K in ((2048, 512, 512), (8192, 512, 512), (8192, 512, 256), (32768, 512, 512), (65536, 512, 512),
                    (131072, 512, 512)):
        g = torch.Generator(device="cpu").manual_seed(M + K)
        A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
        B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
        C = torch.empty(M, N, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            G.gemm_bf16_tn_async(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C.data_ptr(), N, err.data_ptr(), stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            G.gemm_bf16_tn_async(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C.data_ptr(), N, err.data_ptr(), stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if int(err.item()):
            raise RuntimeError("k_gemm_tn: a bounded wait gave up")
        ms = e0.elapsed_time(e1) / args.steps
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        # algorithmic bytes: both operands read once, the FP32 result written once
        nbytes = 2.0 * M * K + 2.0 * N * K + 4.0 * M * N
        res.append({"M": M, "N": N, "K": K, "us": ms * 1e3, "tflops": tf, "frac": tf / peak,
                    "flop_per_byte": 2.0 * M * N * K / nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9})
    top = res[-1]
    # roofline of the largest shape: below the ridge (tensor peak / HBM bandwidth) it is bound by HBM
    hbm = pk.get("hbm_gbs", 6800.0)
    ridge = peak * 1e12 / (hbm * 1e9)
    if top["flop_per_byte"] < ridge:
        roof = {"bound": "hbm", "kernel": "k_gemm_tn (tcgen05)", "achieved": top["gbs"], "peak": hbm, "unit": "GB/s",
                "frac": top["gbs"] / hbm, "traffic": None,
                "peak_source": f"HBM copy bandwidth, {src}",
                "flop_per_byte": top["flop_per_byte"], "ridge_flop_per_byte": ridge,
                "tensor_frac": top["frac"], "attainable_tflops": top["flop_per_byte"] * hbm / 1e3}
    else:
        roof = {"bound": "tensor", "kernel": "k_gemm_tn (tcgen05)", "achieved": top["tflops"], "peak": peak,
                "unit": "TFLOP/s", "frac": top["frac"], "traffic": None,
                "peak_source": f"bf16 dense GEMM burst, {src}", "flop_per_byte": top["flop_per_byte"],
                "ridge_flop_per_byte": ridge}
    if rank == 0:
        print(json.dumps({"metric": "BF16 GEMM TFLOP/s (surrogate layer shapes)", "value": top["tflops"] * ws,
                          "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                          "data": "synthetic", "config": {"workload": "surrogate_gemm", "shapes": "M x 512 x K"},
                          "roofline": roof, "shapes": res}))


def run_po(args, ws, rank, local, pg):
    """The PO sum alone on the aircraft's records at 10 GHz (B = 10, every 5th of the 360 aspects unless
    --aspects): sbr_po_integrate with device outputs, timed with CUDA events on the context's stream over
    args.steps calls after args.warmup, for 1, 2 and 16 frequencies (HH, VV). One and two frequencies run
    the staged kernel (records streamed through shared memory), 16 the register kernel. Roofline at one
    frequency: the 32-byte records read once, against the HBM copy bandwidth."""
    import torch
    import paper_2604_09243_gb300 as G

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the PO-only timing has no oracle leg; the oracle "
                              "sums the same records inside the default workload's reference arm"}))
        return
    torch.cuda.set_device(local)
    case = workload("aircraft10")
    n_asp = args.aspects if args.aspects > 0 else 72
    idx = np.linspace(0, len(case["angles"]) - 1, n_asp).round().astype(int)
    stream = torch.cuda.Stream()
    ctx = G.Context(local, stream=stream)
    ctx.load_mesh(case["xyz"], case["tri"])
    ctx.set_tuning(**({k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(","))} if args.tune
                      else {"po_item": 2048}))
    st = ctx.trace(case["angles"][idx], case["spacing"], eta=case["eta"], max_bounces=case["max_bounces"],
                   offset=case["offset"])
    rec_bytes = 32.0 * st["valid_rays"]
    pk, src = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    res = []
    for nf in (1, 2, 16):
        f = np.linspace(9e9, 11e9, nf)
        E = torch.empty(n_asp, nf, 2, 2, dtype=torch.float64, device="cuda")
        R = torch.empty(n_asp, nf, 2, dtype=torch.float64, device="cuda")
        for _ in range(max(1, args.warmup)):
            ctx.po_integrate(f, "HH,VV", E_out=E, rcs_out=R)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.po_integrate(f, "HH,VV", E_out=E, rcs_out=R)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res.append({"frequencies": nf, "ms": ms, "tube_freqs_per_s": st["valid_rays"] * nf / (ms * 1e-3),
                    "record_gbs": rec_bytes / (ms * 1e-3) / 1e9,
                    "kernel": "k_po_bulk" if nf <= 2 else "k_po"})
    ctx.close()
    one = res[0]
    if rank == 0:
        print(json.dumps({"metric": "PO tube-frequencies/s (one frequency)", "value": one["tube_freqs_per_s"] * ws,
                          "unit": "tube-frequencies/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic",
                          "config": {"workload": f"po_aircraft_10GHz_{n_asp}aspects", "records": st["valid_rays"],
                                     "record_bytes": rec_bytes, "pols": "HH,VV"},
                          "roofline": {"bound": "hbm", "kernel": "k_po_bulk (one frequency)",
                                       "achieved": one["record_gbs"], "peak": hbm, "unit": "GB/s",
                                       "frac": one["record_gbs"] / hbm, "traffic": None,
                                       "peak_source": f"HBM copy bandwidth, {src}",
                                       "note": "time of the whole call: work list, PO sum, final sums"},
                          "frequencies": res}))


def run_sbr(args, case, ws, rank, local, pg):
    import torch

    import paper_2604_09243_gb300 as G
    from paper_2604_09243_gb300 import build

    build.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    ctx = G.Context(local, stream=stream)
    ctx.load_mesh(case["xyz"], case["tri"])
    if args.builder != "ploc":
        ctx.build_bvh(builder=args.builder)
    ang = np.ascontiguousarray(case["angles"], np.float64)
    freqs = np.ascontiguousarray(case["freqs"], np.float64)
    B = case["max_bounces"]
    kw = dict(eta=case["eta"], max_bounces=B, window=case.get("window", 0.0), offset=case.get("offset", (0.0, 0.0)))
    na, nf, npol = len(ang), len(freqs), 2
    E_dev = torch.empty((na, nf, npol, 2), dtype=torch.float64, device=f"cuda:{local}")
    R_dev = torch.empty((na, nf, npol), dtype=torch.float64, device=f"cuda:{local}")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    xf = G.TRACE_REQUIRE_ESCAPE if case.get("escape") else 0

    def step(flags=G.TRACE_TIME_PASSES):
        st = ctx.trace(ang, case["spacing"], flags=flags | xf, **kw)
        ctx.po_integrate(freqs, "HH,VV", E_out=E_dev, rcs_out=R_dev)
        return st

    tune = None
    if args.tune:
        # a fixed setting (e.g. the one the autotuner picked), no tuning runs
        ctx.set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(","))})
        tune = {"best": ctx.tuning(), "fixed": True}
    elif not args.no_autotune:
        # untimed: the autotuner picks blocks per SM, ray tile, stack depth, PO item and chunk size on an
        # evenly spaced sample of the workload's aspects
        # enough aspects for at least 16 M rays, so the sample's passes fill the GPU as the full sweep does
        per = np.mean([(lambda g: g["nu"] * g["nv"])(ctx.ray_grid_for(
            ang[i, 0], ang[i, 1], case["spacing"], eta=case["eta"], window=case.get("window", 0.0),
            offset=case.get("offset", (0.0, 0.0)))) for i in np.linspace(0, na - 1, min(na, 8)).round().astype(int)])
        n_tune = max(args.tune_aspects, int(np.ceil(16e6 / max(1.0, per))))
        pick = np.linspace(0, na - 1, min(na, n_tune)).round().astype(int)
        sample = [dict(az=float(ang[i, 0]), el=float(ang[i, 1]), freqs=freqs, spacing=case["spacing"]) for i in pick]
        best, best_ms, trials = ctx.autotune(sample, reps=5, flags=xf, **kw)
        tune = {"best": best, "start": {k: trials[0][k] for k in best}, "start_ms": trials[0]["ms"],
                "best_ms": best_ms, "trials": len(trials),
                "tried": [[{k: t[k] for k in best if t[k] != best[k]}, round(t["ms"], 4), t["status"]]
                          for t in trials],
                "refused": sum(1 for t in trials if t["status"] != 0),
                "sample": f"{len(pick)} of {na} aspects, fastest of 5 runs per setting"}

    for _ in range(args.warmup):
        step()
    cnt = ctx.trace(ang, case["spacing"], flags=G.TRACE_COUNT_VISITS | xf, **kw)  # counting run, untimed
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize()
    sampler.start()
    stats = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 255)
        ev[k][0].record(stream)
        stats.append(step())
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = max_over_ranks(pg, sum(step_ms) / 1e3)
    bounces = stats[0]["ray_bounces"]
    assert all(s["ray_bounces"] == bounces for s in stats)
    value = ws * bounces * args.steps / t_dev

    # --- end to end through the public API from host buffers
    xyz_p = torch.from_numpy(case["xyz"]).pin_memory()
    tri_p = torch.from_numpy(case["tri"]).pin_memory()
    ang_p = torch.from_numpy(ang).pin_memory()
    E_h = np.empty((na, nf, npol, 2))
    R_h = np.empty((na, nf, npol))
    h2d = xyz_p.numel() * 4 + tri_p.numel() * 4 + ang_p.numel() * 8 + freqs.size * 8
    d2h = E_h.nbytes + R_h.nbytes

    def e2e_step():
        ctx.load_mesh(xyz_p.numpy(), tri_p.numpy())
        if args.builder != "ploc":
            ctx.build_bvh(builder=args.builder)
        ctx.trace(ang_p.numpy(), case["spacing"], flags=xf, **kw)
        E, R = ctx.po_integrate(freqs, "HH,VV")
        E_h[...] = np.stack([E.real, E.imag], -1)
        R_h[...] = R

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier(pg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(pg, time.perf_counter() - t0)
    e2e_value = ws * bounces * args.steps / t_e2e

    # --- roofline of the bounce passes (section 8(d) of the method's measurement plan)
    tun = ctx.tuning()
    wide, octant, raster = tun["bvh_width"] == 4, tun["octant"] == 1, tun["raster"] == 1
    props = torch.cuda.get_device_properties(local)
    n_sm = int(props.multi_processor_count)
    l2_bytes = int(getattr(props, "L2_cache_size", 0) or 0)
    l2_gbs = G.probe_l2_bandwidth(local, nbytes=64 << 20, passes=40)
    fp32_tflops = G.probe_fp32_fma(local)
    pk, src = peaks()
    pass_all_s = float(np.mean([s_["pass_ms"] for s_ in stats])) / 1e3
    primary_s = float(np.mean([s_["primary_ms"] for s_ in stats])) / 1e3
    bounce_s = pass_all_s - primary_s
    q_bounce = cnt["ray_bounces"] - cnt["rays_launched"]  # bounce queries: all queries after the primary one
    tri_bounce = cnt["tri_tests"] - cnt["raster_tests"]
    if q_bounce <= 0 and not raster:  # B = 1 with traversed primary rays: the primary pass is the traversal
        q_bounce, tri_bounce, bounce_s = cnt["rays_launched"], cnt["tri_tests"], primary_s
    n_node = cnt["node_visits"] / max(q_bounce, 1)
    n_tri = tri_bounce / max(q_bounce, 1)
    B_rb = BYTES_NODE * n_node + BYTES_TRI * n_tri
    F_rb = FLOP_NODE * n_node + FLOP_TRI * n_tri
    nt = len(case["tri"])
    tree = ctx.bvh_info()  # nodes reachable from the root (the node array holds no others)
    node_bytes = tree["n_nodes4"] * 128 if wide else tree["n_nodes"] * (8 * 64 if octant else 64)
    set_bytes = node_bytes + nt * 48
    fits = l2_bytes > 0 and set_bytes <= l2_bytes
    bw = l2_gbs if fits else float(pk.get("hbm_gbs", 6800.0))
    r_mem = bw * 1e9 / max(B_rb, 1e-9)
    r_alu = fp32_tflops * 1e12 / max(F_rb, 1e-9)
    measured = q_bounce / bounce_s if bounce_s > 0 else 0.0  # bounce queries per second of the bounce passes
    mem_bound = r_mem <= r_alu
    r_star = min(r_mem, r_alu)
    traffic = None
    for per_q, setting in TRAFFIC_PER_QUERY.get(args.workload, []):
        if all(tun[k] == v for k, v in setting.items()):
            traffic = per_q * q_bounce
    roof = {"bound": ("l2" if fits else "hbm") if mem_bound else "alu",
            "kernel": f"k_bounce (bounce passes, {'4-wide' if wide else ('binary, octant copies' if octant else 'binary')} tree)",
            "achieved": measured * B_rb / 1e9 if mem_bound else measured * F_rb / 1e12,
            "peak": bw if mem_bound else fp32_tflops,
            "unit": "GB/s" if mem_bound else "TFLOP/s",
            "frac": measured / r_star,
            "traffic": traffic,
            "peak_source": ((f"L2 read probe (sbr_probe_l2_bandwidth, 64 MiB x 40 passes)" if fits else
                             f"HBM copy bandwidth, {src}") if mem_bound else
                            "FP32 FMA probe (sbr_probe_fp32_fma, 2 FLOP per FMA)"),
            "ray_bounces_per_s_bound": r_star, "ray_bounces_per_s_measured": measured,
            "memory_side": {"bw_gbs": bw, "what": "l2" if fits else "hbm", "bytes_per_query": B_rb,
                            "ray_bounces_per_s": r_mem, "frac": measured / r_mem},
            "alu_side": {"tflops": fp32_tflops, "flop_per_query": F_rb, "ray_bounces_per_s": r_alu,
                         "frac": measured / r_alu},
            "node_visits_per_query": n_node, "tri_tests_per_query": n_tri, "bounce_queries_per_step": q_bounce,
            "lane_occupancy_bound": cnt["node_visits"] / max(cnt["warp_node_visits"], 1),
            "tree_and_triangle_bytes": set_bytes, "tree_nodes": tree["n_nodes4"] if wide else tree["n_nodes"],
            "l2_bytes": l2_bytes, "sm_count": n_sm,
            "pass_ms_per_step": bounce_s * 1e3,
            "hit_arithmetic": {"bounce_hits": cnt["bounce_hits"], "primary_hits_rebuilt": cnt["listed_hits"],
                               "ops_per_bounce_hit": OPS_HIT, "ops_per_primary_hit": OPS_PRIMARY_HIT,
                               "t_ops_per_s": (OPS_HIT * cnt["bounce_hits"] + OPS_PRIMARY_HIT * cnt["listed_hits"])
                               / max(bounce_s, 1e-12) / 1e12},
            "exact_decisions": {"open_tests": cnt["open_tests"], "fp64_tests": cnt["fp64_tests"],
                                "tri_tests": cnt["tri_tests"]}}
    if q_bounce <= 0:
        # B = 1 with rasterised primary hits: no traversal runs, and the rasterisation is the dominant kernel
        # (ALU: FLOP_CELL per cell test against the FP32 FMA probe)
        ach = cnt["raster_tests"] * FLOP_CELL / primary_s / 1e12
        roof = {"bound": "alu", "kernel": "k_raster+k_raster_big (rasterised primary hits; no bounce pass at B = 1)",
                "achieved": ach, "peak": fp32_tflops, "unit": "TFLOP/s", "frac": ach / fp32_tflops, "traffic": None,
                "peak_source": "FP32 FMA probe (sbr_probe_fp32_fma, 2 FLOP per FMA)",
                "flop_per_cell_test": FLOP_CELL, "cell_tests_per_step": cnt["raster_tests"],
                "primary_ms_per_step": primary_s * 1e3, "sm_count": n_sm,
                "exact_decisions": {"open_tests": cnt["open_tests"], "fp64_tests": cnt["fp64_tests"],
                                    "tri_tests": cnt["tri_tests"]}}
    launches = stats[0]["kernel_launches"] + 3  # + PO work list, PO reduce and PO final
    line = {"metric": "ray-bounces/s", "value": value, "unit": "ray-bounces/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(wl_config(case, args.workload), bvh_builder=args.builder),
            "angles_per_s": ws * na * args.steps / t_dev,
            "rays_launched_per_step": stats[0]["rays_launched"], "ray_bounces_per_step": bounces,
            "valid_rays_per_step": stats[0]["valid_rays"],
            "roofline": roof,
            "probes": {"l2_read_gbs": l2_gbs, "fp32_fma_tflops": fp32_tflops, "sm_count": n_sm, "l2_bytes": l2_bytes},
            "primary": {"kernel": "k_raster+k_raster_big+k_vis_mask+k_primary_vis (rasterised primary hits)" if raster
                        else "k_primary (traversed)", "ms_per_step": primary_s * 1e3,
                        "transport_ms_per_step": pass_all_s * 1e3, "raster_tests": cnt["raster_tests"],
                        "raster_tests_per_s": cnt["raster_tests"] / primary_s if raster and primary_s > 0 else None},
            "e2e": {"value": e2e_value, "unit": "ray-bounces/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * t_e2e / args.steps},
            "gpu_launches": int(launches * args.steps),
            "autotune": tune,
            "clocks": clocks}
    if not args.no_surrogate:
        line["surrogate"] = surrogate_leg(G, torch, local, ctx if args.workload.startswith("aircraft") else None)
    # the legs below make contexts of their own: free the timed workload's buffers first
    ctx.close()
    if args.workload != "trihedral" and not args.no_trihedral:
        line["trihedral"] = sweep_value(G, torch, local, S.trihedral_case(), dict(tile_w=4, octant=1), 20, 3, flush)
    if args.batch_requests > 0:
        line["batched_vs_plain"] = batched_vs_plain(G, torch, local, args.batch_requests)
    if not args.no_precision:
        line["precision"] = precision_report(G, torch, local)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        n, frac = oracle_sample_size(case)
        b, t, idx = oracle_sample(case, min(n, args.ref_angles), threads, frac)
        line["cpu_baseline"] = {"value": b / t, "unit": "ray-bounces/s", "cores": threads, "kind": "oracle",
                                "sample": f"{len(idx)} of {na} aspects (evenly spaced), "
                                          + ("full ray grids" if frac >= 1.0 else
                                             f"a seeded {100 * frac:.3g} % of each aspect's rays")
                                          + f", {b} ray-bounces in {t:.1f} s wall"}
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sbr", choices=["sbr", "reference"])
    ap.add_argument("--workload", default="aircraft10",
                    choices=["trihedral", "sphere", "aircraft1", "aircraft3", "aircraft10", "aircraft3deep",
                             "surrogate", "gemm", "po"])
    ap.add_argument("--ref-angles", type=int, default=24)
    ap.add_argument("--batch-requests", type=int, default=4096,
                    help="mixed requests for the batched-vs-plain comparison (0 = skip)")
    ap.add_argument("--aspects", type=int, default=0,
                    help="use this many evenly spaced aspects of the sweep (small profiling cases); 0 = all")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-trihedral", action="store_true", help="skip the trihedral sweep reported beside the headline")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the bounded surrogate leg beside the headline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tuning")
    ap.add_argument("--no-precision", action="store_true", help="skip the phase-precision report")
    ap.add_argument("--builder", default="ploc", choices=["ploc", "lbvh"], help="BVH builder of the timed workload")
    ap.add_argument("--tune-aspects", type=int, default=24,
                    help="fewest aspects in the autotuner's sample (more where needed for 16 M rays)")
    ap.add_argument("--tune", default="", help="fixed tuning instead of the autotuner, e.g. tile_w=4,stack_depth=32")
    ap.add_argument("--sur-domains", default="full,patch,patch_dense", help="surrogate: domains to evaluate")
    ap.add_argument("--sur-scale", type=float, default=1.0, help="surrogate: fraction of the sample counts")
    ap.add_argument("--sur-epochs", type=int, default=60)
    ap.add_argument("--sur-rpl", type=float, default=0.0,
                    help="surrogate: rays per wavelength of its SBR runs (0: the domain's own, 10 unless set)")
    args = ap.parse_args()
    ws, rank, local, pg = dist_setup()
    if args.workload in ("gemm", "po"):
        (run_gemm if args.workload == "gemm" else run_po)(args, ws, rank, local, pg)
        if pg is not None:
            pg.destroy_process_group()
        return
    if args.workload == "surrogate":
        run_surrogate(args, ws, rank, local, pg)
        if pg is not None:
            pg.destroy_process_group()
        return
    case = workload(args.workload)
    if args.aspects > 0:
        idx = np.linspace(0, len(case["angles"]) - 1, args.aspects).round().astype(int)
        case["angles"] = case["angles"][idx]
        case["name"] += f"_{args.aspects}aspects"
        args.ref_angles = min(args.ref_angles, args.aspects)
    if args.impl == "reference":
        run_reference(args, case, ws, rank, pg)
    else:
        run_sbr(args, case, ws, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
