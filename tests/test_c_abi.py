"""The boundary used from plain C: tests/c/sbr_plate.c includes only
include/sbr.h and links only libsbr.so. It compiles on the CPU (no GPU needed);
on a GPU its output equals the Python binding's, and the plate's normal
incidence RCS equals 4 pi A^2 / lambda^2."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import sbr_inputs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "sbr_plate.c")
LIBDIR = os.path.join(ROOT, "paper_2604_09243_gb300", "lib")


def _compile(tmp_path):
    from paper_2604_09243_gb300 import build

    build.build()
    gcc = shutil.which("gcc") or pytest.skip("gcc not found")
    exe = str(tmp_path / "sbr_plate")
    cuda = "/usr/local/cuda"
    cmd = [gcc, "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC, "-o",
           exe, "-L", LIBDIR, "-lsbr", f"-Wl,-rpath,{LIBDIR}", "-L", os.path.join(cuda, "lib64"),
           f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_against_the_header(tmp_path):
    assert os.path.exists(_compile(tmp_path))


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the Python binding passes across the boundary has the
    size, field offsets and field sizes of its C declaration in the header (a
    small C program prints sizeof and offsetof; no GPU and no library needed)."""
    import ctypes as C

    from paper_2604_09243_gb300 import sbr

    gcc = shutil.which("gcc") or pytest.skip("gcc not found")
    pairs = [("sbr_bvh_opts", sbr.BvhOpts), ("sbr_trace_opts", sbr.TraceOpts), ("sbr_tuning", sbr.Tuning),
             ("sbr_tune_trial", sbr.TuneTrial), ("sbr_bvh_info", sbr.BvhInfo), ("sbr_trace_stats", sbr.TraceStats),
             ("sbr_request", sbr.Request), ("sbr_ray_grid", sbr.RayGrid), ("sbr_surrogate_opts", sbr.SurrogateOpts)]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sbr.h"',
             "#define F(T, m) printf(\"%s %s %zu %zu\\n\", #T, #m, offsetof(T, m), sizeof(((T*)0)->m))",
             "int main(void)", "{"]
    for cname, py in pairs:
        lines.append(f'    printf("%s size %zu 0\\n", "{cname}", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f"    F({cname}, {f});")
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            t, m, a, b = ln.split()
            got[(t, m)] = (int(a), int(b))
    for cname, py in pairs:
        assert got[(cname, "size")][0] == C.sizeof(py), cname
        for f, _ in py._fields_:
            d = getattr(py, f)
            assert got[(cname, f)] == (d.offset, d.size), (cname, f)


@pytest.mark.gpu
def test_c_program_matches_binding_and_closed_form(tmp_path):
    exe = _compile(tmp_path)
    ang = [(0.0, 90.0), (30.0, 70.0), (120.0, 60.0)]
    r = subprocess.run([exe] + [f"{v}" for a in ang for v in a], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rows = np.array([[float(x) for x in line.split()] for line in r.stdout.strip().splitlines()])
    import paper_2604_09243_gb300 as G

    xyz, tri = S.square_plate(1.0, 8)
    with G.Context(0) as c:
        c.load_mesh(xyz, tri)
        st = c.trace(ang, G.spacing_for(10e9, 10.0), eta=0.05, max_bounces=1, window=1.3)
        _, R = c.po_integrate([10e9], "HH,VV")
    assert np.array_equal(rows[:, 2:4], R[:, 0, :])
    assert int(rows[0, 4]) == st["valid_rays"]
    lam = 299_792_458.0 / 10e9
    assert abs(rows[0, 2] - 10 * math.log10(4 * math.pi / lam**2)) < 0.1
