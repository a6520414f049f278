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
