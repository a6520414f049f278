"""The multi-GPU form is replicas only: every rank runs the whole workload on
its own GPU, and the ranks share only the timing barrier and the max of their
times (gloo, host). These tests run those pieces as two gloo ranks on the CPU,
and the oracle reference arm under torchrun, where rank 0 alone prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    ws, r, local, pg = bench.dist_setup()
    bench.barrier(pg)
    m = bench.max_over_ranks(pg, 1.5 + rank)
    bench.barrier(pg)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "max": m}, f)
    pg.destroy_process_group()


def test_barrier_and_max_over_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    ps = [mp.Process(target=_rank, args=(r, port, str(tmp_path))) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d == {"ws": 2, "rank": r, "local": r, "max": 2.5}


def test_reference_arm_under_torchrun_prints_once():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2",
           "--workload", "sphere", "--steps", "1", "--warmup", "1", "--ref-angles", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="1"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
