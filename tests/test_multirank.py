"""The benchmark's multi-rank path on the CPU (gloo, two ranks on 127.0.0.1).

Fields are independent, so N ranks run replicas with no collective in the
data path: the only cross-rank operations are the barriers around the timed
region and the max over ranks of the elapsed time.  Under torchrun the
reference arm runs on rank 0 alone and the other ranks leave without work.
"""
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


def _rank(rank, port, out):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, _ = bench.dist_setup()
    bench.barrier(ws)
    m = bench.max_over_ranks(ws, 1.5 + r)   # rank 0 reports 1.5, rank 1 reports 2.5
    bench.barrier(ws)
    with open(out, "w") as fh:
        json.dump({"ws": ws, "rank": r, "max": m}, fh)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_barrier_and_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    outs = [str(tmp_path / f"r{i}.json") for i in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(i, port, outs[i])) for i in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = [json.load(open(o)) for o in outs]
    assert [r["rank"] for r in res] == [0, 1]
    assert all(r["ws"] == 2 and r["max"] == 2.5 for r in res)


def test_reference_arm_prints_once_under_torchrun(oracle_mod):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "t31_reg_10"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
