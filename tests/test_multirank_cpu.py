"""The N > 1 paths of bench.py on the CPU (gloo, world size 2).

The decomposition is not sharded ("replicas only": every rank decomposes its
own matrix, no collective on the data path); what a multi-rank run adds is the
rank bookkeeping: the job time is the slowest rank's, and only rank 0 prints.
Both are exercised here without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        out[rank] = bench.max_over_ranks(values[rank], dist)
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_ranks():
    import torch.multiprocessing as mp
    port = _free_port()
    values = [3.25, 7.5]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_max_worker, args=(2, port, values, out), nprocs=2, join=True)
        assert dict(out) == {0: 7.5, 1: 7.5}


def test_single_process_passes_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, None) == 4.0


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2", OPENBLAS_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "pd256"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
